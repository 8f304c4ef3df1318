"""The C ABI from a plain C program (host buffers in and out, no CUDA
headers): built with gcc against include/dfb.h and libdfb.so; on the GPU its
output matches the FP64 oracle."""

import os
import subprocess

import numpy as np
import pytest

from harness import scenes
from oracle import dfb_oracle as o
from paper_2305_07083_gb300 import build, dfb as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def compile_client(tmp_path):
    build()
    exe = str(tmp_path / "composite_host")
    pkg = os.path.dirname(D.LIB)
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "composite_host.c"), "-o", exe, "-L", pkg, "-ldfb",
           "-Wl,-rpath," + pkg]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def test_c_client_compiles_and_links(tmp_path):
    exe = compile_client(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 2 and "usage" in r.stderr


@pytest.mark.gpu
def test_c_client_matches_oracle(tmp_path):
    exe = compile_client(tmp_path)
    sc = scenes.scene_data_parallel(160, 96, 32, (3, 2, 2), seed=12, jitter_sigma=0.05)
    frames = [sc.frame_rgba(f) for f in range(3)]
    scene = tmp_path / "scene.bin"
    with open(scene, "wb") as f:
        f.write(np.array([sc.W, sc.H, sc.T, len(frames)], np.int32).tobytes())
        for rgba in frames:
            f.write(np.array([len(sc.tile_ids)], np.int32).tobytes())
            f.write(np.ascontiguousarray(sc.tile_ids, np.int32).tobytes())
            f.write(np.ascontiguousarray(sc.keys, np.float32).tobytes())
            f.write(np.ascontiguousarray(rgba, np.float32).tobytes())
            f.write(np.ascontiguousarray(sc.depth, np.float32).tobytes())
    out = tmp_path / "out.bin"
    r = subprocess.run([exe, str(scene), str(out)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "accumulated 3" in r.stdout
    raw = np.fromfile(out, dtype=np.uint8)
    px = sc.W * sc.H
    rgba8 = raw[:4 * px].view(np.uint32).reshape(sc.H, sc.W)
    mean = raw[4 * px:].view(np.float32).reshape(sc.H, sc.W, 4)
    imgs = [o.composite_frame(sc.W, sc.H, sc.T, o.BLEND_DEPTH, sc.tile_ids, sc.keys,
                              rgba.astype(np.float64), sc.depth) for rgba in frames]
    want = o.accumulate(imgs)
    assert np.max(np.abs(mean - want)) <= 1e-5
    d8 = np.abs(o.unpack_rgba8(rgba8) - o.unpack_rgba8(o.pack_rgba8(want)))
    assert d8.max() <= 1
