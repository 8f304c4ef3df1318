"""Build libdfb.so in-tree with nvcc for sm_103a (GB300), and its checked
twin libdfb_checked.so (-DDFB_CHECKED: device-side bounds checks that report
DFB_ERR_CHECK instead of touching memory out of range).

All translation units of both libraries compile in parallel; the link uses
the static CUDA runtime so the library loads without a GPU driver (its first
CUDA call then reports DFB_ERR_CUDA).
"""

from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdfb.so")
LIB_CHECKED = os.path.join(PKG, "libdfb_checked.so")
VARIANTS = [(LIB, "normal", []), (LIB_CHECKED, "checked", ["-DDFB_CHECKED"])]
SOURCES = ["dfb_composite.cu", "dfb_kernels.cu", "dfb_api.cu", "dfb_noalloc.cu"]
HEADERS = [os.path.join(CSRC, "dfb_internal.h"), os.path.join(CSRC, "dfb_device.cuh"),
           os.path.join(ROOT, "include", "dfb.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-DDFB_BUILDING", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return "nvcc"


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + HEADERS + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    todo = [v for v in VARIANTS if force or _stale(v[0])]
    if not todo:
        return LIB
    jobs = []
    for lib, tag, extra in todo:
        os.makedirs(os.path.join(BUILD, tag), exist_ok=True)
        objs = []
        for src in SOURCES:
            obj = os.path.join(BUILD, tag, src.replace(".cu", ".o"))
            cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
            objs.append(obj)
        jobs.append((lib, objs))
    links = []
    for job in jobs:
        if isinstance(job[1], list):
            links.append(job)
            continue
        cmd, p = job
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: %s\n%s" % (" ".join(cmd), out.decode(errors="replace")))
        if verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
    for lib, objs in links:
        tmp = lib + ".tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("link failed: %s\n%s" % (" ".join(cmd), r.stdout.decode(errors="replace")))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
