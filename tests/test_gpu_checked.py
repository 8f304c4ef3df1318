"""The checked build (libdfb_checked.so, compiled with device-side bounds
checks on the composite's shared-memory ring, its queue, and every output
index): the parity, batch and image-parallel tests pass with it loaded, so
no check fires on any of their cases (a fired check turns the next sync or
read into DFB_ERR_CHECK)."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_is_loaded_and_tests_pass():
    env = dict(os.environ, DFB_CHECKED="1")
    probe = subprocess.run(
        [sys.executable, "-c", "from paper_2305_07083_gb300 import dfb as D; D.lib(); print(D.LIB)"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert probe.returncode == 0, probe.stderr
    assert probe.stdout.strip().endswith("libdfb_checked.so")
    files = ["tests/test_gpu_parity.py", "tests/test_gpu_batch.py",
             "tests/test_gpu_image_parallel.py", "tests/test_gpu_pack.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p",
                        "no:cacheprovider", *files], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
