"""GB300 (sm_103a) implementation of the Distributed FrameBuffer's per-tile
sort-last compositing path: a C-ABI library (libdfb.so, include/dfb.h) with
hand-written CUDA kernels, and a thin ctypes binding (``dfb``)."""

from ._build import build  # noqa: F401
from . import dfb  # noqa: F401
