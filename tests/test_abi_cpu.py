"""The C ABI without a GPU: the library loads, exports every declared entry
point, and its host-side logic (validation, frame state, per-tile dependency
trees of Sec. 3.1.1) answers with the documented status codes.  No kernel is
launched: every case here stops at a host-side check."""

import ctypes as C
import math
import os
import re

import numpy as np
import pytest

from paper_2305_07083_gb300 import build, dfb as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def declared_symbols():
    with open(os.path.join(ROOT, "include", "dfb.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"DFB_API\s+[\w\s\*]+?\b(dfb_\w+)\s*\(", text)))


@pytest.mark.parametrize("lib", ["normal", "checked"])
def test_exports_every_declared_symbol(lib):
    from paper_2305_07083_gb300 import _build
    syms = declared_symbols()
    assert len(syms) >= 25
    L = C.CDLL(_build.LIB if lib == "normal" else _build.LIB_CHECKED)
    for s in syms:
        assert hasattr(L, s), s


def test_error_strings_and_version():
    assert D.dfb_version() >= 10000
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8, -9):
        assert D.dfb_error_string(code) not in ("", "unknown status")
    assert D.dfb_error_string(-99) == "unknown status"


@pytest.mark.parametrize("W,H,T,mode,dtype,flags", [
    (0, 64, 16, 0, 0, 1), (64, -1, 16, 0, 0, 1), (64, 64, 12, 0, 0, 1), (64, 64, 2, 0, 0, 1),
    (64, 64, 512, 0, 0, 1), (64, 64, 16, 4, 0, 1), (64, 64, 16, 0, 4, 1), (64, 64, 16, 0, 0, 64),
    (1 << 16, (1 << 15) + 1, 16, 0, 0, 1),    # more than 2^31 pixels
    ((1 << 24) + 1, 1, 256, 0, 0, 1)])        # whole tiles hold more than 2^32 pixels
def test_create_rejects_bad_config(W, H, T, mode, dtype, flags):
    with pytest.raises(D.DfbError) as e:
        D.dfb_create_ex(W, H, T, mode, dtype, flags)
    assert e.value.code == D.DFB_ERR_INVALID_ARG


def deferred(W=64, H=48, T=16, dtype=D.DFB_F32, mode=D.DFB_BLEND_DEPTH):
    return D.dfb_create_ex(W, H, T, mode, dtype, D.DFB_FLAGS_DEFAULT | D.DFB_FLAG_DEFER_ALLOC)


FAKE = 1 << 20      # aligned fake device addresses: never dereferenced here


def submit(h, tiles, keys=None, rgba=None, depth=None, scales=None):
    n = len(tiles)
    keys = np.zeros(n, np.float32) if keys is None else keys
    rgba = [FAKE + 4096 * i for i in range(n)] if rgba is None else rgba
    depth = [FAKE * 2 + 4096 * i for i in range(n)] if depth is None else depth
    D.dfb_submit_tiles(h, tiles, keys, rgba, depth, scales, D.DFB_PTR_DEVICE)


def code_of(fn, *a):
    with pytest.raises(D.DfbError) as e:
        fn(*a)
    return e.value.code


def ex(h, rows, scale=1.0):
    """dfb_submit_tiles_ex on fake device addresses; rows = (tile, key, gen, children)."""
    D.dfb_submit_tiles_ex(h, [(t, k, FAKE, FAKE, scale, g, c) for t, k, g, c in rows],
                          D.DFB_PTR_DEVICE)


def test_frame_state_machine():
    h = deferred()
    try:
        assert code_of(submit, h, [0]) == D.DFB_ERR_STATE           # no open frame
        assert code_of(D.dfb_set_tile_children, h, 0, 1) == D.DFB_ERR_STATE
        assert code_of(D.dfb_end_frame, h) == D.DFB_ERR_STATE
        D.dfb_begin_frame(h, 0)
        assert code_of(D.dfb_begin_frame, h, 0) == D.DFB_ERR_STATE  # already open
        assert code_of(D.dfb_read_color, h, np.zeros(4, np.float32)) == D.DFB_ERR_STATE
    finally:
        D.dfb_destroy(h)


def test_submit_validation():
    h = deferred(dtype=D.DFB_F32)
    try:
        D.dfb_begin_frame(h, 0)
        tx, ty = D.dfb_get_tiles(h)
        assert (tx, ty) == (4, 3)
        assert code_of(submit, h, [12]) == D.DFB_ERR_TILE_RANGE
        assert code_of(submit, h, [-1]) == D.DFB_ERR_TILE_RANGE
        assert code_of(submit, h, [0], np.array([math.nan], np.float32)) == D.DFB_ERR_INVALID_ARG
        assert code_of(submit, h, [0], None, [FAKE + 4]) == D.DFB_ERR_INVALID_ARG   # rgba 16B
        assert code_of(submit, h, [0], None, None, [FAKE + 2]) == D.DFB_ERR_INVALID_ARG
        assert code_of(submit, h, [0], None, [0]) == D.DFB_ERR_INVALID_ARG          # null
        assert code_of(ex, h, [(0, 0.0, 0, 0)]) == D.DFB_ERR_INVALID_ARG       # generation 0
        assert code_of(ex, h, [(0, 0.0, 1, -1)]) == D.DFB_ERR_INVALID_ARG      # children < 0
    finally:
        D.dfb_destroy(h)
    h8 = deferred(dtype=D.DFB_FP8E4M3)
    try:
        D.dfb_begin_frame(h8, 0)
        assert code_of(D.dfb_submit_tile, h8, 0, 0.0, FAKE, FAKE) == D.DFB_ERR_INVALID_ARG
        assert code_of(submit, h8, [0]) == D.DFB_ERR_INVALID_ARG                  # no scales
        for bad in (0.0, -1.0, math.inf, math.nan):
            assert code_of(submit, h8, [0], None, None, None,
                           np.array([bad], np.float32)) == D.DFB_ERR_INVALID_ARG
        submit(h8, [0], scales=np.array([0.5], np.float32))
        # every tile is streamed with bulk copies: 16-byte alignment for all dtypes
        assert code_of(submit, h8, [0], None, [FAKE + 4], None,
                       np.array([0.5], np.float32)) == D.DFB_ERR_INVALID_ARG
        assert code_of(submit, h8, [0], None, None, [FAKE + 8],
                       np.array([0.5], np.float32)) == D.DFB_ERR_INVALID_ARG
    finally:
        D.dfb_destroy(h8)


def test_dependency_tree_counts():
    """Sec. 3.1.1: the children declared by a generation give the number of
    tiles expected in the next; completion needs every generation."""
    h = deferred()
    try:
        D.dfb_begin_frame(h, 0)
        D.dfb_set_tile_children(h, 5, 3)
        assert code_of(D.dfb_set_tile_children, h, 5, 1) == D.DFB_ERR_STATE   # declared twice
        assert code_of(D.dfb_set_tile_children, h, 99, 1) == D.DFB_ERR_TILE_RANGE
        assert code_of(D.dfb_set_tile_children, h, 1, -2) == D.DFB_ERR_INVALID_ARG
        submit(h, [5, 5])
        assert code_of(D.dfb_end_frame, h) == D.DFB_ERR_INCOMPLETE            # 2 of 3
        submit(h, [5, 5])
        assert code_of(D.dfb_end_frame, h) == D.DFB_ERR_INCOMPLETE            # 4 of 3
    finally:
        D.dfb_destroy(h)


def test_multi_generation_tree():
    h = deferred()
    try:
        D.dfb_begin_frame(h, 0)
        D.dfb_set_tile_children(h, 2, 2)
        # generation 1: two tiles, declaring 1 + 2 children in generation 2;
        # arrival order across generations is arbitrary
        ex(h, [(2, 2.0, 2, 0), (2, 0.0, 1, 1), (2, 3.0, 2, 0), (2, 1.0, 1, 2)])
        assert code_of(D.dfb_end_frame, h) == D.DFB_ERR_INCOMPLETE            # 2 of 3 in gen 2
        ex(h, [(2, 4.0, 2, 0)])
        # a stray generation-3 tile nobody declared
        ex(h, [(2, 5.0, 3, 0)])
        assert code_of(D.dfb_end_frame, h) == D.DFB_ERR_INCOMPLETE
    finally:
        D.dfb_destroy(h)


def test_bulk_submit_is_all_or_nothing():
    h = deferred()
    try:
        D.dfb_begin_frame(h, 0)
        D.dfb_set_tile_children(h, 0, 2)
        assert code_of(submit, h, [0, 0, 77]) == D.DFB_ERR_TILE_RANGE
        # nothing from the rejected call was kept: still 0 of 2 received
        submit(h, [0])
        assert code_of(D.dfb_end_frame, h) == D.DFB_ERR_INCOMPLETE
    finally:
        D.dfb_destroy(h)


@pytest.mark.skipif(_has_gpu(), reason="would launch kernels on the fake addresses")
def test_complete_multi_generation_tree_passes_host_checks():
    h = deferred()
    try:
        D.dfb_begin_frame(h, 0)
        D.dfb_set_tile_children(h, 2, 2)
        ex(h, [(2, 2.0, 2, 0), (2, 0.0, 1, 1), (2, 3.0, 2, 0), (2, 1.0, 1, 2), (2, 4.0, 2, 0)])
        assert code_of(D.dfb_end_frame, h) == D.DFB_ERR_CUDA   # trees fine; no device here
    finally:
        D.dfb_destroy(h)


@pytest.mark.skipif(_has_gpu(), reason="would launch kernels on the fake addresses")
def test_complete_frame_without_device_reports_cuda_error():
    h = deferred()
    try:
        D.dfb_begin_frame(h, 0)
        D.dfb_set_tile_children(h, 0, 1)
        submit(h, [0])
        assert code_of(D.dfb_end_frame, h) == D.DFB_ERR_CUDA
        # the frame stays open, so it can still be ended once a device is present
        assert code_of(D.dfb_begin_frame, h, 0) == D.DFB_ERR_STATE
    finally:
        D.dfb_destroy(h)


def test_wait_limit_and_stall_arguments():
    h = deferred()
    try:
        D.dfb_set_wait_limit(h, 0.01)
        assert code_of(D.dfb_set_wait_limit, h, 0.0) == D.DFB_ERR_INVALID_ARG
        assert code_of(D.dfb_set_wait_limit, h, 1e9) == D.DFB_ERR_INVALID_ARG
        D.dfb_inject_stall(h, 3)
        D.dfb_inject_stall(h, -1)
        assert code_of(D.dfb_inject_stall, h, -5) == D.DFB_ERR_INVALID_ARG
    finally:
        D.dfb_destroy(h)
    # the allocation-free call's process-wide settings
    assert code_of(D.dfb_noalloc_set_wait_limit, 0.0) == D.DFB_ERR_INVALID_ARG
    assert code_of(D.dfb_noalloc_set_wait_limit, -1.0) == D.DFB_ERR_INVALID_ARG
    assert code_of(D.dfb_noalloc_set_wait_limit, 4000.0) == D.DFB_ERR_INVALID_ARG
    assert code_of(D.dfb_noalloc_inject_stall, -2) == D.DFB_ERR_INVALID_ARG
    D.dfb_noalloc_set_wait_limit(2.0)
    D.dfb_noalloc_inject_stall(-1)


def test_null_handle_and_pointers():
    L = D.lib()
    assert L.dfb_destroy(None) == 0
    assert L.dfb_begin_frame(None, 0) == D.DFB_ERR_INVALID_ARG
    assert L.dfb_create_ex(None, None) == D.DFB_ERR_INVALID_ARG
    assert L.dfb_end_frames(None, 1, None) == D.DFB_ERR_INVALID_ARG
    assert L.dfb_convert_tiles(None, None, None, 1, 16, 1, None) == D.DFB_ERR_INVALID_ARG


# --- prepared submissions (validated on the host; nothing is launched) -------
def _deferred(W=128, H=64, T=32, dtype=D.DFB_F32):
    return D.dfb_create_ex(W, H, T, D.DFB_BLEND_DEPTH, dtype,
                           D.DFB_FLAGS_DEFAULT | D.DFB_FLAG_DEFER_ALLOC)


def _fake_pointers(n, tile_bytes, base):
    # addresses are only validated here (alignment), never dereferenced
    return np.uint64(base) + np.arange(n, dtype=np.uint64) * np.uint64(tile_bytes)


def test_tileset_validation():
    h = _deferred()
    tid = np.array([0, 3, 7, 3], np.int32)
    key = np.array([0.5, 1.0, 2.0, 0.25], np.float32)
    rp = _fake_pointers(4, 32 * 32 * 16, 1 << 40)
    dp = _fake_pointers(4, 32 * 32 * 4, 1 << 41)
    s = D.dfb_tileset_create(h, tid, key, rp, dp)
    bad = dict(tid=np.array([0, 8, 1, 2], np.int32))          # 8 tiles: ids 0..7
    with pytest.raises(D.DfbError) as e:
        D.dfb_tileset_create(h, bad["tid"], key, rp, dp)
    assert e.value.code == D.DFB_ERR_TILE_RANGE
    with pytest.raises(D.DfbError) as e:
        D.dfb_tileset_create(h, tid, key, rp + np.uint64(4), dp)   # misaligned
    assert e.value.code == D.DFB_ERR_INVALID_ARG
    with pytest.raises(D.DfbError) as e:
        D.dfb_tileset_create(h, tid, np.array([0, math.nan, 1, 2], np.float32), rp, dp)
    assert e.value.code == D.DFB_ERR_INVALID_ARG
    # FP8 sets need positive finite scales
    h8 = _deferred(dtype=D.DFB_FP8E4M3)
    with pytest.raises(D.DfbError) as e:
        D.dfb_tileset_create(h8, tid, key, rp, dp)
    assert e.value.code == D.DFB_ERR_INVALID_ARG
    s8 = D.dfb_tileset_create(h8, tid, key, rp, dp, np.ones(4, np.float32))
    # submitting: only inside a frame, only into handles of the same shape
    with pytest.raises(D.DfbError) as e:
        D.dfb_submit_tileset(h, s)
    assert e.value.code == D.DFB_ERR_STATE
    D.dfb_begin_frame(h, 0)
    D.dfb_submit_tileset(h, s)
    with pytest.raises(D.DfbError) as e:
        D.dfb_submit_tileset(h, s8)          # other dtype
    assert e.value.code == D.DFB_ERR_INVALID_ARG
    other = _deferred(W=96)
    D.dfb_begin_frame(other, 0)
    with pytest.raises(D.DfbError) as e:
        D.dfb_submit_tileset(other, s)       # other geometry
    assert e.value.code == D.DFB_ERR_INVALID_ARG
    empty = D.dfb_tileset_create(h, [], [], [], [])
    D.dfb_submit_tileset(h, empty)
    for x in (s, s8, empty):
        D.dfb_tileset_destroy(x)
    for x in (h, h8, other):
        D.dfb_destroy(x)


def test_tileset_counts_toward_declared_trees():
    """A set's tiles are generation-1 arrivals: a tile that declared more
    children than the set delivers keeps the frame open (INCOMPLETE is
    returned before any device work)."""
    h = _deferred()
    tid = np.array([2, 2, 5], np.int32)
    s = D.dfb_tileset_create(h, tid, np.zeros(3, np.float32),
                             _fake_pointers(3, 32 * 32 * 16, 1 << 40),
                             _fake_pointers(3, 32 * 32 * 4, 1 << 41))
    D.dfb_begin_frame(h, 0)
    D.dfb_set_tile_children(h, 2, 3)
    D.dfb_submit_tileset(h, s)
    with pytest.raises(D.DfbError) as e:
        D.dfb_end_frame(h)
    assert e.value.code == D.DFB_ERR_INCOMPLETE
    D.dfb_tileset_destroy(s)
    D.dfb_destroy(h)


def test_run_frames_validates_before_beginning():
    a, b = _deferred(), _deferred()
    c = _deferred(dtype=D.DFB_F16)
    mk = lambda h, dt=16: D.dfb_tileset_create(h, [1], [0.0],
                                               _fake_pointers(1, 32 * 32 * dt, 1 << 40),
                                               _fake_pointers(1, 32 * 32 * 4, 1 << 41))
    sa, sc = mk(a), mk(c, 8)
    with pytest.raises(D.DfbError) as e:
        D.dfb_run_frames([a, a], [sa, sa])                   # not distinct
    assert e.value.code == D.DFB_ERR_INVALID_ARG
    with pytest.raises(D.DfbError) as e:
        D.dfb_run_frames([a, c], [sa, sc])                   # mixed dtypes
    assert e.value.code == D.DFB_ERR_INVALID_ARG
    with pytest.raises(D.DfbError) as e:
        D.dfb_run_frames([a, b], [sa, sc])                   # set of another dtype
    assert e.value.code == D.DFB_ERR_INVALID_ARG
    D.dfb_begin_frame(b, 0)
    with pytest.raises(D.DfbError) as e:
        D.dfb_run_frames([a, b], [sa, sa])                   # b is inside a frame
    assert e.value.code == D.DFB_ERR_STATE
    # nothing was begun on `a` by the failed calls
    with pytest.raises(D.DfbError) as e:
        D.dfb_submit_tileset(a, sa)
    assert e.value.code == D.DFB_ERR_STATE
    for x in (sa, sc):
        D.dfb_tileset_destroy(x)
    for x in (a, b, c):
        D.dfb_destroy(x)


def test_tuning_shapes():
    h = _deferred()
    for shape in ((110, 2, 1), (110, 2, 2), (72, 3, 1), (220, 1, 2), (220, 1, 3), (0, 0, 0)):
        D.dfb_set_tuning(h, *shape)
    for shape in ((110, 2, 3), (110, 4, 1), (220, 1, 4), (0, 2, 1), (300, 2, 1), (110, 0, 0),
                  (-1, 2, 1)):
        with pytest.raises(D.DfbError) as e:
            D.dfb_set_tuning(h, *shape)
        assert e.value.code == D.DFB_ERR_INVALID_ARG
    D.dfb_destroy(h)


def test_pixel_op_validation():
    h = _deferred()
    for op, e in ((D.DFB_PIXELOP_NONE, 1.0), (D.DFB_PIXELOP_EXPOSURE, 0.0),
                  (D.DFB_PIXELOP_REINHARD, 4.0)):
        D.dfb_set_pixel_op(h, op, e)
    for op, e in ((4, 1.0), (-1, 1.0), (D.DFB_PIXELOP_EXPOSURE, -1.0),
                  (D.DFB_PIXELOP_REINHARD, math.nan), (D.DFB_PIXELOP_EXPOSURE, math.inf),
                  (D.DFB_PIXELOP_CURVE, -2.0)):
        with pytest.raises(D.DfbError) as e_:
            D.dfb_set_pixel_op(h, op, e)
        assert e_.value.code == D.DFB_ERR_INVALID_ARG
    # the curve operation needs a curve loaded first
    with pytest.raises(D.DfbError) as e_:
        D.dfb_set_pixel_op(h, D.DFB_PIXELOP_CURVE, 1.0)
    assert e_.value.code == D.DFB_ERR_STATE
    D.dfb_destroy(h)
    a = D.dfb_create_ex(64, 64, 16, D.DFB_AVERAGE, D.DFB_F32,
                        D.DFB_FLAGS_DEFAULT | D.DFB_FLAG_DEFER_ALLOC)
    D.dfb_destroy(a)


def test_pixel_curve_validation():
    """Argument checks of dfb_set_pixel_curve, all made before any CUDA call."""
    h = _deferred()
    good = np.linspace(0.0, 1.0, 8, dtype=np.float32)
    bad_cases = [
        (np.stack([good] * 3)[:, :1], 1.0),                       # n = 1
        (np.zeros((3, 4097), np.float32), 1.0),                   # n > 4096
        (np.stack([good] * 3), 0.0),                              # x_max = 0
        (np.stack([good] * 3), -1.0),
        (np.stack([good] * 3), math.nan),
        (np.stack([good] * 3), math.inf),
        (np.stack([good, good, np.where(good > 0.5, np.nan, good)]), 1.0),   # a NaN sample
        (np.stack([good, np.full(8, np.inf, np.float32), good]), 1.0),
    ]
    for curves, xm in bad_cases:
        with pytest.raises(D.DfbError) as e_:
            D.dfb_set_pixel_curve(h, curves, xm)
        assert e_.value.code == D.DFB_ERR_INVALID_ARG
    assert D.lib().dfb_set_pixel_curve(h, None, 8, 1.0) == D.DFB_ERR_INVALID_ARG
    assert D.lib().dfb_set_pixel_curve(None, np.stack([good] * 3).ctypes.data, 8,
                                       1.0) == D.DFB_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        D.dfb_set_pixel_curve(h, good, 1.0)                        # not 3 rows
    # nothing was loaded, so the operation still cannot be selected
    with pytest.raises(D.DfbError) as e_:
        D.dfb_set_pixel_op(h, D.DFB_PIXELOP_CURVE, 1.0)
    assert e_.value.code == D.DFB_ERR_STATE
    D.dfb_destroy(h)


def test_binding_rejects_strided_buffers():
    """The library reads and writes buffers densely, so the binding refuses a
    strided view instead of handing out its base address."""
    import torch
    a = np.zeros((8, 8, 4), np.float32)
    assert D._ptr(a) == a.ctypes.data
    with pytest.raises(ValueError):
        D._ptr(a[:, ::2])
    with pytest.raises(ValueError):
        D._ptr(a.transpose(1, 0, 2))
    t = torch.zeros((8, 8, 4))
    assert D._ptr(t) == t.data_ptr()
    with pytest.raises(ValueError):
        D._ptr(t[:, ::2])
    assert D._ptr(None) is None and D._ptr(1234) == 1234


def _header_constants():
    """Integer constants of include/dfb.h: enumerators and #defines."""
    with open(os.path.join(ROOT, "include", "dfb.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    vals = {}
    for name, v in re.findall(r"\b(DFB_[A-Z0-9_]+)\s*=\s*(-?\d+)", text):
        vals[name] = int(v)
    for name, v in re.findall(r"#define\s+(DFB_[A-Z0-9_]+)\s+(\d+)u?\b", text):
        vals[name] = int(v)
    return vals


def test_binding_and_oracle_constants_match_the_header():
    """The header, the binding and the oracle (which defines its enums on its
    own) agree on every value they share."""
    from oracle import dfb_oracle as o
    hdr = _header_constants()
    assert len(hdr) >= 30
    for name, v in hdr.items():
        assert getattr(D, name) == v, name
    assert D.DFB_FLAGS_DEFAULT == (hdr["DFB_FLAG_ACCUMULATE"] | hdr["DFB_FLAG_WRITE_COLOR"]
                                   | hdr["DFB_FLAG_PACK_RGBA8"])
    pairs = {"BLEND_DEPTH": "DFB_BLEND_DEPTH", "BLEND_ORDERED": "DFB_BLEND_ORDERED",
             "ZCOMPOSITE": "DFB_ZCOMPOSITE", "AVERAGE": "DFB_AVERAGE",
             "PIXELOP_NONE": "DFB_PIXELOP_NONE", "PIXELOP_EXPOSURE": "DFB_PIXELOP_EXPOSURE",
             "PIXELOP_REINHARD": "DFB_PIXELOP_REINHARD", "PIXELOP_CURVE": "DFB_PIXELOP_CURVE",
             "F32": "DFB_F32", "F16": "DFB_F16", "BF16": "DFB_BF16", "FP8E4M3": "DFB_FP8E4M3"}
    for ours, theirs in pairs.items():
        assert getattr(o, ours) == hdr[theirs], ours
