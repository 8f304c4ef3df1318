"""ctypes binding of libdfb.so (include/dfb.h).

Argument marshalling only: every function here has the name of the C entry
point it calls and raises ``DfbError`` on a negative status.  Buffers may be
given as torch tensors (host or device), numpy arrays, or integer addresses.
There is no fallback: if the library is not built, loading it raises.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._build import LIB as _LIB_NORMAL, LIB_CHECKED

# DFB_CHECKED=1 in the environment loads the checked build (device-side bounds
# checks that report DFB_ERR_CHECK); it must be set before the first call.
LIB = LIB_CHECKED if os.environ.get("DFB_CHECKED") == "1" else _LIB_NORMAL

# enums (include/dfb.h)
DFB_BLEND_DEPTH, DFB_BLEND_ORDERED, DFB_ZCOMPOSITE, DFB_AVERAGE = 0, 1, 2, 3
DFB_PIXELOP_NONE, DFB_PIXELOP_EXPOSURE, DFB_PIXELOP_REINHARD, DFB_PIXELOP_CURVE = 0, 1, 2, 3
DFB_F32, DFB_F16, DFB_BF16, DFB_FP8E4M3 = 0, 1, 2, 3
DFB_OK = 0
DFB_ERR_INVALID_ARG, DFB_ERR_TILE_RANGE, DFB_ERR_STATE, DFB_ERR_INCOMPLETE = -1, -2, -3, -4
DFB_ERR_OOM, DFB_ERR_TIMEOUT, DFB_ERR_CUDA, DFB_ERR_CAPACITY = -5, -6, -7, -8
DFB_ERR_CHECK = -9
DFB_FLAG_ACCUMULATE, DFB_FLAG_WRITE_COLOR, DFB_FLAG_PACK_RGBA8, DFB_FLAG_DEFER_ALLOC = 1, 2, 4, 8
DFB_FLAGS_DEFAULT = DFB_FLAG_ACCUMULATE | DFB_FLAG_WRITE_COLOR | DFB_FLAG_PACK_RGBA8
DFB_PTR_AUTO, DFB_PTR_DEVICE, DFB_PTR_HOST, DFB_PTR_HOST_BORROWED = 0, 1, 2, 3

ELEMENT_BYTES = {DFB_F32: 4, DFB_F16: 2, DFB_BF16: 2, DFB_FP8E4M3: 1}


class DfbError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, dfb_error_string(code), code))


class dfb_config(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("tile_size", C.c_int),
                ("mode", C.c_int), ("dtype", C.c_int), ("flags", C.c_uint),
                ("kahan_after", C.c_int), ("max_fragments", C.c_int)]


class dfb_tile_desc(C.Structure):
    _fields_ = [("tile_id", C.c_int), ("order_key", C.c_float), ("rgba", C.c_void_p),
                ("depth", C.c_void_p), ("scale", C.c_float), ("generation", C.c_int),
                ("children", C.c_int)]


class dfb_frame_stats(C.Structure):
    _fields_ = [("fragments", C.c_int64), ("fragment_pixels", C.c_int64),
                ("frame_pixels", C.c_int64), ("fragment_bytes", C.c_int64),
                ("state_bytes", C.c_int64), ("accumulated", C.c_int32), ("tiles", C.c_int32),
                ("kernel_launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class dfb_timing(C.Structure):
    _fields_ = [("launches", C.c_int32), ("bucket_ms", C.c_float), ("composite_ms", C.c_float)]


_lib = None
H = C.c_void_p
P = C.c_void_p


def lib():
    """Load libdfb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError("%s is not built; call paper_2305_07083_gb300.build()" % LIB)
    L = C.CDLL(LIB)
    sig = {
        "dfb_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(H)]),
        "dfb_create_ex": (C.c_int, [C.POINTER(dfb_config), C.POINTER(H)]),
        "dfb_destroy": (C.c_int, [H]),
        "dfb_set_background": (C.c_int, [H, C.c_float, C.c_float, C.c_float, C.c_float]),
        "dfb_set_pixel_op": (C.c_int, [H, C.c_int, C.c_float]),
        "dfb_set_pixel_curve": (C.c_int, [H, P, C.c_int, C.c_float]),
        "dfb_begin_frame": (C.c_int, [H, C.c_int]),
        "dfb_set_tile_children": (C.c_int, [H, C.c_int, C.c_int]),
        "dfb_submit_tile": (C.c_int, [H, C.c_int, C.c_float, P, P]),
        "dfb_submit_tile_ex": (C.c_int, [H, C.POINTER(dfb_tile_desc)]),
        "dfb_submit_tiles": (C.c_int, [H, C.c_int, P, P, P, P, P, C.c_int]),
        "dfb_submit_tiles_ex": (C.c_int, [H, C.c_int, P, C.c_int]),
        "dfb_end_frame": (C.c_int, [H, P]),
        "dfb_end_frames": (C.c_int, [P, C.c_int, P]),
        "dfb_tileset_create": (C.c_int, [H, C.c_int, P, P, P, P, P, C.POINTER(H)]),
        "dfb_tileset_destroy": (C.c_int, [H]),
        "dfb_submit_tileset": (C.c_int, [H, H]),
        "dfb_run_frames": (C.c_int, [P, P, P, C.c_int, P]),
        "dfb_sync": (C.c_int, [H]),
        "dfb_read_color": (C.c_int, [H, P]),
        "dfb_read_accum": (C.c_int, [H, P]),
        "dfb_read_variance": (C.c_int, [H, P, P]),
        "dfb_read_rgba8": (C.c_int, [H, P]),
        "dfb_get_stats": (C.c_int, [H, C.POINTER(dfb_frame_stats)]),
        "dfb_get_tiles": (C.c_int, [H, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "dfb_save_accum": (C.c_int, [H, P, P, P, C.POINTER(C.c_int)]),
        "dfb_load_accum": (C.c_int, [H, P, P, P, C.c_int]),
        "dfb_convert_tiles": (C.c_int, [P, P, P, C.c_int, C.c_int, C.c_int, P]),
        "dfb_set_timing": (C.c_int, [H, C.c_int]),
        "dfb_read_timing": (C.c_int, [H, C.POINTER(dfb_timing), C.c_int]),
        "dfb_composite_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                            P, P, P, P, P, P, P, P, P]),
        "dfb_set_tuning": (C.c_int, [H, C.c_int, C.c_int, C.c_int]),
        "dfb_set_wait_limit": (C.c_int, [H, C.c_double]),
        "dfb_inject_stall": (C.c_int, [H, C.c_int]),
        "dfb_noalloc_set_wait_limit": (C.c_int, [C.c_double]),
        "dfb_noalloc_inject_stall": (C.c_int, [C.c_int]),
        "dfb_graph_create": (C.c_int, [P, C.c_int, C.POINTER(H)]),
        "dfb_graph_launch": (C.c_int, [H, P]),
        "dfb_graph_set_tuning": (C.c_int, [H, C.c_int, C.c_int, C.c_int]),
        "dfb_graph_autotune": (C.c_int, [H, P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(C.c_int),
                                         C.POINTER(C.c_float)]),
        "dfb_graph_destroy": (C.c_int, [H]),
        "dfb_error_string": (C.c_char_p, [C.c_int]),
        "dfb_version": (C.c_int, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(x):
    """Address of a buffer: torch tensor, numpy array, ctypes object, int or None.
    Arrays must be contiguous: the library reads and writes them densely."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("tensor passed to libdfb must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array passed to libdfb must be C-contiguous")
        return x.ctypes.data
    return C.addressof(x)


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st, where):
    if st != DFB_OK:
        raise DfbError(st, where)
    return st


def dfb_error_string(code: int) -> str:
    return lib().dfb_error_string(code).decode()


def dfb_version() -> int:
    return lib().dfb_version()


def dfb_create(width, height, tile_size, mode=DFB_BLEND_DEPTH):
    h = H()
    _check(lib().dfb_create(width, height, tile_size, mode, C.byref(h)), "dfb_create")
    return h


def dfb_create_ex(width, height, tile_size, mode=DFB_BLEND_DEPTH, dtype=DFB_F32,
                  flags=DFB_FLAGS_DEFAULT, kahan_after=0, max_fragments=0):
    cfg = dfb_config(width, height, tile_size, mode, dtype, flags, kahan_after, max_fragments)
    h = H()
    _check(lib().dfb_create_ex(C.byref(cfg), C.byref(h)), "dfb_create_ex")
    return h


def dfb_destroy(h):
    return _check(lib().dfb_destroy(h), "dfb_destroy")


def dfb_set_background(h, r, g, b, a):
    return _check(lib().dfb_set_background(h, r, g, b, a), "dfb_set_background")


def dfb_set_pixel_op(h, op, exposure=1.0):
    return _check(lib().dfb_set_pixel_op(h, int(op), float(exposure)), "dfb_set_pixel_op")


def dfb_set_pixel_curve(h, curves, x_max=1.0):
    """curves: 3 x n samples (one row per channel), copied to the device."""
    c = np.ascontiguousarray(curves, dtype=np.float32)
    if c.ndim != 2 or c.shape[0] != 3:
        raise ValueError("curves must have shape (3, n)")
    return _check(lib().dfb_set_pixel_curve(h, c.ctypes.data, int(c.shape[1]), float(x_max)),
                  "dfb_set_pixel_curve")


def dfb_begin_frame(h, accumulate=0):
    return _check(lib().dfb_begin_frame(h, int(accumulate)), "dfb_begin_frame")


def dfb_set_tile_children(h, tile_id, n_children):
    return _check(lib().dfb_set_tile_children(h, tile_id, n_children), "dfb_set_tile_children")


def dfb_submit_tile(h, tile_id, order_key, rgba, depth):
    return _check(lib().dfb_submit_tile(h, tile_id, order_key, _ptr(rgba), _ptr(depth)),
                  "dfb_submit_tile")


def dfb_submit_tile_ex(h, tile_id, order_key, rgba, depth, scale=1.0, generation=1, children=0):
    d = dfb_tile_desc(tile_id, order_key, _ptr(rgba), _ptr(depth), scale, generation, children)
    return _check(lib().dfb_submit_tile_ex(h, C.byref(d)), "dfb_submit_tile_ex")


def dfb_submit_tiles(h, tile_ids, order_keys, rgba_ptrs, depth_ptrs, scales=None,
                     where=DFB_PTR_AUTO):
    """Bulk setTile.  ``rgba_ptrs``/``depth_ptrs`` are sequences of addresses."""
    tid = np.ascontiguousarray(tile_ids, dtype=np.int32)
    key = np.ascontiguousarray(order_keys, dtype=np.float32)
    rp = np.ascontiguousarray(rgba_ptrs, dtype=np.uint64)
    dp = np.ascontiguousarray(depth_ptrs, dtype=np.uint64)
    sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
    n = len(tid)
    if not (len(key) == len(rp) == len(dp) == n) or (sc is not None and len(sc) != n):
        raise ValueError("array lengths differ")
    st = lib().dfb_submit_tiles(h, n, tid.ctypes.data, key.ctypes.data, rp.ctypes.data,
                                dp.ctypes.data, None if sc is None else sc.ctypes.data, where)
    return _check(st, "dfb_submit_tiles")


def dfb_submit_tiles_ex(h, tiles, where=DFB_PTR_AUTO):
    """Bulk setTile of (tile_id, order_key, rgba, depth, scale, generation, children) tuples."""
    arr = (dfb_tile_desc * len(tiles))(*[
        dfb_tile_desc(t, k, _ptr(r), _ptr(d), s, g, c) for (t, k, r, d, s, g, c) in tiles])
    return _check(lib().dfb_submit_tiles_ex(h, len(tiles), C.addressof(arr), where),
                  "dfb_submit_tiles_ex")


def pool_pointers(base, n, tile_bytes):
    """Addresses of n tiles laid out back to back from ``base``."""
    return np.uint64(_ptr(base)) + np.arange(n, dtype=np.uint64) * np.uint64(tile_bytes)


def dfb_end_frame(h, stream=None):
    return _check(lib().dfb_end_frame(h, _stream(stream)), "dfb_end_frame")


def dfb_end_frames(handles, stream=None):
    arr = (H * len(handles))(*[h.value if isinstance(h, H) else h for h in handles])
    return _check(lib().dfb_end_frames(C.addressof(arr), len(handles), _stream(stream)),
                  "dfb_end_frames")


def dfb_tileset_create(h, tile_ids, order_keys, rgba_ptrs, depth_ptrs, scales=None):
    """Prepared bulk setTile (device pointers) for handles shaped like ``h``."""
    tid = np.ascontiguousarray(tile_ids, dtype=np.int32)
    key = np.ascontiguousarray(order_keys, dtype=np.float32)
    rp = np.ascontiguousarray(rgba_ptrs, dtype=np.uint64)
    dp = np.ascontiguousarray(depth_ptrs, dtype=np.uint64)
    sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
    n = len(tid)
    if not (len(key) == len(rp) == len(dp) == n) or (sc is not None and len(sc) != n):
        raise ValueError("array lengths differ")
    s = H()
    _check(lib().dfb_tileset_create(h, n, tid.ctypes.data, key.ctypes.data, rp.ctypes.data,
                                    dp.ctypes.data, None if sc is None else sc.ctypes.data,
                                    C.byref(s)), "dfb_tileset_create")
    return s


def dfb_tileset_destroy(s):
    return _check(lib().dfb_tileset_destroy(s), "dfb_tileset_destroy")


def dfb_submit_tileset(h, s):
    return _check(lib().dfb_submit_tileset(h, s), "dfb_submit_tileset")


def _addresses(objs):
    return np.array([o.value if isinstance(o, H) else (o or 0) for o in objs], dtype=np.uint64)


def dfb_run_frames(handles, sets, accumulate=None, stream=None):
    """Begin, submit a prepared set and end the frames of several handles in
    one call (one batched launch)."""
    hs = _addresses(handles)
    ss = _addresses(sets)
    if len(hs) != len(ss):
        raise ValueError("one set per handle")
    acc = None if accumulate is None else np.ascontiguousarray(accumulate, dtype=np.int32)
    if acc is not None and len(acc) != len(hs):
        raise ValueError("one accumulate flag per handle")
    return _check(lib().dfb_run_frames(hs.ctypes.data, ss.ctypes.data,
                                       None if acc is None else acc.ctypes.data, len(hs),
                                       _stream(stream)), "dfb_run_frames")


def dfb_sync(h):
    return _check(lib().dfb_sync(h), "dfb_sync")


def dfb_read_color(h, out):
    return _check(lib().dfb_read_color(h, _ptr(out)), "dfb_read_color")


def dfb_read_accum(h, out):
    return _check(lib().dfb_read_accum(h, _ptr(out)), "dfb_read_accum")


def dfb_read_variance(h, per_pixel=None, per_tile=None):
    return _check(lib().dfb_read_variance(h, _ptr(per_pixel), _ptr(per_tile)), "dfb_read_variance")


def dfb_read_rgba8(h, out):
    return _check(lib().dfb_read_rgba8(h, _ptr(out)), "dfb_read_rgba8")


def dfb_get_stats(h) -> dict:
    s = dfb_frame_stats()
    _check(lib().dfb_get_stats(h, C.byref(s)), "dfb_get_stats")
    return s.as_dict()


def dfb_get_tiles(h):
    tx, ty = C.c_int(), C.c_int()
    _check(lib().dfb_get_tiles(h, C.byref(tx), C.byref(ty)), "dfb_get_tiles")
    return tx.value, ty.value


def dfb_save_accum(h, total, comp, m2) -> int:
    n = C.c_int()
    _check(lib().dfb_save_accum(h, _ptr(total), _ptr(comp), _ptr(m2), C.byref(n)), "dfb_save_accum")
    return n.value


def dfb_load_accum(h, total, comp, m2, frames):
    return _check(lib().dfb_load_accum(h, _ptr(total), _ptr(comp), _ptr(m2), frames),
                  "dfb_load_accum")


def dfb_convert_tiles(src, dst, scales, n_tiles, tile_pixels, dtype, stream=None):
    return _check(lib().dfb_convert_tiles(_ptr(src), _ptr(dst), _ptr(scales), n_tiles,
                                          tile_pixels, dtype, _stream(stream)),
                  "dfb_convert_tiles")


def dfb_set_timing(h, enable=True):
    return _check(lib().dfb_set_timing(h, int(enable)), "dfb_set_timing")


def dfb_read_timing(h, reset=True) -> dict:
    t = dfb_timing()
    _check(lib().dfb_read_timing(h, C.byref(t), int(reset)), "dfb_read_timing")
    return {"launches": t.launches, "bucket_ms": t.bucket_ms, "composite_ms": t.composite_ms}


def dfb_composite_noalloc(width, height, tile_size, mode, dtype, tile_ids, order_keys, rgba_ptrs,
                          depth_ptrs, scales=None, background=None, color_out=None,
                          rgba8_out=None, stream=None):
    """One frame without any allocation; outputs are caller-owned device buffers."""
    tid = np.ascontiguousarray(tile_ids, dtype=np.int32)
    key = np.ascontiguousarray(order_keys, dtype=np.float32)
    rp = np.ascontiguousarray(rgba_ptrs, dtype=np.uint64)
    dp = np.ascontiguousarray(depth_ptrs, dtype=np.uint64)
    sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
    bg = None if background is None else np.ascontiguousarray(background, dtype=np.float32)
    n = len(tid)
    if not (len(key) == len(rp) == len(dp) == n) or (sc is not None and len(sc) != n):
        raise ValueError("array lengths differ")
    st = lib().dfb_composite_noalloc(
        width, height, tile_size, mode, dtype, n, tid.ctypes.data, key.ctypes.data,
        rp.ctypes.data, dp.ctypes.data, None if sc is None else sc.ctypes.data,
        None if bg is None else bg.ctypes.data, _ptr(color_out), _ptr(rgba8_out), _stream(stream))
    return _check(st, "dfb_composite_noalloc")


def dfb_set_wait_limit(h, seconds):
    return _check(lib().dfb_set_wait_limit(h, float(seconds)), "dfb_set_wait_limit")


def dfb_inject_stall(h, item):
    return _check(lib().dfb_inject_stall(h, int(item)), "dfb_inject_stall")


def dfb_noalloc_set_wait_limit(seconds):
    return _check(lib().dfb_noalloc_set_wait_limit(float(seconds)), "dfb_noalloc_set_wait_limit")


def dfb_noalloc_inject_stall(item):
    return _check(lib().dfb_noalloc_inject_stall(int(item)), "dfb_noalloc_inject_stall")


def dfb_set_tuning(h, ring_kb=0, ctas_per_sm=0, groups=0):
    return _check(lib().dfb_set_tuning(h, int(ring_kb), int(ctas_per_sm), int(groups)),
                  "dfb_set_tuning")


def dfb_graph_create(handles):
    arr = (H * len(handles))(*[h.value if isinstance(h, H) else h for h in handles])
    g = H()
    _check(lib().dfb_graph_create(C.addressof(arr), len(handles), C.byref(g)), "dfb_graph_create")
    return g


def dfb_graph_launch(g, stream=None):
    return _check(lib().dfb_graph_launch(g, _stream(stream)), "dfb_graph_launch")


def dfb_graph_set_tuning(g, ring_kb, ctas_per_sm, groups):
    return _check(lib().dfb_graph_set_tuning(g, int(ring_kb), int(ctas_per_sm), int(groups)),
                  "dfb_graph_set_tuning")


def dfb_graph_autotune(g, stream=None, reps=5):
    r, c, gr, ms = C.c_int(), C.c_int(), C.c_int(), C.c_float()
    _check(lib().dfb_graph_autotune(g, _stream(stream), int(reps), C.byref(r), C.byref(c),
                                    C.byref(gr), C.byref(ms)), "dfb_graph_autotune")
    return {"ring_kb": r.value, "ctas_per_sm": c.value, "groups": gr.value, "ms": ms.value}


def dfb_graph_destroy(g):
    return _check(lib().dfb_graph_destroy(g), "dfb_graph_destroy")
