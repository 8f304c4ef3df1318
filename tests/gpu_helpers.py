"""Helpers for the GPU parity tests: drive libdfb.so through its C ABI."""

from __future__ import annotations

import numpy as np

from paper_2305_07083_gb300 import dfb as D


def torch():
    import torch as t
    return t


def to_dev(a):
    t = torch()
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        a = a.view(np.int16)          # same bytes; torch's uint16 support is partial
    return t.from_numpy(a).cuda()


class GpuFrameBuffer:
    """One handle plus the device copies of the fragment pools it reads."""

    def __init__(self, W, H, T, mode, dtype=D.DFB_F32, flags=D.DFB_FLAGS_DEFAULT, kahan_after=0,
                 bg=(0.0, 0.0, 0.0, 0.0)):
        self.W, self.H, self.T, self.mode, self.dtype, self.flags = W, H, T, mode, dtype, flags
        self.h = D.dfb_create_ex(W, H, T, mode, dtype, flags, kahan_after)
        D.dfb_set_background(self.h, *bg)
        self.keep = []
        self.tiles_x, self.tiles_y = D.dfb_get_tiles(self.h)

    def close(self):
        if self.h is not None:
            D.dfb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def begin(self, accumulate=0):
        D.dfb_begin_frame(self.h, accumulate)

    def submit_pool(self, tile_ids, keys, rgba_stored, depth, scales=None, where="device"):
        """Submit n tiles stored back to back (device or host arrays)."""
        n = len(tile_ids)
        if n == 0:
            return
        if where == "device":
            r = to_dev(rgba_stored)
            d = to_dev(depth)
            self.keep += [r, d]
            w = D.DFB_PTR_DEVICE
        else:
            r = np.ascontiguousarray(rgba_stored)
            d = np.ascontiguousarray(depth, dtype=np.float32)
            self.keep += [r, d]
            w = D.DFB_PTR_HOST
        rb = self.T * self.T * 4 * D.ELEMENT_BYTES[self.dtype]
        db = self.T * self.T * 4
        D.dfb_submit_tiles(self.h, tile_ids, keys, D.pool_pointers(r, n, rb),
                           D.pool_pointers(d, n, db), scales, w)

    def end(self, stream=None):
        D.dfb_end_frame(self.h, stream)

    def color(self):
        out = np.empty((self.H, self.W, 4), np.float32)
        D.dfb_read_color(self.h, out)
        return out

    def accum(self):
        out = np.empty((self.H, self.W, 4), np.float32)
        D.dfb_read_accum(self.h, out)
        return out

    def variance(self):
        px = np.empty((self.H, self.W, 4), np.float32)
        tv = np.empty(self.tiles_x * self.tiles_y, np.float32)
        D.dfb_read_variance(self.h, px, tv)
        return px, tv

    def rgba8(self):
        out = np.empty((self.H, self.W), np.uint32)
        D.dfb_read_rgba8(self.h, out)
        return out

    def stats(self):
        return D.dfb_get_stats(self.h)


def composite_once(sc, mode, rgba_stored=None, dtype=D.DFB_F32, scales=None, bg=(0, 0, 0, 0),
                   where="device", flags=D.DFB_FLAGS_DEFAULT):
    fb = GpuFrameBuffer(sc.W, sc.H, sc.T, mode, dtype, flags=flags, bg=bg)
    fb.begin(0)
    fb.submit_pool(sc.tile_ids, sc.keys, sc.rgba if rgba_stored is None else rgba_stored,
                   sc.depth, scales, where)
    fb.end()
    D.dfb_sync(fb.h)
    return fb
