"""Maximum sizes: a 32768 x 32768 frame (2^30 pixels, 262,144 tiles of
64 x 64, 4.2 M work items; the library accepts up to 2^31 pixels) with
fragments on a seeded sample of tiles, two accumulated frames.  Pixel,
state and tile indices pass 2^30, so 32-bit overflow anywhere shows up.
Checked against the oracle on the sampled tiles and on empty tiles."""

import numpy as np
import pytest

from oracle import dfb_oracle as o
from paper_2305_07083_gb300 import dfb as D

pytestmark = pytest.mark.gpu


def test_2_pow_30_pixel_frame_sampled_tiles():
    import torch
    W = H = 32768
    T = 64
    tiles_x = W // T
    n_tiles = tiles_x * (H // T)
    rng = np.random.default_rng(90)
    # the last tile of the frame, the first, and a seeded sample in between
    lit = np.unique(np.concatenate([[0, n_tiles - 1, n_tiles - tiles_x],
                                    rng.choice(n_tiles, 509, replace=False)]))
    counts = np.zeros(n_tiles, np.int64)
    counts[lit] = rng.integers(1, 5, len(lit))
    flags = D.DFB_FLAG_ACCUMULATE | D.DFB_FLAG_PACK_RGBA8      # no FP32 colour image
    h = D.dfb_create_ex(W, H, T, D.DFB_BLEND_DEPTH, D.DFB_F32, flags, 0, int(counts.sum()))
    try:
        imgs = {}
        for f in range(2):
            n = int(counts.sum())
            ids = np.repeat(np.arange(n_tiles, dtype=np.int32), counts)
            keys = rng.random(n).astype(np.float32)
            a = rng.uniform(0.0, 0.8, (n, T * T, 1)).astype(np.float32)
            rgba = np.concatenate([rng.random((n, T * T, 3)).astype(np.float32) * a, a], -1)
            depth = rng.random((n, T * T)).astype(np.float32)
            r = torch.from_numpy(rgba).cuda()
            d = torch.from_numpy(depth).cuda()
            D.dfb_begin_frame(h, f > 0)
            D.dfb_submit_tiles(h, ids, keys, D.pool_pointers(r, n, T * T * 16),
                               D.pool_pointers(d, n, T * T * 4), None, D.DFB_PTR_DEVICE)
            D.dfb_end_frame(h)
            D.dfb_sync(h)
            lists, _, _ = o.bucket(ids, keys, n_tiles)
            for t in lit:
                idx = np.array(lists[t], dtype=np.int64)
                imgs.setdefault(int(t), []).append(
                    o.composite_tile(rgba[idx].astype(np.float64), depth[idx], keys[idx], idx,
                                     o.BLEND_DEPTH))
            del r, d
        out = np.empty((H, W), np.uint32)
        D.dfb_read_rgba8(h, out)
        tv = np.empty(n_tiles, np.float32)
        D.dfb_read_variance(h, None, tv)
        for t, frames in imgs.items():
            y0, x0 = (t // tiles_x) * T, (t % tiles_x) * T
            mean = o.accumulate(frames)
            got = o.unpack_rgba8(out[y0:y0 + T, x0:x0 + T].reshape(-1))
            assert np.abs(got - o.unpack_rgba8(o.pack_rgba8(mean))).max() <= 1, t
            want_tv = o.variance(frames)[:, :3].mean()
            assert abs(tv[t] - want_tv) <= 1e-4 * want_tv + 1e-9, t
        empty = np.setdiff1d(rng.choice(n_tiles, 200, replace=False), lit)
        for t in empty:
            y0, x0 = (t // tiles_x) * T, (t % tiles_x) * T
            assert not out[y0:y0 + T, x0:x0 + T].any()
            assert tv[t] == 0.0
        st = D.dfb_get_stats(h)
        assert st["accumulated"] == 2 and st["frame_pixels"] == W * H
    finally:
        D.dfb_destroy(h)
