"""Seeded random configurations through every launch shape the composite is
built for (groups x CTAs per SM, as the autotuner may pick them), all modes
and storage dtypes: small ragged frames with empty, ordinary and long tiles,
a background, and two accumulated frames, each checked against the oracle.

Long tiles (more than 16 fragments) stream through the composite's ring in
several fills.  In BLEND_DEPTH their pixels take a speculative pass in list
order, and the 32-pixel units whose depths are out of list order are redone
exactly by a second kernel; the cases with 64-128 fragments per tile give
their long tiles depths in list order with a few out-of-order pixels, so
both paths run in one launch."""

import numpy as np
import pytest

from harness import scenes
from oracle import dfb_oracle as o
from paper_2305_07083_gb300 import dfb as D

from tests.gpu_helpers import GpuFrameBuffer

pytestmark = pytest.mark.gpu

SHAPES = [(110, 2, 1), (110, 2, 2), (72, 3, 1), (220, 1, 2), (220, 1, 3), (64, 3, 1)]
MODES = [D.DFB_BLEND_DEPTH, D.DFB_BLEND_ORDERED, D.DFB_ZCOMPOSITE, D.DFB_AVERAGE]
DTYPES = [D.DFB_F32, D.DFB_F16, D.DFB_BF16, D.DFB_FP8E4M3]
TOL = {D.DFB_F32: 1e-5, D.DFB_F16: 1e-5, D.DFB_BF16: 1e-5, D.DFB_FP8E4M3: 1e-5}


def fits(shape, dtype):
    """Whether the shape's ring holds the dtype's largest staged item."""
    ring_kb, per, _ = shape
    item = 16 * 256 * (4 + {0: 16, 1: 8, 2: 8, 3: 4}[dtype]) + 3 * 256 * 16
    cap = (233472 // per - 1024 - 12032) & ~127
    return min(ring_kb * 1024, cap) >= item


CASES = []
_rng = np.random.default_rng(2024)
for case in range(48):
    shape = SHAPES[case % len(SHAPES)]
    dtype = DTYPES[(case // len(SHAPES)) % len(DTYPES)]
    mode = MODES[int(_rng.integers(len(MODES)))]
    if not fits(shape, dtype):
        dtype = D.DFB_FP8E4M3 if fits(shape, D.DFB_FP8E4M3) else D.DFB_F32
    CASES.append((case, shape, mode, dtype))


def order_depths(sc, rng, frac_swapped):
    """Give every pixel of every tile depths that ascend in the tile's list
    order (order key, then submit index), then swap two depths at a random
    `frac_swapped` of the pixels of long tiles, so that those pixels (and
    only their 32-pixel units) are out of order."""
    lists, _, _ = o.bucket(sc.tile_ids, sc.keys, sc.n_tiles)
    depth = sc.depth.copy()
    for idx in lists:
        idx = np.asarray(idx, dtype=np.int64)
        if len(idx) < 2:
            continue
        z = np.sort(depth[idx], axis=0)          # NaN (special depths) sort last
        depth[idx] = z
        if len(idx) > 16:
            px = np.nonzero(rng.random(depth.shape[1]) < frac_swapped)[0]
            for p in px:
                a, b = rng.choice(len(idx), 2, replace=False)
                depth[idx[a], p], depth[idx[b], p] = depth[idx[b], p], depth[idx[a], p]
    sc.depth = depth
    return sc


DEEP = []
_rng2 = np.random.default_rng(2025)
for case in range(12):
    shape = SHAPES[case % len(SHAPES)]
    dtype = DTYPES[(case // 3) % len(DTYPES)]
    mode = D.DFB_BLEND_DEPTH if case % 3 else MODES[int(_rng2.integers(len(MODES)))]
    if not fits(shape, dtype):
        dtype = D.DFB_FP8E4M3 if fits(shape, D.DFB_FP8E4M3) else D.DFB_F32
    DEEP.append((case, shape, mode, dtype))


@pytest.mark.parametrize("case,shape,mode,dtype", DEEP,
                         ids=["d%d-%d.%d.%d-m%d-d%d" % (c, *s, m, d) for c, s, m, d in DEEP])
def test_deep_lists_in_order_and_redone(case, shape, mode, dtype):
    rng = np.random.default_rng(5000 + case)
    T = 64 if case % 2 == 0 else 32
    W, H = 3 * T + 17, 2 * T + 5
    n_tiles = (-(-W // T)) * (-(-H // T))
    bg = tuple(float(v) for v in rng.random(4))
    fb = GpuFrameBuffer(W, H, T, mode, dtype, bg=bg)
    D.dfb_set_tuning(fb.h, *shape)
    imgs = []
    for f in range(2):
        counts = rng.integers(0, 9, n_tiles)
        counts[rng.random(n_tiles) < 0.5] = rng.integers(64, 129)     # 64-128 per tile
        sc = scenes.random_scene(W, H, T, counts, seed=case * 10 + f + 500, alpha_max=0.3,
                                 special_depths=case % 4 == 1)
        sc = order_depths(sc, rng, 0.0 if case % 4 == 2 else 0.003)
        stored, scales = scenes.store_rgba(sc.rgba, dtype)
        fb.begin(accumulate=f > 0)
        fb.submit_pool(sc.tile_ids, sc.keys, stored, sc.depth, scales)
        fb.end()
        want = o.composite_frame(W, H, T, mode, sc.tile_ids, sc.keys,
                                 o.dequantize(stored, dtype, scales), sc.depth, bg=bg)
        got = fb.color()
        if mode == D.DFB_ZCOMPOSITE and dtype != D.DFB_FP8E4M3:
            bg_px = np.array([bg[0] * bg[3], bg[1] * bg[3], bg[2] * bg[3], bg[3]])
            exact = ~np.all(np.isclose(want, bg_px, atol=0), axis=-1)
            np.testing.assert_array_equal(got[exact].astype(np.float64), want[exact])
        assert np.max(np.abs(got - want)) <= TOL[dtype]
        imgs.append(want)
    assert np.max(np.abs(fb.accum() - o.accumulate(imgs))) <= 2e-5
    px, _ = fb.variance()
    assert np.max(np.abs(px - o.variance(imgs))) <= 2e-6


@pytest.mark.parametrize("case,shape,mode,dtype", CASES,
                         ids=["c%d-%d.%d.%d-m%d-d%d" % (c, *s, m, d) for c, s, m, d in CASES])
def test_random_configuration(case, shape, mode, dtype):
    if not fits(shape, dtype):
        pytest.skip("the shape's ring cannot hold this dtype's largest item")
    rng = np.random.default_rng(1000 + case)
    T = int(rng.choice([8, 16, 32, 64]))
    W = int(rng.integers(T // 2 + 1, 5 * T))
    H = int(rng.integers(T // 2 + 1, 4 * T))
    n_tiles = (-(-W // T)) * (-(-H // T))
    bg = tuple(float(v) for v in rng.random(4))
    fb = GpuFrameBuffer(W, H, T, mode, dtype, bg=bg)
    D.dfb_set_tuning(fb.h, *shape)
    imgs = []
    for f in range(2):
        counts = rng.integers(0, 6, n_tiles)
        counts[rng.random(n_tiles) < 0.15] = 0
        counts[rng.random(n_tiles) < 0.1] = int(rng.integers(17, 40))   # long tiles
        sc = scenes.random_scene(W, H, T, counts, seed=case * 10 + f, alpha_max=0.7,
                                 special_depths=bool(case % 3 == 0),
                                 depth_levels=4 if case % 5 == 0 else None)
        stored, scales = scenes.store_rgba(sc.rgba, dtype)
        fb.begin(accumulate=f > 0)
        fb.submit_pool(sc.tile_ids, sc.keys, stored, sc.depth, scales)
        fb.end()
        want = o.composite_frame(W, H, T, mode, sc.tile_ids, sc.keys,
                                 o.dequantize(stored, dtype, scales), sc.depth, bg=bg)
        got = fb.color()
        if mode == D.DFB_ZCOMPOSITE and dtype != D.DFB_FP8E4M3:
            # winners copied unchanged (an FP8 value carries one FP32 rounding
            # of code x scale, so it is compared within the tolerance below)
            bg_px = np.array([bg[0] * bg[3], bg[1] * bg[3], bg[2] * bg[3], bg[3]])
            exact = ~np.all(np.isclose(want, bg_px, atol=0), axis=-1)
            np.testing.assert_array_equal(got[exact].astype(np.float64), want[exact])
            assert np.max(np.abs(got - want)) <= 1e-6
        else:
            assert np.max(np.abs(got - want)) <= TOL[dtype]
        imgs.append(want)
    assert np.max(np.abs(fb.accum() - o.accumulate(imgs))) <= 2e-5
    px, tv = fb.variance()
    assert np.max(np.abs(px - o.variance(imgs))) <= 2e-6
    d8 = np.abs(o.unpack_rgba8(fb.rgba8()) - o.unpack_rgba8(o.pack_rgba8(o.accumulate(imgs))))
    assert d8.max() <= 1
