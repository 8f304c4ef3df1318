"""Image-parallel rendering on the GPU: redundantly rendered tiles averaged by
the tile operation (Sec. 4.1.1), the per-tile variance that decides how many
renders a tile gets next, and the pixel operations run before the display
conversion (Sec. 3.1.2)."""

import numpy as np
import pytest

from harness import scenes
from oracle import dfb_oracle as o
from paper_2305_07083_gb300 import adaptive
from paper_2305_07083_gb300 import dfb as D

from tests.gpu_helpers import GpuFrameBuffer

pytestmark = pytest.mark.gpu

TOL = 1e-5


def redundant_frame(W, H, T, counts, seed, dtype=D.DFB_F32):
    """counts[t] renders of image tile t, each a full tile of a noisy estimate
    of the same smooth image (different seeds)."""
    rng = np.random.default_rng(seed)
    tiles_x = -(-W // T)
    yy, xx = np.mgrid[0:T, 0:T] / T
    ids, rgba = [], []
    for t, k in enumerate(counts):
        tx, ty = t % tiles_x, t // tiles_x
        base = np.stack([0.3 + 0.4 * xx + 0.05 * tx, 0.2 + 0.5 * yy, 0.6 - 0.3 * xx * yy], -1)
        for _ in range(k):
            a = np.clip(0.8 + 0.2 * rng.standard_normal((T, T)), 0.0, 1.0)
            c = np.clip(base + 0.1 * rng.standard_normal((T, T, 3)), 0.0, 1.0) * a[..., None]
            rgba.append(np.concatenate([c, a[..., None]], -1).reshape(T * T, 4))
            ids.append(t)
    rgba = np.array(rgba, np.float32).reshape(-1, T * T, 4) if rgba else np.zeros((0, T * T, 4), np.float32)
    ids = np.array(ids, np.int32)
    keys = rng.random(len(ids)).astype(np.float32)      # arbitrary: the average ignores them
    depth = rng.random((len(ids), T * T)).astype(np.float32)
    return ids, keys, rgba, depth


@pytest.mark.parametrize("dtype,tol", [(D.DFB_F32, TOL), (D.DFB_F16, TOL), (D.DFB_BF16, TOL)])
def test_redundant_tiles_average_accumulate_and_pack(dtype, tol):
    W, H, T = 320, 192, 64                    # 5 x 3 tiles, 16 work items each
    counts = np.array([1, 2, 3, 4, 0, 5, 20, 1, 2, 17, 3, 3, 1, 2, 6])
    fb = GpuFrameBuffer(W, H, T, D.DFB_AVERAGE, dtype, bg=(0.2, 0.4, 0.6, 1.0))
    imgs = []
    for f in range(3):
        ids, keys, rgba, depth = redundant_frame(W, H, T, counts, 100 + f)
        stored, scales = scenes.store_rgba(rgba, dtype)
        fb.begin(accumulate=f > 0)
        fb.submit_pool(ids, keys, stored, depth, scales)
        fb.end()
        want = o.composite_frame(W, H, T, o.AVERAGE, ids, keys,
                                 o.dequantize(stored, dtype, scales), depth,
                                 bg=(0.2, 0.4, 0.6, 1.0))
        imgs.append(want)
        assert np.max(np.abs(fb.color() - want)) <= tol
    assert np.max(np.abs(fb.accum() - o.accumulate(imgs))) <= tol
    px, tv = fb.variance()
    assert np.max(np.abs(px - o.variance(imgs))) <= 1e-6
    np.testing.assert_allclose(tv, o.tile_variance(o.variance(imgs), T), rtol=1e-4, atol=1e-9)
    d8 = np.abs(o.unpack_rgba8(fb.rgba8()) - o.unpack_rgba8(o.pack_rgba8(o.accumulate(imgs))))
    assert d8.max() <= 1


def test_average_of_k_renders_equals_k_accumulated_frames_on_gpu():
    """Sec. 4.1.1: k renders averaged in one frame equal the same renders
    accumulated as k frames (both on the GPU, equal counts per tile)."""
    W = H = 128
    T = 64
    k = 4
    ids, keys, rgba, depth = redundant_frame(W, H, T, [k] * 4, 7)
    avg = GpuFrameBuffer(W, H, T, D.DFB_AVERAGE)
    avg.begin(0)
    avg.submit_pool(ids, keys, rgba, depth)
    avg.end()
    acc = GpuFrameBuffer(W, H, T, D.DFB_BLEND_ORDERED)
    for i in range(k):
        sel = np.arange(i, len(ids), k)
        acc.begin(accumulate=i > 0)
        acc.submit_pool(ids[sel], keys[sel], rgba[sel], depth[sel])
        acc.end()
    assert np.max(np.abs(avg.color() - acc.accum())) <= 1e-6


def test_variance_steers_redundancy_then_average():
    """Two refinement passes: the per-tile variance of the first decides how
    many renders each tile gets in the second (adaptive.redundancy), which
    the averaging tile operation composites."""
    W, H, T = 256, 128, 64
    n_tiles = 8
    fb = GpuFrameBuffer(W, H, T, D.DFB_AVERAGE)
    for f in range(2):
        ids, keys, rgba, depth = redundant_frame(W, H, T, [1] * n_tiles, 200 + f)
        fb.begin(accumulate=f > 0)
        fb.submit_pool(ids, keys, rgba, depth)
        fb.end()
    _, tv = fb.variance()
    counts = adaptive.redundancy(tv, k_min=1, k_max=6)
    assert counts.min() >= 1 and counts.max() <= 6
    ids, keys, rgba, depth = redundant_frame(W, H, T, counts, 300)
    fb2 = GpuFrameBuffer(W, H, T, D.DFB_AVERAGE)
    fb2.begin(0)
    fb2.submit_pool(ids, keys, rgba, depth)
    fb2.end()
    want = o.composite_frame(W, H, T, o.AVERAGE, ids, keys, rgba.astype(np.float64), depth)
    assert np.max(np.abs(fb2.color() - want)) <= TOL


@pytest.mark.parametrize("op,e", [(D.DFB_PIXELOP_EXPOSURE, 1.7), (D.DFB_PIXELOP_REINHARD, 2.5),
                                  (D.DFB_PIXELOP_EXPOSURE, 0.0)])
def test_pixel_ops_before_the_pack(op, e):
    sc = scenes.scene_data_parallel(192, 128, 32, (3, 3, 3), seed=9, jitter_sigma=0.05)
    plain = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH)
    fb = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH)
    D.dfb_set_pixel_op(fb.h, op, e)
    imgs = []
    for f in range(3):
        rgba = sc.frame_rgba(f)
        for b in (plain, fb):
            b.begin(accumulate=f > 0)
            b.submit_pool(sc.tile_ids, sc.keys, rgba, sc.depth)
            b.end()
        imgs.append(o.composite_frame(sc.W, sc.H, sc.T, o.BLEND_DEPTH, sc.tile_ids, sc.keys,
                                      rgba.astype(np.float64), sc.depth))
    # the operation changes the display pixels only
    np.testing.assert_array_equal(fb.accum(), plain.accum())
    np.testing.assert_array_equal(fb.color(), plain.color())
    want8 = o.pack_rgba8(o.pixel_op(o.accumulate(imgs), op, e))
    d8 = np.abs(o.unpack_rgba8(fb.rgba8()) - o.unpack_rgba8(want8))
    assert d8.max() <= 1


def _curves(n, x_max, seed):
    """Three seeded tone curves: increasing, decreasing and wiggly, in [0, 1]."""
    rng = np.random.default_rng(seed)
    up = np.cumsum(rng.random(n)); up = (up - up[0]) / (up[-1] - up[0])
    down = 1.0 - up[::-1]
    wig = 0.5 + 0.4 * np.sin(np.linspace(0.0, 7.0, n)) * rng.random(n)
    return np.stack([up, down, wig]).astype(np.float32)


def test_user_tone_curve_before_the_pack():
    """DFB_PIXELOP_CURVE: the user's curves, swapped between frames (with a
    different sample count), and a switch back to a built-in operation."""
    sc = scenes.scene_data_parallel(192, 128, 32, (3, 3, 3), seed=11, jitter_sigma=0.05)
    plain = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH)
    fb = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH)
    settings = [(17, 1.5, 1.3), (5, 0.75, 1.0), (2, 1.0, 2.0), (4096, 3.0, 0.8), (None, None, 2.5)]
    imgs = []
    for f, (n, xm, e) in enumerate(settings):
        if n is None:
            D.dfb_set_pixel_op(fb.h, D.DFB_PIXELOP_REINHARD, e)
        else:
            curves = _curves(n, xm, 60 + f)
            D.dfb_set_pixel_op(fb.h, D.DFB_PIXELOP_EXPOSURE, e)
            D.dfb_set_pixel_curve(fb.h, curves, xm)          # selects the curve, keeps e
        rgba = sc.frame_rgba(f)
        for b in (plain, fb):
            b.begin(accumulate=f > 0)
            b.submit_pool(sc.tile_ids, sc.keys, rgba, sc.depth)
            b.end()
        imgs.append(o.composite_frame(sc.W, sc.H, sc.T, o.BLEND_DEPTH, sc.tile_ids, sc.keys,
                                      rgba.astype(np.float64), sc.depth))
        mean = o.accumulate(imgs)
        if n is None:
            want = o.pixel_op(mean, o.PIXELOP_REINHARD, e)
        else:
            want = o.pixel_op(mean, o.PIXELOP_CURVE, e, curves.astype(np.float64), xm)
        d8 = np.abs(o.unpack_rgba8(fb.rgba8()) - o.unpack_rgba8(o.pack_rgba8(want)))
        assert d8.max() <= 1, (f, n)
        assert np.mean(d8 == 0) > 0.99, (f, n)
        np.testing.assert_array_equal(fb.accum(), plain.accum())
    # with a curve loaded the operation can be selected again
    D.dfb_set_pixel_op(fb.h, D.DFB_PIXELOP_CURVE, 1.0)


def test_identity_curve_matches_no_operation():
    sc = scenes.scene_data_parallel(128, 128, 32, (2, 2, 2), seed=12, jitter_sigma=0.05)
    plain = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH)
    fb = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH)
    D.dfb_set_pixel_curve(fb.h, np.stack([np.linspace(0.0, 1.0, 257)] * 3), 1.0)
    for b in (plain, fb):
        b.begin(accumulate=False)
        b.submit_pool(sc.tile_ids, sc.keys, sc.frame_rgba(0), sc.depth)
        b.end()
    d8 = np.abs(o.unpack_rgba8(fb.rgba8()) - o.unpack_rgba8(plain.rgba8()))
    assert d8.max() <= 1
    assert np.mean(d8 == 0) > 0.999
