"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP32 colour max-abs 1e-5 against the oracle fed the same stored
values; z-composite winners bit-exact; RGBA8 within 1 LSB; variances within
1e-6 absolute (they are below 0.25 and FP32 keeps ~7 digits).
"""

import numpy as np
import pytest

from harness import scenes
from oracle import dfb_oracle as o
from paper_2305_07083_gb300 import dfb as D

from tests.gpu_helpers import GpuFrameBuffer, composite_once, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-5
MODES = [D.DFB_BLEND_DEPTH, D.DFB_BLEND_ORDERED, D.DFB_ZCOMPOSITE, D.DFB_AVERAGE]


def oracle_frame(sc, mode, rgba64=None, bg=(0, 0, 0, 0), tiles=None):
    r = sc.rgba.astype(np.float64) if rgba64 is None else rgba64
    return o.composite_frame(sc.W, sc.H, sc.T, mode, sc.tile_ids, sc.keys, r, sc.depth, bg,
                             tiles=tiles)


def check_color(got, want, mode, tol=TOL, bg=(0, 0, 0, 0)):
    if mode == D.DFB_ZCOMPOSITE:
        # winners are copied unchanged: bit-exact; background pixels carry the
        # FP32 product rgb*a (one rounding) instead of the float64 one
        bgp = np.array([bg[0] * bg[3], bg[1] * bg[3], bg[2] * bg[3], bg[3]])
        is_bg = np.all(want == bgp, axis=-1)
        g = got.astype(np.float64)
        np.testing.assert_array_equal(g[~is_bg], want[~is_bg])
        assert np.max(np.abs(g[is_bg] - want[is_bg]), initial=0.0) <= 1e-7
    else:
        err = np.max(np.abs(got.astype(np.float64) - want)) if got.size else 0.0
        assert err <= tol, "max-abs %.3g > %.1g" % (err, tol)


# --- single frame -------------------------------------------------------------
@pytest.mark.parametrize("mode", MODES)
def test_single_frame_256_eight_bricks(mode):
    sc = scenes.scene_single_frame_256(seed=0)
    fb = composite_once(sc, mode)
    check_color(fb.color(), oracle_frame(sc, mode), mode)
    st = fb.stats()
    assert st["fragments"] == 32 and st["fragment_pixels"] == 131072


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("W,H,T", [(200, 136, 64), (37, 29, 16), (13, 9, 4), (70, 33, 8),
                                   (300, 130, 128), (260, 300, 256)])
def test_ragged_frames_random_counts(mode, W, H, T):
    tiles = (-(-W // T)) * (-(-H // T))
    counts = np.random.default_rng(W * 7 + H).integers(0, 7, tiles)
    counts[0] = 0
    sc = scenes.random_scene(W, H, T, counts, seed=W + H, special_depths=True)
    bg = (0.2, 0.4, 0.6, 0.5)
    fb = composite_once(sc, mode, bg=bg)
    check_color(fb.color(), oracle_frame(sc, mode, bg=bg), mode, bg=bg)


@pytest.mark.parametrize("mode", MODES)
def test_depth_ties_and_equal_keys(mode):
    """Ties in depth and in key are broken by (key, submit index)."""
    W = H = 32
    T = 8
    counts = np.full(16, 6)
    sc = scenes.random_scene(W, H, T, counts, seed=3, depth_levels=3, equal_keys=True,
                             special_depths=True)
    fb = composite_once(sc, mode)
    check_color(fb.color(), oracle_frame(sc, mode), mode)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [17, 40, 300])
def test_long_fragment_lists(mode, n):
    """More fragments than the sort window (16) and the staged pointers (256)."""
    counts = np.array([n, 1, 0, 5])
    sc = scenes.random_scene(32, 32, 16, counts, seed=n, alpha_max=0.2)
    fb = composite_once(sc, mode)
    check_color(fb.color(), oracle_frame(sc, mode), mode, tol=2e-5 if n > 100 else TOL)


@pytest.mark.parametrize("mode", MODES)
def test_long_tiles_of_many_items_with_accumulation(mode):
    """Long tiles (more than 16 fragments) of 64x64 pixels are 16 work items
    each, streamed through the composite in several fills next to ordinary
    tiles (their random depths send them to the exact re-do kernel in
    BLEND_DEPTH); two accumulated frames exercise both kernels' reads of the
    running state."""
    counts = np.array([20, 3, 33, 0, 17, 16, 1, 25])
    fb = GpuFrameBuffer(256, 128, 64, mode)
    imgs = []
    for f in range(2):
        sc = scenes.random_scene(256, 128, 64, counts, seed=80 + f, alpha_max=0.3)
        fb.begin(accumulate=f > 0)
        fb.submit_pool(sc.tile_ids, sc.keys, sc.rgba, sc.depth)
        fb.end()
        imgs.append(oracle_frame(sc, mode))
        check_color(fb.color(), imgs[-1], mode)
    assert np.max(np.abs(fb.accum() - o.accumulate(imgs))) <= TOL
    px, tv = fb.variance()
    assert np.max(np.abs(px - o.variance(imgs))) <= 1e-6
    np.testing.assert_allclose(tv, o.tile_variance(o.variance(imgs), 64), rtol=1e-4, atol=1e-9)


@pytest.mark.parametrize("mode", [D.DFB_BLEND_DEPTH, D.DFB_ZCOMPOSITE])
def test_long_tile_in_a_sparse_frame_with_accumulation(mode):
    """A frame of few fragments per tile (below 2) streams its accumulation
    state through the composite's ring, with the last fill of each item; one
    long tile there spans several fills."""
    counts = np.zeros(32, int)
    counts[[0, 5, 9, 30]] = [1, 2, 1, 1]
    counts[17] = 21
    assert counts.sum() / counts.size < 2.0
    fb = GpuFrameBuffer(512, 256, 64, mode)
    imgs = []
    for f in range(3):
        sc = scenes.random_scene(512, 256, 64, counts, seed=90 + f, alpha_max=0.4)
        fb.begin(accumulate=f > 0)
        fb.submit_pool(sc.tile_ids, sc.keys, sc.rgba, sc.depth)
        fb.end()
        imgs.append(oracle_frame(sc, mode))
        check_color(fb.color(), imgs[-1], mode)
    assert np.max(np.abs(fb.accum() - o.accumulate(imgs))) <= TOL
    px, _ = fb.variance()
    assert np.max(np.abs(px - o.variance(imgs))) <= 1e-6


def test_empty_frame_shows_background():
    sc = scenes.random_scene(64, 64, 16, np.zeros(16, int), seed=1)
    for mode in MODES:
        fb = composite_once(sc, mode, bg=(1.0, 0.5, 0.25, 0.5))
        np.testing.assert_array_equal(fb.color(), np.broadcast_to(     # dyadic: exact
            np.array([0.5, 0.25, 0.125, 0.5], np.float32), (64, 64, 4)))


def test_rank_order_matches_depth_sort_on_gpu():
    """Sec. 4.2: disjoint bricks with keys in visibility order -> same image."""
    sc = scenes.scene_data_parallel(256, 192, 32, (3, 3, 3), seed=5, jitter_sigma=0.0)
    a = composite_once(sc, D.DFB_BLEND_DEPTH).color()
    b = composite_once(sc, D.DFB_BLEND_ORDERED).color()
    np.testing.assert_array_equal(a, b)


def test_host_pointers_equal_device_pointers():
    sc = scenes.scene_data_parallel(256, 256, 64, (2, 2, 2), seed=2, jitter_sigma=0.0)
    a = composite_once(sc, D.DFB_BLEND_DEPTH, where="device").color()
    b = composite_once(sc, D.DFB_BLEND_DEPTH, where="host").color()
    np.testing.assert_array_equal(a, b)


def test_borrowed_host_pointers_back_to_back():
    """DFB_PTR_HOST_BORROWED: host tiles copied asynchronously (the caller
    keeps them until the frame is done); frames ended back to back without a
    sync give the same accumulation as device pointers."""
    sc = scenes.scene_data_parallel(192, 128, 32, (3, 2, 2), seed=14, jitter_sigma=0.05)
    frames = [np.ascontiguousarray(sc.frame_rgba(f)) for f in range(4)]
    depth = np.ascontiguousarray(sc.depth, np.float32)
    rb, db = sc.T * sc.T * 16, sc.T * sc.T * 4
    outs = []
    for where in (D.DFB_PTR_HOST_BORROWED, D.DFB_PTR_DEVICE):
        fb = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH)
        bufs = frames if where != D.DFB_PTR_DEVICE else [to_dev(f) for f in frames]
        dep = depth if where != D.DFB_PTR_DEVICE else to_dev(depth)
        if where == D.DFB_PTR_DEVICE:
            import torch
            torch.cuda.synchronize()
        for f, buf in enumerate(bufs):
            fb.begin(accumulate=f > 0)
            D.dfb_submit_tiles(fb.h, sc.tile_ids, sc.keys, D.pool_pointers(buf, sc.n, rb),
                               D.pool_pointers(dep, sc.n, db), None, where)
            fb.end()
        D.dfb_sync(fb.h)
        outs.append((fb.accum(), fb.rgba8()))
        fb.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def test_repeatable_and_order_independent():
    sc = scenes.scene_data_parallel(256, 256, 32, (3, 3, 3), seed=6, jitter_sigma=0.0)
    a = composite_once(sc, D.DFB_BLEND_DEPTH).color()
    b = composite_once(sc, D.DFB_BLEND_DEPTH).color()
    np.testing.assert_array_equal(a, b)
    perm = np.random.default_rng(0).permutation(sc.n)
    sc2 = scenes.Scene(sc.W, sc.H, sc.T, sc.tile_ids[perm], sc.keys[perm], sc.rgba[perm],
                       sc.depth[perm])
    c = composite_once(sc2, D.DFB_BLEND_DEPTH).color()
    np.testing.assert_array_equal(a, c)     # no equal keys: order does not matter


# --- progressive refinement -------------------------------------------------------
def _frames(sc, n):
    return [sc.frame_rgba(f) for f in range(n)]


def test_accumulation_variance_and_pack():
    sc = scenes.scene_data_parallel(192, 128, 32, (3, 3, 3), seed=7, jitter_sigma=0.05)
    nf = 6
    fb = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH)
    imgs = []
    for f, rgba in enumerate(_frames(sc, nf)):
        fb.begin(accumulate=f > 0)
        fb.submit_pool(sc.tile_ids, sc.keys, rgba, sc.depth)
        fb.end()
        imgs.append(o.composite_frame(sc.W, sc.H, sc.T, o.BLEND_DEPTH, sc.tile_ids, sc.keys,
                                      rgba.astype(np.float64), sc.depth))
        check_color(fb.color(), imgs[-1], D.DFB_BLEND_DEPTH)
    mean = o.accumulate(imgs)
    var = o.variance(imgs)
    assert np.max(np.abs(fb.accum() - mean)) <= TOL
    px, tv = fb.variance()
    assert np.max(np.abs(px - var)) <= 1e-6
    np.testing.assert_allclose(tv, o.tile_variance(var, sc.T), rtol=1e-4, atol=1e-9)
    got8 = o.unpack_rgba8(fb.rgba8())
    want8 = o.unpack_rgba8(o.pack_rgba8(mean))
    assert np.max(np.abs(got8 - want8)) <= 1
    assert fb.stats()["accumulated"] == nf


def test_back_to_back_frames_on_alternating_streams():
    """Frames queued without a read in between (the bucketing of each frame
    overlaps the previous composite on the library's side stream), with
    different fragment sets per frame and the user stream switching every
    frame: every frame's colour and the accumulation match the oracle."""
    torch = pytest.importorskip("torch")
    W, H, T = 160, 96, 16
    n_tiles = (W // T) * (H // T)
    fb = GpuFrameBuffer(W, H, T, D.DFB_BLEND_DEPTH, flags=D.DFB_FLAGS_DEFAULT)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    imgs, colors = [], []
    for f in range(7):
        counts = np.random.default_rng(70 + f).integers(0, 7, n_tiles)
        sc = scenes.random_scene(W, H, T, counts, seed=70 + f)
        fb.begin(accumulate=f > 0)
        fb.submit_pool(sc.tile_ids, sc.keys, sc.rgba, sc.depth)
        streams[f % 2].wait_stream(torch.cuda.current_stream())  # uploads done
        fb.end(streams[f % 2])
        imgs.append(o.composite_frame(W, H, T, o.BLEND_DEPTH, sc.tile_ids, sc.keys,
                                      sc.rgba.astype(np.float64), sc.depth))
        if f in (2, 6):
            colors.append((f, fb.color()))
    for f, c in colors:
        check_color(c, imgs[f], D.DFB_BLEND_DEPTH)
    assert np.max(np.abs(fb.accum() - o.accumulate(imgs))) <= TOL
    px, _ = fb.variance()
    assert np.max(np.abs(px - o.variance(imgs))) <= 1e-6


def test_accumulate_reset_and_single_frame_variance():
    sc = scenes.scene_single_frame_256(seed=1)
    fb = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH)
    for _ in range(2):
        fb.begin(accumulate=0)
        fb.submit_pool(sc.tile_ids, sc.keys, sc.rgba, sc.depth)
        fb.end()
        want = oracle_frame(sc, o.BLEND_DEPTH)
        assert np.max(np.abs(fb.accum() - want)) <= TOL
        px, tv = fb.variance()
        assert not px.any() and not tv.any()
        assert fb.stats()["accumulated"] == 1
        got8 = o.unpack_rgba8(fb.rgba8())
        assert np.max(np.abs(got8 - o.unpack_rgba8(o.pack_rgba8(want)))) <= 1


@pytest.mark.parametrize("grid", [(1, 1, 1), (2, 2, 2)])
def test_kahan_compensated_sum(grid):
    """Past the threshold the running sum is compensated; results stay within
    tolerance of the exact mean (threshold lowered to 2 to exercise it).  One
    brick gives one fragment per tile, whose frames stream the accumulation
    state through the composite's ring; eight bricks give 3.4 per tile, whose
    frames have the consumers load it: both paths, with the compensation."""
    sc = scenes.scene_data_parallel(128, 128, 32, grid, seed=8, jitter_sigma=0.05)
    assert (sc.n / 16 >= 2.0) == (grid == (2, 2, 2))
    nf = 7
    fb = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_ORDERED, kahan_after=2)
    imgs = []
    for f, rgba in enumerate(_frames(sc, nf)):
        fb.begin(accumulate=f > 0)
        fb.submit_pool(sc.tile_ids, sc.keys, rgba, sc.depth)
        fb.end()
        imgs.append(o.composite_frame(sc.W, sc.H, sc.T, o.BLEND_ORDERED, sc.tile_ids, sc.keys,
                                      rgba.astype(np.float64), sc.depth))
        assert np.max(np.abs(fb.accum() - o.accumulate(imgs))) <= TOL
    px, _ = fb.variance()
    assert np.max(np.abs(px - o.variance(imgs))) <= 1e-6


def test_save_and_resume_accumulation():
    sc = scenes.scene_data_parallel(128, 96, 32, (2, 2, 2), seed=9, jitter_sigma=0.05)
    frames = _frames(sc, 5)
    full = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH, kahan_after=2)
    for f, rgba in enumerate(frames):
        full.begin(f > 0)
        full.submit_pool(sc.tile_ids, sc.keys, rgba, sc.depth)
        full.end()
    part = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH, kahan_after=2)
    for f, rgba in enumerate(frames[:3]):
        part.begin(f > 0)
        part.submit_pool(sc.tile_ids, sc.keys, rgba, sc.depth)
        part.end()
    shape = (sc.H, sc.W, 4)
    s, c, m = (np.empty(shape, np.float32) for _ in range(3))
    n = D.dfb_save_accum(part.h, s, c, m)
    assert n == 3
    res = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH, kahan_after=2)
    D.dfb_load_accum(res.h, s, c, m, n)
    for rgba in frames[3:]:
        res.begin(1)
        res.submit_pool(sc.tile_ids, sc.keys, rgba, sc.depth)
        res.end()
    np.testing.assert_array_equal(res.accum(), full.accum())
    np.testing.assert_array_equal(res.variance()[0], full.variance()[0])
    np.testing.assert_array_equal(res.rgba8(), full.rgba8())


# --- storage precision ---------------------------------------------------------------
# Storage error bounds.  FP16 meets the 2e-3 max-abs target.  BF16 keeps an
# 8-bit significand (a stored value in [0.5, 1) is off by up to 2^-9) and
# FP8 e4m3 3 mantissa bits (up to 2^-4 relative near the tile's amax); the
# colour and coverage errors of a pixel's layers add, so the format-derived
# bounds would be 2^-7 and 2^-3.  The asserted max-abs bounds sit just above
# the errors these scenes actually reach (the oracle on the stored values
# against the oracle on the FP32 values: BF16 3.0e-3 here and 4.0e-3 at
# 4096x1024, FP8 4.8e-2 and 6.6e-2), so that a regression fails; the 2e-3
# and 2e-2 targets hold for the RMS error.
STORAGE = [(D.DFB_F16, 2e-3, 2e-3), (D.DFB_BF16, 5e-3, 2e-3), (D.DFB_FP8E4M3, 8e-2, 2e-2)]


@pytest.mark.parametrize("dtype,max_tol,rms_tol", STORAGE)
@pytest.mark.parametrize("mode", MODES)
def test_storage_dtypes(dtype, max_tol, rms_tol, mode):
    sc = scenes.scene_data_parallel(256, 128, 32, (4, 2, 2), seed=10, jitter_sigma=0.0,
                                    extent=(2.0, 1.0, 1.0), radius=1.2)
    stored, scales = scenes.store_rgba(sc.rgba, dtype)
    fb = composite_once(sc, mode, rgba_stored=stored, dtype=dtype, scales=scales)
    got = fb.color().astype(np.float64)
    deq = o.dequantize(stored, dtype, scales)
    want_same_input = oracle_frame(sc, mode, rgba64=deq)
    if mode == D.DFB_ZCOMPOSITE and dtype != D.DFB_FP8E4M3:
        np.testing.assert_array_equal(got, want_same_input)
    else:
        assert np.max(np.abs(got - want_same_input)) <= TOL      # kernel error
    diff = got - oracle_frame(sc, mode)                          # storage error
    assert np.max(np.abs(diff)) <= max_tol, np.max(np.abs(diff))
    assert np.sqrt(np.mean(diff ** 2)) <= rms_tol


@pytest.mark.parametrize("dtype", [D.DFB_F16, D.DFB_BF16, D.DFB_FP8E4M3])
def test_convert_tiles_matches_reference_casts(dtype):
    import torch
    rng = np.random.default_rng(11)
    T = 16
    x = rng.uniform(0, 1, (9, T * T, 4)).astype(np.float32) * rng.uniform(0, 2, (9, 1, 1)).astype(np.float32)
    x[3] = 0.0
    src = torch.from_numpy(x).cuda()
    nb = {D.DFB_F16: 2, D.DFB_BF16: 2, D.DFB_FP8E4M3: 1}[dtype]
    dst = torch.zeros(x.size * nb, dtype=torch.uint8, device="cuda")
    sc = torch.zeros(9, dtype=torch.float32, device="cuda")
    D.dfb_convert_tiles(src, dst, sc, 9, T * T, dtype)
    torch.cuda.synchronize()
    got = dst.cpu().numpy()
    if dtype == D.DFB_F16:
        np.testing.assert_array_equal(got.view(np.float16).reshape(x.shape), x.astype(np.float16))
    elif dtype == D.DFB_BF16:
        ref, _ = scenes.store_rgba(x, 2)
        np.testing.assert_array_equal(got.view(np.uint16).reshape(x.shape), ref)
    else:
        scales = sc.cpu().numpy()
        for t in range(9):
            codes, s = o.fp8_quantize_tile(x[t])
            assert scales[t] == s
            np.testing.assert_array_equal(got.reshape(9, -1)[t], codes.reshape(-1))


# --- dependency trees and errors on the device ---------------------------------------------
def test_declared_children_and_incomplete():
    sc = scenes.scene_single_frame_256(seed=2)
    fb = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH)
    fb.begin(0)
    counts = sc.counts()
    for t in range(16):
        D.dfb_set_tile_children(fb.h, t, int(counts[t]))
    half = sc.n // 2
    fb.submit_pool(sc.tile_ids[:half], sc.keys[:half], sc.rgba[:half], sc.depth[:half])
    with pytest.raises(D.DfbError) as e:
        fb.end()
    assert e.value.code == D.DFB_ERR_INCOMPLETE
    fb.submit_pool(sc.tile_ids[half:], sc.keys[half:], sc.rgba[half:], sc.depth[half:])
    fb.end()                               # tree complete now
    check_color(fb.color(), oracle_frame(sc, o.BLEND_DEPTH), D.DFB_BLEND_DEPTH)


def test_read_before_any_frame_is_state_error():
    fb = GpuFrameBuffer(64, 64, 16, D.DFB_BLEND_DEPTH)
    with pytest.raises(D.DfbError) as e:
        fb.color()
    assert e.value.code == D.DFB_ERR_STATE


# --- the full-size workload, in the launch configuration the benchmark times -------------
@pytest.mark.parametrize("dtype", [D.DFB_F32, D.DFB_F16, D.DFB_BF16, D.DFB_FP8E4M3])
def test_full_size_2048_sampled_tiles(dtype):
    """2048x2048, 64 bricks, 3 accumulated frames in each storage dtype (the
    launch shape the benchmark uses for it): every output of a seeded sample
    of tiles (plus the fullest tile) against the oracle fed the same stored
    values."""
    sc = scenes.scene_2048(seed=0, jitter_sigma=0.02)
    counts = sc.counts()
    rng = np.random.default_rng(1)
    sample = sorted(set(rng.choice(sc.n_tiles, 24, replace=False).tolist()) |
                    {int(np.argmax(counts)), int(np.argmin(counts))})
    fb = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH, dtype)
    imgs = []
    for f in range(3):
        stored, scales = scenes.store_rgba(sc.frame_rgba(f), dtype)
        fb.begin(f > 0)
        fb.submit_pool(sc.tile_ids, sc.keys, stored, sc.depth, scales)
        fb.end()
        imgs.append(o.composite_frame(sc.W, sc.H, sc.T, o.BLEND_DEPTH, sc.tile_ids, sc.keys,
                                      o.dequantize(stored, dtype, scales), sc.depth,
                                      tiles=sample))
        fb.keep.clear()
    col, acc = fb.color(), fb.accum()
    px, tv = fb.variance()
    p8 = fb.rgba8()
    mean, var = o.accumulate(imgs), o.variance(imgs)
    tvo = o.tile_variance(np.nan_to_num(var), sc.T)
    for t in sample:
        y0, x0 = (t // sc.tiles_x) * sc.T, (t % sc.tiles_x) * sc.T
        sl = (slice(y0, y0 + sc.T), slice(x0, x0 + sc.T))
        assert np.max(np.abs(col[sl] - imgs[-1][sl])) <= TOL
        assert np.max(np.abs(acc[sl] - mean[sl])) <= TOL
        assert np.max(np.abs(px[sl] - var[sl])) <= 1e-6
        assert abs(tv[t] - tvo[t]) <= 1e-4 * abs(tvo[t]) + 1e-9
        d8 = np.abs(o.unpack_rgba8(p8[sl]) - o.unpack_rgba8(o.pack_rgba8(mean[sl])))
        assert d8.max() <= 1
    st = fb.stats()
    assert st["fragments"] == sc.n and st["fragment_pixels"] == sc.fragment_pixels()


# --- failure detection: a bounded wait that runs out -------------------------------------
def test_stalled_work_item_times_out_and_context_survives():
    """A work item whose shared-memory stage is never filled (injected on the
    host) makes the kernel's bounded wait run out: the frame reports
    DFB_ERR_TIMEOUT, and the next frame on the same context is correct."""
    sc = scenes.scene_single_frame_256(seed=0)
    fb = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH)
    D.dfb_set_wait_limit(fb.h, 0.05)
    D.dfb_inject_stall(fb.h, 0)
    fb.begin(0)
    fb.submit_pool(sc.tile_ids, sc.keys, sc.rgba, sc.depth)
    fb.end()
    with pytest.raises(D.DfbError) as e:
        D.dfb_sync(fb.h)
    assert e.value.code == D.DFB_ERR_TIMEOUT
    D.dfb_sync(fb.h)                         # the error was reported once
    fb.begin(0)
    fb.submit_pool(sc.tile_ids, sc.keys, sc.rgba, sc.depth)
    fb.end()
    check_color(fb.color(), oracle_frame(sc, o.BLEND_DEPTH), D.DFB_BLEND_DEPTH)
