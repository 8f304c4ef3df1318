"""Batched compositing: several frames of different sizes in one persistent
launch (dfb_end_frames), and the same work replayed from a CUDA graph, must
give exactly the per-frame results (work items are independent and each is
computed the same way), which match the FP64 oracle."""

import numpy as np
import pytest

from harness import scenes
from oracle import dfb_oracle as o
from paper_2305_07083_gb300 import dfb as D

from tests.gpu_helpers import GpuFrameBuffer

pytestmark = pytest.mark.gpu

TOL = 1e-5


def mixed_frames(dtype):
    """(scene, mode) pairs of different sizes, tile sizes and fragment counts,
    including tiles with more fragments than the kernel stages."""
    out = []
    out.append((scenes.scene_data_parallel(256, 192, 64, (3, 3, 3), seed=31, jitter_sigma=0.0),
                D.DFB_BLEND_DEPTH))
    counts = np.random.default_rng(32).integers(0, 6, 13 * 9)
    counts[5] = 40                                   # streamed work items
    out.append((scenes.random_scene(200, 136, 16, counts, seed=32, special_depths=True),
                D.DFB_BLEND_DEPTH))
    out.append((scenes.scene_data_parallel(128, 128, 32, (2, 2, 2), seed=33, jitter_sigma=0.0),
                D.DFB_BLEND_ORDERED))
    counts = np.random.default_rng(34).integers(0, 20, 4)
    out.append((scenes.random_scene(64, 64, 32, counts, seed=34, depth_levels=4),
                D.DFB_ZCOMPOSITE))
    counts = np.random.default_rng(35).integers(0, 5, 12)
    counts[7] = 30                                    # long tile of 16 work items
    out.append((scenes.random_scene(256, 192, 64, counts, seed=35), D.DFB_AVERAGE))
    return out


def make_buffers(frames, dtype):
    fbs = []
    for sc, mode in frames:
        stored, scales = scenes.store_rgba(sc.rgba, dtype)
        fb = GpuFrameBuffer(sc.W, sc.H, sc.T, mode, dtype)
        fb.begin(0)
        fb.submit_pool(sc.tile_ids, sc.keys, stored, sc.depth, scales)
        fb.stored, fb.scales = stored, scales
        fbs.append(fb)
    return fbs


def outputs(fb):
    return fb.color(), fb.rgba8()


@pytest.mark.parametrize("dtype", [D.DFB_F32, D.DFB_F16])
def test_batch_equals_individual_frames_and_oracle(dtype):
    frames = mixed_frames(dtype)
    alone = []
    for fb in make_buffers(frames, dtype):
        fb.end()
        alone.append(outputs(fb))
    fbs = make_buffers(frames, dtype)
    D.dfb_end_frames([fb.h for fb in fbs])
    for (sc, mode), fb, (c0, p0) in zip(frames, fbs, alone):
        c1, p1 = outputs(fb)
        np.testing.assert_array_equal(c1, c0)
        np.testing.assert_array_equal(p1, p0)
        want = o.composite_frame(sc.W, sc.H, sc.T, mode, sc.tile_ids, sc.keys,
                                 o.dequantize(fb.stored, dtype, fb.scales), sc.depth)
        if mode == D.DFB_ZCOMPOSITE:
            np.testing.assert_array_equal(c1.astype(np.float64), want)
        else:
            assert np.max(np.abs(c1 - want)) <= TOL


def test_graph_replays_equal_individual_frames():
    dtype = D.DFB_F16
    frames = mixed_frames(dtype)
    alone = []
    for fb in make_buffers(frames, dtype):
        fb.end()
        alone.append(outputs(fb))
    fbs = make_buffers(frames, dtype)
    g = D.dfb_graph_create([fb.h for fb in fbs])
    try:
        for _ in range(2):
            D.dfb_graph_launch(g)
            for fb, (c0, p0) in zip(fbs, alone):
                c1, p1 = outputs(fb)
                np.testing.assert_array_equal(c1, c0)
                np.testing.assert_array_equal(p1, p0)
        best = D.dfb_graph_autotune(g, None, 2)
        assert best["ring_kb"] > 0 and best["ms"] > 0
        assert (best["groups"], best["ctas_per_sm"]) in ((1, 2), (2, 2), (1, 3), (2, 1), (3, 1))
        D.dfb_graph_launch(g)
        for fb, (c0, p0) in zip(fbs, alone):
            np.testing.assert_array_equal(outputs(fb)[0], c0)
    finally:
        D.dfb_graph_destroy(g)


def test_graph_rejects_mixed_dtypes_and_closed_frames():
    a = GpuFrameBuffer(64, 64, 16, D.DFB_BLEND_DEPTH, D.DFB_F32)
    b = GpuFrameBuffer(64, 64, 16, D.DFB_BLEND_DEPTH, D.DFB_F16)
    a.begin(0)
    b.begin(0)
    with pytest.raises(D.DfbError) as e:
        D.dfb_graph_create([a.h, b.h])
    assert e.value.code == D.DFB_ERR_INVALID_ARG
    c = GpuFrameBuffer(64, 64, 16, D.DFB_BLEND_DEPTH, D.DFB_F32)
    with pytest.raises(D.DfbError) as e:
        D.dfb_graph_create([a.h, c.h])
    assert e.value.code == D.DFB_ERR_STATE


def test_run_frames_with_prepared_sets_equals_individual_frames():
    """dfb_run_frames (prepared tile sets, one call per step) over several
    accumulated steps gives exactly what per-frame dfb_submit_tiles +
    dfb_end_frame give, frame by frame."""
    import torch
    dtype = D.DFB_F16
    frames = mixed_frames(dtype)
    fbs_a = make_buffers(frames, dtype)       # per-frame path
    for fb in fbs_a:
        fb.end()
    fbs_b = []
    sets = []
    for (sc, mode), fa in zip(frames, fbs_a):
        fb = GpuFrameBuffer(sc.W, sc.H, sc.T, mode, dtype)
        r = torch.from_numpy(np.ascontiguousarray(fa.stored).view(np.int16)).cuda()
        d = torch.from_numpy(np.ascontiguousarray(sc.depth)).cuda()
        fb.keep += [r, d]
        n, P = len(sc.tile_ids), sc.T * sc.T
        sets.append(D.dfb_tileset_create(fb.h, sc.tile_ids, sc.keys,
                                         D.pool_pointers(r, n, P * 8), D.pool_pointers(d, n, P * 4)))
        fbs_b.append(fb)
    try:
        for step in range(3):
            if step > 0:
                for (sc, mode), fa in zip(frames, fbs_a):
                    fa.begin(1)
                    fa.submit_pool(sc.tile_ids, sc.keys, fa.stored, sc.depth, fa.scales)
                    fa.end()
            D.dfb_run_frames([fb.h for fb in fbs_b], sets, [1 if step else 0] * len(sets))
            for fa, fb in zip(fbs_a, fbs_b):
                np.testing.assert_array_equal(fb.color(), fa.color())
                np.testing.assert_array_equal(fb.accum(), fa.accum())
                np.testing.assert_array_equal(fb.rgba8(), fa.rgba8())
                assert fb.stats()["accumulated"] == step + 1
                assert fb.stats()["fragment_pixels"] == fa.stats()["fragment_pixels"]
    finally:
        for s in sets:
            D.dfb_tileset_destroy(s)


def test_end_frame_inside_a_stream_capture_is_refused():
    """Capturing dfb_end_frame would replay stale records; the call is
    refused with STATE and the frame stays open for an ordinary end."""
    import torch
    sc = scenes.scene_single_frame_256(seed=2)
    fb = GpuFrameBuffer(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH)
    fb.begin(0)
    fb.submit_pool(sc.tile_ids, sc.keys, sc.rgba, sc.depth)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    code = None
    with torch.cuda.graph(g, stream=s):
        x = torch.zeros(4, device="cuda")
        x += 1                                        # the graph is not empty
        try:
            D.dfb_end_frame(fb.h, s)
        except D.DfbError as e:
            code = e.code
    assert code == D.DFB_ERR_STATE
    fb.end()
    want = o.composite_frame(sc.W, sc.H, sc.T, o.BLEND_DEPTH, sc.tile_ids, sc.keys,
                             sc.rgba.astype(np.float64), sc.depth)
    assert np.max(np.abs(fb.color() - want)) <= TOL


def test_pixel_ops_per_handle_in_one_launch():
    """Each handle's pixel operation (tone curves of different lengths,
    Reinhard, exposure, none) applies to its own frame inside one batched
    launch and one graph replay; the RGBA8 equals the handle alone and the
    oracle within 1 LSB."""
    dtype = D.DFB_F32
    frames = mixed_frames(dtype)
    rng = np.random.default_rng(36)

    def curve(n):
        c = np.sort(rng.random((3, n)), axis=1)
        return c.astype(np.float32)
    ops = [(D.DFB_PIXELOP_CURVE, 1.4, curve(33), 1.25), (D.DFB_PIXELOP_REINHARD, 3.0, None, None),
           (D.DFB_PIXELOP_NONE, 1.0, None, None), (D.DFB_PIXELOP_EXPOSURE, 0.6, None, None),
           (D.DFB_PIXELOP_CURVE, 1.0, curve(5), 2.0)]

    def setup():
        fbs = make_buffers(frames, dtype)
        for fb, (op, e, c, xm) in zip(fbs, ops):
            D.dfb_set_pixel_op(fb.h, D.DFB_PIXELOP_EXPOSURE, e)
            if op == D.DFB_PIXELOP_CURVE:
                D.dfb_set_pixel_curve(fb.h, c, xm)
            else:
                D.dfb_set_pixel_op(fb.h, op, e)
        return fbs
    alone = []
    for fb in setup():
        fb.end()
        alone.append(fb.rgba8())
    fbs = setup()
    D.dfb_end_frames([fb.h for fb in fbs])
    for (sc, mode), fb, p0, (op, e, c, xm) in zip(frames, fbs, alone, ops):
        p1 = fb.rgba8()
        np.testing.assert_array_equal(p1, p0)
        col = o.composite_frame(sc.W, sc.H, sc.T, mode, sc.tile_ids, sc.keys,
                                o.dequantize(fb.stored, dtype, fb.scales), sc.depth)
        want = o.pack_rgba8(o.pixel_op(col, op, e, None if c is None else c.astype(np.float64),
                                       1.0 if xm is None else xm))
        assert np.abs(o.unpack_rgba8(p1) - o.unpack_rgba8(want)).max() <= 1
    fbs = setup()
    g = D.dfb_graph_create([fb.h for fb in fbs])
    try:
        D.dfb_graph_launch(g)
        for fb, p0 in zip(fbs, alone):
            np.testing.assert_array_equal(fb.rgba8(), p0)
    finally:
        D.dfb_graph_destroy(g)
