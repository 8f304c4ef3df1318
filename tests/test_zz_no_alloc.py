"""dfb_composite_noalloc: the single-frame entry point for callers that must
not allocate GPU memory (for instance a simulation that owns the whole device
through its own pool, or real-time code that cannot afford the device-wide
synchronisation a cudaMalloc may cause).

Calls in a row, through the C ABI, are checked against the handle-based path
(dfb_create / dfb_submit_tiles / dfb_end_frame), which allocates its own
buffers, and against the FP64 oracle fed the same stored values.  The second
call is smaller than the first, so leftovers of the first call in the shared
scratch array would show up as wrong pixels; the later calls have tiles with
more than 16 fragments, and one stores its tiles as FP8 with a scale per
tile.  This file is collected last on purpose."""

import numpy as np
import pytest

from harness import scenes
from oracle import dfb_oracle as o
from paper_2305_07083_gb300 import dfb as D

from tests.gpu_helpers import GpuFrameBuffer, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-5


def handle_path(sc, mode, dtype, stored, scales, bg):
    fb = GpuFrameBuffer(sc.W, sc.H, sc.T, mode, dtype,
                        flags=D.DFB_FLAG_WRITE_COLOR | D.DFB_FLAG_PACK_RGBA8, bg=bg)
    fb.begin(0)
    fb.submit_pool(sc.tile_ids, sc.keys, stored, sc.depth, scales)
    fb.end()
    col, p8 = fb.color(), fb.rgba8()
    fb.close()
    return col, p8


def noalloc_path(sc, mode, dtype, stored, scales, bg):
    import torch
    r = to_dev(stored)
    d = to_dev(sc.depth)
    color = torch.full((sc.H, sc.W, 4), -1.0, dtype=torch.float32, device="cuda")
    p8 = torch.zeros((sc.H, sc.W), dtype=torch.int32, device="cuda")
    rb = sc.T * sc.T * 4 * D.ELEMENT_BYTES[dtype]
    D.dfb_composite_noalloc(sc.W, sc.H, sc.T, mode, dtype, sc.tile_ids, sc.keys,
                            D.pool_pointers(r, sc.n, rb), D.pool_pointers(d, sc.n, sc.T * sc.T * 4),
                            scales, bg, color, p8)
    torch.cuda.synchronize()
    return color.cpu().numpy(), p8.cpu().numpy().view(np.uint32)


def test_two_calls_in_a_row_match_the_handle_path():
    calls = []
    big = scenes.scene_data_parallel(512, 384, 32, (4, 4, 4), seed=21, jitter_sigma=0.0)
    calls.append((big, D.DFB_BLEND_DEPTH, D.DFB_F32, (0.0, 0.0, 0.0, 0.0)))
    counts = np.random.default_rng(22).integers(0, 5, (-(-200 // 16)) * (-(-136 // 16)))
    small = scenes.random_scene(200, 136, 16, counts, seed=22, special_depths=True)
    calls.append((small, D.DFB_BLEND_ORDERED, D.DFB_F16, (0.2, 0.4, 0.6, 0.5)))
    assert small.n < big.n
    # long tiles (more than 16 fragments) stream in several fills; their
    # re-do list also lives in the fixed scratch
    counts = np.random.default_rng(23).integers(0, 4, 4 * 3)
    counts[[1, 6, 10]] = [20, 37, 17]
    longs = scenes.random_scene(256, 192, 64, counts, seed=23, alpha_max=0.3)
    calls.append((longs, D.DFB_BLEND_DEPTH, D.DFB_F32, (0.1, 0.2, 0.3, 1.0)))
    calls.append((longs, D.DFB_AVERAGE, D.DFB_BF16, (0.0, 0.0, 0.0, 0.0)))
    calls.append((longs, D.DFB_BLEND_ORDERED, D.DFB_FP8E4M3, (0.3, 0.3, 0.3, 0.25)))
    for sc, mode, dtype, bg in calls:
        stored, scales = scenes.store_rgba(sc.rgba, dtype)
        want_c, want_8 = handle_path(sc, mode, dtype, stored, scales, bg)
        got_c, got_8 = noalloc_path(sc, mode, dtype, stored, scales, bg)
        assert np.max(np.abs(got_c - want_c)) <= TOL
        d8 = np.abs(got_8.view(np.uint8).astype(int) - want_8.view(np.uint8).astype(int))
        assert d8.max() <= 1
        # and the oracle, on the same stored (dequantised) values
        ref = o.composite_frame(sc.W, sc.H, sc.T, mode, sc.tile_ids, sc.keys,
                                o.dequantize(stored, dtype, scales), sc.depth, bg=bg)
        assert np.max(np.abs(got_c.astype(np.float64) - ref)) <= TOL
        r8 = o.unpack_rgba8(o.pack_rgba8(ref)).astype(int)
        assert np.abs(o.unpack_rgba8(got_8).astype(int) - r8).max() <= 1


def test_refuses_host_tiles_and_a_capturing_stream():
    import torch
    sc = scenes.random_scene(64, 64, 16, np.full(16, 2), seed=24)
    out = torch.empty((sc.H, sc.W, 4), dtype=torch.float32, device="cuda")
    host_r = np.ascontiguousarray(sc.rgba, np.float32)
    host_d = np.ascontiguousarray(sc.depth, np.float32)
    dev_d = to_dev(sc.depth)
    tb = sc.T * sc.T
    # ordinary host memory passed as tiles: refused before any GPU work
    with pytest.raises(D.DfbError) as e:
        D.dfb_composite_noalloc(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH, D.DFB_F32, sc.tile_ids,
                                sc.keys, D.pool_pointers(host_r, sc.n, tb * 16),
                                D.pool_pointers(dev_d, sc.n, tb * 4), None, None, out, None)
    assert e.value.code == D.DFB_ERR_INVALID_ARG
    with pytest.raises(D.DfbError) as e:
        D.dfb_composite_noalloc(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH, D.DFB_F32, sc.tile_ids,
                                sc.keys, D.pool_pointers(to_dev(sc.rgba), sc.n, tb * 16),
                                D.pool_pointers(host_d, sc.n, tb * 4), None, None, out, None)
    assert e.value.code == D.DFB_ERR_INVALID_ARG
    # a stream under capture: refused before the stream is touched
    dev_r = to_dev(sc.rgba)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.stream(s):
        g.capture_begin(capture_error_mode="relaxed")
        try:
            D.dfb_composite_noalloc(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH, D.DFB_F32, sc.tile_ids,
                                    sc.keys, D.pool_pointers(dev_r, sc.n, tb * 16),
                                    D.pool_pointers(dev_d, sc.n, tb * 4), None, None, out, None,
                                    stream=s)
        except D.DfbError as err:
            codes.append(err.code)
        finally:
            g.capture_end()
    assert codes == [D.DFB_ERR_STATE]
    # the same call on an ordinary stream then succeeds
    D.dfb_composite_noalloc(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH, D.DFB_F32, sc.tile_ids, sc.keys,
                            D.pool_pointers(dev_r, sc.n, tb * 16),
                            D.pool_pointers(dev_d, sc.n, tb * 4), None, None, out, None)
    ref = o.composite_frame(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH, sc.tile_ids, sc.keys,
                            sc.rgba.astype(np.float64), sc.depth)
    assert np.max(np.abs(out.cpu().numpy().astype(np.float64) - ref)) <= TOL


def test_a_wait_that_runs_out_is_reported_and_the_next_call_is_correct():
    """Failure detection without a GPU fault: the next call leaves work item 0
    unfilled (injected on the host), so its consumers' bounded wait (50 ms
    here) runs out and the kernel gives up; the call returns DFB_ERR_TIMEOUT.
    The following call, on the same context and scratch, matches the
    oracle."""
    import torch
    sc = scenes.random_scene(128, 96, 32, np.full(12, 3), seed=25, alpha_max=0.6)
    dev_r, dev_d = to_dev(sc.rgba), to_dev(sc.depth)
    out = torch.empty((sc.H, sc.W, 4), dtype=torch.float32, device="cuda")
    tb = sc.T * sc.T

    def call():
        D.dfb_composite_noalloc(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH, D.DFB_F32, sc.tile_ids,
                                sc.keys, D.pool_pointers(dev_r, sc.n, tb * 16),
                                D.pool_pointers(dev_d, sc.n, tb * 4), None, None, out, None)

    D.dfb_noalloc_set_wait_limit(0.05)
    try:
        D.dfb_noalloc_inject_stall(0)
        with pytest.raises(D.DfbError) as e:
            call()
        assert e.value.code == D.DFB_ERR_TIMEOUT
        call()                                   # the injected stall was used up
        ref = o.composite_frame(sc.W, sc.H, sc.T, D.DFB_BLEND_DEPTH, sc.tile_ids, sc.keys,
                                sc.rgba.astype(np.float64), sc.depth)
        assert np.max(np.abs(out.cpu().numpy().astype(np.float64) - ref)) <= TOL
    finally:
        D.dfb_noalloc_inject_stall(-1)
        D.dfb_noalloc_set_wait_limit(2.0)


def test_rejects_requests_beyond_the_fixed_scratch():
    import torch
    out = torch.empty((64, 64, 4), dtype=torch.float32, device="cuda")
    n = 65537
    with pytest.raises(D.DfbError) as e:
        D.dfb_composite_noalloc(64, 64, 16, D.DFB_BLEND_DEPTH, D.DFB_F32, np.zeros(n, np.int32),
                                np.zeros(n, np.float32), np.zeros(n, np.uint64),
                                np.zeros(n, np.uint64), None, None, out, None)
    assert e.value.code == D.DFB_ERR_CAPACITY
    with pytest.raises(D.DfbError) as e:      # 257 x 257 tiles of 4 pixels
        D.dfb_composite_noalloc(1028, 1028, 4, D.DFB_BLEND_DEPTH, D.DFB_F32, [], [], [], [],
                                None, None, out, None)
    assert e.value.code == D.DFB_ERR_CAPACITY
