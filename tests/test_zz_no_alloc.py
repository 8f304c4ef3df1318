"""dfb_composite_noalloc: the single-frame entry point for callers that must
not allocate GPU memory (for instance a simulation that owns the whole device
through its own pool, or real-time code that cannot afford the device-wide
synchronisation a cudaMalloc may cause).

Calls in a row, through the C ABI, are checked against the handle-based path
(dfb_create / dfb_submit_tiles / dfb_end_frame), which allocates its own
buffers.  The second call is smaller than the first, so leftovers of the first
call in the shared scratch array would show up as wrong pixels; the last two
have tiles with more than 16 fragments.  This file is collected last on
purpose."""

import numpy as np
import pytest

from harness import scenes
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
    # long tiles (more than 16 fragments) go through the long-tile kernel,
    # whose list also lives in the fixed scratch
    counts = np.random.default_rng(23).integers(0, 4, 4 * 3)
    counts[[1, 6, 10]] = [20, 37, 17]
    longs = scenes.random_scene(256, 192, 64, counts, seed=23, alpha_max=0.3)
    calls.append((longs, D.DFB_BLEND_DEPTH, D.DFB_F32, (0.1, 0.2, 0.3, 1.0)))
    calls.append((longs, D.DFB_AVERAGE, D.DFB_BF16, (0.0, 0.0, 0.0, 0.0)))
    for sc, mode, dtype, bg in calls:
        stored, scales = scenes.store_rgba(sc.rgba, dtype)
        want_c, want_8 = handle_path(sc, mode, dtype, stored, scales, bg)
        got_c, got_8 = noalloc_path(sc, mode, dtype, stored, scales, bg)
        assert np.max(np.abs(got_c - want_c)) <= TOL
        d8 = np.abs(got_8.view(np.uint8).astype(int) - want_8.view(np.uint8).astype(int))
        assert d8.max() <= 1


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
