"""Tile ownership across ranks with the library compositing on each owner
(Sec. 3, 3.2, 4.1.1): DistributedFrameBuffer sends every rank's fragment
tiles to their owners in one all-to-all, each owner composites its tiles on
its GPU through the C ABI, and the display rank gathers the frame.

One GPU serves here: the single-rank case, and two ranks (two processes on
the same GPU, a gloo group whose exchange is staged through host memory;
their kernels never wait on one another).  The second frame goes through
post() / composite_received() with the next frame produced in between.  The gathered colour, RGBA8 and
accumulation are compared with the oracle's composite of the union of the
ranks' fragments in rank order."""

import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from harness import scenes  # noqa: E402
from oracle import dfb_oracle as o  # noqa: E402

pytestmark = pytest.mark.gpu

W, H, T = 300, 200, 32
TOL = 1e-5


def rank_frames(rank, n_tiles, frames=2):
    """A rank's fragment tiles for each frame: any tiles of the frame, some
    long lists, depths in random order."""
    out = []
    for f in range(frames):
        rng = np.random.default_rng([11, rank, f])
        counts = rng.integers(0, 5, n_tiles)
        counts[rng.random(n_tiles) < 0.1] = 12
        out.append(scenes.random_scene(W, H, T, counts, seed=100 * rank + f, alpha_max=0.6))
    return out


def run_rank(rank, world, mode, dtype, scheme):
    """Composite two accumulated frames on this rank; returns the gathered
    (colour of the last frame, RGBA8, accumulation) on rank 0."""
    import torch
    from paper_2305_07083_gb300 import build, dfb as D, distributed as DD
    build()
    torch.cuda.set_device(0)
    fb = DD.DistributedFrameBuffer(W, H, T, mode, dtype, scheme=scheme)
    frames = rank_frames(rank, fb.own.n_tiles)

    def produce(sc):
        stored, scales = scenes.store_rgba(sc.rgba, dtype)
        st = np.ascontiguousarray(stored)
        r = torch.from_numpy(st.view(np.int16) if st.dtype == np.uint16 else st).cuda()
        return r, torch.from_numpy(sc.depth).cuda(), scales

    # frame 0 in one call; frame 1 posted, then the next frame's tiles are
    # produced into other buffers while the tiles travel, then composited
    r, d, scales = produce(frames[0])
    fb.composite(frames[0].tile_ids, frames[0].keys, r, d, scales, accumulate=False)
    D.dfb_sync(fb.h)
    r, d, scales = produce(frames[1])
    pend = fb.post(frames[1].tile_ids, frames[1].keys, r, d, scales)
    nxt = produce(frames[0])
    fb.composite_received(pend, accumulate=True)
    D.dfb_sync(fb.h)
    del nxt
    res = (fb.gather("color"), fb.gather("rgba8"), fb.gather("accum"))
    fb.close()
    return res


def oracle_reference(world, mode, dtype):
    per_rank = [rank_frames(r, (-(-W // T)) * (-(-H // T))) for r in range(world)]
    imgs = []
    for f in range(2):
        frs = [per_rank[r][f] for r in range(world)]
        tid = np.concatenate([x.tile_ids for x in frs])
        key = np.concatenate([x.keys for x in frs])
        deq = []
        for x in frs:
            stored, scales = scenes.store_rgba(x.rgba, dtype)
            deq.append(o.dequantize(stored, dtype, scales))
        dep = np.concatenate([x.depth for x in frs])
        imgs.append(o.composite_frame(W, H, T, mode, tid, key, np.concatenate(deq), dep))
    return imgs


def check(res, imgs):
    color, rgba8, accum = res
    assert np.max(np.abs(color.astype(np.float64) - imgs[-1])) <= TOL
    mean = o.accumulate(imgs)
    assert np.max(np.abs(accum.astype(np.float64) - mean)) <= TOL
    d8 = np.abs(o.unpack_rgba8(rgba8).astype(int) - o.unpack_rgba8(o.pack_rgba8(mean)).astype(int))
    assert d8.max() <= 1


@pytest.mark.parametrize("mode,dtype", [(0, 0), (1, 1)])
def test_single_rank(mode, dtype):
    res = run_rank(0, 1, mode, dtype, "round_robin")
    check(res, oracle_reference(1, mode, dtype))


def _two_rank_main(rank, world, port, mode, dtype, scheme, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = run_rank(rank, world, mode, dtype, scheme)
        if rank == 0:
            q.put(res)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode,dtype,scheme", [(0, 0, "round_robin"), (0, 1, "block"),
                                               (2, 3, "round_robin")])
def test_two_ranks_on_one_gpu(mode, dtype, scheme):
    world = 2
    port = 29901 + 3 * mode + dtype + (1 if scheme == "block" else 0)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_two_rank_main, args=(r, world, port, mode, dtype, scheme, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    imgs = oracle_reference(world, mode, dtype)
    if mode == 2:
        # z-composite: the winners' RGBA are copied exactly (FP8: one FP32
        # rounding of code x scale); the frame is checked within the bar
        assert np.max(np.abs(res[0].astype(np.float64) - imgs[-1])) <= TOL
    check(res, imgs)
