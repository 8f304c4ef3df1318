"""Tile ownership across ranks (Sec. 3, 3.2, 4.1.1) on CPU ranks: the
partition of the tiles, the routing of fragment tiles to their owners
(headers first, then the tiles as asynchronous all-to-alls; gloo, world
size 2 and 3), and the gather of the owners' tiles into the display rank's
frame.

In these CPU tests the owners composite their tiles with the oracle (test
code); the library's own compositing on each owner is covered by
tests/test_gpu_distributed.py.  The gathered frame is compared with the
oracle's composite of the union of every rank's fragments, taken in rank
order (the order that breaks ties of equal keys)."""

import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from harness import scenes  # noqa: E402
from oracle import dfb_oracle as o  # noqa: E402
from paper_2305_07083_gb300 import distributed as DD  # noqa: E402

W, H, T = 150, 100, 16


def rank_fragments(rank, n_tiles, seed):
    """A rank's own fragment tiles: arbitrary tiles of the frame (any rank
    may render for any tile), random depths, some equal keys across ranks."""
    rng = np.random.default_rng([seed, rank])
    counts = rng.integers(0, 4, n_tiles)
    sc = scenes.random_scene(W, H, T, counts, seed=seed * 10 + rank, alpha_max=0.7,
                             equal_keys=True)
    return sc


@pytest.mark.parametrize("scheme", ["round_robin", "block"])
@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_partition_covers_every_tile_once(scheme, world):
    own = DD.TileOwnership(W, H, T, world, scheme)
    allt = np.concatenate(own.owned)
    assert sorted(allt.tolist()) == list(range(own.n_tiles))
    for r in range(world):
        assert (own.owner[own.owned[r]] == r).all()
        np.testing.assert_array_equal(own.local_index[own.owned[r]], np.arange(len(own.owned[r])))
        cols, rows = own.local_grid(r)
        assert cols * rows >= len(own.owned[r])
    sizes = [len(x) for x in own.owned]
    assert max(sizes) - min(sizes) <= 1           # both schemes balance the tile count
    if scheme == "block":                         # contiguous runs
        for r in range(world):
            if len(own.owned[r]):
                assert own.owned[r][-1] - own.owned[r][0] + 1 == len(own.owned[r])


def test_route_is_stable_by_destination():
    own = DD.TileOwnership(W, H, T, 3)
    tiles = np.random.default_rng(1).integers(0, own.n_tiles, 200)
    order, counts = DD.route(tiles, own)
    dest = own.owner[tiles]
    want = [i for r in range(3) for i in range(len(tiles)) if dest[i] == r]   # brute force
    assert order.tolist() == want
    assert counts.tolist() == [int((dest == r).sum()) for r in range(3)]


def test_header_round_trip():
    sc = scenes.random_scene(32, 32, 16, np.array([2, 0, 3, 1]), seed=4, special_depths=True)
    scales = np.linspace(0.5, 2.0, sc.n).astype(np.float32)
    order = np.arange(sc.n)[::-1].copy()
    for sc_in in (None, scales):
        hdr = DD.pack_headers(sc.tile_ids, sc.keys, sc_in, order)
        assert hdr.shape == (sc.n, 4) and hdr.dtype == np.int32
        assert hdr.nbytes == sc.n * DD.HEADER_BYTES
        tid, key, scl = DD.unpack_headers(hdr)
        np.testing.assert_array_equal(tid, sc.tile_ids[order])
        np.testing.assert_array_equal(key.view(np.int32), sc.keys[order].view(np.int32))
        want = np.ones(sc.n, np.float32) if sc_in is None else scales[order]
        np.testing.assert_array_equal(scl, want)


def _owner_composite(own, rank, tid, key, rgba, depth, mode):
    """Test-side stand-in for the owner's compositing: the oracle on the
    fragments this rank received, into the rank's local tile grid."""
    cols, rows = own.local_grid(rank)
    img = np.zeros((rows * T, cols * T, 4))
    lists, _, _ = o.bucket(own.local_index[tid], key, max(1, len(own.owned[rank])))
    for i in range(len(own.owned[rank])):
        idx = np.asarray(lists[i], dtype=np.int64)
        res = o.composite_tile(rgba[idx].astype(np.float64), depth[idx], key[idx], idx, mode)
        r, c = divmod(i, cols)
        img[r * T:(r + 1) * T, c * T:(c + 1) * T] = res.reshape(T, T, 4)
    return img


def _rank_main(rank, world, port, scheme, mode, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        own = DD.TileOwnership(W, H, T, world, scheme)
        sc = rank_fragments(rank, own.n_tiles, 7)
        src_r, src_d = torch.from_numpy(sc.rgba.copy()), torch.from_numpy(sc.depth.copy())
        # the headers over a group of their own, as a DistributedFrameBuffer
        # on an NCCL group does
        meta = dist.new_group(backend="gloo")
        pend = DD.exchange_async(sc.tile_ids, sc.keys, src_r, src_d, own, meta_group=meta)
        # the headers are known at once; the sources may be reused at once
        # (the next frame produced into them) while the tiles travel
        src_r.fill_(-7.0)
        src_d.fill_(-7.0)
        pend.wait()
        tid, key, scl, r, d = pend.tile_ids, pend.keys, pend.scales, pend.rgba, pend.depth
        # every received fragment is owned here, and nothing owned is missing
        assert (own.owner[tid] == rank).all()
        allfr = [rank_fragments(s, own.n_tiles, 7) for s in range(world)]
        want_t, want_k, want_r = [], [], []
        for s, f in enumerate(allfr):                 # (source rank, source order)
            sel = np.nonzero(own.owner[f.tile_ids] == rank)[0]
            want_t.append(f.tile_ids[sel])
            want_k.append(f.keys[sel])
            want_r.append(f.rgba[sel])
        np.testing.assert_array_equal(tid, np.concatenate(want_t))
        np.testing.assert_array_equal(key, np.concatenate(want_k))
        np.testing.assert_array_equal(r.numpy(), np.concatenate(want_r))
        local = _owner_composite(own, rank, tid, key, r.numpy(), d.numpy(), mode)
        frame = DD.gather_tiles(local, own)
        if rank == 0:
            union_t = np.concatenate([f.tile_ids for f in allfr])
            union_k = np.concatenate([f.keys for f in allfr])
            union_r = np.concatenate([f.rgba for f in allfr]).astype(np.float64)
            union_d = np.concatenate([f.depth for f in allfr])
            ref = o.composite_frame(W, H, T, mode, union_t, union_k, union_r, union_d)
            q.put(("frame", float(np.max(np.abs(frame - ref)))))
        else:
            assert frame is None
        q.put(("ok", rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,scheme,mode", [(2, "round_robin", o.BLEND_DEPTH),
                                               (2, "block", o.BLEND_ORDERED),
                                               (3, "round_robin", o.ZCOMPOSITE)])
def test_exchange_and_gather_equal_the_single_process_frame(world, scheme, mode):
    port = 29811 + world + (3 if scheme == "block" else 0) + 7 * mode
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, scheme, mode, q))
             for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=180) for _ in range(world + 1)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    errs = [v for k, v in got if k == "frame"]
    assert len(errs) == 1 and errs[0] == 0.0      # same oracle arithmetic on the same lists
    assert sorted(v for k, v in got if k == "ok") == list(range(world))


def _empty_rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        own = DD.TileOwnership(W, H, T, world)
        full = rank_fragments(0, own.n_tiles, 5)
        if rank == 0:
            sc = full
        else:                                   # this rank rendered nothing this frame
            sc = scenes.Scene(W, H, T, full.tile_ids[:0], full.keys[:0], full.rgba[:0],
                              full.depth[:0])
        pend = DD.exchange_async(sc.tile_ids, sc.keys, torch.from_numpy(sc.rgba),
                                 torch.from_numpy(sc.depth), own).wait()
        mine = np.nonzero(own.owner[full.tile_ids] == rank)[0]
        np.testing.assert_array_equal(pend.tile_ids, full.tile_ids[mine])
        np.testing.assert_array_equal(pend.rgba.numpy(), full.rgba[mine])
        assert pend.depth.shape == (len(mine),) + full.depth.shape[1:]
        q.put(("ok", rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_exchange_with_a_rank_that_sends_nothing():
    world, port = 2, 29871
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_empty_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(v for _, v in got) == [0, 1]
