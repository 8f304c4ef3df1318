"""Tile ownership across ranks (Sec. 3, 3.2, 4.1.1) on CPU ranks: the
partition of the tiles, the routing of fragment tiles to their owners in one
all-to-all exchange (gloo, world size 2 and 3), and the gather of the
owners' tiles into the display rank's frame.

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


def test_pack_unpack_round_trip_all_dtypes():
    for dt in (0, 1, 2, 3):
        sc = scenes.random_scene(32, 32, 16, np.array([2, 0, 3, 1]), seed=4)
        stored, scales = scenes.store_rgba(sc.rgba, dt)
        st = np.ascontiguousarray(stored)
        rgba = torch.from_numpy(st.view(np.int16) if st.dtype == np.uint16 else st)
        depth = torch.from_numpy(sc.depth)
        order = np.arange(sc.n)[::-1].copy()
        buf, rec = DD.pack_records(sc.tile_ids, sc.keys, rgba, depth, scales, order)
        assert rec == DD.HEADER_BYTES + rgba[0].numel() * rgba.element_size() + 16 * 16 * 4
        tid, key, scl, r2, d2 = DD.unpack_records(buf, tuple(rgba.shape[1:]), rgba.dtype,
                                                  tuple(depth.shape[1:]))
        np.testing.assert_array_equal(tid, sc.tile_ids[order])
        np.testing.assert_array_equal(key, sc.keys[order])
        if scales is not None:
            np.testing.assert_array_equal(scl, np.asarray(scales, np.float32)[order])
        assert torch.equal(r2, rgba[order])
        assert torch.equal(d2, depth[order])


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
        tid, key, scl, r, d = DD.exchange(sc.tile_ids, sc.keys, torch.from_numpy(sc.rgba),
                                          torch.from_numpy(sc.depth), own)
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
