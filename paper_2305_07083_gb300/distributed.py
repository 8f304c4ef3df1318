"""Tile ownership across ranks: the distribution of the framebuffer (Sec. 3,
3.2 and 4.1.1), one process per GPU.

Every image tile has exactly one owner rank.  Each rank's producers render
fragment tiles for any image tile; at the end of a frame every rank sends
each of its fragment tiles to the tile's owner in one all-to-all exchange
(the paper sends them as asynchronous messages), so that the fragments land
in the owner's own memory before any kernel reads them.  The owner
composites its tiles with the library (dfb_submit_tiles / dfb_end_frame on
a framebuffer that holds only its tiles), and the finished tiles are
gathered to the display rank (the paper's gather of the final image).
Ownership is independent of which rank renders what (Sec. 4.1.1): any
rank may produce fragments for any tile.

Ownership schemes: "round_robin" (tile t belongs to rank t mod N, which
spreads the frame's dense regions over the ranks) and "block" (contiguous
runs of tiles).  An owner lays its tiles out as a small framebuffer of its
own (owned tile i at local tile i, row-major in a grid of full T x T
tiles); pixels of a frame-edge tile that fall outside the frame are
composited too and cropped by the gather.

Order of equal keys: the owner submits the fragments it receives in
(source rank, the source's own order) order, so the submission index that
breaks ties is the fragment's position in the ranks' lists taken in rank
order.

The exchange and the gather use torch.distributed: on an NCCL group the
device buffers travel as they are; on a gloo group (CPU ranks, tests) they
are staged through host memory.
"""

from __future__ import annotations

import math

import numpy as np

from . import dfb as D

HEADER_BYTES = 16  # tile id (int32), order key (f32), FP8 scale (f32), spare


class TileOwnership:
    """Owner rank of every tile of a W x H frame of T x T tiles."""

    def __init__(self, W, H, T, world, scheme="round_robin"):
        if world < 1:
            raise ValueError("world must be >= 1")
        self.W, self.H, self.T, self.world = W, H, T, world
        self.tiles_x = -(-W // T)
        self.tiles_y = -(-H // T)
        self.n_tiles = self.tiles_x * self.tiles_y
        t = np.arange(self.n_tiles, dtype=np.int64)
        if scheme == "round_robin":
            owner = t % world
        elif scheme == "block":
            owner = (t * world) // self.n_tiles
        else:
            raise ValueError("unknown ownership scheme %r" % scheme)
        self.scheme = scheme
        self.owner = owner.astype(np.int32)
        self.owned = [np.nonzero(self.owner == r)[0].astype(np.int32) for r in range(world)]
        self.local_index = np.empty(self.n_tiles, np.int32)
        for r in range(world):
            self.local_index[self.owned[r]] = np.arange(len(self.owned[r]), dtype=np.int32)

    def local_grid(self, rank):
        """(tiles_x, tiles_y) of rank's own framebuffer (at least 1 x 1)."""
        n = max(1, len(self.owned[rank]))
        cols = int(math.ceil(math.sqrt(n)))
        return cols, -(-n // cols)

    def local_size(self, rank):
        cols, rows = self.local_grid(rank)
        return cols * self.T, rows * self.T

    def destinations(self, tile_ids):
        return self.owner[np.asarray(tile_ids, dtype=np.int64)]


def _rank_world(group):
    import torch.distributed as dist
    if group is None and not dist.is_initialized():
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def _staged(group):
    """Whether collectives of `group` need host tensors (gloo)."""
    import torch.distributed as dist
    return dist.get_backend(group) != "nccl"


def route(tile_ids, own: TileOwnership):
    """Stable order of a rank's fragments by destination rank and the number
    of fragments for every destination."""
    dest = own.destinations(tile_ids)
    order = np.argsort(dest, kind="stable")
    counts = np.bincount(dest, minlength=own.world).astype(np.int64)
    return order, counts


def pack_records(tile_ids, keys, rgba, depth, scales, order):
    """Fixed-size byte records of the fragments in `order`: header (tile id,
    key, scale), then the T*T RGBA values and T*T depths.  `rgba` and
    `depth` are tensors of shape (n, ...) on any device; the result is on
    the same device."""
    import torch
    n = len(order)
    dev = rgba.device
    rb = int(np.prod(rgba.shape[1:])) * rgba.element_size()
    db = int(np.prod(depth.shape[1:])) * depth.element_size()
    rec = HEADER_BYTES + rb + db
    out = torch.empty((n, rec), dtype=torch.uint8, device=dev)
    if n == 0:
        return out, rec
    idx = torch.as_tensor(np.ascontiguousarray(order), dtype=torch.long, device=dev)
    hdr = np.zeros((n, 4), np.float32)
    hdr.view(np.int32)[:, 0] = np.asarray(tile_ids, np.int32)[order]
    hdr[:, 1] = np.asarray(keys, np.float32)[order]
    hdr[:, 2] = 1.0 if scales is None else np.asarray(scales, np.float32)[order]
    out[:, :HEADER_BYTES] = torch.from_numpy(hdr.view(np.uint8).reshape(n, HEADER_BYTES)).to(dev)
    out[:, HEADER_BYTES:HEADER_BYTES + rb] = rgba.index_select(0, idx).reshape(n, -1).view(torch.uint8)
    out[:, HEADER_BYTES + rb:] = depth.index_select(0, idx).reshape(n, -1).view(torch.uint8)
    return out, rec


def unpack_records(buf, rgba_shape, rgba_dtype, depth_shape):
    """Inverse of pack_records: (tile ids, keys, scales) as numpy arrays and
    (rgba, depth) tensors on the buffer's device."""
    import torch
    n = buf.shape[0]
    hdr = buf[:, :HEADER_BYTES].cpu().numpy().reshape(n, 4 * 4).view(np.float32).reshape(n, 4)
    tile_ids = hdr.view(np.int32)[:, 0].copy()
    keys = hdr[:, 1].copy()
    scales = hdr[:, 2].copy()
    esz = torch.empty((), dtype=rgba_dtype).element_size()
    rb = int(np.prod(rgba_shape)) * esz
    rgba = buf[:, HEADER_BYTES:HEADER_BYTES + rb].contiguous().view(rgba_dtype).reshape(n, *rgba_shape)
    depth = buf[:, HEADER_BYTES + rb:].contiguous().view(torch.float32).reshape(n, *depth_shape)
    return tile_ids, keys, scales, rgba, depth


def exchange(tile_ids, keys, rgba, depth, own: TileOwnership, scales=None, group=None):
    """One all-to-all of fragment tiles: every rank sends each fragment to its
    tile's owner.  Returns the fragments this rank owns, in (source rank,
    source order) order, with their global tile ids: (tile ids, keys,
    scales, rgba, depth), rgba/depth on the device of the inputs."""
    import torch
    import torch.distributed as dist
    rank, world = _rank_world(group)
    if world != own.world:
        raise ValueError("ownership is for %d ranks, the group has %d" % (own.world, world))
    if world == 1:  # every tile is this rank's: nothing moves
        sc = np.ones(len(tile_ids), np.float32) if scales is None else np.asarray(scales, np.float32)
        return (np.asarray(tile_ids, np.int32), np.asarray(keys, np.float32), sc, rgba, depth)
    order, counts = route(tile_ids, own)
    packed, rec = pack_records(tile_ids, keys, rgba, depth, scales, order)
    staged = _staged(group)
    dev = torch.device("cpu") if staged else packed.device
    send_counts = torch.as_tensor(counts, dtype=torch.int64, device=dev)
    recv_counts = torch.empty(world, dtype=torch.int64, device=dev)
    dist.all_to_all_single(recv_counts, send_counts, group=group)
    rc = recv_counts.cpu().numpy()
    src = packed.cpu() if staged else packed
    buf = torch.empty((int(rc.sum()), rec), dtype=torch.uint8, device=src.device)
    dist.all_to_all_single(buf, src, [int(v) for v in rc], [int(v) for v in counts],
                           group=group)
    buf = buf.to(rgba.device)
    return unpack_records(buf, tuple(rgba.shape[1:]), rgba.dtype, tuple(depth.shape[1:]))


def gather_tiles(local, own: TileOwnership, group=None, dst=0):
    """Assemble a frame from the tiles every rank owns.  `local` is this
    rank's framebuffer image (H_r x W_r x C or H_r x W_r; numpy array or
    tensor on any device, laid out as TileOwnership.local_grid); returns the
    H x W (x C) frame as a numpy array on `dst` (None on the other ranks).
    The tiles are reordered on the device that holds `local`."""
    import torch
    import torch.distributed as dist
    rank, world = _rank_world(group)
    T = own.T
    loc = local if torch.is_tensor(local) else torch.from_numpy(np.ascontiguousarray(local))
    flat = loc.dim() == 2
    if flat:
        loc = loc.unsqueeze(-1)
    C = loc.shape[2]
    cols, rows = own.local_grid(rank)
    mine = len(own.owned[rank])
    maxn = max(1, max(len(o) for o in own.owned))
    grid = loc[:rows * T, :cols * T].reshape(rows, T, cols, T, C).permute(0, 2, 1, 3, 4)
    tiles = torch.zeros((maxn, T, T, C), dtype=loc.dtype, device=loc.device)
    tiles[:mine] = grid.reshape(rows * cols, T, T, C)[:mine]
    if world == 1:
        parts = [tiles]
    else:
        t = tiles.reshape(-1).view(torch.uint8)
        if _staged(group):
            t = t.cpu()
        elif not t.is_cuda:  # NCCL gathers device buffers
            t = t.to(torch.device("cuda", torch.cuda.current_device()))
        parts_t = [torch.empty_like(t) for _ in range(world)] if rank == dst else None
        dist.gather(t, parts_t, dst=dst, group=group)
        if rank != dst:
            return None
        parts = [p.to(loc.device).view(loc.dtype).reshape(maxn, T, T, C) for p in parts_t]
    by_tile = torch.zeros((own.n_tiles, T, T, C), dtype=loc.dtype, device=loc.device)
    for r in range(world):
        idx = torch.as_tensor(own.owned[r], dtype=torch.long, device=loc.device)
        by_tile.index_copy_(0, idx, parts[r][:len(own.owned[r])])
    frame = by_tile.reshape(own.tiles_y, own.tiles_x, T, T, C).permute(0, 2, 1, 3, 4)
    frame = frame.reshape(own.tiles_y * T, own.tiles_x * T, C)[:own.H, :own.W]
    out = frame.contiguous().cpu().numpy()
    return out[..., 0] if flat else out


class DistributedFrameBuffer:
    """A W x H framebuffer whose tiles are owned by the ranks of `group`.
    Each rank holds a library framebuffer of its own tiles; compositing runs
    on each owner's GPU after one all-to-all of fragment tiles."""

    def __init__(self, W, H, T, mode, dtype=D.DFB_F32, flags=D.DFB_FLAGS_DEFAULT, group=None,
                 scheme="round_robin", background=(0.0, 0.0, 0.0, 0.0), kahan_after=0):
        self.rank, self.world = _rank_world(group)
        self.group = group
        self.own = TileOwnership(W, H, T, self.world, scheme)
        self.W, self.H, self.T, self.mode, self.dtype = W, H, T, mode, dtype
        lw, lh = self.own.local_size(self.rank)
        self.h = D.dfb_create_ex(lw, lh, T, mode, dtype, flags, kahan_after)
        D.dfb_set_background(self.h, *background)
        self.keep = []

    def close(self):
        if self.h is not None:
            D.dfb_destroy(self.h)
            self.h = None

    def composite(self, tile_ids, keys, rgba, depth, scales=None, accumulate=False, stream=None):
        """One frame: this rank's fragment tiles (global tile ids; rgba and
        depth device tensors of shape (n, T*T, 4) and (n, T*T)) go to their
        owners; this rank composites the fragments it owns."""
        tid, key, scl, r, d = exchange(tile_ids, keys, rgba, depth, self.own, scales, self.group)
        if self.keep and (self.keep[0] is not r or self.keep[1] is not d):
            D.dfb_sync(self.h)  # the previous frame's tiles are released below
        self.keep = [r, d]  # the library borrows the device tiles until the frame is done
        n = len(tid)
        P = self.T * self.T
        D.dfb_begin_frame(self.h, 1 if accumulate else 0)
        if n:
            rb = P * 4 * D.ELEMENT_BYTES[self.dtype]
            D.dfb_submit_tiles(self.h, self.own.local_index[tid], key, D.pool_pointers(r, n, rb),
                               D.pool_pointers(d, n, P * 4),
                               scl if self.dtype == D.DFB_FP8E4M3 else None, D.DFB_PTR_DEVICE)
        D.dfb_end_frame(self.h, stream)
        return n

    def _local(self, what):
        """This rank's framebuffer image as a device tensor (RGBA8 as int32)."""
        import torch
        lw, lh = self.own.local_size(self.rank)
        dev = torch.device("cuda", torch.cuda.current_device())
        if what == "rgba8":
            out = torch.empty((lh, lw), dtype=torch.int32, device=dev)
            D.dfb_read_rgba8(self.h, out)
        else:
            out = torch.empty((lh, lw, 4), dtype=torch.float32, device=dev)
            (D.dfb_read_color if what == "color" else D.dfb_read_accum)(self.h, out)
        # the read is queued on the frame's stream; torch works on its own
        torch.cuda.synchronize()
        return out

    def gather(self, what="rgba8", dst=0):
        """The finished frame ("rgba8" as uint32, "color" or "accum" as
        float32 RGBA) as a numpy array on rank `dst` (None elsewhere)."""
        frame = gather_tiles(self._local(what), self.own, self.group, dst)
        return frame.view(np.uint32) if (frame is not None and what == "rgba8") else frame
