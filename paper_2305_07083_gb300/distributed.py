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

The exchange runs in two steps, as the paper's producers send their tiles
asynchronously: the counts and the 16-byte headers (tile id, key, scale) go
first, over a host (gloo) group, so the owner knows what it will receive;
the RGBA and depth tiles follow as asynchronous all-to-alls while the
caller goes on producing (DistributedFrameBuffer.post); the owner's
composite is ordered after their arrival on the GPU stream
(composite_received).  The exchange and the gather use torch.distributed:
on an NCCL group the device buffers travel as they are; on a gloo group
(CPU ranks, tests) they are staged through host memory.
"""

from __future__ import annotations

import math

import numpy as np

from . import dfb as D

HEADER_BYTES = 16  # per fragment: tile id (int32), order key (f32), FP8 scale (f32), spare


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


def pack_headers(tile_ids, keys, scales, order):
    """Header records of the fragments in `order`: (tile id, order key bits,
    scale bits, 0) as an (n, 4) int32 array."""
    order = np.asarray(order, dtype=np.int64)
    n = len(order)
    hdr = np.zeros((n, 4), np.int32)
    hdr[:, 0] = np.asarray(tile_ids, np.int32)[order]
    hdr[:, 1] = np.asarray(keys, np.float32)[order].view(np.int32)
    sc = np.ones(n, np.float32) if scales is None else np.asarray(scales, np.float32)[order]
    hdr[:, 2] = sc.view(np.int32)
    return hdr


def unpack_headers(hdr):
    """Inverse of pack_headers: (tile ids, keys, scales) as numpy arrays."""
    hdr = np.ascontiguousarray(hdr, dtype=np.int32).reshape(-1, 4)
    return (hdr[:, 0].copy(), hdr[:, 1].copy().view(np.float32),
            hdr[:, 2].copy().view(np.float32))


class PendingExchange:
    """The fragments this rank owns after an exchange was started: their
    tile ids, keys and scales (host arrays, final at once) and their RGBA
    and depth tiles (device tensors, valid once wait() has returned; on an
    NCCL group wait() only orders the caller's current stream after the
    transfer, so the host does not block)."""

    def __init__(self, tile_ids, keys, scales, rgba, depth, works=(), device=None):
        self.tile_ids, self.keys, self.scales = tile_ids, keys, scales
        self.rgba, self.depth = rgba, depth
        self._works = list(works)
        self._device = device

    def wait(self, stream=None):
        """Wait for the tiles.  Work that reads them afterwards on the
        caller's current stream, or on `stream` (a torch stream or a raw
        cudaStream_t), is ordered after the transfer."""
        import torch
        moved = bool(self._works)
        for w in self._works:
            w.wait()
        self._works = []
        if self._device is not None and self.rgba.device != self._device:
            # a gloo group received into host memory
            self.rgba = self.rgba.to(self._device)
            self.depth = self.depth.to(self._device)
        if moved and stream is not None and self.rgba.is_cuda:
            s = stream if isinstance(stream, torch.cuda.Stream) else torch.cuda.ExternalStream(stream)
            cur = torch.cuda.current_stream(self.rgba.device)
            if s.cuda_stream != cur.cuda_stream:
                s.wait_stream(cur)
        return self


def exchange_async(tile_ids, keys, rgba, depth, own: TileOwnership, scales=None, group=None,
                   meta_group=None):
    """Start the all-to-all of fragment tiles: every rank sends each fragment
    to its tile's owner.  The 16-byte headers (tile id, key, scale) and the
    counts travel first, over `meta_group` (default: `group`; a gloo group
    keeps this step off the GPU streams), and are known when the call
    returns; the RGBA and depth tiles follow as two asynchronous
    all-to-alls on `group`, so the caller can go on producing the next
    frame.  The owned fragments come in (source rank, source order) order.
    With more than one rank the tiles are copied into send buffers before
    the call returns (in stream order on an NCCL group), so the sources may
    be reused; with one rank nothing moves and the PendingExchange holds
    the sources themselves.  Returns a PendingExchange."""
    import torch
    import torch.distributed as dist
    rank, world = _rank_world(group)
    if world != own.world:
        raise ValueError("ownership is for %d ranks, the group has %d" % (own.world, world))
    if world == 1:  # every tile is this rank's: nothing moves
        sc = np.ones(len(tile_ids), np.float32) if scales is None else np.asarray(scales, np.float32)
        return PendingExchange(np.asarray(tile_ids, np.int32), np.asarray(keys, np.float32), sc,
                               rgba, depth)
    meta = group if meta_group is None else meta_group
    order, counts = route(tile_ids, own)
    # headers and counts
    mdev = torch.device("cpu") if _staged(meta) else rgba.device
    send_counts = torch.as_tensor(counts, dtype=torch.int64, device=mdev)
    recv_counts = torch.empty(world, dtype=torch.int64, device=mdev)
    dist.all_to_all_single(recv_counts, send_counts, group=meta)
    rc = [int(v) for v in recv_counts.cpu().numpy()]
    sc_ = [int(v) for v in counts]
    hdr_out = torch.from_numpy(pack_headers(tile_ids, keys, scales, order)).to(mdev)
    hdr_in = torch.empty((sum(rc), 4), dtype=torch.int32, device=mdev)
    dist.all_to_all_single(hdr_in, hdr_out, rc, sc_, group=meta)
    tid, key, scl = unpack_headers(hdr_in.cpu().numpy())
    # tile payloads, in destination order, as byte rows
    n = len(order)
    idx = torch.as_tensor(np.ascontiguousarray(order), dtype=torch.long, device=rgba.device)
    r_out = rgba.index_select(0, idx).reshape(n, int(np.prod(rgba.shape[1:]))).view(torch.uint8)
    d_out = depth.index_select(0, idx).reshape(n, int(np.prod(depth.shape[1:]))).view(torch.uint8)
    staged = _staged(group)
    pdev = torch.device("cpu") if staged else rgba.device
    if staged:
        r_out, d_out = r_out.cpu(), d_out.cpu()
    r_in = torch.empty((sum(rc), r_out.shape[1]), dtype=torch.uint8, device=pdev)
    d_in = torch.empty((sum(rc), d_out.shape[1]), dtype=torch.uint8, device=pdev)
    works = [dist.all_to_all_single(r_in, r_out, rc, sc_, group=group, async_op=True),
             dist.all_to_all_single(d_in, d_out, rc, sc_, group=group, async_op=True)]
    m = sum(rc)
    r_in = r_in.view(rgba.dtype).reshape(m, *rgba.shape[1:])
    d_in = d_in.view(torch.float32).reshape(m, *depth.shape[1:])
    return PendingExchange(tid, key, scl, r_in, d_in, works, rgba.device)


def exchange(tile_ids, keys, rgba, depth, own: TileOwnership, scales=None, group=None,
             meta_group=None):
    """exchange_async, waited for: (tile ids, keys, scales, rgba, depth) of
    the fragments this rank owns, rgba/depth on the device of the inputs."""
    p = exchange_async(tile_ids, keys, rgba, depth, own, scales, group, meta_group).wait()
    return p.tile_ids, p.keys, p.scales, p.rgba, p.depth


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
    if frame.is_cuda:
        # into pinned host memory (torch caches the block across calls): the
        # read-back runs at the host link's speed, not a pageable copy's
        host = torch.empty(frame.shape, dtype=frame.dtype, pin_memory=True)
        host.copy_(frame)
        out = host.numpy()
    else:
        out = frame.contiguous().numpy()
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
        # headers and counts go over a host (gloo) group when the tiles travel
        # over NCCL, so that starting an exchange never waits on a GPU stream
        self.meta_group = group
        if self.world > 1:
            import torch.distributed as dist
            if not _staged(group):
                self.meta_group = dist.new_group(
                    ranks=dist.get_process_group_ranks(group) if group is not None else None,
                    backend="gloo")

    def close(self):
        if self.h is not None:
            D.dfb_destroy(self.h)
            self.h = None

    def post(self, tile_ids, keys, rgba, depth, scales=None):
        """Start sending this rank's fragment tiles of a frame (global tile
        ids; rgba and depth device tensors of shape (n, T*T, 4) and (n, T*T))
        to their owners; returns the PendingExchange of the fragments this
        rank owns.  The caller may produce the next frame's tiles (into other
        buffers) before passing it to composite_received."""
        return exchange_async(tile_ids, keys, rgba, depth, self.own, scales, self.group,
                              self.meta_group)

    def composite(self, tile_ids, keys, rgba, depth, scales=None, accumulate=False, stream=None):
        """One frame: post() and composite_received() in one call."""
        return self.composite_received(self.post(tile_ids, keys, rgba, depth, scales),
                                       accumulate, stream)

    def composite_received(self, pending, accumulate=False, stream=None):
        """Composite the fragments this rank owns for one frame, once their
        transfer is done (on an NCCL group the composite is ordered after it
        on the stream; the host does not wait)."""
        pending.wait(stream)
        tid, key, scl, r, d = (pending.tile_ids, pending.keys, pending.scales, pending.rgba,
                               pending.depth)
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
