"""Seeded synthetic brick-decomposed scenes: the inputs of the compositing path.

This module only *produces* fragment tiles.  It contains none of the
compositing arithmetic (no blending, sorting of fragments, accumulation or
packing), so that both the FP64 oracle and the CUDA library can take their
inputs from it without sharing any of the method's code.

The scenes follow the data-parallel setting of Sec. 4.2 of the paper: the
volume is split into a grid of disjoint bricks, one producer ("rank") per
brick; each producer finds the tiles its brick projects to (a conservative
screen-space rectangle refined by ray casting the box, as Listing 3 does) and
emits one fragment tile per touched tile.  A fragment tile holds premultiplied
RGBA and a per-pixel depth inside the brick's ray interval; pixels whose ray
misses the brick are empty (RGBA 0, depth +inf).  The order key of a fragment
is the distance from the eye to its brick's centre.

Fragment tiles are stored row-major within the tile (pixel p = y*T + x) and
the frame's tiles are numbered row-major (tile = ty * tilesX + tx).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Camera:
    kind: str                      # "ortho" or "persp"
    W: int
    H: int
    eye: np.ndarray = None
    forward: np.ndarray = None
    right: np.ndarray = None
    up: np.ndarray = None
    vfov_deg: float = 60.0
    ortho_lo: tuple = (0.0, 0.0)   # world (x, y) at pixel (0, 0) corner
    ortho_hi: tuple = (1.0, 1.0)
    ortho_z: float = 2.0           # eye plane, looking down -z

    def rays(self, px, py):
        """Ray origins/directions through pixel centres (px, py integer arrays)."""
        px = np.asarray(px, dtype=np.float64) + 0.5
        py = np.asarray(py, dtype=np.float64) + 0.5
        if self.kind == "ortho":
            x = self.ortho_lo[0] + (self.ortho_hi[0] - self.ortho_lo[0]) * px / self.W
            y = self.ortho_lo[1] + (self.ortho_hi[1] - self.ortho_lo[1]) * py / self.H
            o = np.stack([x, y, np.full_like(x, self.ortho_z)], axis=-1)
            d = np.broadcast_to(np.array([0.0, 0.0, -1.0]), o.shape)
            return o, d
        th = np.tan(np.radians(self.vfov_deg) / 2)
        aspect = self.W / self.H
        u = (2.0 * px / self.W - 1.0) * th * aspect
        v = (1.0 - 2.0 * py / self.H) * th
        d = self.forward[None] + u[..., None] * self.right[None] + v[..., None] * self.up[None]
        d = d / np.linalg.norm(d, axis=-1, keepdims=True)
        o = np.broadcast_to(self.eye, d.shape)
        return o, d

    def project(self, pts):
        """World points -> pixel coordinates (x, y); perspective assumes in front."""
        pts = np.asarray(pts, dtype=np.float64)
        if self.kind == "ortho":
            x = (pts[:, 0] - self.ortho_lo[0]) / (self.ortho_hi[0] - self.ortho_lo[0]) * self.W
            y = (pts[:, 1] - self.ortho_lo[1]) / (self.ortho_hi[1] - self.ortho_lo[1]) * self.H
            return x, y, np.ones(len(pts), dtype=bool)
        rel = pts - self.eye
        zc = rel @ self.forward
        th = np.tan(np.radians(self.vfov_deg) / 2)
        aspect = self.W / self.H
        u = (rel @ self.right) / np.maximum(zc, 1e-9) / (th * aspect)
        v = (rel @ self.up) / np.maximum(zc, 1e-9) / th
        x = (u + 1.0) * 0.5 * self.W
        y = (1.0 - v) * 0.5 * self.H
        return x, y, zc > 1e-6


def look_at(eye, target, W, H, vfov_deg=60.0, world_up=(0.0, 1.0, 0.0)):
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(world_up, dtype=np.float64))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    return Camera("persp", W, H, eye=eye, forward=f, right=r, up=u, vfov_deg=vfov_deg)


@dataclass
class Scene:
    """A set of fragment tiles for one frame (plus what is needed for more frames).

    ``tile_ids``/``keys`` are in submission order; submission index = position.
    ``rgba`` is premultiplied FP32 for frame 0 (shape (n, T*T, 4)); ``depth``
    is FP32 (n, T*T).  ``base_rgb``/``alpha`` hold the unpremultiplied colour
    and coverage so later frames can be drawn with colour jitter.
    """
    W: int
    H: int
    T: int
    tile_ids: np.ndarray
    keys: np.ndarray
    rgba: np.ndarray
    depth: np.ndarray
    base_rgb: np.ndarray = None
    alpha: np.ndarray = None
    hit: np.ndarray = None
    seed: int = 0
    jitter_sigma: float = 0.0
    info: dict = field(default_factory=dict)

    @property
    def n(self):
        return len(self.tile_ids)

    @property
    def tiles_x(self):
        return -(-self.W // self.T)

    @property
    def tiles_y(self):
        return -(-self.H // self.T)

    @property
    def n_tiles(self):
        return self.tiles_x * self.tiles_y

    def in_frame_pixels(self):
        """Per fragment: how many of its tile's pixels lie inside the frame."""
        tx = self.tile_ids % self.tiles_x
        ty = self.tile_ids // self.tiles_x
        w = np.minimum(self.T, self.W - tx * self.T)
        h = np.minimum(self.T, self.H - ty * self.T)
        return (w * h).astype(np.int64)

    def fragment_pixels(self) -> int:
        return int(self.in_frame_pixels().sum())

    def counts(self):
        return np.bincount(self.tile_ids, minlength=self.n_tiles)

    def frame_rgba(self, f: int) -> np.ndarray:
        """Premultiplied FP32 RGBA of frame f (frame 0 is ``rgba``)."""
        if f == 0 or self.jitter_sigma == 0.0:
            return self.rgba
        rng = np.random.default_rng([self.seed, 1000 + f])
        j = rng.standard_normal(self.base_rgb.shape, dtype=np.float32) * np.float32(self.jitter_sigma)
        return _premultiply(np.clip(self.base_rgb + j, 0.0, 1.0), self.alpha, self.hit)


def _premultiply(rgb, alpha, hit):
    out = np.empty(rgb.shape[:-1] + (4,), dtype=np.float32)
    a = np.where(hit, alpha, 0.0).astype(np.float32)
    out[..., :3] = rgb * a[..., None]
    out[..., 3] = a
    return out


def brick_grid(grid, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    gx, gy, gz = grid
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    size = (hi - lo) / np.array(grid)
    boxes = []
    for k in range(gz):
        for j in range(gy):
            for i in range(gx):
                bmin = lo + size * np.array([i, j, k])
                boxes.append((bmin, bmin + size))
    return boxes


def _ray_box(o, d, bmin, bmax):
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t0 = (bmin - o) * inv
        t1 = (bmax - o) * inv
    t0 = np.nan_to_num(t0, nan=-np.inf)
    t1 = np.nan_to_num(t1, nan=np.inf)
    tmin = np.max(np.minimum(t0, t1), axis=-1)
    tmax = np.min(np.maximum(t0, t1), axis=-1)
    tin = np.maximum(tmin, 0.0)
    return tin, tmax, tmax > tin


def brick_scene(W, H, T, boxes, cam: Camera, seed=0, alpha="uniform", alpha_max=0.6,
                jitter_sigma=0.0, max_per_tile=None, shuffle=True):
    """Render every brick's fragment tiles (the producers of Sec. 4.2)."""
    rng = np.random.default_rng(seed)
    tiles_x, tiles_y = -(-W // T), -(-H // T)
    tid_l, key_l, rgb_l, a_l, z_l, hit_l = [], [], [], [], [], []
    ly, lx = np.meshgrid(np.arange(T), np.arange(T), indexing="ij")
    lx = lx.reshape(-1)
    ly = ly.reshape(-1)
    for bmin, bmax in boxes:
        corners = np.array([[x, y, z] for x in (bmin[0], bmax[0])
                            for y in (bmin[1], bmax[1]) for z in (bmin[2], bmax[2])])
        sx, sy, ok = cam.project(corners)
        if not ok.all():
            continue
        x0 = int(np.floor(max(sx.min(), 0)) // T)
        x1 = int(min(np.ceil(sx.max()), W) - 1) // T
        y0 = int(np.floor(max(sy.min(), 0)) // T)
        y1 = int(min(np.ceil(sy.max()), H) - 1) // T
        if x1 < x0 or y1 < y0 or sx.max() <= 0 or sy.max() <= 0:
            continue
        centre = 0.5 * (bmin + bmax)
        if cam.kind == "ortho":
            key = float(cam.ortho_z - centre[2])
        else:
            key = float(np.linalg.norm(centre - cam.eye))
        for ty in range(y0, y1 + 1):
            for tx in range(x0, x1 + 1):
                px = tx * T + lx
                py = ty * T + ly
                o, d = cam.rays(px, py)
                tin, tout, hit = _ray_box(o, d, bmin, bmax)
                hit &= (px < W) & (py < H)
                if not hit.any():
                    continue       # refined by ray casting the box (Listing 3)
                tid_l.append(ty * tiles_x + tx)
                key_l.append(key)
                u = rng.random(len(px))
                z = np.where(hit, tin + u * (tout - tin), np.inf).astype(np.float32)
                if alpha == "beta":
                    a = rng.beta(2.0, 5.0, len(px)).astype(np.float32)
                else:
                    a = (rng.random(len(px)) * alpha_max).astype(np.float32)
                rgb = rng.random((len(px), 3)).astype(np.float32)
                rgb_l.append(rgb)
                a_l.append(a)
                z_l.append(z)
                hit_l.append(hit)
    n = len(tid_l)
    tile_ids = np.array(tid_l, dtype=np.int32)
    keys = np.array(key_l, dtype=np.float32)
    base_rgb = np.stack(rgb_l) if n else np.zeros((0, T * T, 3), np.float32)
    alpha_a = np.stack(a_l) if n else np.zeros((0, T * T), np.float32)
    depth = np.stack(z_l) if n else np.zeros((0, T * T), np.float32)
    hit = np.stack(hit_l) if n else np.zeros((0, T * T), bool)
    if max_per_tile is not None and n:
        keep = np.ones(n, dtype=bool)
        seen = {}
        for i, t in enumerate(tile_ids):
            seen[t] = seen.get(t, 0) + 1
            keep[i] = seen[t] <= max_per_tile
        tile_ids, keys = tile_ids[keep], keys[keep]
        base_rgb, alpha_a, depth, hit = base_rgb[keep], alpha_a[keep], depth[keep], hit[keep]
        n = len(tile_ids)
    if shuffle and n:
        perm = rng.permutation(n)           # arrival order is arbitrary (Sec. 3.1.1)
        tile_ids, keys = tile_ids[perm], keys[perm]
        base_rgb, alpha_a, depth, hit = base_rgb[perm], alpha_a[perm], depth[perm], hit[perm]
    rgb0 = base_rgb
    if jitter_sigma:
        j = np.random.default_rng([seed, 1000]).standard_normal(base_rgb.shape, dtype=np.float32)
        rgb0 = np.clip(base_rgb + j * np.float32(jitter_sigma), 0.0, 1.0)
    rgba = _premultiply(rgb0, alpha_a, hit)
    sc = Scene(W, H, T, tile_ids, keys, rgba, depth, base_rgb=base_rgb, alpha=alpha_a, hit=hit,
               seed=seed, jitter_sigma=jitter_sigma)
    c = sc.counts()
    sc.info = {"fragments": n, "fragment_pixels": sc.fragment_pixels(),
               "min_per_tile": int(c.min()) if len(c) else 0,
               "max_per_tile": int(c.max()) if len(c) else 0,
               "mean_per_tile": float(c.mean()) if len(c) else 0.0}
    return sc


# --- the workloads ------------------------------------------------------------
def scene_single_frame_256(seed=0):
    """256x256 frame, 64x64 tiles, 2x2x2 bricks of the unit cube, orthographic
    camera looking down -z, alpha U(0, 0.6), zero background."""
    cam = Camera("ortho", 256, 256)
    return brick_scene(256, 256, 64, brick_grid((2, 2, 2)), cam, seed=seed,
                       alpha="uniform", alpha_max=0.6)


def orbit_camera(W, H, seed, radius=1.0, lo=(0, 0, 0), hi=(1, 1, 1), vfov=60.0):
    rng = np.random.default_rng([seed, 7])
    th = rng.uniform(0.0, 2.0 * np.pi)
    el = rng.uniform(-0.35, 0.35)
    c = 0.5 * (np.asarray(lo, float) + np.asarray(hi, float))
    eye = c + radius * np.array([np.cos(th) * np.cos(el), np.sin(el), np.sin(th) * np.cos(el)])
    return look_at(eye, c, W, H, vfov)


def scene_data_parallel(W=2048, H=2048, T=64, grid=(4, 4, 4), seed=0, radius=1.0,
                        jitter_sigma=0.02, extent=(1.0, 1.0, 1.0), max_per_tile=None):
    """Perspective (60 deg) brick-grid frame with Beta(2,5) alpha and per-frame
    colour jitter; the data-parallel frame of Sec. 4.2."""
    hi = tuple(float(e) for e in extent)
    cam = orbit_camera(W, H, seed, radius=radius, hi=hi)
    return brick_scene(W, H, T, brick_grid(grid, hi=hi), cam, seed=seed, alpha="beta",
                       jitter_sigma=jitter_sigma, max_per_tile=max_per_tile)


def scene_2048(seed=0, jitter_sigma=0.02):
    """2048x2048, 64x64 tiles, 4x4x4 bricks: the headline data-parallel frame."""
    return scene_data_parallel(2048, 2048, 64, (4, 4, 4), seed=seed, jitter_sigma=jitter_sigma)


def scene_4096x1024(seed=0):
    """4096x1024, 64x64 tiles, 8x4x4 bricks of a 2x1x1 box (precision form)."""
    return scene_data_parallel(4096, 1024, 64, (8, 4, 4), seed=seed, jitter_sigma=0.0,
                               extent=(2.0, 1.0, 1.0), radius=1.2)


def random_scene(W, H, T, counts, seed=0, depth_levels=None, special_depths=False,
                 alpha_max=1.0, equal_keys=False):
    """Fragments with arbitrary (not brick-ordered) depths and keys.

    ``counts`` gives the number of fragments of every tile (len = tiles).
    ``depth_levels`` draws depths from a few integer levels (many ties);
    ``special_depths`` sprinkles NaN, -0.0, +0.0 and +inf depths.
    """
    rng = np.random.default_rng(seed)
    tiles_x, tiles_y = -(-W // T), -(-H // T)
    counts = np.asarray(counts, dtype=np.int64)
    assert len(counts) == tiles_x * tiles_y
    tile_ids = np.repeat(np.arange(len(counts), dtype=np.int32), counts)
    rng.shuffle(tile_ids)
    n, P = len(tile_ids), T * T
    if equal_keys:
        keys = rng.integers(0, 3, n).astype(np.float32)
    else:
        keys = rng.uniform(0.0, 10.0, n).astype(np.float32)
    a = (rng.random((n, P)) * alpha_max).astype(np.float32)
    rgba = np.empty((n, P, 4), np.float32)
    rgba[..., :3] = rng.random((n, P, 3)).astype(np.float32) * a[..., None]
    rgba[..., 3] = a
    if depth_levels:
        depth = rng.integers(0, depth_levels, (n, P)).astype(np.float32)
    else:
        depth = rng.uniform(0.0, 10.0, (n, P)).astype(np.float32)
    if special_depths and n:
        u = rng.random((n, P))
        depth[u < 0.05] = np.nan
        depth[(u >= 0.05) & (u < 0.10)] = -0.0
        depth[(u >= 0.10) & (u < 0.15)] = 0.0
        depth[(u >= 0.15) & (u < 0.20)] = np.inf
    sc = Scene(W, H, T, tile_ids, keys, rgba, depth, seed=seed)
    sc.info = {"fragments": n}
    return sc


def store_rgba(rgba_f32, dtype):
    """Storage form of FP32 fragment tiles, made with library casts.

    dtype 0 FP32 (copy), 1 FP16 (numpy, round to nearest even), 2 BF16 (torch
    CPU cast, bits as uint16), 3 FP8 e4m3 (one FP32 scale per tile =
    amax/448, 1 for an all-zero tile; torch CPU cast of x/scale clamped to
    +-448).  Returns (stored, scales or None).
    """
    x = np.ascontiguousarray(rgba_f32, dtype=np.float32)
    if dtype == 0:
        return x.copy(), None
    if dtype == 1:
        return x.astype(np.float16), None
    import torch
    t = torch.from_numpy(x)
    if dtype == 2:
        return t.to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16), None
    n = x.shape[0]
    amax = np.abs(x.reshape(n, -1)).max(axis=1) if n else np.zeros(0, np.float32)
    scales = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    q = (x / scales.reshape((-1,) + (1,) * (x.ndim - 1))).astype(np.float32)
    q = np.clip(q, -448.0, 448.0)
    codes = torch.from_numpy(q).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    return codes, scales


# --- large workloads generated on the GPU -------------------------------------
def _beta25_torch(torch, shape, gen, device):
    """Beta(2, 5) as X / (X + Y) with X ~ Gamma(2), Y ~ Gamma(5), each Gamma(k)
    drawn as the negative log of a product of k uniforms."""
    u = torch.rand((7,) + tuple(shape), generator=gen, device=device).clamp_min_(1e-12)
    x = -torch.log(u[0] * u[1])
    y = -torch.log(u[2] * u[3] * u[4] * u[5] * u[6])
    return x / (x + y)


def brick_scene_torch(W, H, T, boxes, cam: Camera, seed, device):
    """The recipe of brick_scene (projected brick rectangles refined by ray
    casting the box, per-pixel depth uniform in the ray interval, alpha
    Beta(2,5), colour U(0,1) premultiplied) with the random draws made by a
    seeded torch generator on `device`.  Returns (tile_ids, keys) as numpy
    arrays in a seeded arrival order and (rgba, depth) as device tensors."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 7919 + 17)
    tiles_x = -(-W // T)
    ly, lx = torch.meshgrid(torch.arange(T, device=device), torch.arange(T, device=device),
                            indexing="ij")
    lx = lx.reshape(-1).double()
    ly = ly.reshape(-1).double()
    tid_l, key_l, rgba_l, z_l = [], [], [], []
    for bmin, bmax in boxes:
        corners = np.array([[x, y, z] for x in (bmin[0], bmax[0])
                            for y in (bmin[1], bmax[1]) for z in (bmin[2], bmax[2])])
        sx, sy, ok = cam.project(corners)
        if not ok.all():
            continue
        x0 = int(np.floor(max(sx.min(), 0)) // T)
        x1 = int(min(np.ceil(sx.max()), W) - 1) // T
        y0 = int(np.floor(max(sy.min(), 0)) // T)
        y1 = int(min(np.ceil(sy.max()), H) - 1) // T
        if x1 < x0 or y1 < y0 or sx.max() <= 0 or sy.max() <= 0:
            continue
        tys, txs = np.meshgrid(np.arange(y0, y1 + 1), np.arange(x0, x1 + 1), indexing="ij")
        tys = torch.as_tensor(tys.reshape(-1), device=device)
        txs = torch.as_tensor(txs.reshape(-1), device=device)
        px = txs[:, None].double() * T + lx[None, :]
        py = tys[:, None].double() * T + ly[None, :]
        pxc, pyc = px + 0.5, py + 0.5
        th = np.tan(np.radians(cam.vfov_deg) / 2)
        u = (2.0 * pxc / W - 1.0) * th * (W / H)
        v = (1.0 - 2.0 * pyc / H) * th
        f = torch.as_tensor(cam.forward, device=device)
        r = torch.as_tensor(cam.right, device=device)
        up = torch.as_tensor(cam.up, device=device)
        d = f + u[..., None] * r + v[..., None] * up
        d = d / torch.linalg.norm(d, dim=-1, keepdim=True)
        o = torch.as_tensor(cam.eye, device=device)
        lo = torch.as_tensor(bmin, device=device)
        hi = torch.as_tensor(bmax, device=device)
        with torch.no_grad():
            inv = 1.0 / d
            t0 = (lo - o) * inv
            t1 = (hi - o) * inv
            t0 = torch.nan_to_num(t0, nan=-np.inf)
            t1 = torch.nan_to_num(t1, nan=np.inf)
            tmin = torch.minimum(t0, t1).amax(dim=-1).clamp_min(0.0)
            tmax = torch.maximum(t0, t1).amin(dim=-1)
        hit = (tmax > tmin) & (px < W) & (py < H)
        keep = hit.any(dim=1)
        if not bool(keep.any()):
            continue
        hit, tmin, tmax = hit[keep], tmin[keep], tmax[keep]
        n = int(hit.shape[0])
        tid_l.append((tys[keep] * tiles_x + txs[keep]).cpu().numpy())
        centre = 0.5 * (np.asarray(bmin) + np.asarray(bmax))
        key_l.append(np.full(n, np.linalg.norm(centre - cam.eye), np.float32))
        uu = torch.rand((n, T * T), generator=gen, device=device, dtype=torch.float64)
        z = torch.where(hit, tmin + uu * (tmax - tmin), torch.full_like(uu, float("inf")))
        a = _beta25_torch(torch, (n, T * T), gen, device).float() * hit
        rgb = torch.rand((n, T * T, 3), generator=gen, device=device) * a[..., None]
        rgba_l.append(torch.cat([rgb, a[..., None]], dim=-1))
        z_l.append(z.float())
    tile_ids = np.concatenate(tid_l).astype(np.int32) if tid_l else np.zeros(0, np.int32)
    keys = np.concatenate(key_l).astype(np.float32) if key_l else np.zeros(0, np.float32)
    rgba = torch.cat(rgba_l) if rgba_l else torch.zeros((0, T * T, 4), device=device)
    depth = torch.cat(z_l) if z_l else torch.zeros((0, T * T), device=device)
    perm = np.random.default_rng(seed).permutation(len(tile_ids))
    pt = torch.as_tensor(perm, device=device)
    return tile_ids[perm], keys[perm], rgba[pt].contiguous(), depth[pt].contiguous()


BATCH_SIZES = [(512, 512), (1024, 1024), (2048, 2048), (4096, 1024)]


def batch_frames_torch(n_frames=32, seed=0, device="cuda", T=64):
    """Mixed batch: frame i has the size BATCH_SIZES[i % 4], a brick grid of
    g x g x g (g drawn from 2..8, so 8 to 512 bricks) over a 1 x 1 x 1 cube
    (2 x 1 x 1 for the 4096x1024 frames) and a seeded orbit camera whose
    radius leaves the cube covering the frame."""
    rng = np.random.default_rng([seed, 4])
    out = []
    for i in range(n_frames):
        W, H = BATCH_SIZES[i % len(BATCH_SIZES)]
        g = int(rng.integers(2, 9))
        wide = W > H
        extent = (2.0, 1.0, 1.0) if wide else (1.0, 1.0, 1.0)
        grid = (2 * g, g, g) if wide and g <= 4 else (g, g, g)
        hi = tuple(float(e) for e in extent)
        cam = orbit_camera(W, H, seed * 1000 + i, radius=1.2 if wide else 1.0, hi=hi)
        tid, key, rgba, depth = brick_scene_torch(W, H, T, brick_grid(grid, hi=hi), cam,
                                                  seed * 1000 + i, device)
        out.append({"W": W, "H": H, "T": T, "bricks": int(np.prod(grid)), "tile_ids": tid,
                    "keys": key, "rgba": rgba, "depth": depth})
    return out


# --- serving workload ---------------------------------------------------------
def serving_templates(device, seed=0, T=64, convert=None):
    """Job templates resident on the device.

    blend: data-parallel brick frames of 1024x1024, 2048x2048 and 4096x1024
    with g x g x g bricks, g in 4..10 (64 to 1000 bricks);
    accumulate: image-parallel frames of 1024x1024 and 2048x1024 with exactly
    one opaque fragment tile per image tile, 8 distinct passes each (the
    64-pass jobs cycle through them).
    ``convert(rgba_f32, n, P)`` turns FP32 tiles into the storage dtype.
    Returns {"blend": [(W, H, bricks, frame_dict)], "accumulate": [(W, H, [frame_dict])]}.
    """
    import torch
    out = {"blend": [], "accumulate": []}
    specs = [(1024, 1024, 4), (2048, 2048, 6), (4096, 1024, 8), (1024, 1024, 10),
             (2048, 2048, 10), (4096, 1024, 5)]
    for i, (W, H, g) in enumerate(specs):
        wide = W > H
        hi = (2.0, 1.0, 1.0) if wide else (1.0, 1.0, 1.0)
        grid = (g, g, g)
        cam = orbit_camera(W, H, 7000 + seed * 100 + i, radius=1.2 if wide else 1.0, hi=hi)
        tid, key, rgba, depth = brick_scene_torch(W, H, T, brick_grid(grid, hi=hi), cam,
                                                  7000 + seed * 100 + i, device)
        n = len(tid)
        stored = convert(rgba, n, T * T) if convert else rgba
        out["blend"].append((W, H, g ** 3, {"tile_ids": tid, "keys": key, "rgba": stored,
                                              "depth": depth, "fragment_pixels": n * T * T}))
        del rgba
    gen = torch.Generator(device=device)
    for j, (W, H) in enumerate([(1024, 1024), (2048, 1024)]):
        nt = (W // T) * (H // T)
        passes = []
        for f in range(8):
            gen.manual_seed(seed * 991 + j * 31 + f)
            rgb = torch.rand((nt, T * T, 3), generator=gen, device=device)
            rgba = torch.cat([rgb, torch.ones((nt, T * T, 1), device=device)], dim=-1)
            depth = torch.ones((nt, T * T), device=device)
            stored = convert(rgba, nt, T * T) if convert else rgba
            passes.append({"tile_ids": np.arange(nt, dtype=np.int32),
                           "keys": np.zeros(nt, np.float32), "rgba": stored, "depth": depth,
                           "fragment_pixels": nt * T * T})
            del rgba, rgb
        out["accumulate"].append((W, H, passes))
    return out
