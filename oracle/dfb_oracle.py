"""FP64 CPU oracle for the Distributed FrameBuffer compositing path.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain definition that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library under
``paper_2305_07083_gb300`` never does, and this module imports nothing from it.

Everything is computed in float64 with numpy (vectorised along the pixel axis
only: every pixel goes through the same sequence of steps a per-pixel loop
would take) or in plain Python.  Each function cites the passage of Usher et
al., "Scalable Ray Tracing Using the Distributed FrameBuffer" (EuroVis 2019)
that it follows.  Where the paper is silent the reading taken is written next
to the code; the list of readings is:

* Tile colour is premultiplied RGBA (Listing 1 stores ``float color[4*T*T]``
  without saying which).
* Blending is the Porter-Duff "over" operator applied front to back (Sec. 4.2
  names the depth ordering of AlphaBlend but not its blend operator).
* Ties in depth are broken by (order key, submit index); NaN depth reads as
  +inf; -0.0 reads as +0.0.
* The background (the generation-0 tile of Sec. 4.2 / Listing 3) is blended
  behind every fragment as ``rgb*a`` with coverage ``a``.
* Z-compositing (depth compositing, Sec. 2.1) outputs the RGBA of the
  nearest fragment unchanged; a pixel no fragment covers (nearest depth +inf,
  or no fragment at all) shows the premultiplied background.
* The accumulation buffer of Listing 1 holds the running sum of frames; the
  displayed value is that sum divided by the frame count.  The variance
  buffer holds the per-pixel, per-channel sample variance (ddof = 1, 0 for a
  single frame); the per-tile variance that drives adaptive sampling
  (Sec. 4.1.1) is the mean of the per-pixel RGB variances over the tile's
  in-frame pixels.
* The RGBA8 display format (Sec. 3.1) encodes RGB with the IEC 61966-2-1 sRGB
  curve and A linearly, rounding half up; a NaN channel packs to 0.
* FP16 / BF16 storage upcasts exactly; FP8 e4m3 storage decodes the code and
  multiplies by the fragment's FP32 scale.
* The image-parallel tile operation with redundantly assigned tiles
  (Sec. 4.1.1: renders of one tile made with different seeds are averaged,
  which amounts to rendering it with more samples) weighs every tile of an image
  tile equally: the per-pixel mean of the k tiles' RGBA, ignoring depth.  The
  mean then goes over the background like the other tile operations; a tile
  that received nothing shows the background.
* Pixel operations (Sec. 3.1.2) run on the finished value just before the
  display conversion; the paper leaves their formula to the user.  Two
  standard operators are provided, on premultiplied RGB with alpha
  unchanged: an exposure scale ``e * rgb`` and Reinhard's global operator
  per channel, ``e*rgb / (1 + e*rgb)``.  A third is the user's own tone
  curve per channel, given as n samples over [0, x_max] (sample j at
  x_max * j / (n - 1)) and read piecewise linearly at ``e * rgb`` clamped to
  [0, x_max], NaN read as 0.
"""

from __future__ import annotations

import math
from fractions import Fraction  # noqa: F401  (re-exported for the pins)

import numpy as np

# --- enumerations (defined here independently of the C header) -------------
BLEND_DEPTH = 0      # per-pixel depth sort, then blend (Sec. 4.2, Listing 4)
BLEND_ORDERED = 1    # blend in order-key order: the "list" tree of Sec. 4.2
ZCOMPOSITE = 2       # nearest fragment wins (Sec. 2.1, depth compositing)
AVERAGE = 3          # mean of redundantly rendered tiles (Sec. 4.1.1)

PIXELOP_NONE, PIXELOP_EXPOSURE, PIXELOP_REINHARD, PIXELOP_CURVE = 0, 1, 2, 3

F32, F16, BF16, FP8E4M3 = 0, 1, 2, 3

FP8_MAX = 448.0


# --- storage formats ---------------------------------------------------------
def fp8_e4m3_decode(codes) -> np.ndarray:
    """Decode e4m3 codes (uint8) to float64 from the bit layout.

    Layout: 1 sign bit, 4 exponent bits (bias 7), 3 mantissa bits.  Exponent
    field 0 is subnormal (m/8 * 2^-6); code S.1111.111 is NaN; there is no
    infinity.  Storage format of the precision form; not in the paper.
    """
    c = np.asarray(codes, dtype=np.uint8).astype(np.int64)
    sign = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = c & 0x7
    normal = (1.0 + m / 8.0) * np.power(2.0, e - 7.0)
    sub = (m / 8.0) * 2.0 ** -6
    v = np.where(e == 0, sub, normal) * sign
    v = np.where((e == 15) & (m == 7), np.nan, v)
    return v.astype(np.float64)


def _fp8_positive_table():
    codes = np.arange(0, 0x7F, dtype=np.uint8)          # 0x00 .. 0x7E, finite
    return codes, fp8_e4m3_decode(codes)


def fp8_e4m3_encode(x) -> np.ndarray:
    """Round float64 values to e4m3 codes: nearest, ties to even, saturating.

    Magnitudes above 448 saturate to 448, the sign bit is kept (so -0.0 and
    negatives that round to zero give 0x80) and NaN gives 0x7F.  The value
    rounded is the exact float64 given, so the decision is exact.
    """
    x = np.asarray(x, dtype=np.float64)
    codes, vals = _fp8_positive_table()
    mag = np.minimum(np.abs(np.nan_to_num(x, nan=0.0)), FP8_MAX)
    hi = np.searchsorted(vals, mag, side="left")         # first vals[hi] >= mag
    exact = vals[hi] == mag
    lo = np.maximum(hi - 1, 0)                           # vals[lo] < mag unless exact
    dlo = mag - vals[lo]
    dhi = vals[hi] - mag
    pick_hi = exact | (dhi < dlo) | ((dhi == dlo) & (codes[hi] % 2 == 0))
    out = np.where(pick_hi, codes[hi], codes[lo]).astype(np.uint8)
    out = np.where(np.signbit(x), out | np.uint8(0x80), out)
    out = np.where(np.isnan(x), np.uint8(0x7F), out)
    return out.astype(np.uint8)


def bf16_bits_to_f64(bits) -> np.ndarray:
    """BF16 is the top half of an IEEE binary32: widen the bits exactly."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)
    return b.view(np.float32).astype(np.float64)


def dequantize(stored, dtype: int, scale=None) -> np.ndarray:
    """Stored fragment RGBA -> float64 (step 1 of the per-pixel definition).

    ``stored`` has shape (n, P, 4); ``scale`` has shape (n,) for FP8.
    """
    if dtype == F32:
        return np.asarray(stored, dtype=np.float32).astype(np.float64)
    if dtype == F16:
        return np.asarray(stored, dtype=np.float16).astype(np.float64)
    if dtype == BF16:
        return bf16_bits_to_f64(stored)
    if dtype == FP8E4M3:
        v = fp8_e4m3_decode(stored)
        s = np.asarray(scale, dtype=np.float32).astype(np.float64)
        return v * s.reshape((-1,) + (1,) * (v.ndim - 1))
    raise ValueError("unknown dtype")


def fp8_tile_scale(rgba_f32) -> np.float32:
    """Per-fragment FP8 scale: amax / 448 in FP32, 1 when the tile is all zero."""
    amax = np.float32(np.max(np.abs(np.asarray(rgba_f32, dtype=np.float32))))
    if amax == 0:
        return np.float32(1.0)
    return np.float32(amax / np.float32(FP8_MAX))


def fp8_quantize_tile(rgba_f32):
    """FP32 fragment tile -> (e4m3 codes, scale).

    The quotient x / scale is formed in FP32 (one correctly rounded division)
    and then rounded to e4m3 exactly, so the code is decided in FP32.
    """
    x = np.asarray(rgba_f32, dtype=np.float32)
    s = fp8_tile_scale(x)
    q = (x / s).astype(np.float32)
    return fp8_e4m3_encode(q.astype(np.float64)), s


# --- depth and key canonicalisation ----------------------------------------
def canonical_depth(depth_f32) -> np.ndarray:
    """FP32 depth -> float64 with NaN read as +inf and -0 read as +0."""
    z = np.asarray(depth_f32, dtype=np.float32).astype(np.float64)
    z = np.where(np.isnan(z), np.inf, z)
    return z + 0.0            # -0.0 + 0.0 == +0.0


def canonical_key(key) -> float:
    k = float(np.float32(key))
    if math.isnan(k):
        raise ValueError("NaN order key")
    return k + 0.0


# --- bucketing (setTile routing + the key sort of Sec. 4.2) -----------------
def bucket(tile_ids, keys, n_tiles: int):
    """Group fragments by tile, each list sorted by (order key, submit index).

    setTile routes a tile to its owner's operation (Sec. 3.1); the rank-order
    "list" tree of Sec. 4.2 orders a tile's inputs by key.  Returns
    (lists, counts, offsets): ``lists[t]`` holds submit indices.
    """
    lists = [[] for _ in range(n_tiles)]
    for s, t in enumerate(tile_ids):
        t = int(t)
        if not 0 <= t < n_tiles:
            raise ValueError("tile id out of range")
        lists[t].append(s)
    ck = [canonical_key(k) for k in keys]
    for t in range(n_tiles):
        lists[t].sort(key=lambda s: (ck[s], s))
    counts = np.array([len(l) for l in lists], dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    return lists, counts, offsets


# --- compositing (AlphaBlend tile operation, Listing 4) ---------------------
def over_front_to_back(C, A, c, a):
    """One step of front-to-back premultiplied "over": the fragment goes behind
    what has been accumulated so far."""
    t = 1.0 - A
    return C + t[..., None] * c, A + t * a


def average_tiles(rgba):
    """Per-pixel mean of n redundantly rendered tiles, equal weights
    (Sec. 4.1.1): (n, P, 4) -> (P, 4)."""
    rgba = np.asarray(rgba, dtype=np.float64)
    return rgba.sum(axis=0) / rgba.shape[0]


def composite_tile(rgba, depth, keys, sidx, mode: int, bg=(0.0, 0.0, 0.0, 0.0)):
    """Composite one tile's fragments.

    rgba: (n, P, 4) float64 premultiplied; depth: (n, P) FP32 values;
    keys: (n,) order keys; sidx: (n,) submit indices.  Returns (P, 4).

    BLEND_DEPTH: per pixel, sort the fragments by (depth, key, submit index)
    and blend front to back (Sec. 4.2: depth order, then blending), then the
    background.  BLEND_ORDERED: blend in (key, submit index)
    order for every pixel (Sec. 4.2, tree built as a list).  ZCOMPOSITE: the
    RGBA of the per-pixel minimum of (depth, key, submit index), or the
    premultiplied background where that depth is +inf.  AVERAGE: the mean of
    the n fragments' RGBA, then the background (Sec. 4.1.1).
    """
    rgba = np.asarray(rgba, dtype=np.float64)
    n = rgba.shape[0]
    P = rgba.shape[1] if n else np.asarray(depth).shape[-1]
    bg = np.asarray(bg, dtype=np.float64)
    bg_c = bg[:3] * bg[3]
    out = np.zeros((P, 4), dtype=np.float64)
    if n == 0:
        out[:, :3] = bg_c
        out[:, 3] = bg[3]
        return out
    if mode == AVERAGE:
        mean = average_tiles(rgba)
        C, A = over_front_to_back(mean[:, :3], mean[:, 3], np.broadcast_to(bg_c, (P, 3)),
                                  np.full(P, bg[3]))
        out[:, :3] = C
        out[:, 3] = A
        return out
    keys = np.array([canonical_key(k) for k in keys], dtype=np.float64)
    sidx = np.asarray(sidx, dtype=np.int64)
    K = np.broadcast_to(keys[:, None], (n, P))
    S = np.broadcast_to(sidx[:, None], (n, P))
    pix = np.arange(P)
    if mode == BLEND_ORDERED:
        order = np.broadcast_to(np.lexsort((sidx, keys))[:, None], (n, P))
    else:
        z = canonical_depth(depth)
        # np.lexsort: last key is primary -> ascending (z, key, submit index)
        order = np.lexsort((S, K, z), axis=0)
    if mode == ZCOMPOSITE:
        win = order[0]
        res = rgba[win, pix].copy()
        empty = np.isinf(z[win, pix])
        res[empty, :3] = bg_c
        res[empty, 3] = bg[3]
        return res
    C = np.zeros((P, 3), dtype=np.float64)
    A = np.zeros(P, dtype=np.float64)
    for j in range(n):
        f = rgba[order[j], pix]
        C, A = over_front_to_back(C, A, f[:, :3], f[:, 3])
    C, A = over_front_to_back(C, A, np.broadcast_to(bg_c, (P, 3)), np.full(P, bg[3]))
    out[:, :3] = C
    out[:, 3] = A
    return out


def tile_origin(tile_id: int, W: int, T: int):
    tiles_x = -(-W // T)
    return (tile_id % tiles_x) * T, (tile_id // tiles_x) * T


def composite_frame(W, H, T, mode, tile_ids, keys, rgba64, depth, bg=(0, 0, 0, 0),
                    tiles=None):
    """Composite a whole frame: (H, W, 4) float64.

    Each tile is owned by one operation (Sec. 3) and composited from its own
    fragments only; pixels of a submitted tile that fall outside the frame
    are ignored.  ``tiles`` restricts the work to a subset of tile ids (the
    other pixels are left NaN).
    """
    tiles_x, tiles_y = -(-W // T), -(-H // T)
    n_tiles = tiles_x * tiles_y
    lists, _, _ = bucket(tile_ids, keys, n_tiles)
    img = np.full((H, W, 4), np.nan if tiles is not None else 0.0)
    todo = range(n_tiles) if tiles is None else tiles
    for t in todo:
        idx = np.array(lists[t], dtype=np.int64)
        if len(idx):
            res = composite_tile(rgba64[idx], depth[idx], np.asarray(keys)[idx], idx, mode, bg)
        else:
            res = composite_tile(np.zeros((0, T * T, 4)), np.zeros((0, T * T)), [], [], mode, bg)
        x0, y0 = tile_origin(t, W, T)
        res = res.reshape(T, T, 4)
        h, w = min(T, H - y0), min(T, W - x0)
        img[y0:y0 + h, x0:x0 + w] = res[:h, :w]
    return img


# --- progressive refinement (Listing 1: accumulation / variance tiles) -------
def accumulate(frames):
    """Running sum over frames f = 1..n divided by n (float64, frame order)."""
    frames = [np.asarray(f, dtype=np.float64) for f in frames]
    S = np.zeros_like(frames[0])
    for f in frames:
        S = S + f
    return S / len(frames)


def variance(frames):
    """Per-pixel, per-channel sample variance (ddof = 1); 0 for one frame."""
    frames = [np.asarray(f, dtype=np.float64) for f in frames]
    n = len(frames)
    if n < 2:
        return np.zeros_like(frames[0])
    mean = accumulate(frames)
    acc = np.zeros_like(mean)
    for f in frames:
        d = f - mean
        acc = acc + d * d
    return acc / (n - 1)


def tile_variance(var_img, T):
    """Per-tile error estimate: mean of the RGB variances over in-frame pixels."""
    H, W = var_img.shape[:2]
    tiles_x, tiles_y = -(-W // T), -(-H // T)
    out = np.zeros(tiles_x * tiles_y, dtype=np.float64)
    for ty in range(tiles_y):
        for tx in range(tiles_x):
            blk = var_img[ty * T:(ty + 1) * T, tx * T:(tx + 1) * T, :3]
            out[ty * tiles_x + tx] = blk.mean()
    return out


# --- display conversion (Sec. 3.1, RGBA8 format) -----------------------------
def srgb_encode(x):
    """IEC 61966-2-1 sRGB transfer function on [0, 1]."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(x <= 0.0031308, 12.92 * x, 1.055 * np.power(np.maximum(x, 0.0), 1.0 / 2.4) - 0.055)


def pack_rgba8(img):
    """(..., 4) float -> (...,) uint32 with bytes R, G, B, A in memory order."""
    img = np.nan_to_num(np.asarray(img, dtype=np.float64), nan=0.0)
    v = np.clip(img, 0.0, 1.0)
    rgb = np.floor(255.0 * srgb_encode(v[..., :3]) + 0.5)
    a = np.floor(255.0 * v[..., 3] + 0.5)
    b = np.concatenate([rgb, a[..., None]], axis=-1).astype(np.uint32)
    return b[..., 0] | (b[..., 1] << 8) | (b[..., 2] << 16) | (b[..., 3] << 24)


def tone_curve(x, samples, x_max: float):
    """A user tone curve (Sec. 3.1.2 leaves the operation to the user): the
    polyline through (x_max * j / (n - 1), samples[j]), j = 0 .. n-1, at x
    clamped to [0, x_max]; NaN reads as 0."""
    t = np.asarray(samples, dtype=np.float64)
    n = t.shape[0]
    x = np.asarray(x, dtype=np.float64)
    x = np.where(np.isnan(x), 0.0, x)
    x = np.minimum(np.maximum(x, 0.0), x_max)
    f = x * ((n - 1) / x_max)               # position in sample steps
    j = np.minimum(np.floor(f).astype(np.int64), n - 2)
    return t[j] + (f - j) * (t[j + 1] - t[j])


def pixel_op(img, op: int, exposure: float = 1.0, curves=None, x_max: float = 1.0):
    """A pixel operation on finished pixels (Sec. 3.1.2), before the display
    conversion: RGB transformed, alpha unchanged.  ``curves`` (3 x n
    samples, one row per channel) and ``x_max`` define PIXELOP_CURVE."""
    img = np.array(img, dtype=np.float64)
    if op == PIXELOP_NONE:
        return img
    x = exposure * img[..., :3]
    if op == PIXELOP_EXPOSURE:
        img[..., :3] = x
    elif op == PIXELOP_REINHARD:
        img[..., :3] = x / (1.0 + x)
    elif op == PIXELOP_CURVE:
        for c in range(3):
            img[..., c] = tone_curve(x[..., c], curves[c], x_max)
    else:
        raise ValueError("unknown pixel operation")
    return img


def unpack_rgba8(u32):
    u = np.asarray(u32, dtype=np.uint32)
    return np.stack([(u >> s) & 0xFF for s in (0, 8, 16, 24)], axis=-1).astype(np.int64)
