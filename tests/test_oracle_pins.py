"""Pins for the FP64 oracle: closed forms, exact rationals, brute force and
library routines, each independent of the oracle's own code."""

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import dfb_oracle as o
from harness import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frags(rgba, depth, keys=None):
    rgba = np.asarray(rgba, dtype=np.float64)
    n = rgba.shape[0]
    keys = np.arange(n, dtype=np.float32) if keys is None else np.asarray(keys, np.float32)
    return rgba, np.asarray(depth, dtype=np.float32), keys, np.arange(n)


# --- the over operator ------------------------------------------------------
@pytest.mark.parametrize("a", [0.05, 0.3, 0.5, 0.9])
@pytest.mark.parametrize("n", [1, 2, 5, 16, 40])
def test_equal_layers_closed_form(a, n):
    """n layers of coverage a: A = 1-(1-a)^n and C = c(1-(1-a)^n)."""
    c = np.array([0.2, 0.7, 1.0])
    P = 3
    rgba = np.zeros((n, P, 4))
    rgba[..., :3] = c * a
    rgba[..., 3] = a
    depth = np.tile(np.arange(n, dtype=np.float32)[:, None], (1, P))[::-1]
    for mode in (o.BLEND_DEPTH, o.BLEND_ORDERED):
        out = o.composite_tile(*_frags(rgba, depth), mode)
        cover = 1.0 - (1.0 - a) ** n
        np.testing.assert_allclose(out[:, 3], cover, rtol=0, atol=1e-13)
        np.testing.assert_allclose(out[:, :3], np.tile(c * cover, (P, 1)), rtol=0, atol=1e-13)


def test_opaque_front_hides_everything():
    rng = np.random.default_rng(1)
    n, P = 7, 50
    a = rng.uniform(0, 1, (n, P))
    rgba = np.concatenate([rng.uniform(0, 1, (n, P, 3)) * a[..., None], a[..., None]], -1)
    depth = rng.uniform(1, 2, (n, P)).astype(np.float32)
    front = rng.integers(0, n, P)
    rgba[front, np.arange(P), 3] = 1.0
    depth[front, np.arange(P)] = 0.5
    out = o.composite_tile(*_frags(rgba, depth), o.BLEND_DEPTH, bg=(0.3, 0.3, 0.3, 1.0))
    np.testing.assert_array_equal(out, rgba[front, np.arange(P)])


def test_single_fragment_is_identity():
    rng = np.random.default_rng(2)
    a = rng.uniform(0, 1, (1, 64))
    rgba = np.concatenate([rng.uniform(0, 1, (1, 64, 3)) * a[..., None], a[..., None]], -1)
    depth = rng.uniform(0, 1, (1, 64)).astype(np.float32)
    for mode in (o.BLEND_DEPTH, o.BLEND_ORDERED, o.ZCOMPOSITE):
        np.testing.assert_array_equal(o.composite_tile(*_frags(rgba, depth), mode), rgba[0])


def _exact_tree_over(frs):
    """Binary-swap style grouping of "over" on exact rationals."""
    layers = [(list(f[:3]), f[3]) for f in frs]
    while len(layers) > 1:
        nxt = []
        for i in range(0, len(layers) - 1, 2):
            (cf, af), (cb, ab) = layers[i], layers[i + 1]
            nxt.append(([x + (1 - af) * y for x, y in zip(cf, cb)], af + (1 - af) * ab))
        if len(layers) % 2:
            nxt.append(layers[-1])
        layers = nxt
    c, a = layers[0]
    return [*c, a]


@pytest.mark.parametrize("seed", range(6))
def test_tree_grouping_equals_sequential_exactly(seed):
    """Associativity: pairwise (binary-swap) grouping on Fractions vs the oracle."""
    rng = np.random.default_rng(10 + seed)
    n, P = int(rng.integers(1, 9)), 16
    num = rng.integers(0, 256, (n, P, 4))
    a = num[..., 3] / 256.0
    rgba = np.concatenate([(num[..., :3] / 256.0) * a[..., None], a[..., None]], -1)
    depth = rng.permuted(np.tile(np.arange(n, dtype=np.float32)[:, None], (1, P)), axis=0)
    out = o.composite_tile(*_frags(rgba, depth), o.BLEND_DEPTH)
    for p in range(P):
        order = sorted(range(n), key=lambda i: (float(depth[i, p]), i))
        fr = [[Fraction(float(v)) for v in rgba[i, p]] for i in order]
        exact = _exact_tree_over(fr)
        assert max(abs(float(e) - out[p, c]) for c, e in enumerate(exact)) < 1e-14


def test_golden_hand_derived_pixels():
    with open(os.path.join(GOLDEN, "over_worked_pixels.json")) as f:
        cases = json.load(f)["cases"]
    for cs in cases:
        rgba = np.array(cs["rgba"], dtype=np.float64)[:, None, :]
        depth = np.array(cs["depth"], dtype=np.float32)[:, None]
        keys = np.array(cs["keys"], dtype=np.float32)
        out = o.composite_tile(rgba, depth, keys, np.arange(len(keys)),
                               {"depth": o.BLEND_DEPTH, "ordered": o.BLEND_ORDERED,
                                "z": o.ZCOMPOSITE}[cs["mode"]], bg=cs.get("bg", (0, 0, 0, 0)))
        np.testing.assert_array_equal(out[0], np.array(cs["expect"]), err_msg=cs["name"])


def test_background_behind_all():
    rgba = np.zeros((1, 1, 4))
    rgba[0, 0] = [0.25, 0.0, 0.0, 0.5]
    out = o.composite_tile(rgba, np.zeros((1, 1), np.float32), [0.0], [0], o.BLEND_DEPTH,
                           bg=(0.0, 1.0, 0.0, 1.0))
    np.testing.assert_array_equal(out[0], [0.25, 0.5, 0.0, 1.0])
    empty = o.composite_tile(np.zeros((0, 4, 4)), np.zeros((0, 4)), [], [], o.BLEND_DEPTH,
                             bg=(0.5, 0.5, 0.5, 0.5))
    np.testing.assert_array_equal(empty, np.tile([0.25, 0.25, 0.25, 0.5], (4, 1)))
    ez = o.composite_tile(np.zeros((0, 4, 4)), np.zeros((0, 4)), [], [], o.ZCOMPOSITE,
                          bg=(0.5, 0.5, 0.5, 0.5))
    np.testing.assert_array_equal(ez, np.tile([0.25, 0.25, 0.25, 0.5], (4, 1)))
    # a pixel that no fragment covers (depth +inf) shows the background in Z mode
    rg = np.array([[[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.5]]])
    zz = o.composite_tile(rg, np.array([[np.inf, 1.0]], np.float32), [0.0], [0], o.ZCOMPOSITE,
                          bg=(1.0, 1.0, 1.0, 0.5))
    np.testing.assert_array_equal(zz, [[0.5, 0.5, 0.5, 0.5], [0.5, 0.0, 0.0, 0.5]])


# --- ordering ----------------------------------------------------------------
def _small_scene(seed=0, persp=False):
    if persp:
        return scenes.scene_data_parallel(64, 48, 16, (2, 2, 2), seed=seed, jitter_sigma=0.0)
    return scenes.brick_scene(64, 64, 16, scenes.brick_grid((2, 2, 2)),
                              scenes.Camera("ortho", 64, 64), seed=seed)


def _frame(sc, mode, order=None, bg=(0, 0, 0, 0)):
    idx = np.arange(sc.n) if order is None else order
    return o.composite_frame(sc.W, sc.H, sc.T, mode, sc.tile_ids[idx], sc.keys[idx],
                             sc.rgba[idx].astype(np.float64), sc.depth[idx], bg)


@pytest.mark.parametrize("persp", [False, True])
def test_rank_order_equals_depth_sort_for_disjoint_bricks(persp):
    """Sec. 4.2: for disjoint bricks with keys in visibility order, the list
    (rank-order) tree gives the same image as the per-pixel depth sort."""
    sc = _small_scene(3, persp)
    np.testing.assert_array_equal(_frame(sc, o.BLEND_DEPTH), _frame(sc, o.BLEND_ORDERED))


def test_arrival_order_does_not_matter():
    """Sec. 3.1.1: tiles may arrive in any order."""
    sc = _small_scene(4, persp=True)
    perm = np.random.default_rng(5).permutation(sc.n)
    for mode in (o.BLEND_DEPTH, o.BLEND_ORDERED, o.ZCOMPOSITE):
        np.testing.assert_array_equal(_frame(sc, mode), _frame(sc, mode, perm))


def test_zcomposite_brute_force():
    rng = np.random.default_rng(6)
    n, P = 9, 200
    rgba = rng.uniform(0, 1, (n, P, 4))
    depth = rng.integers(0, 4, (n, P)).astype(np.float32)        # many ties
    depth[rng.uniform(size=(n, P)) < 0.1] = np.nan
    depth[rng.uniform(size=(n, P)) < 0.1] = -0.0
    keys = rng.integers(0, 3, n).astype(np.float32)
    out = o.composite_tile(rgba, depth, keys, np.arange(n), o.ZCOMPOSITE)
    for p in range(P):
        cand = []
        for i in range(n):
            z = float(depth[i, p])
            z = math.inf if math.isnan(z) else (0.0 if z == 0 else z)
            cand.append((z, float(keys[i]), i))
        zb, _, best = min(cand)
        want = rgba[best, p] if zb != math.inf else np.zeros(4)
        np.testing.assert_array_equal(out[p], want)


def test_depth_sort_ties_and_nan_brute_force():
    rng = np.random.default_rng(7)
    n, P = 6, 300
    a = rng.uniform(0, 1, (n, P))
    rgba = np.concatenate([rng.uniform(0, 1, (n, P, 3)) * a[..., None], a[..., None]], -1)
    depth = rng.integers(0, 3, (n, P)).astype(np.float32)
    depth[rng.uniform(size=(n, P)) < 0.15] = np.nan
    keys = rng.integers(0, 2, n).astype(np.float32)
    out = o.composite_tile(rgba, depth, keys, np.arange(n), o.BLEND_DEPTH)
    for p in range(P):
        def zf(i):
            z = float(depth[i, p])
            return math.inf if math.isnan(z) else z
        order = sorted(range(n), key=lambda i: (zf(i), float(keys[i]), i))
        C = [0.0, 0.0, 0.0]
        A = 0.0
        for i in order:
            t = 1.0 - A
            C = [C[c] + t * rgba[i, p, c] for c in range(3)]
            A = A + t * rgba[i, p, 3]
        np.testing.assert_allclose(out[p], [*C, A], rtol=0, atol=1e-15)


def test_bucket_brute_force():
    rng = np.random.default_rng(8)
    n, nt = 500, 37
    tids = rng.integers(0, nt, n)
    keys = rng.integers(0, 5, n).astype(np.float32)
    keys[rng.uniform(size=n) < 0.1] = -0.0
    lists, counts, offsets = o.bucket(tids, keys, nt)
    assert counts.sum() == n
    assert offsets[0] == 0 and all(offsets[1:] == np.cumsum(counts)[:-1])
    for t in range(nt):
        members = [i for i in range(n) if tids[i] == t]
        assert sorted(lists[t]) == members
        pairs = [(float(keys[i]) + 0.0, i) for i in lists[t]]
        assert pairs == sorted(pairs)
    with pytest.raises(ValueError):
        o.bucket([nt], [0.0], nt)
    with pytest.raises(ValueError):
        o.bucket([0], [float("nan")], nt)


def test_frame_edge_tiles_brute_force():
    """Ragged frames: pixels of a submitted tile outside the frame are ignored."""
    W, H, T = 23, 17, 8
    rng = np.random.default_rng(9)
    tiles_x = 3
    tids = np.array([0, 2, 5, 5, 4], dtype=np.int32)
    keys = np.array([1, 2, 3, 0.5, 1], dtype=np.float32)
    a = rng.uniform(0, 1, (5, T * T))
    rgba = np.concatenate([rng.uniform(0, 1, (5, T * T, 3)) * a[..., None], a[..., None]], -1)
    depth = rng.uniform(0, 1, (5, T * T)).astype(np.float32)
    img = o.composite_frame(W, H, T, o.BLEND_DEPTH, tids, keys, rgba, depth)
    for y in range(H):
        for x in range(W):
            t = (y // T) * tiles_x + (x // T)
            p = (y % T) * T + (x % T)
            fr = [i for i in range(5) if tids[i] == t]
            fr.sort(key=lambda i: (float(depth[i, p]), float(keys[i]), i))
            C, A = np.zeros(3), 0.0
            for i in fr:
                C = C + (1 - A) * rgba[i, p, :3]
                A = A + (1 - A) * rgba[i, p, 3]
            np.testing.assert_allclose(img[y, x], [*C, A], atol=1e-15)


# --- accumulation, variance ---------------------------------------------------
def test_accumulate_fsum_and_constant():
    rng = np.random.default_rng(11)
    frames = [rng.uniform(0, 1, (5, 4)) for _ in range(37)]
    m = o.accumulate(frames)
    for i in range(5):
        for c in range(4):
            ref = math.fsum(f[i, c] for f in frames) / 37
            assert abs(m[i, c] - ref) < 1e-15
    const = [np.full((3, 4), 0.3)] * 1000
    np.testing.assert_allclose(o.accumulate(const), 0.3, atol=1e-14)


def test_redundant_passes_average_equals_accumulation():
    """Sec. 4.1.1: averaging k redundantly rendered tiles equals accumulating
    k passes (more samples per pixel)."""
    rng = np.random.default_rng(12)
    k = 6
    passes = [rng.uniform(0, 1, (16, 4)) for _ in range(k)]
    stacked = np.mean(np.stack(passes), axis=0)
    np.testing.assert_allclose(o.accumulate(passes), stacked, atol=1e-15)


def test_variance_library_and_closed_forms():
    rng = np.random.default_rng(13)
    frames = [rng.uniform(0, 1, (7, 4)) for _ in range(9)]
    np.testing.assert_allclose(o.variance(frames), np.var(np.stack(frames), axis=0, ddof=1),
                               atol=1e-15)
    assert np.all(o.variance([np.full((2, 4), 0.7)] * 5) == 0)
    assert np.all(o.variance([frames[0]]) == 0)
    a, b = frames[0], frames[1]
    np.testing.assert_allclose(o.variance([a, b]), (a - b) ** 2 / 2, atol=1e-15)


def test_tile_variance_brute_force():
    rng = np.random.default_rng(14)
    H, W, T = 13, 21, 8
    v = rng.uniform(0, 1, (H, W, 4))
    tv = o.tile_variance(v, T)
    tiles_x = 3
    for t in range(len(tv)):
        vals = [v[y, x, c] for y in range(H) for x in range(W) for c in range(3)
                if (y // T) * tiles_x + x // T == t]
        assert abs(tv[t] - math.fsum(vals) / len(vals)) < 1e-14


# --- display conversion -----------------------------------------------------
def _srgb_decode(v):
    v = np.asarray(v, dtype=np.float64)
    return np.where(v <= 0.04045, v / 12.92, ((v + 0.055) / 1.055) ** 2.4)


def test_srgb_pack_fixed_points():
    def px(r, g, b, a):
        return o.unpack_rgba8(o.pack_rgba8(np.array([r, g, b, a], float)))
    assert list(px(0, 0, 0, 0)) == [0, 0, 0, 0]
    assert list(px(1, 1, 1, 1)) == [255, 255, 255, 255]
    assert list(px(0.5, -3, 7, 0.5)) == [188, 0, 255, 128]   # linear 0.5 -> sRGB 188
    assert list(px(np.nan, 0, 0, 1)) == [0, 0, 0, 255]
    # linear segment: 12.92 x below 0.0031308
    x = 0.0031308
    assert px(x, 0, 0, 0)[0] == math.floor(255 * 12.92 * x + 0.5)


def test_srgb_pack_against_inverse_thresholds():
    """Code c covers the linear interval [dec((c-.5)/255), dec((c+.5)/255))."""
    thr = _srgb_decode((np.arange(1, 256) - 0.5) / 255.0)
    for eps, want in ((1e-9, 0), (-1e-9, -1)):
        x = thr * (1 + eps)
        got = o.unpack_rgba8(o.pack_rgba8(np.stack([x, x, x, np.zeros_like(x)], -1)))[:, 0]
        np.testing.assert_array_equal(got, np.arange(1, 256) + want)
    # 2^24 seeded uniform samples, in chunks to bound the memory
    rng = np.random.default_rng(15)
    for _ in range(4):
        x = rng.uniform(0, 1, 1 << 22)
        got = o.unpack_rgba8(o.pack_rgba8(np.stack([x, x, x, x], -1)))
        np.testing.assert_array_equal(got[:, 0], np.searchsorted(thr, x, side="right"))
        np.testing.assert_array_equal(got[:, 3], np.floor(255 * x + 0.5).astype(int))


# --- storage formats --------------------------------------------------------
def test_fp8_decode_all_codes():
    torch = pytest.importorskip("torch")
    codes = np.arange(256, dtype=np.uint8)
    mine = o.fp8_e4m3_decode(codes)
    ref = torch.from_numpy(codes.copy()).view(torch.float8_e4m3fn).double().numpy()
    np.testing.assert_array_equal(np.isnan(mine), np.isnan(ref))
    np.testing.assert_array_equal(mine[~np.isnan(mine)], ref[~np.isnan(ref)])


def test_fp8_decode_known_values():
    d = o.fp8_e4m3_decode(np.array([0x7E, 0x08, 0x01, 0x38, 0x00, 0xB8, 0x07], np.uint8))
    np.testing.assert_array_equal(d, [448.0, 2 ** -6, 2 ** -9, 1.0, 0.0, -1.0, 7 * 2 ** -9])
    assert np.isnan(o.fp8_e4m3_decode(np.array([0x7F, 0xFF], np.uint8))).all()


def test_fp8_encode_rne_satfinite():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(16)
    x = rng.uniform(-448, 448, 50000)
    vals = o.fp8_e4m3_decode(np.arange(0x7F, dtype=np.uint8))
    mids = (vals[1:] + vals[:-1]) / 2                              # exact ties
    x = np.concatenate([x, mids, -mids, vals, rng.uniform(-1e-2, 1e-2, 5000)])
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(o.fp8_e4m3_encode(x), ref)
    # ties go to the even code
    for i, m in enumerate(mids):
        assert o.fp8_e4m3_encode(np.array([m]))[0] % 2 == 0
    np.testing.assert_array_equal(o.fp8_e4m3_encode(np.array([1000.0, -1e30, 448.0, 464.0])),
                                  [0x7E, 0xFE, 0x7E, 0x7E])
    assert o.fp8_e4m3_encode(np.array([np.nan]))[0] == 0x7F


def test_fp8_quantize_tile_hits_amax():
    rng = np.random.default_rng(17)
    x = rng.uniform(0, 0.9, (64, 4)).astype(np.float32)
    codes, s = o.fp8_quantize_tile(x)
    amax_code = codes.reshape(-1)[np.argmax(x)]
    assert amax_code == 0x7E
    deq = o.dequantize(codes[None], o.FP8E4M3, np.array([s]))[0]
    assert np.max(np.abs(deq - x) / np.maximum(np.abs(x), 2 ** -6 * s)) <= 2 ** -4 + 1e-12
    z, s0 = o.fp8_quantize_tile(np.zeros((4, 4), np.float32))
    assert s0 == 1.0 and not z.any()


def test_half_and_bf16_upcast_exact():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(18)
    x = rng.uniform(-2, 2, 4096).astype(np.float32)
    h = x.astype(np.float16)
    np.testing.assert_array_equal(o.dequantize(h, o.F16), h.astype(np.float64))
    tb = torch.from_numpy(x).to(torch.bfloat16)
    bits = tb.view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(o.dequantize(bits, o.BF16), tb.double().numpy())


# --- redundant tiles averaged by the image-parallel tile operation (Sec. 4.1.1) --
def test_average_of_identical_tiles_is_the_tile():
    rng = np.random.default_rng(41)
    tile = rng.integers(0, 64, (16, 4)) / 64.0          # dyadic: every step is exact
    for k in (1, 2, 3, 7):
        rgba = np.broadcast_to(tile, (k, 16, 4))
        out = o.composite_tile(*_frags(rgba, np.zeros((k, 16))), o.AVERAGE)
        np.testing.assert_array_equal(out, tile)


def test_average_closed_form():
    """Constant tiles v_1..v_k average to (v_1 + ... + v_k) / k (dyadic, exact)."""
    vals = [0.125, 0.5, 0.75, 0.25]
    rgba = np.stack([np.full((8, 4), v) for v in vals])
    out = o.composite_tile(*_frags(rgba, np.zeros((4, 8))), o.AVERAGE)
    np.testing.assert_array_equal(out, np.full((8, 4), sum(vals) / 4))
    two = o.composite_tile(*_frags(rgba[:3], np.zeros((3, 8))), o.AVERAGE)
    np.testing.assert_array_equal(two, np.full((8, 4), (0.125 + 0.5 + 0.75) / 3))


def test_average_goes_over_background_and_empty_tile_shows_it():
    rgba = np.stack([np.full((4, 4), 0.25), np.full((4, 4), 0.75)])   # mean: c = 0.5, a = 0.5
    bg = (1.0, 0.5, 0.25, 0.5)                                        # premultiplied 0.5, 0.25, 0.125
    out = o.composite_tile(*_frags(rgba, np.zeros((2, 4))), o.AVERAGE, bg)
    want = np.array([0.5 + 0.5 * 0.5, 0.5 + 0.5 * 0.25, 0.5 + 0.5 * 0.125, 0.5 + 0.5 * 0.5])
    np.testing.assert_array_equal(out, np.broadcast_to(want, (4, 4)))
    empty = o.composite_tile(np.zeros((0, 4, 4)), np.zeros((0, 4)), [], [], o.AVERAGE, bg)
    np.testing.assert_array_equal(empty, np.broadcast_to([0.5, 0.25, 0.125, 0.5], (4, 4)))


def test_average_ignores_depth_and_order():
    rng = np.random.default_rng(42)
    rgba = rng.random((5, 32, 4))
    a = o.composite_tile(rgba, rng.random((5, 32)).astype(np.float32), np.zeros(5), np.arange(5),
                         o.AVERAGE)
    perm = rng.permutation(5)
    b = o.composite_tile(rgba[perm], rng.random((5, 32)).astype(np.float32), rng.random(5),
                         np.arange(5), o.AVERAGE)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)
    np.testing.assert_allclose(a, np.array([[math.fsum(rgba[:, p, c]) / 5 for c in range(4)]
                                            for p in range(32)]), rtol=0, atol=1e-15)


def test_average_of_k_tiles_equals_k_accumulated_frames():
    """Sec. 4.1.1: averaging k redundantly rendered tiles gives the tile
    rendered with k times the samples, i.e. what accumulating the k renders as
    k frames gives."""
    rng = np.random.default_rng(43)
    k = 6
    rgba = rng.random((k, 64, 4))
    avg = o.composite_tile(*_frags(rgba, np.zeros((k, 64))), o.AVERAGE)
    frames = [o.composite_tile(*_frags(rgba[i:i + 1], np.zeros((1, 64))), o.BLEND_ORDERED)
              for i in range(k)]
    np.testing.assert_allclose(avg, o.accumulate(frames), rtol=0, atol=1e-15)


# --- pixel operations (Sec. 3.1.2) ------------------------------------------------
def test_pixel_op_identities():
    rng = np.random.default_rng(44)
    img = rng.random((8, 8, 4))
    np.testing.assert_array_equal(o.pixel_op(img, o.PIXELOP_NONE, 3.0), img)
    np.testing.assert_array_equal(o.pixel_op(img, o.PIXELOP_EXPOSURE, 1.0), img)
    dy = rng.integers(0, 256, (4, 4, 4)) / 256.0
    got = o.pixel_op(dy, o.PIXELOP_EXPOSURE, 2.0)
    np.testing.assert_array_equal(got[..., :3], 2.0 * dy[..., :3])
    np.testing.assert_array_equal(got[..., 3], dy[..., 3])


def test_reinhard_closed_forms():
    img = np.array([[1.0, 3.0, 0.0, 0.25], [0.5, 1.5, 7.0, 1.0]])
    got = o.pixel_op(img, o.PIXELOP_REINHARD, 1.0)
    np.testing.assert_array_equal(got, [[0.5, 0.75, 0.0, 0.25], [1.0 / 3.0, 0.6, 0.875, 1.0]])
    got = o.pixel_op(img, o.PIXELOP_REINHARD, 2.0)
    np.testing.assert_array_equal(got[0], [2.0 / 3.0, 6.0 / 7.0, 0.0, 0.25])
    np.testing.assert_array_equal(got[1, :3], [0.5, 0.75, 14.0 / 15.0])
    big = o.pixel_op(np.array([[1e300, 1e300, 1e300, 1.0]]), o.PIXELOP_REINHARD, 1.0)
    np.testing.assert_allclose(big[0, :3], 1.0, rtol=1e-15)


# --- user tone curve (Sec. 3.1.2: the pixel operation is the user's) -----------
def test_tone_curve_samples_clamp_and_identity():
    # x_max = 2 and n = 9 put the samples at exact multiples of 1/4
    t = np.array([0.1, 0.7, -0.2, 3.0, 0.5, 0.5, 1.25, 0.0, 2.0])
    xs = np.arange(9) / 4.0
    np.testing.assert_array_equal(o.tone_curve(xs, t, 2.0), t)
    # halfway between two samples: their mean
    np.testing.assert_allclose(o.tone_curve(xs[:-1] + 0.125, t, 2.0), 0.5 * (t[:-1] + t[1:]),
                               rtol=0, atol=1e-15)
    # below 0, NaN -> the first sample; above x_max -> the last
    got = o.tone_curve(np.array([-3.0, np.nan, 2.0, 7.5, np.inf]), t, 2.0)
    np.testing.assert_array_equal(got, [0.1, 0.1, 2.0, 2.0, 2.0])
    # the identity polyline is the clamp
    rng = np.random.default_rng(45)
    x = rng.uniform(-1.0, 4.0, 1000)
    ident = np.linspace(0.0, 3.0, 33)
    np.testing.assert_allclose(o.tone_curve(x, ident, 3.0), np.clip(x, 0.0, 3.0), rtol=0,
                               atol=1e-15)


def test_tone_curve_chord_bound_on_a_parabola():
    # the polyline through samples of x^2 (spacing h) lies above the parabola
    # by at most h^2 / 4 (the chord error of a function with f'' = 2)
    n, xm = 17, 2.0
    h = xm / (n - 1)
    t = np.linspace(0.0, xm, n) ** 2
    x = np.random.default_rng(46).uniform(0.0, xm, 5000)
    err = o.tone_curve(x, t, xm) - x * x
    assert err.min() >= -1e-15
    assert err.max() <= h * h / 4 + 1e-15
    assert err.max() >= 0.9 * h * h / 4         # the bound is reached between samples


def test_pixel_op_curve_per_channel_after_exposure():
    rng = np.random.default_rng(47)
    img = rng.random((6, 6, 4))
    xm = 4.0
    curves = np.stack([np.linspace(0.0, xm, 5),               # identity
                       np.linspace(1.0, 0.0, 5),              # 1 - x / 4
                       np.full(5, 0.25)])                     # constant
    got = o.pixel_op(img, o.PIXELOP_CURVE, 3.0, curves, xm)
    np.testing.assert_allclose(got[..., 0], np.clip(3.0 * img[..., 0], 0.0, xm), rtol=0,
                               atol=1e-15)
    np.testing.assert_allclose(got[..., 1], 1.0 - np.clip(3.0 * img[..., 1], 0.0, xm) / xm,
                               rtol=0, atol=1e-15)
    np.testing.assert_array_equal(got[..., 2], 0.25)
    np.testing.assert_array_equal(got[..., 3], img[..., 3])


def test_tone_curve_sampled_from_reinhard():
    # Reinhard's curve x / (1 + x) sampled finely reproduces PIXELOP_REINHARD
    # within the chord bound (|f''| <= 2 on x >= 0)
    n, xm = 4096, 8.0
    h = xm / (n - 1)
    xs = np.linspace(0.0, xm, n)
    curves = np.stack([xs / (1.0 + xs)] * 3)
    img = np.random.default_rng(48).random((16, 16, 4)) * np.array([2.0, 2.0, 2.0, 1.0])
    a = o.pixel_op(img, o.PIXELOP_CURVE, 1.5, curves, xm)
    b = o.pixel_op(img, o.PIXELOP_REINHARD, 1.5)
    assert np.abs(a - b).max() <= h * h / 4 + 1e-15
