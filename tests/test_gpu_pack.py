"""The RGBA8 pack on the GPU against its definition: the sRGB code of a linear
value x is the number of code boundaries <= x (x clamped to [0, 1], NaN as
0), the boundaries being the inverse IEC 61966-2-1 curve at (c - 0.5) / 255
rounded to FP32 (Sec. 3.1's display format; the oracle's own formula agrees
with this within 1 LSB, pinned on the CPU).  The kernel reads the code from a
bucket table; this checks it bit for bit on values packed around every
boundary and every bucket edge."""

import numpy as np
import pytest

from oracle import dfb_oracle as o
from paper_2305_07083_gb300 import dfb as D

from tests.gpu_helpers import GpuFrameBuffer

pytestmark = pytest.mark.gpu


def boundaries_f32():
    v = (np.arange(1, 256) - 0.5) / 255.0
    lin = np.where(v <= 0.04045, v / 12.92, ((v + 0.055) / 1.055) ** 2.4)
    return lin.astype(np.float32)


def expected_codes(x):
    thr = boundaries_f32()
    c = np.clip(np.nan_to_num(x, nan=0.0), 0.0, 1.0).astype(np.float32)
    return np.searchsorted(thr, c, side="right").astype(np.uint32)


def fixed_probes():
    """Every code boundary and bucket start of the table, their neighbours,
    and special values."""
    thr = boundaries_f32()
    near = [np.nextafter(thr, np.float32(np.inf * s)) for s in (1, -1)]
    vals = [thr, near[0], near[1], np.nextafter(near[0], np.float32(np.inf)),
            np.nextafter(near[1], np.float32(-np.inf))]
    # every bucket start of the table (exponent + 7 mantissa bits) and its neighbours
    starts = ((np.arange(13 * 128 + 1) + ((127 - 13) << 7)) << 16).astype(np.uint32).view(np.float32)
    vals += [starts, np.nextafter(starts, np.float32(0)), np.nextafter(starts, np.float32(2))]
    special = np.array([0.0, -0.0, 1.0, 1.5, np.inf, -np.inf, -1.0, np.nan, 1e-45, 1e-38,
                        2.0 ** -13, 2.0 ** -14, 0.0031308, 0.04045 / 12.92], np.float32)
    vals.append(special)
    return np.concatenate(vals).astype(np.float32)


def probe_values(n, seed=0):
    rng = np.random.default_rng(seed)
    fixed = fixed_probes()
    rest = n - len(fixed)
    u = rng.random(rest // 2, dtype=np.float32)
    logu = np.exp2(rng.uniform(-24, 0, rest - rest // 2)).astype(np.float32)
    return np.concatenate([fixed, u, logu]).astype(np.float32)


def pack_on_gpu(rgb, W, H, T=64):
    """RGBA8 of an opaque frame whose colour is `rgb` (H, W, 3): one opaque
    fragment per tile at depth 0, so the composited colour is rgb itself."""
    n_tiles = (W // T) * (H // T)
    tiles = np.zeros((n_tiles, T * T, 4), np.float32)
    for t in range(n_tiles):
        ty, tx = divmod(t, W // T)
        tiles[t, :, :3] = rgb[ty * T:(ty + 1) * T, tx * T:(tx + 1) * T].reshape(T * T, 3)
    tiles[:, :, 3] = 1.0
    depth = np.zeros((n_tiles, T * T), np.float32)
    fb = GpuFrameBuffer(W, H, T, D.DFB_BLEND_DEPTH)
    fb.begin(0)
    fb.submit_pool(np.arange(n_tiles, dtype=np.int32), np.zeros(n_tiles, np.float32), tiles, depth)
    fb.end()
    out = fb.rgba8()
    fb.close()
    return out


def test_rgb_codes_match_boundary_definition():
    W = H = 1024
    x = probe_values(3 * W * H)
    rgb = x.reshape(H, W, 3)
    got = pack_on_gpu(rgb, W, H).view(np.uint8).reshape(H, W, 4)
    want = expected_codes(x).reshape(H, W, 3)
    bad = np.argwhere(got[..., :3] != want)
    assert len(bad) == 0, "first mismatches: %s" % [
        (float(rgb[tuple(b)]), int(got[tuple(b)]), int(want[tuple(b)])) for b in bad[:5]]
    assert (got[..., 3] == 255).all()


def test_rgb_codes_against_the_oracle():
    """2^24 seeded uniform samples in [0, 1] (as in the CPU pin of the oracle's
    pack) plus the boundary probes, packed on the GPU, against the oracle's
    float64 sRGB formula: within 1 LSB."""
    W, H = 4096, 2048
    x = np.random.default_rng(15).uniform(0, 1, 3 * W * H).astype(np.float32)
    probes = fixed_probes()
    x[:len(probes)] = probes
    rgb = x.reshape(H, W, 3)
    got = o.unpack_rgba8(pack_on_gpu(rgb, W, H)).reshape(H, W, 4).astype(np.int64)
    img = np.concatenate([rgb.astype(np.float64), np.ones((H, W, 1))], -1)
    want = o.unpack_rgba8(o.pack_rgba8(img)).reshape(H, W, 4).astype(np.int64)
    assert np.abs(got - want).max() <= 1
    assert (got[..., 3] == 255).all()


def test_alpha_codes():
    """Linear alpha: floor(255 a + 0.5) with a clamped to [0, 1]."""
    W, H, T = 256, 256, 64
    n_tiles = 16
    a = np.linspace(0.0, 1.0, W * H, dtype=np.float32).reshape(H, W)
    a.flat[:4] = [0.0, 1.0, 0.5 / 255, 254.5 / 255]
    tiles = np.zeros((n_tiles, T * T, 4), np.float32)
    for t in range(n_tiles):
        ty, tx = divmod(t, W // T)
        tiles[t, :, 3] = a[ty * T:(ty + 1) * T, tx * T:(tx + 1) * T].reshape(-1)
    fb = GpuFrameBuffer(W, H, T, D.DFB_BLEND_DEPTH)
    fb.begin(0)
    fb.submit_pool(np.arange(n_tiles, dtype=np.int32), np.zeros(n_tiles, np.float32), tiles,
                   np.zeros((n_tiles, T * T), np.float32))
    fb.end()
    got = fb.rgba8().view(np.uint8).reshape(H, W, 4)[..., 3].astype(np.int64)
    want = np.floor(255.0 * a.astype(np.float64) + 0.5)
    assert np.max(np.abs(got - want)) <= 1          # FP32 fma vs exact product
    exact = np.abs(255.0 * a.astype(np.float64) + 0.5 - np.round(255.0 * a + 0.5)) > 1e-4
    np.testing.assert_array_equal(got[exact], want[exact])
