"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins
catch every one of them."""

import numpy as np
import pytest

from oracle import dfb_oracle as o
import tests.test_oracle_pins as pins


def _wrong_sign(C, A, c, a):
    t = 1.0 + A
    return C + t[..., None] * c, A + t * a


def _back_to_front_formula(C, A, c, a):
    # treats the new fragment as being in front
    return c + (1.0 - a)[..., None] * C, a + (1.0 - a) * A


def _dropped_alpha_term(C, A, c, a):
    t = 1.0 - A
    return C + t[..., None] * c, A + a


def _unsorted_accumulate(frames):
    return sum(np.asarray(f, float) for f in frames) / max(len(frames) - 1, 1)


def _population_variance(frames):
    return np.var(np.stack(frames), axis=0)


def _srgb_no_offset(x):
    x = np.asarray(x, dtype=np.float64)
    return np.where(x <= 0.0031308, 12.92 * x, 1.055 * np.power(np.maximum(x, 0.0), 1.0 / 2.4))


def _average_wrong_divisor(rgba):
    rgba = np.asarray(rgba, dtype=np.float64)
    return rgba.sum(axis=0) / max(rgba.shape[0] - 1, 1)


def _average_first_tile_only(rgba):
    return np.asarray(rgba, dtype=np.float64)[0]


_real_pixel_op = o.pixel_op


def _reinhard_without_exposure(img, op, exposure=1.0):
    if op == o.PIXELOP_REINHARD:
        img = np.array(img, dtype=np.float64)
        img[..., :3] = img[..., :3] / (1.0 + img[..., :3])
        return img
    return _real_pixel_op(img, op, exposure)


def _exposure_on_alpha(img, op, exposure=1.0):
    img = np.array(img, dtype=np.float64)
    if op == o.PIXELOP_EXPOSURE:
        return img * exposure
    return _real_pixel_op(img, op, exposure)


_real_tone_curve = o.tone_curve


def _curve_nearest_sample(x, samples, x_max):
    t = np.asarray(samples, dtype=np.float64)
    n = t.shape[0]
    x = np.minimum(np.maximum(np.nan_to_num(np.asarray(x, float)), 0.0), x_max)
    return t[np.rint(x * (n - 1) / x_max).astype(np.int64)]


def _curve_no_clamp_above(x, samples, x_max):
    x = np.asarray(x, dtype=np.float64)
    inside = _real_tone_curve(x, samples, x_max)
    t = np.asarray(samples, dtype=np.float64)
    n = t.shape[0]
    slope = (t[-1] - t[-2]) * (n - 1) / x_max
    return np.where(x > x_max, t[-1] + (x - x_max) * slope, inside)


def _curve_step_count_n(x, samples, x_max):
    # spaces the samples x_max / n apart instead of x_max / (n - 1)
    t = np.asarray(samples, dtype=np.float64)
    n = t.shape[0]
    return _real_tone_curve(x, t, x_max * (n - 1) / n)


def _exposure_after_curve(img, op, exposure=1.0, curves=None, x_max=1.0):
    if op == o.PIXELOP_CURVE:
        img = np.array(img, dtype=np.float64)
        for c in range(3):
            img[..., c] = exposure * _real_tone_curve(img[..., c], curves[c], x_max)
        return img
    return _real_pixel_op(img, op, exposure, curves, x_max)


MUTANTS = [
    ("over_front_to_back", _wrong_sign, [pins.test_equal_layers_closed_form]),
    ("over_front_to_back", _back_to_front_formula, [pins.test_golden_hand_derived_pixels]),
    ("over_front_to_back", _dropped_alpha_term, [pins.test_equal_layers_closed_form]),
    ("accumulate", _unsorted_accumulate, [pins.test_accumulate_fsum_and_constant]),
    ("variance", _population_variance, [pins.test_variance_library_and_closed_forms]),
    ("srgb_encode", _srgb_no_offset, [pins.test_srgb_pack_fixed_points]),
    ("average_tiles", _average_wrong_divisor, [pins.test_average_of_identical_tiles_is_the_tile,
                                               pins.test_average_closed_form]),
    ("average_tiles", _average_first_tile_only, [pins.test_average_closed_form]),
    ("pixel_op", _reinhard_without_exposure, [pins.test_reinhard_closed_forms]),
    ("pixel_op", _exposure_on_alpha, [pins.test_pixel_op_identities]),
    ("tone_curve", _curve_nearest_sample, [pins.test_tone_curve_samples_clamp_and_identity,
                                           pins.test_tone_curve_chord_bound_on_a_parabola]),
    ("tone_curve", _curve_no_clamp_above, [pins.test_tone_curve_samples_clamp_and_identity]),
    ("tone_curve", _curve_step_count_n, [pins.test_tone_curve_samples_clamp_and_identity,
                                         pins.test_tone_curve_chord_bound_on_a_parabola]),
    ("pixel_op", _exposure_after_curve, [pins.test_pixel_op_curve_per_channel_after_exposure]),
]


@pytest.mark.parametrize("name,bad,tests", MUTANTS, ids=[m[1].__name__ for m in MUTANTS])
def test_pins_catch_mutant(monkeypatch, name, bad, tests):
    monkeypatch.setattr(o, name, bad)
    for t in tests:
        with pytest.raises(AssertionError):
            if t is pins.test_equal_layers_closed_form:
                t(0.3, 5)
            else:
                t()


def test_pins_catch_wrong_depth_tiebreak(monkeypatch):
    real = np.lexsort

    def lexsort_reverse_submit(keys, axis=-1):
        keys = list(keys)
        if len(keys) == 3:
            keys[0] = -np.asarray(keys[0])       # submit index descending
        return real(tuple(keys), axis=axis)

    monkeypatch.setattr(o.np, "lexsort", lexsort_reverse_submit)
    with pytest.raises(AssertionError):
        pins.test_golden_hand_derived_pixels()
