"""Pins of the oracle's coefficient precision tiers."""
import numpy as np
import pytest

from oracle import mlp, precision


def test_round_sig_matches_numpy_half_including_subnormals():
    g = np.random.default_rng(5)
    x = np.concatenate([g.standard_normal(2000) * 10.0 ** g.uniform(-9, 4, 2000),
                        [6.1e-5, 6.0e-5, 2.0 ** -24, 3 * 2.0 ** -25, 2.0 ** -25, 65504.0, -1e-7]])
    got = precision.round_sig(x, 11, -24)
    ref = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(got, ref)


def test_round_sig_bf16_known_values_and_float32_bit_trick():
    assert precision.round_sig(1 + 2.0 ** -8, 8, -133) == 1.0          # tie -> even
    assert precision.round_sig(1 + 3 * 2.0 ** -9, 8, -133) == 1 + 2.0 ** -7
    # in [2, 4) the BF16 spacing is 2^-6: ties at odd multiples of 2^-7
    assert precision.round_sig(-(2 + 2.0 ** -7), 8, -133) == -2.0
    assert precision.round_sig(-(2 + 3 * 2.0 ** -7), 8, -133) == -(2 + 2.0 ** -5)
    x = np.random.default_rng(6).standard_normal(5000).astype(np.float32).astype(np.float64)
    assert np.array_equal(precision.round_sig(x, 8, -133), mlp.bf16(x))


def test_channel_scale_rule():
    assert precision.channel_scale([0.75, -0.2]) == 2.0 ** -15          # 0.75 < 2^0
    assert precision.channel_scale([1.0]) == 2.0 ** -14                 # 1 < 2^1
    assert precision.channel_scale([-3000.0]) == 2.0 ** -3              # 3000 < 2^12
    c = np.random.default_rng(7).standard_normal(100) * 1e3
    assert np.max(np.abs(c)) / precision.channel_scale(c) < 2 ** 15


@pytest.mark.parametrize("tier", ["f16", "bf16"])
def test_quantize_error_within_unit_roundoff(tier):
    g = np.random.default_rng(8)
    coefs = np.stack([g.standard_normal(4000) * np.exp(g.uniform(-12, 6, 4000)) for _ in range(3)])
    q, s = precision.quantize(coefs, tier)
    u = precision.unit_roundoff(tier)
    err = np.abs(q - coefs)
    # normal range: relative bound; below it the absolute quantum of the tier
    floor = s[:, None] * 2.0 ** (precision.TIERS[tier][1] - 1)
    assert np.all(err <= u * np.abs(coefs) + floor)
    assert np.all(np.abs(coefs / s[:, None]) < 2 ** 15)
