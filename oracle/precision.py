"""Precision tiers of the stored B-spline coefficients.

Oracle (test infrastructure).  The paper stores its grids in single
precision; the reduced tiers are not in the paper.  Definitions (the same
rule the library states for its FP16 / BF16 storage):

    scale of a channel   s = 2^(e - 15),  max |c| < 2^e  (frexp exponent)
    stored value         round(c / s) to the nearest FP16 (11 significant
                         bits, quantum >= 2^-24) or BF16 (8 significant bits,
                         quantum >= 2^-133) number, ties to even
    value used           s * stored value

Computed exactly in float64: x / q is exact for a power of two q and
numpy's rint rounds ties to even.
"""
from __future__ import annotations

import numpy as np

TIERS = {"f32": None, "f16": (11, -24), "bf16": (8, -133)}
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}


def round_sig(x, bits: int, min_exp: int):
    """Nearest value with `bits` significant bits (ties to even), quantum at
    least 2^min_exp."""
    x = np.asarray(x, np.float64)
    m, e = np.frexp(x)
    qe = np.maximum(e - bits, min_exp)
    q = np.ldexp(1.0, qe)
    return np.where(x == 0, 0.0, np.rint(x / q) * q)


def channel_scale(c) -> float:
    m = float(np.max(np.abs(c)))
    if m == 0.0:
        return 1.0
    _, e = np.frexp(m)
    return float(np.ldexp(1.0, int(e) - 15))


def quantize(coefs, tier: str):
    """(coefficients as the kernels see them, per-channel scales)."""
    coefs = np.asarray(coefs, np.float64)
    if TIERS[tier] is None:
        return coefs.astype(np.float32).astype(np.float64), np.ones(len(coefs))
    bits, min_exp = TIERS[tier]
    out = np.empty_like(coefs)
    scales = np.empty(len(coefs))
    for k, c in enumerate(coefs):
        s = channel_scale(c)
        out[k] = round_sig(c / s, bits, min_exp) * s
        scales[k] = s
    return out, scales


def unit_roundoff(tier: str) -> float:
    """Relative rounding bound of a normal stored value."""
    return {"f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}[tier]
