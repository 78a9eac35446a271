"""Coefficients of the log2 polynomial used by the tensor-core epilogue.

The batched kernel evaluates, for every event and parameter set,
log2 I = k + log2(1 + z) with I = 2^k (1 + z), 1 + z in [sqrt(1/2), sqrt(2)).
log2(1 + z) is approximated by P(z) = sum_{j=1..D} a_j z^j (P(0) = 0 exactly).
The coefficients come from a near-minimax fit (iteratively reweighted least
squares on Chebyshev nodes) in float64; each coefficient is then rounded to
float32 in turn and the remaining ones refitted, so that the polynomial with
the float32 coefficients the kernel uses is itself near-minimax.

Run as a script to print the coefficients (scaled by 2^19, the fixed-point
resolution of the kernel's log sums) in the form the kernel embeds.
"""
from __future__ import annotations

import numpy as np

DEGREE = 11
Z_LO = float(np.float32(0.70710677)) - 1.0    # float with bits 0x3F3504F3, minus 1
Z_HI = float(np.float32(1.4142135)) - 1.0     # largest float below 2 * 0x3F3504F3
SCALE = 2.0 ** 19


def _fit(fixed, degree, n=6000, iters=80):
    """Fit a_{len(fixed)+1..degree} with a_1..a_len(fixed) fixed."""
    t = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    z = (Z_LO + Z_HI) / 2 + (Z_HI - Z_LO) / 2 * t
    y = np.log1p(z) / np.log(2.0)
    for j, a in enumerate(fixed, start=1):
        y = y - a * z ** j
    j0 = len(fixed) + 1
    if j0 > degree:
        return []
    A = np.stack([z ** j for j in range(j0, degree + 1)], 1)
    w = np.ones(n)
    coef = None
    for _ in range(iters):
        coef, *_ = np.linalg.lstsq(A * w[:, None], y * w, rcond=None)
        e = A @ coef - y
        w = w * (np.abs(e) / np.abs(e).max() + 1e-3) ** 0.5
        w /= w.max()
    return list(coef)


def coefficients(degree=DEGREE):
    """float32 coefficients a_1..a_D of P(z) ~ log2(1 + z)."""
    fixed = []
    for _ in range(degree):
        rest = _fit(fixed, degree)
        fixed.append(float(np.float32(rest[0])))
    return fixed


def max_error(coef, n=400001):
    """Max |P(z) - log2(1 + z)| over the interval, P evaluated in float64."""
    z = np.linspace(Z_LO, Z_HI, n)
    p = np.zeros_like(z)
    for a in reversed(coef):
        p = (p + a) * z
    return float(np.abs(p - np.log1p(z) / np.log(2.0)).max())


if __name__ == "__main__":
    c = coefficients()
    print("// log2(1+z) ~ sum_j a_j z^j, a_j * 2^19 (max error %.2e)" % max_error(c))
    print("constexpr float kLog2Poly[%d] = {" % len(c))
    for a in c:
        print("    %.9ef," % (a * SCALE))
    print("};")
