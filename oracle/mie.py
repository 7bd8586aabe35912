"""Scalar Mie series for a penetrable sphere (test infrastructure only).

Exact solution of the scalar Helmholtz equation for a plane wave exp(i k z)
(k = k0 n0) hitting a homogeneous sphere of index n1 and radius a centred at
the origin: outside, psi = sum_l i^l (2l+1) [j_l(k r) + A_l h_l(k r)] P_l(cos t),
inside, psi = sum_l i^l (2l+1) C_l j_l(k1 r) P_l(cos t), k1 = k0 n1, with A_l,
C_l from the continuity of psi and d psi / d r at r = a:

    A_l = (k1 j_l'(k1 a) j_l(k a) - k j_l'(k a) j_l(k1 a))
          / (k h_l'(k a) j_l(k1 a) - k1 h_l(k a) j_l'(k1 a)),

h_l = j_l + i y_l.  Used by tests/test_oracle_mie.py to compare the oracle's
forward-only BPM field behind a sphere with this exact solution, as a report
on the physics of the method (the paper validates against analytically
tractable scattering models, method paragraph), not as a parity gate.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def coefficients(k0: float, n0: float, n1: float, a: float, lmax: int) -> np.ndarray:
    k, k1 = k0 * n0, k0 * n1
    ls = np.arange(lmax + 1)
    j = special.spherical_jn(ls, k * a)
    jd = special.spherical_jn(ls, k * a, derivative=True)
    y = special.spherical_yn(ls, k * a)
    yd = special.spherical_yn(ls, k * a, derivative=True)
    j1 = special.spherical_jn(ls, k1 * a)
    j1d = special.spherical_jn(ls, k1 * a, derivative=True)
    h, hd = j + 1j * y, jd + 1j * yd
    return (k1 * j1d * j - k * jd * j1) / (k * hd * j1 - k1 * h * j1d)


def field_outside(k0: float, n0: float, n1: float, a: float, x, y, z, lmax: int | None = None) -> np.ndarray:
    """Total field at points (x, y, z) outside the sphere (arrays of equal shape)."""
    k = k0 * n0
    if lmax is None:
        lmax = int(k * a + 4 * (k * a) ** (1 / 3) + 10)
    A = coefficients(k0, n0, n1, a, lmax)
    r = np.sqrt(x * x + y * y + z * z)
    c = z / r
    scat = np.zeros(r.shape, complex)
    for l in range(lmax + 1):
        h = special.spherical_jn(l, k * r) + 1j * special.spherical_yn(l, k * r)
        scat += (1j ** l) * (2 * l + 1) * A[l] * h * special.eval_legendre(l, c)
    return np.exp(1j * k * z) + scat
