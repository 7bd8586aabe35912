"""Pins of the complex-index screen (absorption, n = n0 + dn + i kappa):
kappa = 0 reproduces the lossless method, a uniform kappa attenuates the
power exactly by exp(-2 k0 kappa dz) per slice (Beer-Lambert), and the phase
is untouched by kappa."""
import numpy as np

import oracle

LAM, N0, D = 0.5, 1.33, 0.1


def test_zero_kappa_is_the_lossless_method():
    rng = np.random.default_rng(3)
    dn = rng.uniform(0, 0.05, (5, 64, 64))
    E0 = np.exp(1j * rng.uniform(0, 6, (64, 64)))
    A, IA = oracle.bpm(dn, E0, D, D, D, LAM, N0)
    B, IB = oracle.bpm(dn, E0, D, D, D, LAM, N0, kappa=np.zeros_like(dn))
    assert np.array_equal(A, B) and np.array_equal(IA, IB)


def test_uniform_kappa_follows_beer_lambert():
    n, nz = 64, 12
    k0 = 2 * np.pi / LAM
    kap = 0.002
    x = (np.arange(n) - n / 2) * D
    X, Y = np.meshgrid(x, x)
    E0 = np.exp(-(X ** 2 + Y ** 2) / 0.5).astype(complex)     # inside the propagating band, nil at the box edge
    # power: in a homogeneous medium nothing else is lost (the beam stays in
    # the propagating band)
    _, I = oracle.bpm(np.zeros((nz, n, n)), E0, D, D, D, LAM, N0, kappa=np.full((nz, n, n), kap))
    P0 = np.sum(np.abs(E0) ** 2)
    for z in range(nz):
        assert abs(np.sum(I[z]) / P0 - np.exp(-2 * k0 * kap * D * (z + 1))) < 1e-12
    # through any index volume the field is the lossless one scaled by the
    # total attenuation (a uniform kappa commutes with every step)
    rng = np.random.default_rng(4)
    dn = rng.uniform(0, 0.05, (nz, n, n))
    E, _ = oracle.bpm(dn, E0, D, D, D, LAM, N0, kappa=np.full((nz, n, n), kap))
    L, _ = oracle.bpm(dn, E0, D, D, D, LAM, N0)
    assert np.max(np.abs(E - L * np.exp(-k0 * kap * D * nz))) < 1e-12
