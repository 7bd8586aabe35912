"""Pins for the oracle's split-step BPM (Biobeam, arXiv:1706.02261, method
paragraph: beam-propagation model with the exact propagator and a phase screen
per slice) against closed forms and invariants that do not depend on how the
oracle is written:

* an on-grid plane wave in a homogeneous medium is an exact Helmholtz solution,
  E(z) = E(0) exp(i kz z), kz = sqrt((k0 n0)^2 - kx^2 - ky^2);
* a wave beyond the propagating disc (including the tie kz^2 = 0) is removed;
* propagation is a semigroup: m slices of dz equal one slice of m dz;
* a uniform index step c is a pure global phase exp(i k0 c dz nz);
* energy is conserved for a band-limited field in a homogeneous medium and
  never increases with a phase screen;
* a Gaussian beam matches an independent angular-spectrum (Hankel) quadrature
  of the continuous problem, slice by slice.
"""
import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_1706_02261_b300 import inputs

LAM, N0 = 0.5, 1.33
K = 2 * np.pi / LAM * N0


def test_tilted_plane_wave_closed_form():
    nx, ny, dx, dy, dz, nz = 48, 32, 0.1, 0.15, 0.2, 7
    mx, my = 5, -3
    E0 = inputs.plane_wave(nx, ny, mx, my, dtype=np.complex128)
    E, I = oracle.bpm(np.zeros((nz, ny, nx)), E0, dx, dy, dz, LAM, N0)
    kx = 2 * np.pi * mx / (nx * dx)
    ky = 2 * np.pi * my / (ny * dy)
    kz = np.sqrt(K * K - kx * kx - ky * ky)
    expect = E0 * np.exp(1j * kz * nz * dz)
    assert np.max(np.abs(E - expect)) < 1e-12
    assert np.max(np.abs(I - 1.0)) < 1e-12


def test_evanescent_wave_is_cut():
    nx, dx = 32, 0.1
    m = 12                                # kx = 2 pi 12 / 3.2 = 23.6 > K = 16.7
    E0 = inputs.plane_wave(nx, nx, m, 0, dtype=np.complex128)
    E, I = oracle.bpm(np.zeros((1, nx, nx)), E0, dx, dx, 0.1, LAM, N0)
    assert np.max(np.abs(E)) < 1e-14


def test_exact_tie_at_kz_zero_is_cut():
    # lambda = 0.5, n0 = 1: K = 4 pi exactly; n dx = 8 and the Nyquist bin
    # (m = 16 of 32) gives |kx| = 4 pi exactly, so kz^2 = 0 with no rounding.
    nx, dx = 32, 0.25
    H = oracle.propagator(nx, nx, dx, dx, 0.1, 0.5, 1.0)
    assert H[0, 16] == 0
    assert H[16, 0] == 0
    assert abs(H[0, 15]) == pytest.approx(1.0)


def test_semigroup():
    n, dx, dz, m = 32, 0.1, 0.13, 5
    rng = np.random.default_rng(5)
    E0 = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Em, _ = oracle.bpm(np.zeros((m, n, n)), E0, dx, dx, dz, LAM, N0, want_intensity=False)
    E1, _ = oracle.bpm(np.zeros((1, n, n)), E0, dx, dx, m * dz, LAM, N0, want_intensity=False)
    assert np.max(np.abs(Em - E1)) < 1e-12 * np.max(np.abs(E0)) * m


def test_uniform_index_is_global_phase():
    n, dx, dz, nz, c = 32, 0.1, 0.1, 6, 0.037
    rng = np.random.default_rng(6)
    E0 = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Eh, Ih = oracle.bpm(np.zeros((nz, n, n)), E0, dx, dx, dz, LAM, N0)
    Ec, Ic = oracle.bpm(np.full((nz, n, n), c), E0, dx, dx, dz, LAM, N0)
    k0 = 2 * np.pi / LAM
    assert np.max(np.abs(Ec - Eh * np.exp(1j * k0 * c * dz * nz))) < 1e-12 * np.max(np.abs(Eh))
    assert np.max(np.abs(Ic - Ih)) < 1e-12 * np.max(Ih)


def _bandlimited_field(n, dx, frac, seed):
    rng = np.random.default_rng(seed)
    k = 2 * np.pi * np.fft.fftfreq(n, dx)
    kp = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)
    spec = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * (kp < frac * K)
    return np.fft.ifft2(spec)


def test_energy_conserved_homogeneous_and_nonincreasing_with_screen():
    n, dx, dz, nz = 64, 0.1, 0.1, 12
    E0 = _bandlimited_field(n, dx, 0.6, 8)
    e0 = np.sum(np.abs(E0) ** 2)
    _, I = oracle.bpm(np.zeros((nz, n, n)), E0, dx, dx, dz, LAM, N0)
    assert np.max(np.abs(I.sum(axis=(1, 2)) / e0 - 1)) < 1e-12
    rng = np.random.default_rng(9)
    dn = rng.uniform(0, 0.05, size=(nz, n, n))
    _, I = oracle.bpm(dn, E0, dx, dx, dz, LAM, N0)
    energy = np.concatenate([[e0], I.sum(axis=(1, 2))])
    assert np.all(np.diff(energy) <= 1e-12 * e0)
    assert energy[-1] < energy[0]          # the screen scatters some light past the cut


def _hankel_gaussian(rho, z, w0):
    """Continuous angular-spectrum solution for E(rho, 0) = exp(-rho^2 / w0^2):
    E(rho, z) = (w0^2 / 2) int_0^K exp(-k^2 w0^2 / 4) J0(k rho) exp(i kz z) k dk."""
    kmax = min(K, 2.0 * 9.0 / w0)        # the envelope is < 1e-35 beyond this

    def f(k, part):
        kz = np.sqrt(K * K - k * k)
        v = np.exp(-(k * w0 / 2) ** 2) * special.j0(k * rho) * np.exp(1j * kz * z) * k
        return v.real if part == 0 else v.imag

    re = integrate.quad(f, 0, kmax, args=(0,), limit=400, epsabs=1e-14, epsrel=1e-12)[0]
    im = integrate.quad(f, 0, kmax, args=(1,), limit=400, epsabs=1e-14, epsrel=1e-12)[0]
    return 0.5 * w0 * w0 * (re + 1j * im)


def test_gaussian_beam_matches_angular_spectrum_quadrature():
    n, dx, dz, nz, w0 = 128, 0.1, 0.1, 30, 1.5
    c = (n // 2) * dx
    x = np.arange(n) * dx - c
    E0 = np.exp(-(x[None, :] ** 2 + x[:, None] ** 2) / w0 ** 2)
    E, I = oracle.bpm(np.zeros((nz, n, n)), E0, dx, dx, dz, LAM, N0)
    pts = [(0, 0), (0, 7), (11, 0), (9, 13), (-20, 5)]
    for (oy, ox) in pts:
        rho = np.hypot(ox * dx, oy * dx)
        ref_out = _hankel_gaussian(rho, nz * dz, w0)
        assert abs(E[n // 2 + oy, n // 2 + ox] - ref_out) < 1e-9
        # I[z] is recorded after slice z, i.e. at depth (z + 1) dz
        ref_mid = _hankel_gaussian(rho, 10 * dz, w0)
        assert abs(I[9, n // 2 + oy, n // 2 + ox] - abs(ref_mid) ** 2) < 1e-9


def test_screen_acts_after_diffraction_within_a_slice():
    """Step order: each slice diffracts first, then applies its screen.  A
    phase screen present only in the last slice is then a pure phase on the
    final field, so the last intensity slice equals that of the homogeneous
    run pointwise; applied before the diffraction it would change it."""
    n, dx, dz, nz, w0 = 64, 0.1, 0.1, 6, 1.0
    x = (np.arange(n) - n // 2) * dx
    E0 = np.exp(-(x[None, :] ** 2 + x[:, None] ** 2) / w0 ** 2)
    dn = np.zeros((nz, n, n))
    dn[-1] = 0.5 * (np.sin(2 * np.pi * x / 0.8)[None, :] > 0)          # strong binary grating
    _, Ih = oracle.bpm(np.zeros((nz, n, n)), E0, dx, dx, dz, LAM, N0)
    _, Ig = oracle.bpm(dn, E0, dx, dx, dz, LAM, N0)
    assert np.max(np.abs(Ig[-1] - Ih[-1])) < 1e-12 * np.max(Ih[-1])
    # and the grating does change the slices after it when it is not last
    dn2 = np.zeros((nz, n, n))
    dn2[-2] = dn[-1]
    _, Ig2 = oracle.bpm(dn2, E0, dx, dx, dz, LAM, N0)
    assert np.max(np.abs(Ig2[-1] - Ih[-1])) > 1e-3 * np.max(Ih[-1])
