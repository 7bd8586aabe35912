"""Pins of reading B of the locally adapted expansion (oracle_bpm_adaptive):
per slice the mean index step delta_z is the reference, the propagator is the
exact one of the medium n0 + delta_z to first order in delta_z, and the
screen acts on dn - delta_z (Biobeam, arXiv:1706.02261, method paragraph)."""
import numpy as np

import oracle

LAM, N0, D = 0.5, 1.33, 0.1


def test_zero_mean_slices_give_reading_a():
    rng = np.random.default_rng(1)
    dn = rng.uniform(-0.02, 0.05, (6, 64, 64))
    dn -= dn.mean(axis=(1, 2), keepdims=True)
    E0 = np.exp(1j * rng.uniform(0, 6, (64, 64)))
    A, IA = oracle.bpm(dn, E0, D, D, D, LAM, N0)
    B, IB = oracle.bpm(dn, E0, D, D, D, LAM, N0, adaptive=True)
    assert np.max(np.abs(A - B)) < 1e-12 and np.max(np.abs(IA - IB)) < 1e-12


def test_uniform_slices_tilted_plane_wave_closed_forms():
    """A plane wave on DFT bin (m, 0) through slices of uniform index steps
    c_z: reading B multiplies by exp(i (kz0 + c_z k0^2 n0 / kz0) dz) per slice,
    reading A by exp(i (kz0 + k0 c_z) dz)."""
    n, m, nz = 64, 9, 7
    k0 = 2 * np.pi / LAM
    K = k0 * N0
    kx = 2 * np.pi * m / (n * D)
    kz0 = np.sqrt(K * K - kx * kx)
    c = 0.01 + 0.004 * np.arange(nz)
    x = np.arange(n) * D
    E0 = np.tile(np.exp(1j * kx * x), (n, 1))
    dn = np.broadcast_to(c[:, None, None], (nz, n, n)).copy()
    B, _ = oracle.bpm(dn, E0, D, D, D, LAM, N0, adaptive=True)
    A, _ = oracle.bpm(dn, E0, D, D, D, LAM, N0)
    phase_b = np.sum((kz0 + c * k0 * k0 * N0 / kz0) * D)
    phase_a = np.sum((kz0 + k0 * c) * D)
    assert np.max(np.abs(B - E0 * np.exp(1j * phase_b))) < 1e-11
    assert np.max(np.abs(A - E0 * np.exp(1j * phase_a))) < 1e-11
    # and the two differ by the first-order obliquity term k0 c (k0 n0 / kz0 - 1) dz
    assert abs(phase_b - phase_a - np.sum(k0 * c * (K / kz0 - 1) * D)) < 1e-12


def test_reading_b_beats_reading_a_in_a_uniform_medium():
    """A Gaussian beam (waist 1 um) through 40 slices of n = 1.36: the exact
    answer is the background-free propagation with n0 = 1.36; reading B's
    error is second order in the index step, reading A's first order."""
    n, nz = 128, 40
    x = (np.arange(n) - n / 2) * D
    X, Y = np.meshgrid(x, x)
    E0 = np.exp(-(X ** 2 + Y ** 2)).astype(complex)
    dn = np.full((nz, n, n), 0.03)
    exact, _ = oracle.bpm(np.zeros((nz, n, n)), E0, D, D, D, LAM, N0 + 0.03, want_intensity=False)
    A, _ = oracle.bpm(dn, E0, D, D, D, LAM, N0, want_intensity=False)
    B, _ = oracle.bpm(dn, E0, D, D, D, LAM, N0, want_intensity=False, adaptive=True)
    ea = np.linalg.norm(A - exact) / np.linalg.norm(exact)
    eb = np.linalg.norm(B - exact) / np.linalg.norm(exact)
    print(f"uniform n = 1.36, Gaussian w0 = 1 um, 4 um: reading A {ea:.2e}, reading B {eb:.2e}")
    assert eb < ea / 20
