"""Pins of the annular-pupil synthesis (Bessel beams and lattices, an
illumination modality of the paper: light-sheet modalities paragraph):
spectral support and flatness, unit energy per emitter, and exact
propagation invariance when every pupil bin has the same |k_perp|."""
import numpy as np

import oracle

LAM, N0 = 0.5, 1.33


def test_annular_spectrum_is_flat_on_the_annulus_and_zero_elsewhere():
    n, d = 64, 0.1
    k = 2 * np.pi * np.fft.fftfreq(n, d)
    kp = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)
    k0 = 2 * np.pi / LAM
    na_in, na_out = 0.4, 0.6
    E = oracle.multiplex_annular(n, n, d, d, LAM, N0, [10], [23], [0.7], [0.0], na_in, na_out)
    F = np.fft.fft2(E)
    ring = (kp >= k0 * na_in) & (kp <= k0 * na_out)
    amp = np.sqrt(n * n / ring.sum())
    assert np.allclose(np.abs(F[ring]), amp, rtol=1e-12)
    assert np.max(np.abs(F[~ring])) < 1e-10
    assert abs(np.sum(np.abs(E) ** 2) - 1.0) < 1e-12                 # unit energy


def test_lattice_of_bessel_beams_has_unit_energy_per_emitter_far_apart():
    n, d = 128, 0.1
    ix = np.array([16, 48, 80, 112])
    E = oracle.multiplex_annular(n, n, d, d, LAM, N0, ix, np.full(4, 64), np.zeros(4), [0.0], 0.45, 0.55)
    single = oracle.multiplex_annular(n, n, d, d, LAM, N0, [16], [64], [0.0], [0.0], 0.45, 0.55)
    assert abs(np.sum(np.abs(single) ** 2) - 1.0) < 1e-12
    # the coherent sum is the sum of the shifted single beams (linearity)
    shifted = sum(np.roll(single, x - 16, axis=1) for x in ix)
    assert np.max(np.abs(E - shifted)) < 1e-12


def test_single_ring_of_bins_propagates_without_change():
    """An annulus containing only DFT bins with kx^2 + ky^2 = (5 dk)^2
    ((+-5, 0), (0, +-5), (+-3, +-4), (+-4, +-3)) has a single kz: its
    intensity is the same at every depth; a disk pupil of the same outer
    radius diffracts."""
    n, d = 64, 0.1
    dk = 2 * np.pi / (n * d)
    k0 = 2 * np.pi / LAM
    na_in, na_out = 4.99 * dk / k0, 5.01 * dk / k0
    E0 = oracle.multiplex_annular(n, n, d, d, LAM, N0, [20], [33], [0.0], [0.0], na_in, na_out)
    Ez, _ = oracle.bpm(np.zeros((40, n, n)), E0, d, d, d, LAM, N0, want_intensity=False)
    assert np.max(np.abs(np.abs(Ez) ** 2 - np.abs(E0) ** 2)) < 1e-12
    D0 = oracle.multiplex_psf(n, n, d, d, LAM, N0, [20], [33], [0.0], [0.0], na_out)
    Dz, _ = oracle.bpm(np.zeros((40, n, n)), D0, d, d, d, LAM, N0, want_intensity=False)
    assert np.max(np.abs(np.abs(Dz) ** 2 - np.abs(D0) ** 2)) > 1e-3
