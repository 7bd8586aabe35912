"""Pins for the oracle's input-field synthesis (Biobeam, arXiv:1706.02261,
method paragraph: one input field multiplexes many mutually independent,
non-overlapping focused PSFs; Fig. 2a: a cylindrical light sheet, NA 0.15).

* the FFT-based multiplexed synthesis equals a direct O(M J) sum of every
  emitter's pupil-limited, defocused angular spectrum;
* each focused field carries unit energy;
* after forward propagation by its focal depth a single emitter focuses back on
  its own grid point, and that depth is where its on-axis intensity peaks;
* the light sheet reaches |E|^2 = 1 at its centre after propagating to its
  focus, is uniform along y, and there has the Gaussian profile
  exp(-2 (x - x_c)^2 / w0^2), w0 = lambda / (pi NA).
"""
import numpy as np
import pytest

import oracle

LAM, N0 = 0.5, 1.33
K0 = 2 * np.pi / LAM
K = K0 * N0


def _direct_multiplex(nx, ny, dx, dy, ix, iy, phase, zf, NA):
    kx = 2 * np.pi * np.fft.fftfreq(nx, dx)
    ky = 2 * np.pi * np.fft.fftfreq(ny, dy)
    fx = np.fft.fftfreq(nx) * nx          # integer bin frequencies
    fy = np.fft.fftfreq(ny) * ny
    out = np.zeros((ny, nx), complex)
    kp2 = kx[None, :] ** 2 + ky[:, None] ** 2
    pupil = (kp2 <= (K0 * NA) ** 2) & (K * K - kp2 > 0)
    amp = np.sqrt(nx * ny / pupil.sum())
    X = np.arange(nx)
    Y = np.arange(ny)
    for j in range(len(ix)):
        kz = np.sqrt(np.where(pupil, K * K - kp2, 0.0))
        spec = amp * np.exp(1j * phase[j]) * np.exp(-1j * kz * zf[j]) * pupil
        # spectrum of a unit spike at (ix, iy), then a direct inverse sum
        spec = spec * np.exp(-2j * np.pi * (fx[None, :] * ix[j] / nx + fy[:, None] * iy[j] / ny))
        ex = np.exp(2j * np.pi * np.outer(fx, X) / nx)      # [kx, x]
        ey = np.exp(2j * np.pi * np.outer(Y, fy) / ny)      # [y, ky]
        out += ey @ spec @ ex / (nx * ny)
    return out


def test_multiplex_equals_direct_sum():
    nx, ny, dx, dy, NA = 32, 24, 0.1, 0.12, 0.6
    ix = np.array([3, 17, 28, 10])
    iy = np.array([5, 20, 2, 11])
    phase = np.array([0.3, 2.0, 4.4, 5.9])
    zf = np.array([1.2, 1.2, 0.7, 1.2])
    got = oracle.multiplex_psf(nx, ny, dx, dy, LAM, N0, ix, iy, phase, zf, NA)
    ref = _direct_multiplex(nx, ny, dx, dy, ix, iy, phase, zf, NA)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_each_focus_has_unit_energy():
    n, dx = 64, 0.1
    E = oracle.multiplex_psf(n, n, dx, dx, LAM, N0, [20], [40], [1.0], 2.0, 0.6)
    assert np.sum(np.abs(E) ** 2) == pytest.approx(1.0, rel=1e-12)


def test_single_focus_forms_at_its_depth_and_position():
    n, dx, dz, NA = 64, 0.1, 0.1, 0.6
    nz_f = 15
    zf = nz_f * dz
    ix, iy = 21, 40
    E0 = oracle.multiplex_psf(n, n, dx, dx, LAM, N0, [ix], [iy], [0.0], zf, NA)
    _, I = oracle.bpm(np.zeros((2 * nz_f, n, n)), E0, dx, dx, dz, LAM, N0)
    at_focus = I[nz_f - 1]                 # after slice nz_f - 1, depth nz_f dz
    assert np.unravel_index(np.argmax(at_focus), at_focus.shape) == (iy, ix)
    assert int(np.argmax(I[:, iy, ix])) == nz_f - 1
    # at the focus every pupil component arrives in phase, so the peak equals
    # the Cauchy-Schwarz bound n_pupil / M for a unit-energy field
    k = 2 * np.pi * np.fft.fftfreq(n, dx)
    kp2 = k[None, :] ** 2 + k[:, None] ** 2
    n_pupil = np.count_nonzero((kp2 <= (K0 * NA) ** 2) & (K * K - kp2 > 0))
    assert at_focus[iy, ix] == pytest.approx(n_pupil / (n * n), rel=1e-12)


def test_light_sheet_focus_profile():
    n, dx, dz, NA = 256, 0.1, 0.1, 0.15
    nzf = 40
    zf = nzf * dz
    E0 = oracle.light_sheet(n, n, dx, dx, LAM, N0, NA, zf)
    assert np.allclose(E0, E0[:1, :], atol=1e-14)        # uniform along y
    _, I = oracle.bpm(np.zeros((nzf, n, n)), E0, dx, dx, dz, LAM, N0)
    prof = I[-1, 7, :]
    xc = n // 2
    assert int(np.argmax(prof)) == xc
    assert prof[xc] == pytest.approx(1.0, abs=1e-12)
    w0 = LAM / (np.pi * NA)
    x = (np.arange(n) - xc) * dx
    assert np.max(np.abs(prof - np.exp(-2 * x ** 2 / w0 ** 2))) < 1e-9
