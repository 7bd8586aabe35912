"""Shared helpers for the GPU parity tests (imported only by tests)."""
import numpy as np


def field_rel_l2(got, ref) -> float:
    got = np.asarray(got, np.complex128)
    ref = np.asarray(ref, np.complex128)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def intensity_rel_max(got, ref) -> float:
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref)) / np.max(ref))


# Tolerances: relative L2 error of the field after up to 256 slices and the
# peak-normalised maximum intensity error, FP32 path against the FP64 oracle on
# the same FP16 index values.
FIELD_TOL = 1e-4
INTENSITY_TOL = 1e-3


def bandlimited_field(n, dx, frac, seed, lam=0.5, n0=1.33):
    """Random complex field whose spectrum lies inside |k| < frac k0 n0."""
    rng = np.random.default_rng(seed)
    k = 2 * np.pi * np.fft.fftfreq(n, dx)
    kp = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)
    K = 2 * np.pi / lam * n0
    spec = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * (kp < frac * K)
    e = np.fft.ifft2(spec)
    e /= np.sqrt(np.mean(np.abs(e) ** 2))
    return e.astype(np.complex64)


def bandlimited_field_rect(nx, ny, dx, frac, seed, lam=0.5, n0=1.33, dy=None):
    """As bandlimited_field on an ny x nx grid (rows of nx points)."""
    dy = dx if dy is None else dy
    rng = np.random.default_rng(seed)
    kx = 2 * np.pi * np.fft.fftfreq(nx, dx)
    ky = 2 * np.pi * np.fft.fftfreq(ny, dy)
    kp = np.sqrt(kx[None, :] ** 2 + ky[:, None] ** 2)
    K = 2 * np.pi / lam * n0
    spec = (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))) * (kp < frac * K)
    e = np.fft.ifft2(spec)
    e /= np.sqrt(np.mean(np.abs(e) ** 2))
    return e.astype(np.complex64)
