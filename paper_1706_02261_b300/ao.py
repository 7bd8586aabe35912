"""Adaptive optics by guide-star phase conjugation (Biobeam, arXiv:1706.02261,
adaptive-optics paragraph, Fig. 2c): a point-like guide star inside the
sample emits; its wave, propagated through the sample back to the surface,
is phase-conjugated there and launched forward, and refocuses at the star
through the scattering tissue.  All arithmetic runs in libbpm.so:

    bpm_multiplex_psf        the guide star: one pupil-limited point (NA) at
                             its own plane (focal depth 0)
    bpm_propagate_reverse    slices iz .. 0, star plane -> surface
    bpm_phase_conjugate      the corrected input wavefront
    bpm_propagate_window     forward to the star plane, |E|^2 of that plane

The uncorrected reference is a focused wave aimed at the star from the
surface (bpm_multiplex_psf with the star's depth), propagated the same way.
A star "at slice iz" sits at the exit plane of slice iz, depth (iz + 1) dz.
"""
from __future__ import annotations

import numpy as np

from . import bpm as B


def focus_planes(plan, dn, star, NA: float, d: float, stream=None):
    """(corrected input field, corrected |E|^2 at the star plane, uncorrected
    |E|^2 at the star plane) as device tensors, for star = (ix, iy, iz)."""
    import torch
    ix, iy, iz = (int(v) for v in star)
    n = dn.shape[-1]
    dev = dn.device
    e_star = torch.empty((n, n), dtype=torch.complex64, device=dev)
    B.bpm_multiplex_psf(plan, 0, np.array([[ix * d, iy * d, 0.0]]), np.zeros(1), NA, e_star, stream)
    e_corr = torch.empty_like(e_star)
    B.bpm_propagate_reverse(plan, dn, e_star, e_corr, None, 0, iz + 1, stream)
    B.bpm_phase_conjugate(plan, 0, e_corr, stream)
    out = torch.empty_like(e_star)
    i_corr = torch.empty((1, n, n), dtype=torch.float32, device=dev)
    B.bpm_propagate_window(plan, dn, e_corr, out, i_corr, iz, iz + 1, 0, iz + 1, stream)
    e_plain = torch.empty_like(e_star)
    B.bpm_multiplex_psf(plan, 0, np.array([[ix * d, iy * d, (iz + 1) * d]]), np.zeros(1), NA, e_plain, stream)
    i_plain = torch.empty_like(i_corr)
    B.bpm_propagate_window(plan, dn, e_plain, out, i_plain, iz, iz + 1, 0, iz + 1, stream)
    return e_corr, i_corr[0], i_plain[0]


def encircled(I: np.ndarray, ix: int, iy: int, radius_px: float) -> float:
    """Fraction of the plane's power within radius_px of (ix, iy), periodic."""
    n = I.shape[0]
    y = (np.arange(n) - iy + n // 2) % n - n // 2
    x = (np.arange(n) - ix + n // 2) % n - n // 2
    r2 = y[:, None] ** 2 + x[None, :] ** 2
    return float(I[r2 <= radius_px ** 2].sum() / I.sum())
