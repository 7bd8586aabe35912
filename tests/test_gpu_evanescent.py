"""GPU parity with evanescent content: the propagator's cut of kz^2 <= 0
(method paragraph: the exact propagator keeps propagating waves only).

Every other GPU input is band-limited inside the cut, so these cases feed the
device a white spectrum, whose bins beyond |k_perp| = k0 n0 must be removed in
the first slice exactly as the oracle removes them, and a grid on which some
bins sit exactly on the cut (kz^2 = 0 in FP64), which both sides must drop.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1706_02261_b300 import inputs  # noqa: E402
from tests.gpu_util import FIELD_TOL, INTENSITY_TOL, field_rel_l2, intensity_rel_max  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_02261_b300 import bpm
    return bpm


def white_field(n, seed):
    """Complex Gaussian noise per pixel: every DFT bin populated, the
    evanescent ones included."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)


def run_gpu(B, dn16, E0, d, lam, n0, flags=0):
    nz, n, _ = dn16.shape
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d, lam, n0), flags=flags)
    try:
        e_in = torch.from_numpy(E0).to(dev)
        e_out = torch.empty_like(e_in)
        I = torch.zeros((nz, n, n), dtype=torch.float32, device=dev)
        B.bpm_propagate(plan, torch.from_numpy(dn16).to(dev), e_in, e_out, I)
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        return e_out.cpu().numpy(), I.cpu().numpy()
    finally:
        B.bpm_free(plan)


@pytest.mark.parametrize("n", [64, 128, 192, 256, 384, 512, 1024])
@pytest.mark.parametrize("flags", [0, 2])
def test_white_spectrum_every_size(B, n, flags):
    # dx = 0.1 um at lambda 0.5 um, n0 1.33: k0 n0 = 16.7 rad/um against a
    # Nyquist wavenumber of 31.4 rad/um, so the propagating disk holds
    # pi 16.7^2 / 62.8^2 = 22 % of the bins and about 78 % of the input's
    # power is evanescent
    nz, d, lam, n0 = 4, 0.1, 0.5, 1.33
    rng = np.random.default_rng(5 * n + flags)
    dn16 = rng.uniform(0, 0.05, size=(nz, n, n)).astype(np.float16)
    E0 = white_field(n, n + 11)
    Eg, Ig = run_gpu(B, dn16, E0, d, lam, n0, flags)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, lam, n0)
    # the cut removed most of the input's power on both sides
    kept = float(np.sum(np.abs(Er) ** 2) / np.sum(np.abs(E0.astype(np.complex128)) ** 2))
    assert 0.15 < kept < 0.3, kept
    assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10
    assert intensity_rel_max(Ig, Ir) <= INTENSITY_TOL / 10


def _tie_grid():
    # N = 64, dx = 0.125 um, lambda = 0.5 um, n0 = 1: k0 n0 = 4 pi and the DFT
    # bin 16 has |kx| = 2 pi 16 / (64 * 0.125) = 4 pi, both exact in FP64, so
    # the bins (+-16, 0) and (0, +-16) have kz^2 = 0 exactly
    n, d, lam, n0 = 64, 0.125, 0.5, 1.0
    k = 2 * np.pi * np.fft.fftfreq(n, d)
    K = 2 * np.pi / lam * n0
    assert K * K - k[16] ** 2 == 0.0
    return n, d, lam, n0


@pytest.mark.parametrize("flags", [0, 2])
def test_exact_tie_bins_are_cut_homogeneous(B, flags):
    """In a homogeneous medium the output spectrum at the tie bins must be
    zero (the screen is a constant phase and cannot refill them)."""
    n, d, lam, n0 = _tie_grid()
    nz = 3
    dn16 = np.zeros((nz, n, n), np.float16)
    E0 = white_field(n, 77)
    Eg, _ = run_gpu(B, dn16, E0, d, lam, n0, flags)
    Fg = np.fft.fft2(Eg.astype(np.complex128))
    tie = np.array([abs(Fg[0, 16]), abs(Fg[0, 48]), abs(Fg[16, 0]), abs(Fg[48, 0])])
    near = np.array([abs(Fg[0, 15]), abs(Fg[0, 49]), abs(Fg[15, 0]), abs(Fg[49, 0])])
    assert np.all(near > 1.0)                       # the neighbours inside the cut carry power
    assert np.all(tie <= 1e-5 * np.abs(Fg).max())   # the tie bins carry none
    Er, _ = oracle.bpm(np.zeros((nz, n, n)), E0, d, d, d, lam, n0)
    assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10


@pytest.mark.parametrize("flags", [0, 2])
def test_exact_tie_grid_through_index_steps(B, flags):
    n, d, lam, n0 = _tie_grid()
    nz = 6
    rng = np.random.default_rng(91 + flags)
    dn16 = rng.uniform(0, 0.05, size=(nz, n, n)).astype(np.float16)
    E0 = white_field(n, 78)
    Eg, Ig = run_gpu(B, dn16, E0, d, lam, n0, flags)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, lam, n0)
    assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10
    assert intensity_rel_max(Ig, Ir) <= INTENSITY_TOL / 10
