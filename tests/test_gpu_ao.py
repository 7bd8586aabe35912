"""Adaptive optics by guide-star phase conjugation on the GPU: reverse
propagation against the oracle (slices in reverse order), the refocusing
identity in a homogeneous medium, the whole chain against the same chain in
the oracle, and focus recovery in Perlin-noise tissue (n = 1.36 +- 0.03)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1706_02261_b300 import inputs  # noqa: E402
from tests.gpu_util import (FIELD_TOL, INTENSITY_TOL, bandlimited_field,  # noqa: E402
                            field_rel_l2, intensity_rel_max)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_02261_b300 import bpm
    return bpm


@pytest.mark.parametrize("n,flags", [(128, 0), (128, 2), (1024, 0)])
def test_reverse_propagation_matches_oracle_on_flipped_slices(B, n, flags):
    nz, zb, ze = 9, 2, 8
    d = 0.1625 if n == 1024 else 0.1
    rng = np.random.default_rng(n + flags)
    dn16 = rng.uniform(0, 0.05, size=(nz, n, n)).astype(np.float16)
    E0 = bandlimited_field(n, d, 0.8, 5)
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d), flags=flags)
    try:
        e0 = torch.from_numpy(E0).to(dev)
        e1 = torch.empty_like(e0)
        I = torch.full((nz, n, n), -1.0, device=dev)
        B.bpm_propagate_reverse(plan, torch.from_numpy(dn16).to(dev), e0, e1, I, zb, ze)
        assert B.bpm_check(plan) == 0, B.bpm_last_error()
        Eg, Ig = e1.cpu().numpy(), I.cpu().numpy()
    finally:
        B.bpm_free(plan)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16[zb:ze][::-1]), E0, d, d, d, 0.5, 1.33)
    assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10
    assert intensity_rel_max(Ig[zb:ze][::-1], Ir) <= INTENSITY_TOL / 10
    assert np.all(Ig[:zb] == -1.0) and np.all(Ig[ze:] == -1.0)


def run_chain(B, dn16, star, NA, d):
    from paper_1706_02261_b300 import ao
    nz, n, _ = dn16.shape
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d))
    try:
        e_corr, i_corr, i_plain = ao.focus_planes(plan, torch.from_numpy(dn16).to(dev), star, NA, d)
        assert B.bpm_check(plan) == 0, B.bpm_last_error()
        return e_corr.cpu().numpy(), i_corr.cpu().numpy(), i_plain.cpu().numpy()
    finally:
        B.bpm_free(plan)


def oracle_chain(dn16, star, NA, d):
    ix, iy, iz = star
    n = dn16.shape[-1]
    dn64 = inputs.dn_to_f64(dn16[:iz + 1])
    s = oracle.multiplex_psf(n, n, d, d, 0.5, 1.33, [ix], [iy], [0.0], [0.0], NA)
    es, _ = oracle.bpm(dn64[::-1], s, d, d, d, 0.5, 1.33, want_intensity=False)
    _, I = oracle.bpm(dn64, np.conj(es), d, d, d, 0.5, 1.33)
    return np.conj(es), I[iz], np.abs(s) ** 2


def test_homogeneous_medium_refocuses_to_the_guide_star(B):
    n, nz, d = 128, 40, 0.1
    star = (40, 70, 30)
    dn16 = np.zeros((nz, n, n), np.float16)
    _, i_corr, _ = run_chain(B, dn16, star, 0.6, d)
    _, _, point = oracle_chain(dn16, star, 0.6, d)
    # conj(P^-1 s) propagated by P is s itself on the propagating band
    assert intensity_rel_max(i_corr, point) <= INTENSITY_TOL


def test_chain_matches_oracle_in_tissue(B):
    n, nz, d = 128, 40, 0.1
    star = (64, 64, 34)
    dn16 = inputs.perlin_phantom_dn((nz, n, n), d, seed=11)
    e_corr, i_corr, _ = run_chain(B, dn16, star, 0.6, d)
    er, ir, _ = oracle_chain(dn16, star, 0.6, d)
    assert field_rel_l2(e_corr, er) <= FIELD_TOL
    assert intensity_rel_max(i_corr, ir) <= INTENSITY_TOL


def test_focus_recovery_in_perlin_tissue(B):
    """256^2 x 150 slices of 0.1 um Perlin tissue, star 15 um deep: the
    conjugated wavefront forms a diffraction-limited focus on the star (the
    peak and encircled power of the same focus without tissue), the focus
    aimed at the star through the tissue does not."""
    from paper_1706_02261_b300 import ao
    n, nz, d = 256, 150, 0.1
    star = (128, 128, 149)
    dn16 = inputs.perlin_phantom_dn((nz, n, n), d, seed=4)
    _, i_corr, i_plain = run_chain(B, dn16, star, 0.6, d)
    _, i_free, _ = run_chain(B, np.zeros_like(dn16), star, 0.6, d)
    peak = lambda I: float(I[star[1], star[0]])
    ec, ep, ef = (ao.encircled(I, star[0], star[1], 3) for I in (i_corr, i_plain, i_free))
    print(f"star peak: corrected {peak(i_corr):.3e}, uncorrected {peak(i_plain):.3e}, no tissue {peak(i_free):.3e}; "
          f"power within 3 px: {ec:.3f} / {ep:.3f} / {ef:.3f}")
    # diffraction-limited focus through the tissue with the conjugated
    # wavefront; the focus aimed at the star without correction is degraded
    assert peak(i_corr) > 0.9 * peak(i_free)
    assert peak(i_plain) < 0.6 * peak(i_free)
    assert ec > 0.9 * ef and ep < 0.6 * ef
    my, mx = np.unravel_index(np.argmax(i_corr), i_corr.shape)
    assert abs(int(mx) - star[0]) <= 1 and abs(int(my) - star[1]) <= 1
