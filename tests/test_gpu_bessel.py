"""Annular-pupil synthesis (Bessel beams and lattices) on the GPU against the
FP64 oracle, and the propagation invariance of a single ring of bins."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from tests.gpu_util import field_rel_l2  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_02261_b300 import bpm
    return bpm


def synth(B, n, d, ix, iy, phase, zf, na_in, na_out, annular=True):
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, 8, d, d))
    try:
        e = torch.empty((n, n), dtype=torch.complex64, device=dev)
        xyz = np.stack([np.asarray(ix) * d, np.asarray(iy) * d, np.broadcast_to(zf, len(ix))], axis=1)
        if annular:
            B.bpm_multiplex_annular(plan, 0, xyz, np.asarray(phase, float), na_in, na_out, e)
        else:
            B.bpm_multiplex_psf(plan, 0, xyz, np.asarray(phase, float), na_out, e)
        assert B.bpm_check(plan) == 0, B.bpm_last_error()
        return e.cpu().numpy()
    finally:
        B.bpm_free(plan)


@pytest.mark.parametrize("n,d", [(256, 0.1), (1024, 0.1625)])
def test_bessel_lattice_matches_oracle(B, n, d):
    rng = np.random.default_rng(n)
    ix = np.arange(8) * (n // 8) + n // 16
    iy = np.full(8, n // 2)
    ph = rng.uniform(0, 2 * np.pi, 8)
    Eg = synth(B, n, d, ix, iy, ph, 3.0, 0.5, 0.55)
    Er = oracle.multiplex_annular(n, n, d, d, 0.5, 1.33, ix, iy, ph, [3.0], 0.5, 0.55)
    assert field_rel_l2(Eg, Er) <= 1e-5


def test_zero_inner_na_is_the_disk_pupil(B):
    n, d = 256, 0.1
    ix, iy, ph = [30, 200], [40, 100], [0.3, 1.7]
    a = synth(B, n, d, ix, iy, ph, 2.0, 0.0, 0.6)
    b = synth(B, n, d, ix, iy, ph, 2.0, 0.0, 0.6, annular=False)
    assert np.array_equal(a, b)


def test_single_ring_is_propagation_invariant_on_the_gpu(B):
    n, d, nz = 64, 0.1, 40
    dk = 2 * np.pi / (n * d)
    k0 = 2 * np.pi / 0.5
    E0 = synth(B, n, d, [20], [33], [0.0], 0.0, 4.99 * dk / k0, 5.01 * dk / k0)
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d))
    try:
        e0 = torch.from_numpy(E0).to(dev)
        e1 = torch.empty_like(e0)
        I = torch.empty((nz, n, n), device=dev)
        B.bpm_propagate(plan, torch.zeros((nz, n, n), dtype=torch.float16, device=dev), e0, e1, I)
        assert B.bpm_check(plan) == 0
        Ig = I.cpu().numpy()
    finally:
        B.bpm_free(plan)
    i0 = np.abs(E0.astype(np.complex128)) ** 2
    assert np.max(np.abs(Ig - i0[None])) <= 1e-5 * i0.max()
