"""Reading B of the locally adapted expansion (BPM_FLAG_ADAPTIVE) on the GPU
against the FP64 oracle's oracle_bpm_adaptive, and its accuracy against
reading A in a uniform medium (Biobeam, arXiv:1706.02261, method paragraph)."""
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


def run(B, dn16, E0, d, flags, n0=1.33):
    nz, n, _ = dn16.shape
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d, 0.5, n0), flags=flags)
    try:
        e0 = torch.from_numpy(np.ascontiguousarray(E0, np.complex64)).to(dev)
        e1 = torch.empty_like(e0)
        I = torch.empty((nz, n, n), device=dev)
        B.bpm_propagate(plan, torch.from_numpy(dn16).to(dev), e0, e1, I)
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        return e1.cpu().numpy(), I.cpu().numpy()
    finally:
        B.bpm_free(plan)


@pytest.mark.parametrize("n", [64, 128, 192, 256, 384, 512, 1024])
@pytest.mark.parametrize("multi", [False, True])
def test_every_size_matches_adaptive_oracle(B, n, multi):
    nz = 5
    d = 0.1625 if n == 1024 else 0.1
    rng = np.random.default_rng(100 + n)
    dn16 = rng.uniform(0, 0.05, size=(nz, n, n)).astype(np.float16)     # mean step 0.025 per slice
    E0 = bandlimited_field(n, d, 0.9, n + 7)
    flags = B.BPM_FLAG_ADAPTIVE | (B.BPM_FLAG_MULTI_LAUNCH if multi else 0)
    Eg, Ig = run(B, dn16, E0, d, flags)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33, adaptive=True)
    assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10
    assert intensity_rel_max(Ig, Ir) <= INTENSITY_TOL / 10


def test_light_sheet_256_adaptive_whole_volume(B):
    w = inputs.light_sheet_256()
    dn16 = w.dn()
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(w.n, w.nz, w.d, w.d, w.lam, w.n0), flags=B.BPM_FLAG_ADAPTIVE)
    try:
        e0 = torch.empty((w.n, w.n), dtype=torch.complex64, device=dev)
        B.bpm_light_sheet(plan, 0, w.sheet_NA, w.sheet_zf(), e0)
        e1 = torch.empty_like(e0)
        I = torch.empty((w.nz, w.n, w.n), device=dev)
        B.bpm_propagate(plan, torch.from_numpy(dn16).to(dev), e0, e1, I)
        assert B.bpm_check(plan) == 0, B.bpm_last_error()
        Eg, Ig = e1.cpu().numpy(), I.cpu().numpy()
    finally:
        B.bpm_free(plan)
    E0 = oracle.light_sheet(w.n, w.n, w.d, w.d, w.lam, w.n0, w.sheet_NA, w.sheet_zf())
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, w.d, w.d, w.d, w.lam, w.n0, adaptive=True)
    assert field_rel_l2(Eg, Er) <= FIELD_TOL
    assert intensity_rel_max(Ig, Ir) <= INTENSITY_TOL


def test_uniform_medium_reading_b_beats_reading_a(B):
    n, nz, d = 128, 40, 0.1
    x = (np.arange(n) - n / 2) * d
    X, Y = np.meshgrid(x, x)
    E0 = np.exp(-(X ** 2 + Y ** 2)).astype(np.complex64)
    dn16 = np.full((nz, n, n), 0.03, np.float16)
    c = float(np.float16(0.03))
    exact, _ = oracle.bpm(np.zeros((nz, n, n)), E0, d, d, d, 0.5, 1.33 + c, want_intensity=False)
    EA, _ = run(B, dn16, E0, d, 0)
    EB, _ = run(B, dn16, E0, d, B.BPM_FLAG_ADAPTIVE)
    ea, eb = field_rel_l2(EA, exact), field_rel_l2(EB, exact)
    print(f"GPU, uniform n0 + {c:.5f}: reading A {ea:.2e}, reading B {eb:.2e}")
    assert eb < ea / 20


def test_adaptive_rejects_batched_plans(B):
    with pytest.raises(RuntimeError):
        B.bpm_plan([B.Instance(64, 4, 0.1, 0.1)] * 2, flags=B.BPM_FLAG_ADAPTIVE)
