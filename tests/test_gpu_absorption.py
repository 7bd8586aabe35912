"""Complex refractive index (absorption) on the GPU against the FP64 oracle,
Beer-Lambert decay, and the combinations the library rejects."""
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


def run(B, dn16, kap16, E0, d, flags=0):
    nz, n, _ = dn16.shape
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d), flags=flags)
    try:
        e0 = torch.from_numpy(np.ascontiguousarray(E0, np.complex64)).to(dev)
        e1 = torch.empty_like(e0)
        I = torch.empty((nz, n, n), device=dev)
        B.bpm_propagate_absorbing(plan, torch.from_numpy(dn16).to(dev), torch.from_numpy(kap16).to(dev), e0, e1, I)
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        return e1.cpu().numpy(), I.cpu().numpy()
    finally:
        B.bpm_free(plan)


@pytest.mark.parametrize("n,flags", [(64, 0), (256, 0), (256, 2), (1024, 0)])
def test_absorbing_matches_oracle(B, n, flags):
    nz = 6
    d = 0.1625 if n == 1024 else 0.1
    rng = np.random.default_rng(7 * n + flags)
    dn16 = rng.uniform(0, 0.05, size=(nz, n, n)).astype(np.float16)
    kap16 = rng.uniform(0, 0.004, size=(nz, n, n)).astype(np.float16)
    E0 = bandlimited_field(n, d, 0.9, n + 3)
    Eg, Ig = run(B, dn16, kap16, E0, d, flags)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33, kappa=inputs.dn_to_f64(kap16))
    assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10
    assert intensity_rel_max(Ig, Ir) <= INTENSITY_TOL / 10


def test_beer_lambert_on_the_gpu(B):
    n, nz, d = 128, 30, 0.1
    x = (np.arange(n) - n / 2) * d
    X, Y = np.meshgrid(x, x)
    E0 = np.exp(-(X ** 2 + Y ** 2) / 0.5).astype(np.complex64)
    kap = np.float16(0.002)
    _, I = run(B, np.zeros((nz, n, n), np.float16), np.full((nz, n, n), kap), E0, d)
    k0 = 2 * np.pi / 0.5
    P = I.astype(np.float64).sum(axis=(1, 2)) / np.sum(np.abs(E0.astype(np.complex128)) ** 2)
    expect = np.exp(-2 * k0 * float(kap) * d * (np.arange(nz) + 1))
    assert np.max(np.abs(P / expect - 1)) < 1e-5


def test_absorption_rejections(B):
    dev = torch.device("cuda")
    z = torch.zeros((2, 64, 64), dtype=torch.float16, device=dev)
    e = torch.zeros((64, 64), dtype=torch.complex64, device=dev)
    plan = B.bpm_plan(B.Instance(64, 2, 0.1, 0.1), flags=B.BPM_FLAG_ADAPTIVE)
    try:
        with pytest.raises(RuntimeError):
            B.bpm_propagate_absorbing(plan, z, z, e, e)
    finally:
        B.bpm_free(plan)
