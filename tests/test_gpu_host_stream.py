"""bpm_propagate_host (host index/intensity volumes streamed in chunks through
device ring buffers) against bpm_propagate on device buffers, and once against
the FP64 oracle directly (also on a rectangular grid)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1706_02261_b300 import inputs  # noqa: E402
from tests.gpu_util import (FIELD_TOL, INTENSITY_TOL, bandlimited_field, bandlimited_field_rect,  # noqa: E402
                            field_rel_l2, intensity_rel_max)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_02261_b300 import bpm
    return bpm


@pytest.mark.parametrize("chunk,on_device,pinned", [(3, False, True), (4, True, True), (64, False, False)])
def test_host_streaming_matches_device_path(B, chunk, on_device, pinned):
    n, nz, d = 256, 10, 0.1
    rng = np.random.default_rng(chunk)
    dn16 = rng.uniform(0, 0.05, size=(nz, n, n)).astype(np.float16)
    E0 = bandlimited_field(n, d, 0.8, chunk + 1)
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d))
    try:
        e_in = torch.from_numpy(E0).to(dev)
        e_ref = torch.empty_like(e_in)
        i_ref = torch.zeros((nz, n, n), dtype=torch.float32, device=dev)
        B.bpm_propagate(plan, torch.from_numpy(dn16).to(dev), e_in, e_ref, i_ref)
        assert B.bpm_check(plan) == 0
        dn_h = torch.from_numpy(dn16)
        e_h = torch.empty((n, n), dtype=torch.complex64)
        i_h = torch.full((nz, n, n), -1.0, dtype=torch.float32)
        if pinned:
            dn_h, e_h, i_h = dn_h.pin_memory(), e_h.pin_memory(), i_h.pin_memory()
        src = e_in if on_device else torch.from_numpy(E0)
        assert B.bpm_propagate_host(plan, dn_h, src, e_h, i_h, chunk) == B.BPM_OK
        assert field_rel_l2(e_h.numpy(), e_ref.cpu().numpy()) <= 1e-6
        assert intensity_rel_max(i_h.numpy(), i_ref.cpu().numpy()) <= 1e-6
        # the field-only variant (no intensity volume)
        e2 = torch.empty((n, n), dtype=torch.complex64)
        assert B.bpm_propagate_host(plan, dn_h, src, e2, None, chunk) == B.BPM_OK
        assert field_rel_l2(e2.numpy(), e_ref.cpu().numpy()) <= 1e-6
    finally:
        B.bpm_free(plan)


@pytest.mark.parametrize("nx,ny", [(256, 256), (512, 256)])
def test_host_streaming_matches_oracle(B, nx, ny):
    nz, d, chunk = 9, 0.1, 4
    rng = np.random.default_rng(nx + ny)
    dn16 = rng.uniform(0, 0.05, size=(nz, ny, nx)).astype(np.float16)
    E0 = bandlimited_field_rect(nx, ny, d, 0.85, 17)
    plan = B.bpm_plan(B.Instance(nx, nz, d, d, ny=ny))
    try:
        e_h = torch.empty((ny, nx), dtype=torch.complex64).pin_memory()
        i_h = torch.empty((nz, ny, nx), dtype=torch.float32).pin_memory()
        assert B.bpm_propagate_host(plan, torch.from_numpy(dn16).pin_memory(), torch.from_numpy(E0), e_h, i_h,
                                    chunk) == B.BPM_OK
    finally:
        B.bpm_free(plan)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33)
    assert field_rel_l2(e_h.numpy(), Er) <= FIELD_TOL / 10
    assert intensity_rel_max(i_h.numpy(), Ir) <= INTENSITY_TOL / 10
