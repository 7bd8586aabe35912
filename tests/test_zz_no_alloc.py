"""The allocation-free entry point bpm_propagate_static against bpm_propagate.

bpm_propagate_static serves callers that cannot allocate device memory (a
host application whose allocator owns the device, a loop that cannot afford
cudaMalloc's synchronisation, code that must not fail on memory after
start-up).  It keeps its tables in one fixed device array inside the library,
shared by every call, so this test makes calls in a row with different
grids and spacings (every grid it accepts) and checks that each matches the
plan-based entry point within the parity tolerances; one more call is checked
against the FP64 oracle directly.  The file is named to be collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1706_02261_b300 import inputs  # noqa: E402
from tests.gpu_util import FIELD_TOL, INTENSITY_TOL, bandlimited_field, field_rel_l2, intensity_rel_max  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_02261_b300 import bpm
    return bpm


def _case(n, nz, d, seed):
    rng = np.random.default_rng(seed)
    dn16 = rng.uniform(0, 0.05, size=(nz, n, n)).astype(np.float16)
    return dn16, bandlimited_field(n, d, 0.85, seed + 1)


def _with_plan(B, inst, dn, e0):
    plan = B.bpm_plan(inst)
    try:
        out = torch.empty_like(e0)
        inten = torch.zeros((inst.nz, inst.n, inst.n), dtype=torch.float32, device=e0.device)
        B.bpm_propagate(plan, dn, e0, out, inten)
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        return out.cpu().numpy(), inten.cpu().numpy()
    finally:
        B.bpm_free(plan)


def test_static_entry_point_matches_plan_path_twice(B):
    dev = torch.device("cuda")
    # every grid the entry point accepts (the rolled-loop 64, the unrolled 128,
    # 192 and 256 transforms, whose twiddle tables differ in layout), called
    # back to back with different grids and spacings on the one shared array
    cases = [(B.Instance(256, 6, 0.1, 0.1), 21), (B.Instance(192, 5, 0.12, 0.15), 22),
             (B.Instance(64, 7, 0.1, 0.1), 23), (B.Instance(128, 4, 0.11, 0.1), 24),
             (B.Instance(64, 3, 0.09, 0.12), 25)]
    for inst, seed in cases:
        dn16, E0 = _case(inst.n, inst.nz, inst.dx, seed)
        dn = torch.from_numpy(dn16).to(dev)
        e0 = torch.from_numpy(E0).to(dev)
        out = torch.empty_like(e0)
        inten = torch.zeros((inst.nz, inst.n, inst.n), dtype=torch.float32, device=dev)
        assert B.bpm_propagate_static(inst, dn, e0, out, inten) == B.BPM_OK
        Es, Is = out.cpu().numpy(), inten.cpu().numpy()
        Ep, Ip = _with_plan(B, inst, dn, e0)
        assert field_rel_l2(Es, Ep) <= FIELD_TOL
        assert intensity_rel_max(Is, Ip) <= INTENSITY_TOL


def test_static_entry_point_matches_oracle(B):
    """One call checked against the FP64 oracle directly (not only through
    the plan path), on the rolled-loop size."""
    dev = torch.device("cuda")
    inst = B.Instance(64, 12, 0.1, 0.1)
    dn16, E0 = _case(inst.n, inst.nz, inst.dx, 31)
    e0 = torch.from_numpy(E0).to(dev)
    out = torch.empty_like(e0)
    inten = torch.zeros((inst.nz, inst.n, inst.n), dtype=torch.float32, device=dev)
    assert B.bpm_propagate_static(inst, torch.from_numpy(dn16).to(dev), e0, out, inten) == B.BPM_OK
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, inst.dx, inst.dx, inst.dz, inst.lam, inst.n0)
    assert field_rel_l2(out.cpu().numpy(), Er) <= FIELD_TOL
    assert intensity_rel_max(inten.cpu().numpy(), Ir) <= INTENSITY_TOL


def test_static_entry_point_rejects_large_grids(B):
    dev = torch.device("cuda")
    inst = B.Instance(512, 2, 0.1, 0.1)
    dn = torch.zeros((2, 512, 512), dtype=torch.float16, device=dev)
    e = torch.zeros((512, 512), dtype=torch.complex64, device=dev)
    with pytest.raises(B.BpmError) as ei:
        B.bpm_propagate_static(inst, dn, e, e, None)
    assert ei.value.code == B.BPM_ERR_UNSUPPORTED
    assert "256" in str(ei.value)
