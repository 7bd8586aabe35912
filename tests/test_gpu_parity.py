"""GPU parity: the CUDA split-step BPM (through the C ABI) against the FP64
oracle on identical seeded inputs (Biobeam, arXiv:1706.02261, method
paragraph).  Gates: field relative L2 error <= 1e-4, peak-normalised intensity
error <= 1e-3."""
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


def run_gpu(B, dn16, E0, d, lam=0.5, n0=1.33, flags=0, want_I=True, z_begin=0, z_end=None):
    nz, n, _ = dn16.shape
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d, lam, n0), flags=flags)
    try:
        dn_t = torch.from_numpy(dn16).to(dev)
        e_in = torch.from_numpy(np.ascontiguousarray(E0, np.complex64)).to(dev)
        e_out = torch.empty_like(e_in)
        I = torch.zeros((nz, n, n), dtype=torch.float32, device=dev) if want_I else None
        B.bpm_propagate(plan, dn_t, e_in, e_out, I, z_begin, nz if z_end is None else z_end)
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        torch.cuda.synchronize()
        return e_out.cpu().numpy(), (I.cpu().numpy() if want_I else None)
    finally:
        B.bpm_free(plan)


def test_sphere64_full(B):
    w = inputs.single_sphere_64()
    dn16 = w.dn()
    E0 = inputs.plane_wave(w.n, w.n)
    Eg, Ig = run_gpu(B, dn16, E0, w.d)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, w.d, w.d, w.d, w.lam, w.n0)
    ef, ei = field_rel_l2(Eg, Er), intensity_rel_max(Ig, Ir)
    print(f"64^3 sphere: field rel L2 {ef:.2e}, intensity max rel {ei:.2e}")
    assert ef <= FIELD_TOL
    assert ei <= INTENSITY_TOL


@pytest.mark.parametrize("n", [64, 128, 192, 256, 384, 512, 1024])
@pytest.mark.parametrize("flags", [0, 2])
def test_every_size_random_inputs(B, n, flags):
    nz = 5
    d = 0.1625 if n == 1024 else 0.1
    rng = np.random.default_rng(n)
    dn16 = rng.uniform(0, 0.05, size=(nz, n, n)).astype(np.float16)
    E0 = bandlimited_field(n, d, 0.9, n + 1)
    Eg, Ig = run_gpu(B, dn16, E0, d, flags=flags)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33)
    assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10
    assert intensity_rel_max(Ig, Ir) <= INTENSITY_TOL / 10


@pytest.mark.parametrize("n", [64, 128, 192, 256, 384, 512, 1024])
def test_every_size_every_phasor_form(B, n):
    """The screen picks its phasor per warp from the largest |k0 dn dz| of the
    warp's elements: the short series (<= 1/8), the long one (<= pi/4) or
    sincosf.  Slice 0 stays in the first, slice 1 reaches the second, slice 2
    mixes rows of small steps with rows of steps up to +-1.4 rad, negative
    ones included, so that warps of every form (and warps whose rows need
    different forms) meet in one propagation."""
    nz, d = 3, 0.1
    rng = np.random.default_rng(7 * n + 1)
    dn = np.empty((nz, n, n))
    dn[0] = rng.uniform(0.0, 0.05, size=(n, n))
    dn[1] = rng.uniform(0.0, 0.4, size=(n, n))
    dn[2] = rng.uniform(-1.1, 1.1, size=(n, n))
    dn[2, ::3] = rng.uniform(0.0, 0.05, size=dn[2, ::3].shape)
    dn16 = dn.astype(np.float16)
    k0dz = 2 * np.pi / 0.5 * d
    ph = np.abs(dn16.astype(np.float64)) * k0dz
    assert ph[0].max() <= 0.125 and 0.125 < ph[1].max() <= np.pi / 4 and ph[2].max() > np.pi / 4
    E0 = bandlimited_field(n, d, 0.9, n + 3)
    Eg, Ig = run_gpu(B, dn16, E0, d)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33)
    assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10
    assert intensity_rel_max(Ig, Ir) <= INTENSITY_TOL / 10


def test_multiplex_synthesis_1024(B):
    w = inputs.multiplex_1024(nz=64)
    f = w.foci()
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(w.n, w.nz, w.d, w.d))
    try:
        e = torch.empty((w.n, w.n), dtype=torch.complex64, device=dev)
        B.bpm_multiplex_psf(plan, 0, f.xyz_um(w.d, w.d), f.phase, f.NA, e)
        assert B.bpm_check(plan) == 0
        Eg = e.cpu().numpy()
    finally:
        B.bpm_free(plan)
    Er = oracle.multiplex_psf(w.n, w.n, w.d, w.d, w.lam, w.n0, f.ix, f.iy, f.phase, f.zf, f.NA)
    ef = field_rel_l2(Eg, Er)
    print(f"1024^2 multiplexed synthesis (32 x 32 foci): field rel L2 {ef:.2e}")
    assert ef <= 1e-5


def test_multiplex_two_depths_and_outside_emitters(B):
    n, d = 128, 0.1
    ix = np.array([10, 70, 100, 40, 500])        # the last one lies outside the grid
    iy = np.array([20, 64, 3, 99, 5])
    ph = np.array([0.1, 1.2, 2.3, 3.4, 4.5])
    zf = np.array([2.0, 2.0, 3.5, 2.0, 2.0])
    xyz = np.stack([ix * d, iy * d, zf], axis=1)
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, 8, d, d))
    try:
        e = torch.empty((n, n), dtype=torch.complex64, device=dev)
        B.bpm_multiplex_psf(plan, 0, xyz, ph, 0.6, e)
        assert B.bpm_check(plan) == 0
        Eg = e.cpu().numpy()
    finally:
        B.bpm_free(plan)
    keep = ix < n
    Er = oracle.multiplex_psf(n, n, d, d, 0.5, 1.33, ix[keep], iy[keep], ph[keep], zf[keep], 0.6)
    assert field_rel_l2(Eg, Er) <= 1e-5


def test_light_sheet_256(B):
    w = inputs.light_sheet_256()
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(w.n, w.nz, w.d, w.d))
    try:
        e = torch.empty((w.n, w.n), dtype=torch.complex64, device=dev)
        B.bpm_light_sheet(plan, 0, w.sheet_NA, w.sheet_zf(), e)
        assert B.bpm_check(plan) == 0
        Eg = e.cpu().numpy()
    finally:
        B.bpm_free(plan)
    Er = oracle.light_sheet(w.n, w.n, w.d, w.d, w.lam, w.n0, w.sheet_NA, w.sheet_zf())
    assert field_rel_l2(Eg, Er) <= 1e-5


def test_split_run_and_in_place(B):
    n, nz, d = 128, 12, 0.1
    rng = np.random.default_rng(11)
    dn16 = rng.uniform(0, 0.05, size=(nz, n, n)).astype(np.float16)
    E0 = bandlimited_field(n, d, 0.8, 12)
    Efull, Ifull = run_gpu(B, dn16, E0, d)
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d))
    try:
        dn_t = torch.from_numpy(dn16).to(dev)
        e = torch.from_numpy(E0).to(dev)
        I = torch.full((nz, n, n), -1.0, dtype=torch.float32, device=dev)
        B.bpm_propagate(plan, dn_t, e, e, I, 0, 5)      # in place
        B.bpm_propagate(plan, dn_t, e, e, I, 5, nz)
        assert B.bpm_check(plan) == 0
        Esplit, Isplit = e.cpu().numpy(), I.cpu().numpy()
        # empty range: output equals input
        e2 = torch.empty_like(e)
        B.bpm_propagate(plan, dn_t, e, e2, None, 3, 3)
        assert torch.equal(e2, e)
    finally:
        B.bpm_free(plan)
    assert field_rel_l2(Esplit, Efull) <= 1e-6
    assert intensity_rel_max(Isplit, Ifull) <= 1e-6


def test_nan_in_index_is_reported(B):
    n, nz, d = 64, 3, 0.1
    dn16 = np.zeros((nz, n, n), np.float16)
    dn16[1, 5, 7] = np.float16(np.nan)
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d))
    try:
        e = torch.ones((n, n), dtype=torch.complex64, device=dev)
        out = torch.empty_like(e)
        B.bpm_propagate(plan, torch.from_numpy(dn16).to(dev), e, out, None)
        assert B.bpm_check(plan) == B.BPM_ERR_NAN
        assert B.bpm_check(plan) == B.BPM_OK          # cleared after reporting
    finally:
        B.bpm_free(plan)


def test_barrier_timeout_is_reported_and_context_survives(B):
    # One barrier waits for an arrival that never comes; the bounded wait runs
    # out after 2 ms, every CTA leaves the kernel and the status says so.
    n, nz, d = 256, 4, 0.1
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d))
    try:
        B.bpm_debug_set_barrier_timeout(plan, 2_000_000, 1)
        dn_t = torch.zeros((nz, n, n), dtype=torch.float16, device=dev)
        e = torch.ones((n, n), dtype=torch.complex64, device=dev)
        out = torch.empty_like(e)
        B.bpm_propagate(plan, dn_t, e, out, None)
        assert B.bpm_check(plan) == B.BPM_ERR_TIMEOUT
        B.bpm_debug_set_barrier_timeout(plan, 2_000_000_000, 0)
        B.bpm_propagate(plan, dn_t, e, out, None)
        assert B.bpm_check(plan) == B.BPM_OK
    finally:
        B.bpm_free(plan)
    torch.cuda.synchronize()


@pytest.mark.parametrize("n", [256, 1024])
def test_exchange_timeout_is_reported_and_context_survives(B, n):
    # The entrance field carries the parity the row half-steps write, so the
    # first column half-step polls for elements that never arrive; the bounded
    # wait runs out after 2 ms, every CTA leaves the kernel and the status says
    # so.  The same plan then propagates correctly.
    nz, d = 4, 0.1
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d))
    try:
        assert B.bpm_plan_info(plan)["persistent"] == 1
        rng = np.random.default_rng(n)
        dn16 = rng.uniform(0.0, 0.05, size=(nz, n, n)).astype(np.float16)
        dn_t = torch.from_numpy(dn16).to(dev)
        E0 = bandlimited_field(n, d, 0.9, n + 1)
        e = torch.from_numpy(np.ascontiguousarray(E0, np.complex64)).to(dev)
        out = torch.empty_like(e)
        B.bpm_debug_set_barrier_timeout(plan, 2_000_000, 0)
        B.bpm_debug_stall_exchange(plan, True)
        B.bpm_propagate(plan, dn_t, e, out, None)
        assert B.bpm_check(plan) == B.BPM_ERR_TIMEOUT
        B.bpm_debug_stall_exchange(plan, False)
        B.bpm_debug_set_barrier_timeout(plan, 2_000_000_000, 0)
        B.bpm_propagate(plan, dn_t, e, out, None)
        assert B.bpm_check(plan) == B.BPM_OK
        Er, _ = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33)
        assert field_rel_l2(out.cpu().numpy(), Er) <= FIELD_TOL / 10
    finally:
        B.bpm_free(plan)
    torch.cuda.synchronize()


def test_argument_errors(B):
    dev = torch.device("cuda")
    with pytest.raises(B.BpmError) as ei:
        B.bpm_plan(B.Instance(100, 4, 0.1, 0.1))
    assert ei.value.code == B.BPM_ERR_UNSUPPORTED
    with pytest.raises(B.BpmError) as ei:
        B.bpm_plan(B.Instance(64, 4, -0.1, 0.1))
    assert ei.value.code == B.BPM_ERR_ARG
    plan = B.bpm_plan(B.Instance(64, 4, 0.1, 0.1))
    try:
        buf = torch.zeros(64 * 64 + 1, dtype=torch.complex64, device=dev)
        dn_t = torch.zeros((4, 64, 64), dtype=torch.float16, device=dev)
        with pytest.raises(B.BpmError) as ei:
            B.bpm_propagate(plan, dn_t, buf[1:], buf[1:], None)
        assert ei.value.code == B.BPM_ERR_ALIGN
        with pytest.raises(B.BpmError) as ei:
            B.bpm_propagate(plan, dn_t, buf[:4096], buf[:4096], None, 3, 1)
        assert ei.value.code == B.BPM_ERR_ARG
    finally:
        B.bpm_free(plan)


@pytest.mark.parametrize("n", [256, 512, 1024])
def test_every_transform_schedule_matches_oracle(B, n):
    """Every transform schedule of a size (set by bpm_set_schedule; the
    autotuner picks among them) against the oracle, with index steps that need
    every phasor form, and the multi-launch path of the same schedule."""
    nz = 3
    d = 0.1625 if n == 1024 else 0.1
    rng = np.random.default_rng(11 * n)
    dn = np.empty((nz, n, n))
    dn[0] = rng.uniform(0.0, 0.05, size=(n, n))
    dn[1] = rng.uniform(0.0, 0.3, size=(n, n))
    dn[2] = rng.uniform(-1.0, 1.0, size=(n, n))
    dn[2, ::3] = rng.uniform(0.0, 0.05, size=dn[2, ::3].shape)
    dn16 = dn.astype(np.float16)
    E0 = bandlimited_field(n, d, 0.9, n + 5)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33)
    dev = torch.device("cuda")
    dn_t = torch.from_numpy(dn16).to(dev)
    e_in = torch.from_numpy(np.ascontiguousarray(E0, np.complex64)).to(dev)
    for flags in (0, B.BPM_FLAG_MULTI_LAUNCH):
        plan = B.bpm_plan(B.Instance(n, nz, d, d), flags=flags)
        try:
            count = B.bpm_plan_info(plan)["schedules"]
            assert count >= 2
            for sc in range(count):
                B.bpm_set_schedule(plan, sc)
                assert B.bpm_plan_info(plan)["schedule"] == sc
                e_out = torch.empty_like(e_in)
                I = torch.zeros((nz, n, n), dtype=torch.float32, device=dev)
                B.bpm_propagate(plan, dn_t, e_in, e_out, I)
                assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
                ef = field_rel_l2(e_out.cpu().numpy(), Er)
                ei = intensity_rel_max(I.cpu().numpy(), Ir)
                assert ef <= FIELD_TOL / 10, (sc, flags, ef)
                assert ei <= INTENSITY_TOL / 10, (sc, flags, ei)
            with pytest.raises(RuntimeError):
                B.bpm_set_schedule(plan, count)
        finally:
            B.bpm_free(plan)


def test_autotune_picks_a_schedule_of_a_single_field_plan(B):
    n, nz, d = 512, 8, 0.1
    rng = np.random.default_rng(21)
    dn16 = rng.uniform(0, 0.05, size=(nz, n, n)).astype(np.float16)
    E0 = bandlimited_field(n, d, 0.9, 77)
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d))
    try:
        dn_t = torch.from_numpy(dn16).to(dev)
        e_in = torch.from_numpy(E0).to(dev)
        e_out = torch.empty_like(e_in)
        I = torch.zeros((nz, n, n), dtype=torch.float32, device=dev)
        assert B.bpm_plan_info(plan)["schedule"] == 2          # the size's measured-best start
        B.bpm_autotune(plan, dn_t, e_in, e_out, I, 4)
        info = B.bpm_plan_info(plan)
        assert 0 <= info["schedule"] < info["schedules"] == 3
        B.bpm_propagate(plan, dn_t, e_in, e_out, I)
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33)
        assert field_rel_l2(e_out.cpu().numpy(), Er) <= FIELD_TOL / 10
        assert intensity_rel_max(I.cpu().numpy(), Ir) <= INTENSITY_TOL / 10
    finally:
        B.bpm_free(plan)
