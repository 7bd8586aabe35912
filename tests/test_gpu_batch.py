"""Batched propagation (many instances of mixed grid sizes in one persistent
cluster launch) against the FP64 oracle, per instance, on seeded inputs."""
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


def _mixed_batch():
    specs = [(512, 4), (128, 6), (384, 3), (64, 5), (256, 4), (192, 5), (128, 0), (1024, 2)]
    cases = []
    for k, (n, nz) in enumerate(specs):
        rng = np.random.default_rng(100 + k)
        dn16 = rng.uniform(0, 0.05, size=(max(nz, 1), n, n)).astype(np.float16)
        d = 0.1625 if n == 1024 else 0.1
        cases.append((n, nz, d, dn16, bandlimited_field(n, d, 0.85, 200 + k)))
    return cases


def _run_batch(B, cases, flags=0, tune=False, z=(0, 2 ** 31 - 1), sched=None):
    dev = torch.device("cuda")
    plan = B.bpm_plan([B.Instance(n, nz, d, d) for (n, nz, d, _, _) in cases], flags=flags)
    try:
        if sched is not None:
            B.bpm_set_schedule(plan, sched)
            assert B.bpm_plan_info(plan)["schedule"] == sched
        dn = [torch.from_numpy(c[3]).to(dev) for c in cases]
        ein = [torch.from_numpy(c[4]).to(dev) for c in cases]
        eout = [torch.empty_like(e) for e in ein]
        inten = [torch.zeros((max(c[1], 1), c[0], c[0]), dtype=torch.float32, device=dev) for c in cases]
        if tune:
            B.bpm_autotune(plan, dn, ein, eout, inten, 2)
            info = B.bpm_plan_info(plan)
            assert info["team_ctas"] in (2, 4, 8, 16)
            assert info["schedules"] == 3 and 0 <= info["schedule"] < 3    # schedule sets of the batched kernel
        B.bpm_propagate(plan, dn, ein, eout, inten, *z)
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        out1 = [e.cpu().numpy() for e in eout]
        # a second call with the same arguments (replays the graph when captured)
        for e in eout:
            e.zero_()
        B.bpm_propagate(plan, dn, ein, eout, inten, *z)
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        out2 = [e.cpu().numpy() for e in eout]
        for a, b in zip(out1, out2):
            assert np.array_equal(a, b)
        return out2, [i.cpu().numpy() for i in inten]
    finally:
        B.bpm_free(plan)


@pytest.mark.parametrize("flags,tune,sched", [(0, False, 0), (4, False, 0), (4, True, None), (4, False, 1),
                                              (0, False, 2)])
def test_mixed_batch_matches_oracle(B, flags, tune, sched):
    """Every schedule set of the batched kernel (and the autotuned one)."""
    cases = _mixed_batch()
    E, I = _run_batch(B, cases, flags=flags, tune=tune, sched=sched)
    for (n, nz, d, dn16, E0), Eg, Ig in zip(cases, E, I):
        if nz == 0:
            assert np.array_equal(Eg, E0)            # empty slice range copies the input
            continue
        Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16[:nz]), E0, d, d, d, 0.5, 1.33)
        assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10, (n, nz)
        assert intensity_rel_max(Ig[:nz], Ir) <= INTENSITY_TOL / 10, (n, nz)


def test_batch_equals_single_instance_runs(B):
    cases = _mixed_batch()[:4]
    E, I = _run_batch(B, cases)
    dev = torch.device("cuda")
    for (n, nz, d, dn16, E0), Eg, Ig in zip(cases, E, I):
        plan = B.bpm_plan(B.Instance(n, nz, d, d))
        try:
            # the transform schedule the batched kernel is compiled with (a
            # single 512^2 plan starts on another one, equal to FP32 rounding)
            B.bpm_set_schedule(plan, 0)
            e = torch.from_numpy(E0).to(dev)
            out = torch.empty_like(e)
            inten = torch.zeros((nz, n, n), dtype=torch.float32, device=dev)
            B.bpm_propagate(plan, torch.from_numpy(dn16).to(dev), e, out, inten)
            assert B.bpm_check(plan) == 0
            assert field_rel_l2(Eg, out.cpu().numpy()) <= 1e-6
            assert intensity_rel_max(Ig, inten.cpu().numpy()) <= 1e-6
        finally:
            B.bpm_free(plan)


def test_seeded_batch_instances_with_their_inputs(B):
    """The first instances of the seeded 64-instance workload (tilted plane
    waves and 8 x 8 multiplexed foci), truncated to 6 slices."""
    ws = inputs.batch_64()[:5]
    dev = torch.device("cuda")
    nzs = [6] * len(ws)
    plan = B.bpm_plan([B.Instance(w.n, nz, w.d, w.d) for w, nz in zip(ws, nzs)], flags=B.BPM_FLAG_GRAPH)
    try:
        dns, eins, refs_in = [], [], []
        for w, nz in zip(ws, nzs):
            dn16 = inputs.sphere_phantom_dn((nz, w.n, w.n), w.d, max(1, w.n_spheres * nz // w.nz), w.seed)
            dns.append(dn16)
            if w.input_kind == "plane":
                E0 = inputs.plane_wave(w.n, w.n, *w.tilt_bins)
                refs_in.append(E0.astype(np.complex128))
                eins.append(torch.from_numpy(E0).to(dev))
            else:
                f = w.foci()
                e = torch.empty((w.n, w.n), dtype=torch.complex64, device=dev)
                B.bpm_multiplex_psf(plan, len(eins), f.xyz_um(w.d, w.d), f.phase, f.NA, e)
                refs_in.append(oracle.multiplex_psf(w.n, w.n, w.d, w.d, w.lam, w.n0, f.ix, f.iy, f.phase,
                                                    f.zf, f.NA))
                eins.append(e)
        dn_t = [torch.from_numpy(x).to(dev) for x in dns]
        eout = [torch.empty_like(e) for e in eins]
        inten = [torch.zeros((nz, w.n, w.n), dtype=torch.float32, device=dev) for w, nz in zip(ws, nzs)]
        B.bpm_propagate(plan, dn_t, eins, eout, inten)
        assert B.bpm_check(plan) == 0, B.bpm_last_error()
        for w, dn16, E0r, eg, ig in zip(ws, dns, refs_in, eout, inten):
            Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0r, w.d, w.d, w.d, w.lam, w.n0)
            assert field_rel_l2(eg.cpu().numpy(), Er) <= FIELD_TOL
            assert intensity_rel_max(ig.cpu().numpy(), Ir) <= INTENSITY_TOL
    finally:
        B.bpm_free(plan)


def test_batch_every_phasor_form(B):
    """The batched kernel's screen (scalar form) with index steps that need
    each phasor evaluation: small steps, steps up to 0.5 rad, and rows of
    steps up to +-1.4 rad next to rows of small ones."""
    cases = []
    for k, n in enumerate([128, 256, 512, 192]):
        rng = np.random.default_rng(300 + k)
        dn = np.empty((3, n, n))
        dn[0] = rng.uniform(0.0, 0.05, size=(n, n))
        dn[1] = rng.uniform(0.0, 0.4, size=(n, n))
        dn[2] = rng.uniform(-1.1, 1.1, size=(n, n))
        dn[2, ::3] = rng.uniform(0.0, 0.05, size=dn[2, ::3].shape)
        cases.append((n, 3, 0.1, dn.astype(np.float16), bandlimited_field(n, 0.1, 0.85, 400 + k)))
    E, I = _run_batch(B, cases)
    for (n, nz, d, dn16, E0), Eg, Ig in zip(cases, E, I):
        Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33)
        assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10, n
        assert intensity_rel_max(Ig, Ir) <= INTENSITY_TOL / 10, n


def test_batch_every_instance_exactly_once_with_fill_teams(B):
    """Many small instances behind two large ones: the main cluster teams take
    positions from the large end of the queue while the fill launch's two-CTA
    teams take small ones from the other end.  Every output must be its own
    instance's propagation (an instance taken twice or never would leave a
    wrong or untouched output; outputs start as NaN)."""
    cases = []
    for k in range(2):
        rng = np.random.default_rng(500 + k)
        cases.append((512, 8, 0.1, rng.uniform(0, 0.05, size=(8, 512, 512)).astype(np.float16),
                      bandlimited_field(512, 0.1, 0.85, 600 + k)))
    for k in range(40):
        rng = np.random.default_rng(700 + k)
        cases.append((64, 3, 0.1, rng.uniform(0, 0.05, size=(3, 64, 64)).astype(np.float16),
                      bandlimited_field(64, 0.1, 0.85, 800 + k)))
    dev = torch.device("cuda")
    plan = B.bpm_plan([B.Instance(n, nz, d, d) for (n, nz, d, _, _) in cases], flags=B.BPM_FLAG_GRAPH)
    try:
        dn = [torch.from_numpy(c[3]).to(dev) for c in cases]
        ein = [torch.from_numpy(c[4]).to(dev) for c in cases]
        for rep in range(2):
            eout = [torch.full_like(e, float("nan")) for e in ein]
            B.bpm_propagate(plan, dn, ein, eout, None)
            assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
            for (n, nz, d, dn16, E0), eg in zip(cases, eout):
                Er, _ = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33, want_intensity=False)
                assert field_rel_l2(eg.cpu().numpy(), Er) <= FIELD_TOL / 10, (n, rep)
    finally:
        B.bpm_free(plan)


def test_batched_exchange_timeout_is_reported_and_context_survives(B):
    # Small instances hand the field between half-steps through tagged
    # elements; with the entrance field carrying the wrong parity their waits
    # run out after 2 ms, the batch reports BPM_ERR_TIMEOUT, and the same plan
    # then propagates correctly (a larger instance, on the cluster barrier,
    # rides along).
    cases = []
    for k, (n, nz) in enumerate([(128, 4), (192, 3), (256, 3), (64, 4)]):
        rng = np.random.default_rng(300 + k)
        dn16 = rng.uniform(0, 0.05, size=(nz, n, n)).astype(np.float16)
        cases.append((n, nz, 0.1, dn16, bandlimited_field(n, 0.1, 0.85, 400 + k)))
    dev = torch.device("cuda")
    plan = B.bpm_plan([B.Instance(n, nz, d, d) for (n, nz, d, _, _) in cases])
    try:
        dn = [torch.from_numpy(c[3]).to(dev) for c in cases]
        ein = [torch.from_numpy(c[4]).to(dev) for c in cases]
        eout = [torch.empty_like(e) for e in ein]
        B.bpm_debug_set_barrier_timeout(plan, 2_000_000, 0)
        B.bpm_debug_stall_exchange(plan, True)
        B.bpm_propagate(plan, dn, ein, eout, None)
        assert B.bpm_check(plan) == B.BPM_ERR_TIMEOUT
        B.bpm_debug_stall_exchange(plan, False)
        B.bpm_debug_set_barrier_timeout(plan, 2_000_000_000, 0)
        B.bpm_propagate(plan, dn, ein, eout, None)
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        for (n, nz, d, dn16, E0), e in zip(cases, eout):
            Er, _ = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33)
            assert field_rel_l2(e.cpu().numpy(), Er) <= FIELD_TOL / 10
    finally:
        B.bpm_free(plan)
    torch.cuda.synchronize()
