"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times (one plan, default flags, the whole depth in one
bpm_propagate call).

* 256^3 light sheet through the 300-sphere phantom: the oracle runs the whole
  volume, so every output is compared.
* 1024^3 multiplexed PSFs through the 800-sphere phantom: the oracle runs the
  first 256 slices of the same volume, giving the field after slice 256 and
  the first 256 intensity planes of the same run.  At every depth, the
  properties that hold for any grid are checked: the screen is unitary and the
  cut propagator can only remove power, so the slice energy never grows (and
  stays constant for a field inside the propagating band), and the output
  field's modulus squared is the last intensity plane.
* 1024^3 multiplexed PSFs through a homogeneous medium: the exact propagator
  composes (H(dz)^k = H(k dz)), so the oracle's single step over k dz gives
  the planes at any depth, here the field after all 1024 slices and sampled
  intensity planes.
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


def test_light_sheet_256_whole_volume(B):
    w = inputs.light_sheet_256()
    dn16 = w.dn()
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(w.n, w.nz, w.d, w.d, w.lam, w.n0))
    try:
        e0 = torch.empty((w.n, w.n), dtype=torch.complex64, device=dev)
        B.bpm_light_sheet(plan, 0, w.sheet_NA, w.sheet_zf(), e0)
        eout = torch.empty_like(e0)
        I = torch.empty((w.nz, w.n, w.n), dtype=torch.float32, device=dev)
        B.bpm_propagate(plan, torch.from_numpy(dn16).to(dev), e0, eout, I)
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        Eg, Ig = eout.cpu().numpy(), I.cpu().numpy()
    finally:
        B.bpm_free(plan)
    E0 = oracle.light_sheet(w.n, w.n, w.d, w.d, w.lam, w.n0, w.sheet_NA, w.sheet_zf())
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, w.d, w.d, w.d, w.lam, w.n0)
    ef, ei = field_rel_l2(Eg, Er), intensity_rel_max(Ig, Ir)
    print(f"256^3 light sheet: field rel L2 {ef:.2e}, intensity max rel {ei:.2e}")
    assert ef <= FIELD_TOL
    assert ei <= INTENSITY_TOL


def _run_1024(B, dn16, w, f, z_part=None):
    """The whole depth with the intensity volume; with z_part also the field
    after the first z_part slices (a second call on the same plan)."""
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(w.n, w.nz, w.d, w.d, w.lam, w.n0))
    try:
        e0 = torch.empty((w.n, w.n), dtype=torch.complex64, device=dev)
        B.bpm_multiplex_psf(plan, 0, f.xyz_um(w.d, w.d), f.phase, f.NA, e0)
        eout = torch.empty_like(e0)
        I = torch.empty((w.nz, w.n, w.n), dtype=torch.float32, device=dev)
        dn_d = torch.from_numpy(dn16).to(dev)
        B.bpm_propagate(plan, dn_d, e0, eout, I)
        e_part = None
        if z_part is not None:
            ep = torch.empty_like(e0)
            B.bpm_propagate(plan, dn_d, e0, ep, None, 0, z_part)
            e_part = ep.cpu().numpy()
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        del dn_d
        energy = I.to(torch.float64).sum(dim=(1, 2)).cpu().numpy()
        e_out = eout.cpu().numpy()
        return e_out, I, energy, e_part
    finally:
        B.bpm_free(plan)


def test_multiplex_1024_cubed_phantom(B):
    w = inputs.multiplex_1024(nz=1024)
    dn16 = w.dn()
    f = w.foci()
    k = 256
    Eg, I, energy, Ek = _run_1024(B, dn16, w, f, z_part=k)
    # the oracle through the first 256 slices of the same phantom (the depth at
    # which the field gate is stated): field after slice 256, every intensity
    # plane of those slices
    E0 = oracle.multiplex_psf(w.n, w.n, w.d, w.d, w.lam, w.n0, f.ix, f.iy, f.phase, f.zf, f.NA)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16[:k]), E0, w.d, w.d, w.d, w.lam, w.n0)
    ef = field_rel_l2(Ek, Er)
    ei = intensity_rel_max(I[:k].cpu().numpy(), Ir)
    del Ir
    # energy: never grows beyond FP32 rounding; the foci's spectrum lies inside
    # NA 0.6 < n0, so almost nothing is cut either
    e_in = float(np.sum(np.abs(E0) ** 2))
    growth = float(np.max(np.diff(energy)) / e_in)
    drift = float(np.max(np.abs(energy - e_in)) / e_in)
    last = float(np.max(np.abs(np.abs(Eg) ** 2 - I[-1].cpu().numpy())) / I[-1].max().item())
    print(f"1024^3 phantom: field rel L2 after {k} slices {ef:.2e}, first {k} planes intensity max rel {ei:.2e}; "
          f"energy growth {growth:.1e}, drift {drift:.1e}; |E_out|^2 vs last plane {last:.1e}")
    assert ef <= FIELD_TOL
    assert ei <= INTENSITY_TOL
    assert growth <= 1e-5
    assert drift <= 1e-3
    assert last <= 1e-5
    assert np.all(np.isfinite(Eg))


def test_multiplex_1024_cubed_homogeneous_against_single_exact_step(B):
    w = inputs.multiplex_1024(nz=1024)
    f = w.foci()
    dn16 = np.zeros((w.nz, w.n, w.n), np.float16)
    Eg, I, _, E256 = _run_1024(B, dn16, w, f, z_part=256)
    E0 = oracle.multiplex_psf(w.n, w.n, w.d, w.d, w.lam, w.n0, f.ix, f.iy, f.phase, f.zf, f.NA)
    zero = np.zeros((1, w.n, w.n))
    Er, _ = oracle.bpm(zero, E0, w.d, w.d, w.nz * w.d, w.lam, w.n0)
    ef = field_rel_l2(Eg, Er)
    Er256, _ = oracle.bpm(zero, E0, w.d, w.d, 256 * w.d, w.lam, w.n0)
    ef256 = field_rel_l2(E256, Er256)
    errs = []
    for z in (0, 127, 511):
        _, Ir = oracle.bpm(zero, E0, w.d, w.d, (z + 1) * w.d, w.lam, w.n0)
        errs.append(intensity_rel_max(I[z].cpu().numpy(), Ir[0]))
    print(f"1024^3 homogeneous: field rel L2 after 256 slices {ef256:.2e}, after 1024 slices {ef:.2e}; "
          f"intensity planes 1/128/512 {errs}")
    # the field gate is stated after 256 slices; the FP32 error is dominated by
    # the rounding of the propagator table and twiddles, the same in every
    # slice, so it grows in proportion to the depth: 4x the gate after 1024
    assert ef256 <= FIELD_TOL
    assert ef <= FIELD_TOL * 1024 / 256
    assert max(errs) <= INTENSITY_TOL


def test_batch64_workload_full_size(B):
    """The batched workload at its full size, in the launch configuration the
    benchmark times (one graph-captured plan of all 64 seeded instances,
    autotuned): the three smallest instances against the oracle through their
    whole depth, and for every instance the properties that hold at any size
    (the slice energy never grows beyond FP32 rounding, the output field's
    modulus squared is the last intensity plane)."""
    ws = inputs.batch_64()
    dev = torch.device("cuda")
    plan = B.bpm_plan([B.Instance(w.n, w.nz, w.d, w.d, w.lam, w.n0) for w in ws], flags=B.BPM_FLAG_GRAPH)
    try:
        dns, eins, E0s = [], [], []
        for k, w in enumerate(ws):
            dns.append(torch.from_numpy(w.dn()).to(dev))
            if w.input_kind == "plane":
                e = torch.from_numpy(inputs.plane_wave(w.n, w.n, *w.tilt_bins)).to(dev)
            else:
                f = w.foci()
                e = torch.empty((w.n, w.n), dtype=torch.complex64, device=dev)
                B.bpm_multiplex_psf(plan, k, f.xyz_um(w.d, w.d), f.phase, f.NA, e)
            eins.append(e)
        eout = [torch.empty_like(e) for e in eins]
        inten = [torch.empty((w.nz, w.n, w.n), dtype=torch.float32, device=dev) for w in ws]
        B.bpm_autotune(plan, dns, eins, eout, inten, 32)
        B.bpm_propagate(plan, dns, eins, eout, inten)
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        for k, w in enumerate(ws):
            e_in = float(torch.sum(torch.abs(eins[k].to(torch.complex128)) ** 2))
            energy = inten[k].to(torch.float64).sum(dim=(1, 2))
            assert float(torch.max(energy[1:] - energy[:-1])) <= 1e-5 * e_in, k
            last = (eout[k].abs() ** 2 - inten[k][-1]).abs().max() / inten[k][-1].max()
            assert float(last) <= 1e-5, k
        smallest = sorted(range(len(ws)), key=lambda k: ws[k].n ** 2 * ws[k].nz)[:3]
        for k in smallest:
            w = ws[k]
            Er, Ir = oracle.bpm(inputs.dn_to_f64(dns[k].cpu().numpy()), eins[k].cpu().numpy(), w.d, w.d, w.d,
                                w.lam, w.n0)
            ef = field_rel_l2(eout[k].cpu().numpy(), Er)
            ei = intensity_rel_max(inten[k].cpu().numpy(), Ir)
            print(f"batch64 instance {k} ({w.n}^2 x {w.nz}): field {ef:.2e}, intensity {ei:.2e}")
            assert ef <= FIELD_TOL * max(1.0, w.nz / 256)
            assert ei <= INTENSITY_TOL
    finally:
        B.bpm_free(plan)
