"""PSF sweep on the GPU (intensity windows, de-multiplexing, the whole
multiplexed sweep) against the FP64 oracle and exact index arithmetic."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1706_02261_b300 import inputs  # noqa: E402
from tests.gpu_util import INTENSITY_TOL, bandlimited_field, intensity_rel_max  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_02261_b300 import bpm
    return bpm


def crop(I, w0, foci, patch):
    """Reference crop: plain indexing with periodic lateral wrap, zeros
    outside the window (the definition of the patches)."""
    px, py, pz = patch
    nwz, n, _ = I.shape
    out = np.zeros((len(foci), pz, py, px), I.dtype)
    for j, (ix, iy, iz) in enumerate(foci):
        for k in range(pz):
            z = iz - pz // 2 + k - w0
            if 0 <= z < nwz:
                ys = (iy - py // 2 + np.arange(py)) % n
                xs = (ix - px // 2 + np.arange(px)) % n
                out[j, k] = I[z][np.ix_(ys, xs)]
    return out


def test_window_equals_full_volume_slices(B):
    n, nz, d = 128, 16, 0.1
    rng = np.random.default_rng(21)
    dn16 = rng.uniform(0, 0.05, size=(nz, n, n)).astype(np.float16)
    E0 = bandlimited_field(n, d, 0.8, 22)
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, nz, d, d))
    try:
        dn = torch.from_numpy(dn16).to(dev)
        e0 = torch.from_numpy(E0).to(dev)
        e1 = torch.empty_like(e0)
        full = torch.zeros((nz, n, n), device=dev)
        B.bpm_propagate(plan, dn, e0, e1, full)
        win = torch.full((9, n, n), -7.0, device=dev)
        e2 = torch.empty_like(e0)
        B.bpm_propagate_window(plan, dn, e0, e2, win, 5, 12)           # 7 of the 9 slices
        assert B.bpm_check(plan) == 0, B.bpm_last_error()
        w, f = win.cpu().numpy(), full.cpu().numpy()
        assert np.array_equal(w[:7], f[5:12])
        assert np.all(w[7:] == -7.0)                                    # nothing outside the window
        assert torch.equal(e1, e2)
    finally:
        B.bpm_free(plan)
    _, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33)
    assert intensity_rel_max(w[:7], Ir[5:12]) <= INTENSITY_TOL


def test_batched_windows(B):
    n, d = 128, 0.1
    rng = np.random.default_rng(31)
    dev = torch.device("cuda")
    insts = [B.Instance(n, 12, d, d), B.Instance(n, 20, d, d)]
    plan = B.bpm_plan(insts)
    try:
        dns = [rng.uniform(0, 0.05, size=(i.nz, n, n)).astype(np.float16) for i in insts]
        E0s = [bandlimited_field(n, d, 0.8, 40 + k) for k in range(2)]
        wins = [(3, 9), (10, 20)]
        outs = [torch.empty((n, n), dtype=torch.complex64, device=dev) for _ in insts]
        Is = [torch.full((w1 - w0, n, n), -1.0, device=dev) for w0, w1 in wins]
        B.bpm_propagate_window(plan, [torch.from_numpy(x).to(dev) for x in dns],
                               [torch.from_numpy(x).to(dev) for x in E0s], outs, Is,
                               [w[0] for w in wins], [w[1] for w in wins])
        assert B.bpm_check(plan) == 0, B.bpm_last_error()
        for k, (w0, w1) in enumerate(wins):
            _, Ir = oracle.bpm(inputs.dn_to_f64(dns[k]), E0s[k], d, d, d, 0.5, 1.33)
            assert intensity_rel_max(Is[k].cpu().numpy(), Ir[w0:w1]) <= INTENSITY_TOL
    finally:
        B.bpm_free(plan)


def test_demultiplex_index_arithmetic_is_exact(B):
    n, w0, wnz = 64, 10, 6
    z, y, x = np.meshgrid(np.arange(wnz), np.arange(n), np.arange(n), indexing="ij")
    I = ((z + w0) * 10000 + y * 100 + x).astype(np.float32)     # exact in float32
    foci = np.array([[0, 0, 12], [63, 5, 10], [30, 62, 15], [7, 40, 3], [20, 20, 30]], np.int32)
    patch = (5, 4, 7)
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(n, 32, 0.1, 0.1))
    try:
        out = torch.full((len(foci), patch[2], patch[1], patch[0]), -1.0, device=dev)
        B.bpm_demultiplex(plan, 0, torch.from_numpy(I).to(dev), w0, foci, patch, out)
        assert B.bpm_check(plan) == 0
        got = out.cpu().numpy()
    finally:
        B.bpm_free(plan)
    assert np.array_equal(got, crop(I, w0, foci.tolist(), patch))
    with pytest.raises(RuntimeError):
        plan = B.bpm_plan(B.Instance(n, 32, 0.1, 0.1))
        try:
            B.bpm_demultiplex(plan, 0, torch.from_numpy(I).to(dev), w0, [[64, 0, 0]], patch, out)
        finally:
            B.bpm_free(plan)


def test_sweep_against_oracle(B):
    from paper_1706_02261_b300.psf import Runner, Sweep
    s = Sweep(n=128, nz=40, d=0.1, pitch=32, depths=[14, 30], patch=(16, 16, 12), seed=5)
    dn16 = inputs.sphere_phantom_dn((s.nz, s.n, s.n), s.d, 6, 9)
    dev = torch.device("cuda")
    r = Runner(s, torch.from_numpy(dn16).to(dev))
    try:
        outs = []
        for k in range(len(s.depths)):
            o = torch.empty((s.foci_per_field,) + s.patch[::-1], device=dev)
            r.field(k, o)
            outs.append(o.cpu().numpy())
        r.check()
    finally:
        r.free()
    dn64 = inputs.dn_to_f64(dn16)
    for k, iz in enumerate(s.depths):
        xyz, ph, foci = s.field_inputs(k)
        w0, w1 = s.window(iz)
        E0 = oracle.multiplex_psf(s.n, s.n, s.d, s.d, s.lam, s.n0, foci[:, 0], foci[:, 1], ph,
                                  xyz[:, 2], s.NA)
        _, Ir = oracle.bpm(dn64[:w1], E0, s.d, s.d, s.d, s.lam, s.n0)
        ref = crop(Ir[w0:w1], w0, foci.tolist(), s.patch)
        assert intensity_rel_max(outs[k], ref) <= INTENSITY_TOL
        # each patch holds its own focus: the brightest voxel of the patch
        # lies within 2 px of its centre laterally
        m = ref.reshape(len(foci), -1).argmax(1)
        _, yy, xx = np.unravel_index(m, s.patch[::-1])
        assert np.all(np.abs(yy - s.patch[1] // 2) <= 2) and np.all(np.abs(xx - s.patch[0] // 2) <= 2)
