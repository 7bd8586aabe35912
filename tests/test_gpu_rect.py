"""GPU parity on rectangular grids and on the transform lengths 96, 768, 1536
and 2048 (nx, ny products of 2 and 3, nx ny <= 2^22), against the FP64
oracle on the same seeded inputs (method paragraph; the paper's 10^6-PSF
calculation runs on a 1024 x 2048 lateral grid, light-sheet paragraph)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1706_02261_b300 import inputs  # noqa: E402
from tests.gpu_util import (FIELD_TOL, INTENSITY_TOL, bandlimited_field_rect,  # noqa: E402
                            field_rel_l2, intensity_rel_max)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_02261_b300 import bpm
    return bpm


def run_gpu(B, inst, dn16, E0, flags=0, kappa16=None):
    dev = torch.device("cuda")
    plan = B.bpm_plan(inst, flags=flags)
    try:
        info = B.bpm_plan_info(plan)
        e_in = torch.from_numpy(np.ascontiguousarray(E0, np.complex64)).to(dev)
        e_out = torch.empty_like(e_in)
        I = torch.zeros(dn16.shape, dtype=torch.float32, device=dev)
        dn_t = torch.from_numpy(dn16).to(dev)
        if kappa16 is None:
            B.bpm_propagate(plan, dn_t, e_in, e_out, I)
        else:
            B.bpm_propagate_absorbing(plan, dn_t, torch.from_numpy(kappa16).to(dev), e_in, e_out, I)
        assert B.bpm_check(plan) == B.BPM_OK, B.bpm_last_error()
        return e_out.cpu().numpy(), I.cpu().numpy(), info
    finally:
        B.bpm_free(plan)


# grids with a persistent kernel (square, or sides differing by a factor of
# two) and grids that run one launch per half-step
PERSISTENT = [(64, 128), (128, 64), (96, 192), (192, 96), (128, 256), (256, 128), (192, 384), (384, 192),
              (256, 512), (512, 256), (384, 768), (768, 384), (512, 1024), (1024, 512), (768, 1536),
              (1536, 768), (1024, 2048), (2048, 1024), (96, 96), (768, 768), (1536, 1536), (2048, 2048)]
MULTI_ONLY = [(96, 256), (1024, 192), (2048, 64), (1536, 2048)]


@pytest.mark.parametrize("nx,ny", PERSISTENT + MULTI_ONLY)
@pytest.mark.parametrize("flags", [0, 2])
def test_grid_random_inputs(B, nx, ny, flags):
    nz, d = 4, 0.1
    rng = np.random.default_rng(nx * 7 + ny)
    dn16 = rng.uniform(0, 0.05, size=(nz, ny, nx)).astype(np.float16)
    E0 = bandlimited_field_rect(nx, ny, d, 0.9, nx + 3 * ny)
    Eg, Ig, info = run_gpu(B, B.Instance(nx, nz, d, d, ny=ny), dn16, E0, flags)
    assert info["persistent"] == (1 if flags == 0 and (nx, ny) in PERSISTENT else 0)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33)
    assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10
    assert intensity_rel_max(Ig, Ir) <= INTENSITY_TOL / 10


@pytest.mark.parametrize("nx,ny", [(1024, 2048), (2048, 1024), (96, 192)])
def test_grid_every_phasor_form(B, nx, ny):
    """Index steps that reach the long series and sincosf (see the square
    test of the same name), with unequal spacings dx != dy."""
    nz, dx, dy = 3, 0.1, 0.125
    rng = np.random.default_rng(nx + ny)
    dn = np.empty((nz, ny, nx))
    dn[0] = rng.uniform(0.0, 0.05, size=(ny, nx))
    dn[1] = rng.uniform(0.0, 0.4, size=(ny, nx))
    dn[2] = rng.uniform(-1.1, 1.1, size=(ny, nx))
    dn16 = dn.astype(np.float16)
    E0 = bandlimited_field_rect(nx, ny, dx, 0.85, 5, dy=dy)
    Eg, Ig, _ = run_gpu(B, B.Instance(nx, nz, dx, dx, dy=dy, ny=ny), dn16, E0)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, dx, dy, dx, 0.5, 1.33)
    assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10
    assert intensity_rel_max(Ig, Ir) <= INTENSITY_TOL / 10


@pytest.mark.parametrize("nx,ny", [(1024, 2048), (2048, 1024), (192, 96), (1536, 768)])
def test_multiplex_synthesis_rect(B, nx, ny):
    """Multiplexed foci on a rectangular grid (pitch 32 px, NA 0.6) against the
    oracle's synthesis."""
    d = 0.1625
    ix, iy = np.meshgrid(np.arange(16, nx, 32), np.arange(16, ny, 32))
    ix, iy = ix.ravel(), iy.ravel()
    rng = np.random.default_rng(nx ^ ny)
    ph = rng.uniform(0, 2 * np.pi, ix.size)
    zf = 20.0
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(nx, 8, d, d, ny=ny))
    try:
        e = torch.empty((ny, nx), dtype=torch.complex64, device=dev)
        B.bpm_multiplex_psf(plan, 0, np.stack([ix * d, iy * d, np.full(ix.size, zf)], 1), ph, 0.6, e)
        assert B.bpm_check(plan) == 0, B.bpm_last_error()
        Eg = e.cpu().numpy()
    finally:
        B.bpm_free(plan)
    Er = oracle.multiplex_psf(nx, ny, d, d, 0.5, 1.33, ix, iy, ph, zf, 0.6)
    assert field_rel_l2(Eg, Er) <= 1e-5


@pytest.mark.parametrize("nx,ny", [(2048, 1024), (96, 192)])
def test_light_sheet_rect(B, nx, ny):
    d = 0.1
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(nx, 8, d, d, ny=ny))
    try:
        e = torch.empty((ny, nx), dtype=torch.complex64, device=dev)
        B.bpm_light_sheet(plan, 0, 0.15, 4.0, e)
        assert B.bpm_check(plan) == 0, B.bpm_last_error()
        Eg = e.cpu().numpy()
    finally:
        B.bpm_free(plan)
    Er = oracle.light_sheet(nx, ny, d, d, 0.5, 1.33, 0.15, 4.0)
    assert field_rel_l2(Eg, Er) <= 1e-5


def test_psf_grid_1024x2048_through_phantom(B):
    """The paper's 10^6-PSF lateral grid: multiplexed foci through a seeded
    sphere phantom, 24 slices, every output against the oracle."""
    nx, ny, nz, d = 1024, 2048, 24, 0.1625
    dn16 = inputs.sphere_phantom_dn((nz, ny, nx), d, 60, 11)
    ix, iy = np.meshgrid(np.arange(16, nx, 32), np.arange(16, ny, 32))
    ix, iy = ix.ravel(), iy.ravel()
    ph = np.random.default_rng(12).uniform(0, 2 * np.pi, ix.size)
    zf = 2.0
    dev = torch.device("cuda")
    plan = B.bpm_plan(B.Instance(nx, nz, d, d, ny=ny))
    try:
        assert B.bpm_plan_info(plan)["persistent"] == 1
        e0 = torch.empty((ny, nx), dtype=torch.complex64, device=dev)
        B.bpm_multiplex_psf(plan, 0, np.stack([ix * d, iy * d, np.full(ix.size, zf)], 1), ph, 0.6, e0)
        eout = torch.empty_like(e0)
        I = torch.empty((nz, ny, nx), dtype=torch.float32, device=dev)
        B.bpm_propagate(plan, torch.from_numpy(dn16).to(dev), e0, eout, I)
        assert B.bpm_check(plan) == 0, B.bpm_last_error()
        Eg, Ig = eout.cpu().numpy(), I.cpu().numpy()
    finally:
        B.bpm_free(plan)
    E0 = oracle.multiplex_psf(nx, ny, d, d, 0.5, 1.33, ix, iy, ph, zf, 0.6)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33)
    ef, ei = field_rel_l2(Eg, Er), intensity_rel_max(Ig, Ir)
    print(f"1024 x 2048 x {nz} multiplexed through the phantom: field rel L2 {ef:.2e}, intensity max rel {ei:.2e}")
    assert ef <= FIELD_TOL / 10
    assert ei <= INTENSITY_TOL / 10


def test_adaptive_and_absorbing_rect(B):
    nx, ny, nz, d = 512, 256, 5, 0.1
    rng = np.random.default_rng(44)
    dn16 = rng.uniform(0.0, 0.05, size=(nz, ny, nx)).astype(np.float16)
    kap16 = rng.uniform(0.0, 0.002, size=(nz, ny, nx)).astype(np.float16)
    E0 = bandlimited_field_rect(nx, ny, d, 0.85, 45)
    inst = B.Instance(nx, nz, d, d, ny=ny)
    Eg, Ig, _ = run_gpu(B, inst, dn16, E0, B.BPM_FLAG_ADAPTIVE)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33, adaptive=True)
    assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10
    assert intensity_rel_max(Ig, Ir) <= INTENSITY_TOL / 10
    Eg, Ig, _ = run_gpu(B, inst, dn16, E0, 0, kappa16=kap16)
    Er, Ir = oracle.bpm(inputs.dn_to_f64(dn16), E0, d, d, d, 0.5, 1.33, kappa=kap16.astype(np.float64))
    assert field_rel_l2(Eg, Er) <= FIELD_TOL / 10
    assert intensity_rel_max(Ig, Ir) <= INTENSITY_TOL / 10


def test_demultiplex_rect(B):
    """Per-focus patches of a rectangular window: exact gather with the
    periodic wrap of each side."""
    nx, ny, w_nz = 256, 128, 6
    dev = torch.device("cuda")
    vol = np.arange(w_nz * ny * nx, dtype=np.float32).reshape(w_nz, ny, nx)
    foci = np.array([[0, 0, 12], [255, 127, 14], [100, 3, 13]], np.int32)
    px, py, pz = 8, 6, 4
    plan = B.bpm_plan(B.Instance(nx, 20, 0.1, 0.1, ny=ny))
    try:
        out = torch.empty((len(foci), pz, py, px), dtype=torch.float32, device=dev)
        B.bpm_demultiplex(plan, 0, torch.from_numpy(vol).to(dev), 11, foci, (px, py, pz), out)
        assert B.bpm_check(plan) == 0
        got = out.cpu().numpy()
    finally:
        B.bpm_free(plan)
    for j, (fx, fy, fz) in enumerate(foci):
        for k in range(pz):
            z = fz - pz // 2 + k - 11
            for y in range(py):
                for x in range(px):
                    want = vol[z, (fy - py // 2 + y) % ny, (fx - px // 2 + x) % nx] if 0 <= z < w_nz else 0.0
                    assert got[j, k, y, x] == want
