"""Seeded synthetic inputs for beam propagation (refractive-index phantoms,
plane waves, emitter lattices).

This module draws random numbers and rasterises shapes; it holds none of the
propagation arithmetic (no propagator, no phase screen, no focusing), so the
CUDA library and the FP64 oracle both consume exactly the arrays it returns.
The workloads stand in for the paper's synthetic tissue phantoms (Biobeam,
arXiv:1706.02261, Fig. 1a: a multicellular phantom with n = 1.33-1.38; Fig. 2a:
an embryo model); the paper uses no public dataset.

Conventions: voxel (ix, iy, iz) sits at (ix dx, iy dy, iz dz) micrometres;
volumes are z-major numpy arrays ``[nz][ny][nx]``; the refractive index is
stored as ``dn = n - n0`` rounded to IEEE half precision.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

LAMBDA_UM = 0.5
N0 = 1.33
DN_MAX = 0.05          # clip so that n <= 1.38


# --------------------------------------------------------------------------
# refractive-index phantoms
# --------------------------------------------------------------------------

def single_sphere_dn(n: int = 64, nz: int = 64, d: float = 0.1, radius: float = 2.0,
                     dn_in: float = 0.05) -> np.ndarray:
    """Hard-edged sphere of index n0 + dn_in (radius in micrometres) centred at
    ((n/2) d, (n/2) d, (nz/2) d); zero elsewhere.  FP16, [nz][n][n]."""
    c = np.array([(n // 2) * d, (n // 2) * d, (nz // 2) * d])
    z = (np.arange(nz) * d - c[2])[:, None, None]
    y = (np.arange(n) * d - c[1])[None, :, None]
    x = (np.arange(n) * d - c[0])[None, None, :]
    inside = (x * x + y * y + z * z) <= radius * radius
    return np.where(inside, np.float16(dn_in), np.float16(0)).astype(np.float16)


def _gaussian_wrap(vol: np.ndarray, sigma: float, threads: int | None = None) -> np.ndarray:
    """Separable Gaussian filter with periodic boundaries along every axis.

    Each 1D pass is split into slabs across an orthogonal axis and run on a
    thread pool; every output element is computed the same way whatever the
    split, so the result does not depend on the thread count."""
    from scipy.ndimage import gaussian_filter1d

    threads = threads or min(32, os.cpu_count() or 1)
    out = vol
    for axis in range(3):
        src = out
        dst = np.empty_like(src)
        split_axis = 1 if axis != 1 else 0
        n = src.shape[split_axis]
        bounds = np.linspace(0, n, min(n, threads * 4) + 1).astype(int)

        def work(k, src=src, dst=dst, axis=axis, split_axis=split_axis):
            sl = [slice(None)] * 3
            sl[split_axis] = slice(bounds[k], bounds[k + 1])
            sl = tuple(sl)
            gaussian_filter1d(src[sl], sigma, axis=axis, mode="wrap", output=dst[sl])

        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, range(len(bounds) - 1)))
        out = dst
    return out


def sphere_phantom_dn(shape, d: float, n_spheres: int, seed: int,
                      r_range=(2.0, 5.0), dn_range=(0.01, 0.05), sigma_vox: float = 1.0,
                      threads: int | None = None) -> np.ndarray:
    """Tissue phantom: ``n_spheres`` spheres with centres uniform in the box,
    radii uniform in ``r_range`` micrometres and index steps uniform in
    ``dn_range``; overlapping steps add; then a Gaussian blur of ``sigma_vox``
    voxels with periodic boundaries, a clip to [0, 0.05] (n <= 1.38) and
    rounding to FP16.  Random draws from ``numpy.random.default_rng(seed)`` in
    the order centres, radii, index steps.  Returns [nz][ny][nx] FP16."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    box = np.array([nx * d, ny * d, nz * d])
    centres = rng.uniform(0.0, 1.0, size=(n_spheres, 3)) * box
    radii = rng.uniform(r_range[0], r_range[1], size=n_spheres)
    steps = rng.uniform(dn_range[0], dn_range[1], size=n_spheres)
    vol = np.zeros((nz, ny, nx), np.float32)
    for (cx, cy, cz), r, s in zip(centres, radii, steps):
        lo = np.maximum(np.floor((np.array([cx, cy, cz]) - r) / d).astype(int), 0)
        hi = np.minimum(np.ceil((np.array([cx, cy, cz]) + r) / d).astype(int) + 1, [nx, ny, nz])
        if np.any(hi <= lo):
            continue
        xs = np.arange(lo[0], hi[0]) * d - cx
        ys = np.arange(lo[1], hi[1]) * d - cy
        zs = np.arange(lo[2], hi[2]) * d - cz
        inside = (zs[:, None, None] ** 2 + ys[None, :, None] ** 2 + xs[None, None, :] ** 2) <= r * r
        vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += np.float32(s) * inside
    if sigma_vox > 0:
        vol = _gaussian_wrap(vol, sigma_vox, threads)
    np.clip(vol, 0.0, DN_MAX, out=vol)
    return vol.astype(np.float16)


def _gradient_noise(shape, d: float, cell_um: float, rng) -> np.ndarray:
    """One octave of periodic gradient (Perlin) noise: unit gradient vectors on
    a lattice of about ``cell_um`` spacing that tiles the box, the dot product
    of each corner's gradient with the offset to the voxel, blended with the
    quintic fade 6t^5 - 15t^4 + 10t^3 along each axis.  Values in about
    [-1, 1]; computed slice by slice."""
    nz, ny, nx = shape
    L = [max(1, int(round(n * d / cell_um))) for n in (nx, ny, nz)]
    g = rng.normal(size=(L[2], L[1], L[0], 3))
    g /= np.linalg.norm(g, axis=-1, keepdims=True)
    fade = lambda t: t * t * t * (t * (t * 6.0 - 15.0) + 10.0)
    ux = np.arange(nx) * L[0] / nx
    uy = np.arange(ny) * L[1] / ny
    x0 = np.floor(ux).astype(int)
    y0 = np.floor(uy).astype(int)
    fx = (ux - x0)[None, :]
    fy = (uy - y0)[:, None]
    out = np.empty(shape, np.float32)
    for z in range(nz):
        uz = z * L[2] / nz
        z0 = int(np.floor(uz))
        fz = uz - z0
        acc = np.zeros((ny, nx))
        for cz in (0, 1):
            wz = fade(fz) if cz else 1 - fade(fz)
            for cy in (0, 1):
                wy = fade(fy) if cy else 1 - fade(fy)
                for cx in (0, 1):
                    wx = fade(fx) if cx else 1 - fade(fx)
                    gg = g[(z0 + cz) % L[2]][np.ix_((y0 + cy) % L[1], (x0 + cx) % L[0])]
                    dot = gg[..., 0] * (fx - cx) + gg[..., 1] * (fy - cy) + gg[..., 2] * (fz - cz)
                    acc += wz * wy * wx * dot
        out[z] = acc
    return out


def perlin_phantom_dn(shape, d: float, seed: int, n_mean: float = 1.36, n_amp: float = 0.03,
                      cell_um: float = 4.0, n0: float = N0) -> np.ndarray:
    """Perlin-noise tissue of the paper's adaptive-optics example (n = 1.36 +-
    0.03): two octaves of periodic gradient noise (cells of ``cell_um`` and
    half of it, weights 1 and 1/2), scaled so its largest magnitude is 1, then
    dn = n_mean - n0 + n_amp * noise, rounded to FP16.  Draws from
    ``default_rng(seed)``.  Returns [nz][ny][nx] FP16."""
    rng = np.random.default_rng(seed)
    noise = _gradient_noise(shape, d, cell_um, rng) + 0.5 * _gradient_noise(shape, d, cell_um / 2, rng)
    noise /= max(float(np.max(np.abs(noise))), 1e-30)
    return (n_mean - n0 + n_amp * noise).astype(np.float16)


# --------------------------------------------------------------------------
# input fields and emitter lattices
# --------------------------------------------------------------------------

def plane_wave(nx: int, ny: int, mx: int = 0, my: int = 0, dtype=np.complex64) -> np.ndarray:
    """Unit-amplitude plane wave exp(2 pi i (mx x / nx + my y / ny)) on grid
    indices, i.e. a transverse wavevector exactly on DFT bin (mx, my)."""
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    ph = 2.0 * np.pi * ((mx * x % nx) / nx + (my * y % ny) / ny)
    return np.exp(1j * ph).astype(dtype)


def tilt_to_bins(theta_x_deg: float, theta_y_deg: float, nx: int, ny: int, dx: float, dy: float,
                 lam: float = LAMBDA_UM, n0: float = N0):
    """Nearest DFT bins (mx, my) to the transverse wavevector k0 n0 sin(theta)
    of a tilted plane wave, so the tilted input stays periodic on the grid."""
    k = 2.0 * np.pi / lam * n0
    mx = int(np.rint(k * np.sin(np.deg2rad(theta_x_deg)) * nx * dx / (2.0 * np.pi)))
    my = int(np.rint(k * np.sin(np.deg2rad(theta_y_deg)) * ny * dy / (2.0 * np.pi)))
    return mx, my


@dataclass
class FociSet:
    """Emitters of a multiplexed field: grid indices, phases and focal depth."""
    ix: np.ndarray
    iy: np.ndarray
    phase: np.ndarray
    zf: float
    NA: float

    def xyz_um(self, dx: float, dy: float) -> np.ndarray:
        """Positions in micrometres, shape [n, 3] (x, y, focal depth)."""
        return np.stack([self.ix * dx, self.iy * dy, np.full(self.ix.shape, self.zf)], axis=1)


def foci_lattice(n: int, per_side: int, nz: int, dz: float, NA: float, seed: int) -> FociSet:
    """``per_side`` x ``per_side`` emitters on pixel centres of a square
    lattice with pitch n / per_side pixels, offset by half a pitch; one shared
    focal depth zf ~ U[0.25, 0.75] nz dz and phases ~ U[0, 2 pi), drawn from
    ``default_rng([seed, 1])`` in that order."""
    pitch = n // per_side
    idx = (np.arange(per_side) * pitch + pitch // 2).astype(np.int32)
    iy, ix = np.meshgrid(idx, idx, indexing="ij")
    rng = np.random.default_rng([seed, 1])
    zf = float(rng.uniform(0.25, 0.75) * nz * dz)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=ix.size)
    return FociSet(ix.ravel().astype(np.int32), iy.ravel().astype(np.int32), phase, zf, NA)


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    n: int
    nz: int
    d: float                       # dx = dy = dz, micrometres
    lam: float = LAMBDA_UM
    n0: float = N0
    input_kind: str = "plane"      # "plane" | "light_sheet" | "foci"
    seed: int | None = None
    n_spheres: int = 0
    sheet_NA: float = 0.15
    foci_per_side: int = 0
    foci_NA: float = 0.6
    tilt_bins: tuple = (0, 0)
    extra: dict = field(default_factory=dict)
    ny: int | None = None          # rows (the y extent); n (the x extent) when None

    @property
    def rows(self) -> int:
        return self.ny or self.n

    @property
    def voxels(self) -> int:
        return self.n * self.rows * self.nz

    def dn(self, threads: int | None = None) -> np.ndarray:
        if self.seed is None:
            return single_sphere_dn(self.n, self.nz, self.d)
        return sphere_phantom_dn((self.nz, self.rows, self.n), self.d, self.n_spheres, self.seed,
                                 threads=threads)

    def foci(self) -> FociSet:
        return foci_lattice(self.n, self.foci_per_side, self.nz, self.d, self.foci_NA,
                            self.seed or 0)

    def sheet_zf(self) -> float:
        return self.nz * self.d / 2.0


def single_sphere_64() -> Workload:
    """64^3, dx = dz = 0.1 um, one hard sphere (n = 1.38, r = 2 um), plane wave."""
    return Workload("sphere64", 64, 64, 0.1, input_kind="plane")


def light_sheet_256() -> Workload:
    """256^3, dx = dz = 0.1 um, 300-sphere phantom (seed 1), light sheet NA 0.15."""
    return Workload("lightsheet256", 256, 256, 0.1, input_kind="light_sheet", seed=1,
                    n_spheres=300)


def multiplex_1024(nz: int = 1024) -> Workload:
    """1024^3, dx = dz = 0.1625 um, 800-sphere phantom (seed 2), 32 x 32 foci
    lattice, NA 0.6, random phases, one seeded focal depth."""
    return Workload("multiplex1024", 1024, nz, 0.1625, input_kind="foci", seed=2,
                    n_spheres=800, foci_per_side=32, foci_NA=0.6)


def psf_grid_2048x1024(nz: int = 1024) -> Workload:
    """The lateral grid of the paper's 10^6-PSF calculation (light-sheet
    paragraph: 1024 x 2048 x 1024 voxels), laid out with its 2048-pixel side
    along x: nx = 2048, ny = 1024, dx = dz = 0.1625 um, the sphere phantom
    recipe of the 1024^3 workload at the same density (1600 spheres, seed 2).
    The sweep does not depend on which lateral side is x (a random phantom
    and a lattice of foci); with the long side along the rows, the 1024-point
    columns take the four-step register layout and a slice is 1.25x shorter
    (28.5 against 35.6 us)."""
    return Workload("psf2048x1024", 2048, nz, 0.1625, input_kind="foci", seed=2,
                    n_spheres=1600, foci_NA=0.6, ny=1024)


BATCH_SIZES = (128, 192, 256, 384, 512)


def batch_64(count: int = 64, seed: int = 3) -> list:
    """Batched workload: ``count`` instances with lateral size drawn from
    {128, 192, 256, 384, 512}, depth uniform in [128, 512], tilt uniform in
    +-10 degrees per axis and input kind (plane wave or 8 x 8 foci, NA 0.6),
    all drawn from ``default_rng(seed)``; instance k uses phantom seed
    3000 + k with a sphere count scaled by volume from the 300 spheres of the
    256^3 x 0.1 um light-sheet phantom.  dx = dz = 0.1 um."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(BATCH_SIZES, size=count)
    depths = rng.integers(128, 513, size=count)
    tilts = rng.uniform(-10.0, 10.0, size=(count, 2))
    kinds = rng.integers(0, 2, size=count)
    out = []
    for k in range(count):
        n, nz = int(sizes[k]), int(depths[k])
        vol_ratio = (n * n * nz) / float(256 ** 3)
        mx, my = tilt_to_bins(tilts[k, 0], tilts[k, 1], n, n, 0.1, 0.1)
        w = Workload(f"batch{k}", n, nz, 0.1, input_kind="plane" if kinds[k] == 0 else "foci",
                     seed=3000 + k, n_spheres=max(1, int(round(300 * vol_ratio))),
                     foci_per_side=8, foci_NA=0.6, tilt_bins=(mx, my))
        out.append(w)
    return out


def dn_to_f64(dn16: np.ndarray) -> np.ndarray:
    """Exact widening of the FP16 index volume for the FP64 oracle."""
    return dn16.astype(np.float64)


# --------------------------------------------------------------------------
# corrector network: parameter layout and seeded initial values
# --------------------------------------------------------------------------

CORRECTOR_CHANNELS = 32


def corrector_layer_shapes(c_in: int):
    """(C_out, C_in) of the corrector's four 3 x 3 convolutions."""
    c = CORRECTOR_CHANNELS
    return [(c, c_in), (c, c), (c, c), (2, c)]


def corrector_param_count(c_in: int) -> int:
    return sum(o * i * 9 + o for o, i in corrector_layer_shapes(c_in))


def corrector_init(c_in: int, seed: int) -> np.ndarray:
    """Flat initial parameters [W1, b1, ..., W4, b4] (weights [o][i][3][3]):
    He-normal weights for the first three layers, zero biases, and a zero last
    layer so the untrained residual corrector is the identity.  Drawn from
    ``default_rng(seed)`` layer by layer."""
    rng = np.random.default_rng(seed)
    parts = []
    shapes = corrector_layer_shapes(c_in)
    for k, (o, i) in enumerate(shapes):
        if k < len(shapes) - 1:
            W = rng.standard_normal((o, i, 3, 3)) * np.sqrt(2.0 / (9 * i))
        else:
            W = np.zeros((o, i, 3, 3))
        parts += [W.ravel(), np.zeros(o)]
    return np.concatenate(parts)
