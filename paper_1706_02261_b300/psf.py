"""Multiplexed PSF sweep and de-multiplexing (Biobeam, arXiv:1706.02261,
method paragraph and the light-sheet simulation paragraph).

The paper computes 1e5-1e6 spatially varying PSFs by propagating highly
multiplexed fields: one field carries hundreds to thousands of mutually
independent, non-overlapping focused waves, and after one propagation the
intensity around each focus is that focus' PSF.  A sweep repeats this for a
set of focal depths.  Per field here:

    bpm_multiplex_psf      the multiplexed input (foci on a lattice, random phases)
    bpm_propagate_window   slices [0, window end), |E|^2 only inside the window
                           of pz slices around the focal slice
    bpm_demultiplex        one (pz, py, px) patch per focus

so a field costs the slices down to its window (not the whole depth) and
writes pz intensity slices (not nz).  All arithmetic runs in libbpm.so; this
module only chooses lattices, windows and buffers.

Depth convention: intensity slice z is recorded after slice z, at depth
(z + 1) dz, so a focus aimed at slice iz has focal depth (iz + 1) dz.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import bpm as B


@dataclass
class Sweep:
    n: int                      # lateral grid: n points along x (ny rows along y)
    nz: int                     # slices of the volume
    d: float                    # dx = dy = dz, um
    pitch: int                  # lattice pitch of the foci, pixels
    depths: list                # focal slice indices, one multiplexed field each
    patch: tuple = (32, 32, 64)  # (px, py, pz) voxels per PSF
    NA: float = 0.6
    lam: float = 0.5
    n0: float = 1.33
    seed: int = 0
    offset: int = field(default=-1)   # lattice offset in pixels (default pitch // 2)
    ny: int | None = None       # rows along y (n when None)

    @property
    def rows(self) -> int:
        return self.ny or self.n

    def lattice(self):
        """(ix, iy) of the foci of one field: a pitch-spaced lattice over the grid."""
        off = self.pitch // 2 if self.offset < 0 else self.offset
        ax = np.arange(off, self.n, self.pitch)
        ay = np.arange(off, self.rows, self.pitch)
        iy, ix = np.meshgrid(ay, ax, indexing="ij")
        return ix.ravel().astype(np.int64), iy.ravel().astype(np.int64)

    @property
    def foci_per_field(self) -> int:
        return len(self.lattice()[0])

    def window(self, iz: int):
        """Intensity window [w0, w1) of the field focused at slice iz: the
        patch's slices clipped to the volume; the propagation stops at w1."""
        pz = self.patch[2]
        w0 = min(self.nz, max(0, iz - pz // 2))
        w1 = min(self.nz, iz - pz // 2 + pz)
        return w0, max(w0, w1)

    def field_inputs(self, k: int):
        """Emitters of field k: (xyz in um, phases, (ix, iy, iz) triples)."""
        ix, iy = self.lattice()
        iz = int(self.depths[k])
        rng = np.random.default_rng([self.seed, k])
        phase = rng.uniform(0, 2 * np.pi, size=ix.size)
        xyz = np.stack([ix * self.d, iy * self.d, np.full(ix.size, (iz + 1) * self.d)], axis=1)
        foci = np.stack([ix, iy, np.full(ix.size, iz)], axis=1).astype(np.int32)
        return xyz, phase, foci


class Runner:
    """Device buffers and plan for a sweep through one index volume."""

    def __init__(self, s: Sweep, dn, stream=None):
        import torch
        self.s = s
        self.dn = dn
        self.stream = stream
        dev = dn.device
        self.plan = B.bpm_plan(B.Instance(s.n, s.nz, s.d, s.d, s.lam, s.n0, ny=s.rows))
        self.e0 = torch.empty((s.rows, s.n), dtype=torch.complex64, device=dev)
        self.e1 = torch.empty_like(self.e0)
        self.win = torch.empty((s.patch[2], s.rows, s.n), dtype=torch.float32, device=dev)

    def field(self, k: int, out) -> None:
        """PSF patches of field k into out [foci_per_field][pz][py][px]."""
        s = self.s
        xyz, phase, foci = s.field_inputs(k)
        w0, w1 = s.window(int(s.depths[k]))
        B.bpm_multiplex_psf(self.plan, 0, xyz, phase, s.NA, self.e0, self.stream)
        B.bpm_propagate_window(self.plan, self.dn, self.e0, self.e1, self.win[:max(w1 - w0, 1)], w0, w1,
                               0, w1, self.stream)
        B.bpm_demultiplex(self.plan, 0, self.win[:w1 - w0], w0, foci, s.patch, out, self.stream)

    def check(self) -> None:
        rc = B.bpm_check(self.plan)
        if rc != B.BPM_OK:
            raise RuntimeError(f"device error {rc}: {B.bpm_last_error()}")

    def free(self) -> None:
        B.bpm_free(self.plan)
