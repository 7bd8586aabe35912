"""Learned coarse-step corrector: data generation, training and evaluation.

Coarse split-steps of length 4 dz with the index screen averaged over the four
fine slices (bpm_coarsen_index) need a quarter of the transforms of the fine
method but add splitting error.  A small convolutional network f
(include/bpm_corrector.h) corrects the field after every coarse step,
E <- E + f(E).  Training pairs are produced by the propagation kernels
themselves: the input is one coarse step from the fine-step field at plane 4j,
the target is the fine-step field at plane 4j + 4, both divided by the RMS
amplitude of the input so the network sees fields of unit size.  Fine-step BPM is both the
fallback and the judge of the corrector's error.

This module only orchestrates calls into libbpm.so (all arithmetic runs in its
kernels); torch provides device memory and batching of tensors.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import bpm as B
from . import inputs

FACTOR = 4


@dataclass
class Setup:
    n: int = 128            # lateral grid
    nz: int = 64            # fine slices per field
    d: float = 0.1          # dx = dz of the fine grid, um
    lam: float = 0.5
    n0: float = 1.33
    c_in: int = 2           # 2: field only; 3: field and averaged index step

    @property
    def dn_scale(self) -> float:
        """Scale of the index channel: the coarse step's screen phase per unit dn."""
        return 2 * math.pi / self.lam * self.d * FACTOR

    def spheres(self) -> int:
        """Sphere count of the 256^3 x 0.1 um light-sheet phantom (300), scaled by volume."""
        return max(1, int(round(300 * self.n * self.n * self.nz / 256 ** 3)))


def input_field(s: Setup, seed: int, plan, dev):
    """Seeded input: tilted plane wave, light sheet or 4 x 4 multiplexed foci (by seed mod 3)."""
    import torch
    rng = np.random.default_rng([seed, 7])
    kind = seed % 3
    if kind == 0:
        tx, ty = rng.uniform(-10, 10, size=2)
        mx, my = inputs.tilt_to_bins(tx, ty, s.n, s.n, s.d, s.d, s.lam, s.n0)
        return torch.from_numpy(inputs.plane_wave(s.n, s.n, mx, my)).to(dev)
    e = torch.empty((s.n, s.n), dtype=torch.complex64, device=dev)
    if kind == 1:
        B.bpm_light_sheet(plan, 0, 0.15, s.nz * s.d / 2, e)
    else:
        f = inputs.foci_lattice(s.n, 4, s.nz, s.d, 0.6, seed)
        B.bpm_multiplex_psf(plan, 0, f.xyz_um(s.d, s.d), f.phase, f.NA, e)
    return e


def make_pairs(s: Setup, seeds, corr: "B.Corrector", dev):
    """Training pairs (packed coarse-step inputs X, fine targets T) for every
    coarse step of every seed's field."""
    import torch
    fine = B.bpm_plan(B.Instance(s.n, s.nz, s.d, s.d, s.lam, s.n0))
    coarse = B.bpm_plan(B.Instance(s.n, s.nz // FACTOR, s.d, s.d * FACTOR, s.lam, s.n0))
    xs, ts = [], []
    try:
        for seed in seeds:
            dn = torch.from_numpy(inputs.sphere_phantom_dn((s.nz, s.n, s.n), s.d, s.spheres(), seed)).to(dev)
            dnc = torch.empty((s.nz // FACTOR, s.n, s.n), dtype=torch.float16, device=dev)
            B.bpm_coarsen_index(dn, FACTOR, dnc)
            E = input_field(s, seed, fine, dev)
            planes = [E.clone()]
            for j in range(s.nz // FACTOR):
                B.bpm_propagate(fine, dn, E, E, None, FACTOR * j, FACTOR * (j + 1))
                planes.append(E.clone())
            ein = torch.stack(planes[:-1])
            ec = torch.empty_like(ein)
            for j in range(s.nz // FACTOR):
                B.bpm_propagate(coarse, dnc, ein[j], ec[j], None, j, j + 1)
            x = torch.empty((ein.shape[0], s.c_in, s.n, s.n), dtype=torch.float32, device=dev)
            t = torch.empty((ein.shape[0], 2, s.n, s.n), dtype=torch.float32, device=dev)
            corr.pack(ec, dnc if s.c_in == 3 else None, s.dn_scale, x, targets=torch.stack(planes[1:]), t=t)
            xs.append(x)
            ts.append(t)
        assert B.bpm_check(fine) == 0 and B.bpm_check(coarse) == 0, B.bpm_last_error()
    finally:
        B.bpm_free(fine)
        B.bpm_free(coarse)
    return torch.cat(xs), torch.cat(ts)


def residual_scale(corr: "B.Corrector", X, T, batch: int = 16) -> float:
    """RMS size of the corrections over the training pairs, measured with the
    network's own loss kernel while its last layer is still zero (f = 0)."""
    total, count = 0.0, 0
    for k in range(0, X.shape[0], batch):
        xb, tb = X[k:k + batch], T[k:k + batch]
        total += corr.loss_grad(xb, tb) * xb.shape[0]
        count += xb.shape[0]
    return math.sqrt(total / count)


def train(corr: "B.Corrector", X, T, steps: int, batch: int = 16, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0):
    """Adam on random mini-batches; returns the losses that were read back."""
    import torch
    rng = np.random.default_rng(seed)
    losses = []
    for k in range(steps):
        idx = torch.from_numpy(rng.choice(X.shape[0], size=min(batch, X.shape[0]), replace=False)).to(X.device)
        want = log_every and (k % log_every == 0 or k == steps - 1)
        loss = corr.train_step(X[idx], T[idx], lr, want_loss=bool(want))
        if want:
            losses.append((k, loss))
    return losses


def evaluate(s: Setup, seeds, corr: "B.Corrector | None", dev):
    """Relative L2 error against fine-step BPM of the field after the whole
    volume, for coarse steps with the corrector (when given) and without."""
    import torch
    fine = B.bpm_plan(B.Instance(s.n, s.nz, s.d, s.d, s.lam, s.n0))
    coarse = B.bpm_plan(B.Instance(s.n, s.nz // FACTOR, s.d, s.d * FACTOR, s.lam, s.n0))
    out = []
    try:
        for seed in seeds:
            dn = torch.from_numpy(inputs.sphere_phantom_dn((s.nz, s.n, s.n), s.d, s.spheres(), seed)).to(dev)
            dnc = torch.empty((s.nz // FACTOR, s.n, s.n), dtype=torch.float16, device=dev)
            B.bpm_coarsen_index(dn, FACTOR, dnc)
            E0 = input_field(s, seed, fine, dev)
            ef = torch.empty_like(E0)
            B.bpm_propagate(fine, dn, E0, ef, None)
            ec = E0.clone()
            B.bpm_propagate(coarse, dnc, ec, ec, None)
            row = {"seed": seed, "coarse": float(torch.linalg.vector_norm(ec - ef) / torch.linalg.vector_norm(ef))}
            if corr is not None:
                e = E0.clone()
                for j in range(s.nz // FACTOR):
                    B.bpm_propagate(coarse, dnc, e, e, None, j, j + 1)
                    corr.apply(e, dnc[j] if s.c_in == 3 else None, s.dn_scale)
                row["corrected"] = float(torch.linalg.vector_norm(e - ef) / torch.linalg.vector_norm(ef))
            out.append(row)
        assert B.bpm_check(fine) == 0 and B.bpm_check(coarse) == 0, B.bpm_last_error()
    finally:
        B.bpm_free(fine)
        B.bpm_free(coarse)
    return out
