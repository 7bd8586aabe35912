"""Learned coarse-step corrector: data generation, training and evaluation.

Coarse split-steps of length 4 dz with the index screen averaged over the four
fine slices (bpm_coarsen_index) need a quarter of the transforms of the fine
method but add splitting error.  A small convolutional network f
(include/bpm_corrector.h) corrects the field after every coarse step,
E <- E + f(E).  Training pairs are produced by the propagation kernels
themselves: the input is one coarse step from the fine-step field at plane 4j,
the target is the fine-step field at plane 4j + 4, both divided by the RMS
amplitude of the input so the network sees fields of unit size.  Fine-step BPM is both the
fallback and the reference the corrector's error is measured against.

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


# --------------------------------------------------------------------------
# the 512^3 learned-corrector workload: training pairs as crops of full-size
# fine-step fields, evaluation of whole volumes
# --------------------------------------------------------------------------

@dataclass
class CropSetup:
    """Training pairs as 128^2 crops of full fine-step fields on the grid the
    corrector is applied to (512^2 x 512 slices of 0.1 um, the light-sheet
    phantom recipe scaled by volume), so that the pairs carry the depths,
    fields and phantoms of the evaluation workload."""
    n: int = 512
    nz: int = 512
    d: float = 0.1
    crop: int = 128
    lam: float = 0.5
    n0: float = 1.33
    c_in: int = 2

    def field_setup(self) -> Setup:
        return Setup(n=self.n, nz=self.nz, d=self.d, lam=self.lam, n0=self.n0, c_in=self.c_in)

    def phantom(self, seed: int):
        s = self.field_setup()
        return inputs.sphere_phantom_dn((s.nz, s.n, s.n), s.d, s.spheres(), seed)


def make_crop_pairs(cs: CropSetup, seeds, corr: "B.Corrector", dev, pairs_per_seed: int, rng_seed: int = 0,
                    phantoms=None):
    """For each seed: the fine-step field at every fourth plane 4j (one
    propagation through the phantom), one coarse step from each of those
    planes, both packed (divided by the RMS amplitude of the whole coarse
    field), then pairs_per_seed random (plane, crop) pairs of cs.crop^2
    crops on the crop lattice.  Returns (X, T) as float tensors."""
    import torch
    s = cs.field_setup()
    nzc = s.nz // FACTOR
    per = s.n // cs.crop
    rng = np.random.default_rng(rng_seed)
    fine = B.bpm_plan(B.Instance(s.n, s.nz, s.d, s.d, s.lam, s.n0))
    coarse = B.bpm_plan(B.Instance(s.n, nzc, s.d, s.d * FACTOR, s.lam, s.n0))
    xs, ts = [], []
    try:
        for si, seed in enumerate(seeds):
            dn_h = phantoms[si] if phantoms is not None else cs.phantom(seed)
            dn = torch.from_numpy(dn_h).to(dev)
            dnc = torch.empty((nzc, s.n, s.n), dtype=torch.float16, device=dev)
            B.bpm_coarsen_index(dn, FACTOR, dnc)
            E = input_field(s, seed, fine, dev)
            planes = torch.empty((nzc + 1, s.n, s.n), dtype=torch.complex64, device=dev)
            planes[0] = E
            for j in range(nzc):
                B.bpm_propagate(fine, dn, planes[j], planes[j + 1], None, FACTOR * j, FACTOR * (j + 1))
            ec = torch.empty((nzc, s.n, s.n), dtype=torch.complex64, device=dev)
            for j in range(nzc):
                B.bpm_propagate(coarse, dnc, planes[j], ec[j], None, j, j + 1)
            pick = rng.choice(nzc * per * per, size=min(pairs_per_seed, nzc * per * per), replace=False)
            j_of, c_of = pick // (per * per), pick % (per * per)
            X = torch.empty((nzc, s.c_in, s.n, s.n), dtype=torch.float32, device=dev)
            T = torch.empty((nzc, 2, s.n, s.n), dtype=torch.float32, device=dev)
            step = 16
            for j0 in range(0, nzc, step):
                j1 = min(nzc, j0 + step)
                corr.pack(ec[j0:j1], dnc[j0:j1] if s.c_in == 3 else None, s.dn_scale, X[j0:j1],
                          targets=planes[j0 + 1:j1 + 1], t=T[j0:j1])
            jj = torch.from_numpy(j_of).to(dev)
            cy = torch.from_numpy((c_of // per) * cs.crop).to(dev)
            cx = torch.from_numpy((c_of % per) * cs.crop).to(dev)
            ar = torch.arange(cs.crop, device=dev)
            ys = (cy[:, None] + ar[None, :])[:, :, None]            # [k][crop][1]
            xs_ = (cx[:, None] + ar[None, :])[:, None, :]           # [k][1][crop]
            xsel = X[jj]                                            # [k][c][n][n]
            tsel = T[jj]
            kk = torch.arange(len(pick), device=dev)[:, None, None]
            xs.append(torch.stack([xsel[:, c][kk, ys, xs_] for c in range(s.c_in)], 1).contiguous())
            ts.append(torch.stack([tsel[:, c][kk, ys, xs_] for c in range(2)], 1).contiguous())
            del X, T, xsel, tsel, planes, ec, dn, dnc
        assert B.bpm_check(fine) == 0 and B.bpm_check(coarse) == 0, B.bpm_last_error()
    finally:
        B.bpm_free(fine)
        B.bpm_free(coarse)
    return torch.cat(xs), torch.cat(ts)


def evaluate_volume(cs: CropSetup, seed: int, corr: "B.Corrector | None", dev, dn_h=None):
    """One held-out phantom through the whole volume by fine-step BPM (the
    reference), plain coarse steps, and coarse steps with the corrector.
    Errors against fine-step BPM: field relative L2 after the volume, and the
    peak-normalised maximum intensity error over the coarse planes (coarse
    plane j against fine slice 4j + 3, both after their last screen).  Times
    are CUDA events around each whole-volume propagation (intensity volumes
    written)."""
    import torch
    s = cs.field_setup()
    nzc = s.nz // FACTOR
    fine = B.bpm_plan(B.Instance(s.n, s.nz, s.d, s.d, s.lam, s.n0))
    coarse = B.bpm_plan(B.Instance(s.n, nzc, s.d, s.d * FACTOR, s.lam, s.n0))
    try:
        dn = torch.from_numpy(dn_h if dn_h is not None else cs.phantom(seed)).to(dev)
        dnc = torch.empty((nzc, s.n, s.n), dtype=torch.float16, device=dev)
        B.bpm_coarsen_index(dn, FACTOR, dnc)
        E0 = input_field(s, seed, fine, dev)
        If = torch.empty((s.nz, s.n, s.n), dtype=torch.float32, device=dev)
        Ic = torch.empty((nzc, s.n, s.n), dtype=torch.float32, device=dev)
        ef, ec = torch.empty_like(E0), torch.empty_like(E0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        # warm both plans once
        B.bpm_propagate(fine, dn, E0, ef, If)
        B.bpm_propagate(coarse, dnc, E0, ec, Ic)
        ev[0].record()
        B.bpm_propagate(fine, dn, E0, ef, If)
        ev[1].record()
        ev[2].record()
        B.bpm_propagate(coarse, dnc, E0, ec, Ic)
        ev[3].record()
        ref_planes = If[FACTOR - 1::FACTOR]
        peak = ref_planes.max()
        nrm = torch.linalg.vector_norm(ef)
        row = {"seed": seed,
               "coarse_field": float(torch.linalg.vector_norm(ec - ef) / nrm),
               "coarse_intensity": float((Ic - ref_planes).abs().max() / peak)}
        if corr is not None:
            # one corrected step outside the timed region (first-use set-up of
            # the kernels it launches)
            e = E0.clone()
            Icor = torch.empty_like(Ic)
            B.bpm_propagate(coarse, dnc, e, e, None, 0, 1)
            corr.apply(e, dnc[0] if s.c_in == 3 else None, s.dn_scale)
            torch.mul(e.real, e.real, out=Icor[0]).addcmul_(e.imag, e.imag)
            e = E0.clone()
            ev[4].record()
            for j in range(nzc):
                B.bpm_propagate(coarse, dnc, e, e, None, j, j + 1)
                corr.apply(e, dnc[j] if s.c_in == 3 else None, s.dn_scale)
                torch.mul(e.real, e.real, out=Icor[j]).addcmul_(e.imag, e.imag)
            ev[5].record()
            torch.cuda.synchronize()
            corr.check()
            row["corrected_field"] = float(torch.linalg.vector_norm(e - ef) / nrm)
            row["corrected_intensity"] = float((Icor - ref_planes).abs().max() / peak)
            row["corrected_ms"] = ev[4].elapsed_time(ev[5])
        torch.cuda.synchronize()
        row["fine_ms"] = ev[0].elapsed_time(ev[1])
        row["coarse_ms"] = ev[2].elapsed_time(ev[3])
        assert B.bpm_check(fine) == 0 and B.bpm_check(coarse) == 0, B.bpm_last_error()
        return row
    finally:
        B.bpm_free(fine)
        B.bpm_free(coarse)


def choose_path(held_out_rows, gate: float = 1e-3) -> str:
    """Fine-step BPM is the fallback and the reference: the corrected coarse path
    is used only when its intensity error against fine-step BPM on every
    held-out volume is within the gate, else propagation stays fine-step."""
    ok = all(r.get("corrected_intensity", np.inf) <= gate for r in held_out_rows)
    return "coarse+corrector" if ok else "fine"
