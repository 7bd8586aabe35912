#!/usr/bin/env python3
"""Benchmark of the split-step beam-propagation hot path on B300.

Workload (the paper's headline case, Biobeam arXiv:1706.02261 method
paragraph: a ~1000-PSF multiplexed field through 1024^3 voxels): a
1024 x 1024 x 1024 grid, dx = dz = 0.1625 um, lambda = 0.5 um, n0 = 1.33, a
seeded 800-sphere FP16 tissue phantom, and an input field of 32 x 32 focused
emitters (NA 0.6, random phases, one seeded focal depth).  Inputs are synthetic
(paper_1706_02261_b300.inputs); the paper uses no public dataset.

One step = the multiplexed input synthesis (bpm_multiplex_psf) plus the
propagation through all 1024 slices with the FP32 intensity volume written
(bpm_propagate).  The plan (propagator table, twiddles) is built once outside
the timed region, as a user reuses it for every field.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank propagates its own
replica of the workload on its own GPU (the path has no data exchange between
fields); the elapsed time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
# Slices per host-streaming chunk of the end-to-end leg.  The copies run at the
# host link's limit (pinned: 55 GB/s in, 57 GB/s out, 74.5 GB/s both at once on
# B300); what a smaller chunk saves is the pipeline's fill (first index chunk
# in) and drain (last intensity chunk out): 82.2 ms per 1024^3 step at 64
# slices, 80.9 ms at 16.
E2E_CHUNK = 16
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxel-steps/s (1024^3 multiplexed-PSF propagation)"
UNIT = "voxel-steps/s"
PAPER_VOXEL_STEPS_PER_S = 1024 ** 3 / 0.5     # "< 500 ms" per 1024^3 field (context)
FP32_LANES_PER_SM = 128


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["multiplex1024", "batch64", "corrector512", "psf1e6"],
                    default="multiplex1024",
                    help="multiplex1024: the headline 1024^3 multiplexed-PSF field (default); "
                         "batch64: 64 seeded instances of mixed sizes in one launch; "
                         "corrector512: 512^3 coarse steps with the learned corrector vs fine-step BPM")
    ap.add_argument("--nz", type=int, default=1024, help="slices (default: the full 1024)")
    ap.add_argument("--cpu-slices", type=int, default=128, help="slices in the oracle's timed sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT slice-loop comparison")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the batched workload that the default run also measures (one GPU)")
    ap.add_argument("--psf-fields", type=int, default=489,
                    help="psf1e6: multiplexed fields of 2048 foci (489 give 1.0e6 PSFs)")
    return ap.parse_args()


def step_flops(n: int, nz: int) -> float:
    """Algorithmic FLOPs of one propagation: per slice a forward and an inverse
    2D FFT credited 5 M log2 M each, the propagator and screen complex
    multiplies (6 M each) and |E|^2 (3 M)."""
    M = n * n
    return nz * (10.0 * M * math.log2(M) + 15.0 * M)


def step_bytes(n: int, nz: int) -> float:
    """Algorithmic HBM bytes of one propagation: FP16 index and FP32 intensity
    per voxel, plus the input and output fields."""
    M = n * n
    return nz * M * (2 + 4) + 2 * M * 8


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, device=None, ws: int = 1):
    """Each entry's largest value over the ranks (the slowest replica sets the
    job's time); the values themselves on a single rank."""
    if ws <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def shard_range(n: int, rank: int, ws: int):
    """Contiguous share [lo, hi) of n independent units for this rank (shares
    differ by at most one unit and cover [0, n) exactly)."""
    return (n * rank) // ws, (n * (rank + 1)) // ws


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


def make_workload(nz: int):
    from paper_1706_02261_b300 import inputs
    w = inputs.multiplex_1024(nz=nz)
    dn = w.dn()
    return w, dn, w.foci()


def cpu_baseline(w, dn16, foci, slices: int, want_output: bool = False):
    """The FP64 oracle, as it stands, on the first ``slices`` slices of the
    same workload (synthesis of the same multiplexed field + propagation).
    With ``want_output`` also returns the oracle's field after the sample and
    its intensity planes, for the parity figures of the bench line."""
    import oracle
    from paper_1706_02261_b300 import inputs
    dn64 = inputs.dn_to_f64(dn16[:slices])
    t0 = time.perf_counter()
    E0 = oracle.multiplex_psf(w.n, w.n, w.d, w.d, w.lam, w.n0, foci.ix, foci.iy, foci.phase, foci.zf, foci.NA)
    Er, Ir = oracle.bpm(dn64, E0, w.d, w.d, w.d, w.lam, w.n0)
    dt = time.perf_counter() - t0
    res = {"value": w.n * w.n * slices / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{w.n}x{w.n}x{slices} slices of the 1024^3 workload incl. the multiplexed synthesis "
                     f"({dt:.1f} s)"}
    return (res, Er, Ir) if want_output else res


def parity_figures(Eg, Ig, Er, Ir, slices: int):
    """Error of the GPU's results against the FP64 oracle on the same inputs:
    field relative L2 after the sample's last slice, and the peak-normalised
    maximum intensity error over the sample's planes."""
    Eg = np.asarray(Eg, np.complex128)
    field = float(np.linalg.norm(Eg - Er) / np.linalg.norm(Er))
    num, peak = 0.0, 0.0
    for z in range(slices):
        num = max(num, float(np.max(np.abs(np.asarray(Ig[z], np.float64) - Ir[z]))))
        peak = max(peak, float(np.max(Ir[z])))
    return {"slices": slices, "field_rel_l2": field, "intensity_rel_max": num / peak,
            "gates": {"field_rel_l2": 1e-4, "intensity_rel_max": 1e-3},
            "reference": "FP64 CPU oracle (oracle/bpm_oracle.c) on the same FP16 index values and emitter list"}


def workload_name(w, nz: int) -> str:
    """The headline workload as both arms name it in their config."""
    return (f"multiplex1024: {w.n}x{w.n}x{nz} voxels, dx=dz={w.d} um, lambda={w.lam} um, "
            f"n0={w.n0}, 800-sphere FP16 phantom (seed 2), 32x32 foci NA 0.6")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w, dn16, foci = make_workload(args.nz)
    k = max(1, args.cpu_slices // 8)      # a bounded sample per step
    for _ in range(max(0, min(args.warmup, 1))):
        cpu_baseline(w, dn16, foci, 1)
    times = []
    cores = 1
    for _ in range(args.steps):
        r = cpu_baseline(w, dn16, foci, k)
        cores = r["cores"]
        times.append(w.n * w.n * k / r["value"])
    t = statistics.mean(times)
    value = w.n * w.n * k / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(w, dn16.shape[0]), "parallelism": "single host (FP64 CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{k} slices of {w.n}x{w.n} per step of that workload, with the "
                                       f"multiplexed synthesis"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cufft_slice_loop(w, dn_d, e0, eout_ours, stream):
    """Comparison only: the same split-step through torch.fft (cuFFT) and
    torch pointwise kernels, one slice at a time, timed once over the whole
    depth with the intensity volume written.  Not part of the product path."""
    import torch
    n, nz = w.n, dn_d.shape[0]
    dev = dn_d.device
    k0 = 2 * math.pi / w.lam
    K = k0 * w.n0
    k = 2 * math.pi * np.fft.fftfreq(n, w.d)
    kz2 = K * K - k[None, :] ** 2 - k[:, None] ** 2
    H = np.where(kz2 > 0, np.exp(1j * np.sqrt(np.maximum(kz2, 0)) * w.d), 0)
    Hd = torch.from_numpy(H.astype(np.complex64)).to(dev)
    inten = torch.empty((nz, n, n), dtype=torch.float32, device=dev)
    scale = k0 * w.d

    def volume(zn):
        e = e0.clone()
        for z in range(zn):
            e = torch.fft.ifft2(torch.fft.fft2(e) * Hd)
            phase = dn_d[z].float() * scale
            e = e * torch.polar(torch.ones_like(phase), phase)
            inten[z] = e.real * e.real + e.imag * e.imag
        return e

    with torch.cuda.stream(stream):
        volume(8)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        e = volume(nz)
        b.record(stream)
        torch.cuda.synchronize(dev)
    t = a.elapsed_time(b) / 1e3
    err = float(torch.linalg.vector_norm(e - eout_ours) / torch.linalg.vector_norm(eout_ours))
    return {"ms_per_volume": t * 1e3, "value": float(n) * n * nz / t, "unit": UNIT,
            "kind": "torch.fft (cuFFT) fft2/ifft2 + torch pointwise per slice, eager, FP32",
            "field_rel_l2_vs_ours": err}


def _kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("bpm_kernels.cuh", "fft.cuh", "bpm_args.cuh", "bpm_ops.cuh", "ops_1024.cu"):
        with open(os.path.join(ROOT, "paper_1706_02261_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the CUDA library is the only compute path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=dev)
    from paper_1706_02261_b300 import build as build_mod
    build_mod.build()
    from paper_1706_02261_b300 import bpm as B

    w, dn16, foci = make_workload(args.nz)
    n, nz = w.n, w.nz
    xyz = foci.xyz_um(w.d, w.d)
    stream = torch.cuda.current_stream(dev)

    t0 = time.perf_counter()
    plan = B.bpm_plan(B.Instance(n, nz, w.d, w.d, w.lam, w.n0))
    plan_ms = (time.perf_counter() - t0) * 1e3
    info = B.bpm_plan_info(plan)
    dn_d = torch.from_numpy(dn16).to(dev)
    e0 = torch.empty((n, n), dtype=torch.complex64, device=dev)
    eout = torch.empty_like(e0)
    inten = torch.empty((nz, n, n), dtype=torch.float32, device=dev)

    kev = []

    def step(record=False):
        B.bpm_multiplex_psf(plan, 0, xyz, foci.phase, foci.NA, e0, stream)
        if record:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            B.bpm_propagate(plan, dn_d, e0, eout, inten, 0, nz, stream)
            b.record(stream)
            kev.append((a, b))
        else:
            B.bpm_propagate(plan, dn_d, e0, eout, inten, 0, nz, stream)

    for _ in range(args.warmup):
        step()
    if B.bpm_check(plan) != 0:
        raise SystemExit(f"device error during warm-up: {B.bpm_last_error()}")

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    with ClockSampler(local) as clocks:
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step(record=True)
        ev1.record(stream)
        barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    if B.bpm_check(plan) != 0:
        raise SystemExit(f"device error in the timed region: {B.bpm_last_error()}")
    kern_s = statistics.mean(a.elapsed_time(b) for a, b in kev) / 1e3
    elapsed, kern_s = max_over_ranks([elapsed, kern_s], dev, ws)
    vox = float(n) * n * nz
    value = vox * args.steps * ws / elapsed

    # end to end through the C ABI with host buffers: every step synthesises
    # the input on the device from the host emitter list and runs
    # bpm_propagate_host, which streams the index volume in and the intensity
    # volume out (pinned host memory) overlapping the propagation
    e2e = None
    e2e_window = None
    if not args.no_e2e:
        dn_h = torch.from_numpy(dn16).pin_memory()
        i_h = torch.empty((nz, n, n), dtype=torch.float32).pin_memory()
        e_h = torch.empty((n, n), dtype=torch.complex64).pin_memory()

        def e2e_step():
            B.bpm_multiplex_psf(plan, 0, xyz, foci.phase, foci.NA, e0, stream)
            B.bpm_propagate_host(plan, dn_h, e0, e_h, i_h, E2E_CHUNK, stream)

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e_s, = max_over_ranks([e2e_s], dev, ws)
        e2e = {"value": vox * args.steps * ws / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(dn_h.numel() * dn_h.element_size() + xyz.nbytes + foci.phase.nbytes),
               "d2h_bytes_per_step": int(i_h.numel() * 4 + e_h.numel() * 8),
               "ms_per_step": e2e_s / args.steps * 1e3, "api": f"bpm_multiplex_psf + bpm_propagate_host (chunk {E2E_CHUNK})"}
        del dn_h, i_h

        # the reduced form a multiplexed-PSF user needs: the index volume stays
        # on the device (one sample, many fields), each step sends the emitter
        # list and reads back the 64 intensity slices around the focal depth
        # (the PSFs) and the output field
        WIN = 64
        zf_slice = int(round(foci.zf / w.d)) - 1
        w0 = max(0, min(nz - WIN, zf_slice - WIN // 2))
        win_d = torch.empty((WIN, n, n), dtype=torch.float32, device=dev)
        win_h = torch.empty((WIN, n, n), dtype=torch.float32).pin_memory()
        xyz_h = torch.from_numpy(np.ascontiguousarray(xyz)).pin_memory().numpy()
        ph_h = torch.from_numpy(np.ascontiguousarray(foci.phase)).pin_memory().numpy()

        def e2e_win_step():
            B.bpm_multiplex_psf(plan, 0, xyz_h, ph_h, foci.NA, e0, stream)
            B.bpm_propagate_window(plan, dn_d, e0, eout, win_d, w0, w0 + WIN, 0, nz, stream)
            win_h.copy_(win_d, non_blocking=True)
            e_h.copy_(eout, non_blocking=True)
            stream.synchronize()

        e2e_win_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_win_step()
        barrier()
        ew_s = time.perf_counter() - t0
        ew_s, = max_over_ranks([ew_s], dev, ws)
        e2e_window = {"value": vox * args.steps * ws / ew_s, "unit": UNIT,
                      "h2d_bytes_per_step": int(xyz.nbytes + foci.phase.nbytes),
                      "d2h_bytes_per_step": int(win_h.numel() * 4 + e_h.numel() * 8),
                      "ms_per_step": ew_s / args.steps * 1e3,
                      "api": f"bpm_multiplex_psf + bpm_propagate_window (index volume resident on the device, "
                             f"|E|^2 of slices [{w0}, {w0 + WIN}) around the focal depth read back)"}

    peaks, peak_src = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    props = torch.cuda.get_device_properties(dev)
    alu_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = step_flops(n, nz) / kern_s / 1e12
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "persistent1024_traffic.json")
    if os.path.exists(tfile):
        with open(tfile) as f:
            tj = json.load(f)
        if tj.get("kernel_source_hash") == _kernel_hash():
            traffic = tj.get("bytes_per_full_launch")
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": traffic,
                "peak_source": f"derived: {props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 "
                               f"x {sm_max:.0f} MHz ({peak_src} max SM clock)",
                "kernel": "bpm_persistent_kernel<1024>", "kernel_ms": kern_s * 1e3,
                "algorithmic_flops": step_flops(n, nz), "algorithmic_bytes": step_bytes(n, nz),
                "hbm_achieved_gbs": step_bytes(n, nz) / kern_s / 1e9, "hbm_peak_gbs": hbm_peak,
                "hbm_frac_of_measured": step_bytes(n, nz) / kern_s / 1e9 / hbm_peak}

    cufft = None
    if not args.no_cufft:
        cufft = cufft_slice_loop(w, dn_d, e0, eout, stream)

    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu:
        ks = min(args.cpu_slices, nz)
        cpu, Er, Ir = cpu_baseline(w, dn16, foci, ks, want_output=True)
        # the same sample on the GPU: the timed steps' intensity planes
        # [0, ks) and the field after slice ks (one more call, untimed)
        ek = torch.empty_like(e0)
        B.bpm_propagate(plan, dn_d, e0, ek, None, 0, ks, stream)
        if B.bpm_check(plan) != 0:
            raise SystemExit(f"device error in the parity call: {B.bpm_last_error()}")
        parity = parity_figures(ek.cpu().numpy(), inten[:ks].cpu().numpy(), Er, Ir, ks)
        del Er, Ir

    # the batched workload in the same run (driver-visible), timed after the
    # headline's own measurements
    secondary = None
    if rank == 0 and ws == 1 and not args.no_secondary:
        sec_args = argparse.Namespace(**vars(args))
        sec_args.steps, sec_args.warmup = 5, 3
        bl = batch_line(sec_args)
        secondary = {"batch64": {k: bl[k] for k in ("metric", "value", "unit", "ms_per_step", "steps", "warmup",
                                                    "config", "sequential_single_plans", "roofline", "clocks")}}

    launches_per_step = 6     # pupil count, scatter, 3 synthesis half-steps, persistent propagation (device leg)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": value / (PAPER_VOXEL_STEPS_PER_S * ws), "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(w, nz),
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": "inputs larger than L2 (2 GiB index volume, 4 GiB intensity volume per step)",
                       "team_ctas": info["team_ctas"], "plan_ms": plan_ms},
            "roofline": roofline, "clocks": clocks.summary(), "gpu_launches": launches_per_step * args.steps,
            "e2e": e2e, "e2e_window": e2e_window, "cpu_baseline": cpu, "parity": parity, "cufft_comparison": cufft,
            "secondary": secondary}
    if rank == 0:
        print(json.dumps(line), flush=True)
    B.bpm_free(plan)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def batch_line(args):
    """64 seeded instances (128^2..512^2, 128-512 slices, tilted plane waves or
    8 x 8 multiplexed foci) propagated in one graph-captured persistent launch,
    and the same instances propagated one plan at a time for comparison;
    returns the JSON line of this workload."""
    import torch
    from paper_1706_02261_b300 import build as build_mod
    from paper_1706_02261_b300 import inputs
    build_mod.build()
    from paper_1706_02261_b300 import bpm as B

    dev = torch.device("cuda", 0)
    ws = inputs.batch_64()
    stream = torch.cuda.current_stream(dev)
    plan = B.bpm_plan([B.Instance(w.n, w.nz, w.d, w.d, w.lam, w.n0) for w in ws], flags=B.BPM_FLAG_GRAPH)
    dns, eins = [], []
    for k, w in enumerate(ws):
        dns.append(torch.from_numpy(w.dn()).to(dev))
        if w.input_kind == "plane":
            eins.append(torch.from_numpy(inputs.plane_wave(w.n, w.n, *w.tilt_bins)).to(dev))
        else:
            f = w.foci()
            e = torch.empty((w.n, w.n), dtype=torch.complex64, device=dev)
            B.bpm_multiplex_psf(plan, k, f.xyz_um(w.d, w.d), f.phase, f.NA, e, stream)
            eins.append(e)
    eout = [torch.empty_like(e) for e in eins]
    inten = [torch.empty((w.nz, w.n, w.n), dtype=torch.float32, device=dev) for w in ws]
    t0 = time.perf_counter()
    B.bpm_autotune(plan, dns, eins, eout, inten, 32, stream)
    tune_s = time.perf_counter() - t0
    info = B.bpm_plan_info(plan)
    for _ in range(args.warmup):
        B.bpm_propagate(plan, dns, eins, eout, inten, 0, 2 ** 31 - 1, stream)
    if B.bpm_check(plan) != 0:
        raise SystemExit(B.bpm_last_error())
    with ClockSampler(0) as clocks:
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            B.bpm_propagate(plan, dns, eins, eout, inten, 0, 2 ** 31 - 1, stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    if B.bpm_check(plan) != 0:
        raise SystemExit(B.bpm_last_error())
    t_batch = ev0.elapsed_time(ev1) / 1e3 / args.steps
    vox = float(sum(w.n * w.n * w.nz for w in ws))
    flops = sum(step_flops(w.n, w.nz) for w in ws)
    B.bpm_free(plan)
    # the same instances, one single-instance plan (cooperative persistent launch) each
    plans = [B.bpm_plan(B.Instance(w.n, w.nz, w.d, w.d, w.lam, w.n0)) for w in ws]
    def seq():
        for p, dn, ei, eo, it in zip(plans, dns, eins, eout, inten):
            B.bpm_propagate(p, dn, ei, eo, it, 0, 2 ** 31 - 1, stream)
    seq()
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(max(1, args.steps // 2)):
        seq()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    t_seq = ev0.elapsed_time(ev1) / 1e3 / max(1, args.steps // 2)
    for p in plans:
        B.bpm_free(p)
    peaks, peak_src = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    props = torch.cuda.get_device_properties(dev)
    alu_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    line = {"metric": "voxel-steps/s (64 batched instances, 128^2-512^2 x 128-512 slices)", "value": vox / t_batch,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch64: 64 seeded instances (default_rng(3)), sizes {128,192,256,384,512}^2, "
                                   "128-512 slices, tilted plane waves or 8x8 foci NA 0.6, phantoms seeds 3000+k",
                       "voxel_steps": vox, "cluster_ctas": info["team_ctas"], "schedule_set": info["schedule"],
                       "autotune_s": tune_s,
                       "graph": True},
            "sequential_single_plans": {"ms_per_step": t_seq * 1e3, "value": vox / t_seq,
                                        "speedup_batched": t_seq / t_batch},
            "roofline": {"bound": "alu", "achieved": flops / t_batch / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": flops / t_batch / 1e12 / alu_peak, "traffic": None,
                         "kernel": "bpm_batch_kernel", "peak_source": f"derived ({peak_src} max SM clock)"},
            "clocks": clocks.summary(), "gpu_launches": args.steps, "e2e": None, "cpu_baseline": None}
    return line


def run_batch(args):
    print(json.dumps(batch_line(args)), flush=True)
    return 0


def run_psf(args):
    """The paper's 10^6-PSF calculation on its grid (light-sheet paragraph:
    1024 x 2048 x 1024 voxels, laid out as 2048 x 1024 lateral pixels, the
    long side along the rows): multiplexed fields of 64 x 32 foci (pitch 32
    px, NA 0.6) swept over focal depths through the sphere phantom; per field
    the synthesis, the propagation down to the end of the 64-slice window
    around the focal depth with |E|^2 written only in that window, and the
    de-multiplexing into one 32 x 32 x 64 patch per focus."""
    import torch
    from paper_1706_02261_b300 import build as build_mod
    from paper_1706_02261_b300 import inputs
    build_mod.build()
    from paper_1706_02261_b300 import psf

    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)
    w = inputs.psf_grid_2048x1024(nz=1024)
    dn = torch.from_numpy(w.dn()).to(dev)
    F = args.psf_fields
    # focal slices spread evenly over [32, 992) so that every window lies inside the volume
    depths = [32 + (k * 960) // max(F, 1) for k in range(F)]
    s = psf.Sweep(n=w.n, nz=w.nz, d=w.d, pitch=32, depths=depths, patch=(32, 32, 64), NA=0.6, seed=2, ny=w.rows)
    r = psf.Runner(s, dn, stream)
    # the fields are independent: each rank takes a contiguous share of the
    # depths (no collective on the data path; the slowest rank sets the time)
    k0, k1 = shard_range(F, rank, ws)
    outs = [torch.empty((s.foci_per_field, 64, 32, 32), dtype=torch.float32, device=dev) for _ in range(2)]
    for k in range(args.warmup):
        r.field(k0 + k % max(1, k1 - k0), outs[k & 1])
    r.check()
    with ClockSampler(local) as clocks:
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev0.record(stream)
        for k in range(k0, k1):
            r.field(k, outs[k & 1])
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        wall = time.perf_counter() - t0
    r.check()
    r.free()
    t, wall = max_over_ranks([ev0.elapsed_time(ev1) / 1e3, wall], dev, ws)
    n_psf = F * s.foci_per_field
    slices = sum(s.window(z)[1] for z in depths)
    line = {"metric": "PSFs/s (multiplexed PSF sweep through 2048x1024x1024, 32x32x64-voxel patches)",
            "value": n_psf / t, "unit": "PSFs/s", "n_gpus": ws, "steps": F, "warmup": args.warmup,
            "ms_per_step": t / F * 1e3, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"psf1e6: {F} fields x {s.foci_per_field} foci (pitch 32 px, NA 0.6) through the "
                                   f"{w.n}x{w.rows}x{w.nz} 1600-sphere phantom (seed 2), focal slices 32..991, "
                                   "window 64 slices",
                       "psfs": n_psf, "slices_propagated": slices, "voxel_steps": float(slices) * w.n * w.rows,
                       "seconds_for_1e6_psfs": t * 1e6 / n_psf, "wall_s": wall,
                       "paper": "10^6 PSFs 'in well under 10 minutes' on one graphics card (context)"},
            "voxel_steps_per_s": float(slices) * w.n * w.rows / t,
            "clocks": clocks.summary(), "gpu_launches": F * 7, "e2e": None, "cpu_baseline": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_corrector(args):
    """The learned coarse-step corrector at 512^3 (lambda 0.5 um, n0 1.33, the
    light-sheet phantom recipe): a 2-channel network (field only, the
    specified one) and a 3-channel one (field and averaged index step, a
    deviation) trained on 20480 pairs of 128^2 crops cut from fine-step BPM
    fields of 20 seeded 512^3 phantoms (seeds 4000-4019, 1024 pairs each),
    then fine-step BPM (512 x 0.1 um), plain coarse steps (128 x 0.4 um) and
    coarse steps with the corrector on 10 held-out phantoms (seeds
    5000-5009), errors against fine-step BPM and times per volume."""
    import torch
    from paper_1706_02261_b300 import build as build_mod
    from paper_1706_02261_b300 import inputs
    build_mod.build()
    from paper_1706_02261_b300 import bpm as B
    from paper_1706_02261_b300 import corrector as C

    dev = torch.device("cuda", 0)
    train_seeds = list(range(4000, 4020))
    held_out = list(range(5000, 5010))
    cs0 = C.CropSetup()
    t0 = time.perf_counter()
    train_ph = [cs0.phantom(sd) for sd in train_seeds]
    test_ph = [cs0.phantom(sd) for sd in held_out]
    phantom_s = time.perf_counter() - t0
    res = {}
    for c_in in (2, 3):
        cs = C.CropSetup(c_in=c_in)
        corr = B.Corrector(c_in, 32, cs.n, cs.n)
        corr.set_params(inputs.corrector_init(c_in, 0).astype(np.float32))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        X, T = C.make_crop_pairs(cs, train_seeds, corr, dev, 1024, rng_seed=c_in, phantoms=train_ph)
        torch.cuda.synchronize(dev)
        gen_s = time.perf_counter() - t0
        corr.set_residual_scale(C.residual_scale(corr, X, T, batch=32))
        # time of one training step (batch 32 of 128^2) on each engine, then
        # the training itself on the tensor cores
        step_ms = {}
        for tc_on in (False, True):
            corr.set_train_tensor_cores(tc_on)
            C.train(corr, X[:32], T[:32], steps=3, batch=32, lr=1e-12, seed=0)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            C.train(corr, X, T, steps=50, batch=32, lr=1e-12, seed=0)
            torch.cuda.synchronize(dev)
            step_ms["tensor_cores" if tc_on else "fp32_pipes"] = (time.perf_counter() - t0) / 50 * 1e3
        corr.set_params(inputs.corrector_init(c_in, 0).astype(np.float32))
        corr.set_train_tensor_cores(True)
        t0 = time.perf_counter()
        losses = C.train(corr, X, T, steps=6000, batch=32, lr=1e-3, seed=1, log_every=1000)
        losses += C.train(corr, X, T, steps=2000, batch=32, lr=2.5e-4, seed=2, log_every=1000)
        torch.cuda.synchronize(dev)
        corr.check()
        train_s = time.perf_counter() - t0
        del X, T
        rows = [C.evaluate_volume(cs, sd, corr, dev, dn_h=ph) for sd, ph in zip(held_out, test_ph)]
        corr.free()
        mean = lambda k: float(np.mean([r[k] for r in rows]))
        res[f"c_in={c_in}"] = {"pairs": 20480, "pair_generation_s": gen_s, "train_s": train_s, "train_steps": 8000,
                               "batch": 32, "train_engine": "tensor cores (tcgen05, BF16 operands)",
                               "train_step_ms": step_ms, "loss_trace": losses, "held_out_512": rows,
                               "mean": {k: mean(k) for k in ("coarse_field", "coarse_intensity", "corrected_field",
                                                             "corrected_intensity", "fine_ms", "coarse_ms",
                                                             "corrected_ms")},
                               "path_chosen_at_1e-3": C.choose_path(rows, 1e-3)}
    m2 = res["c_in=2"]["mean"]
    t_corr = m2["corrected_ms"] / 1e3
    line = {"metric": "fine-equivalent voxel-steps/s of 512^3 coarse steps with the learned corrector",
            "value": 512.0 ** 3 / t_corr, "unit": UNIT, "n_gpus": 1, "steps": len(held_out), "warmup": 1,
            "ms_per_step": t_corr * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (BF16 weights)", "data": "synthetic",
            "config": {"workload": "corrector512: 512^3, dz 0.1 um fine / 0.4 um coarse, light-sheet phantom recipe "
                                   "(2400 spheres), training seeds 4000-4019 (20480 crops of 128^2), held-out "
                                   "seeds 5000-5009", "phantom_generation_s": phantom_s},
            "fine_bpm_ms": m2["fine_ms"], "coarse_bpm_ms": m2["coarse_ms"],
            "errors_vs_fine_2ch": {k: m2[k] for k in ("coarse_field", "coarse_intensity", "corrected_field",
                                                      "corrected_intensity")},
            "intensity_gate": 1e-3,
            "network": "tcgen05 kind::f16 implicit-GEMM convolutions (BF16 activations, FP32 accumulation)",
            "results": res, "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "corrector512":
        return run_corrector(args)
    if args.workload == "psf1e6":
        return run_psf(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
