"""Wall-clock time of the FP64 CPU oracle on the paper's synthetic workloads
(test infrastructure: times the oracle, never the CUDA library).

    python -m oracle.time_configs [--skip-1024]

Prints one JSON line per workload: the 64^3 single sphere (plane wave), the
256^3 light sheet through the 300-sphere phantom, and the whole 1024^3
multiplexed-PSF propagation through the 800-sphere phantom (synthesis
included), each with voxel-steps/s and the OpenMP thread count.  The index
volumes are built before the clock starts; the intensity volume is computed
(the oracle stores |E|^2 of every slice, as the method does).
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

import oracle
from paper_1706_02261_b300 import inputs


def _time(fn):
    t0 = time.perf_counter()
    fn()
    return time.perf_counter() - t0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--skip-1024", action="store_true", help="only the 64^3 and 256^3 workloads")
    args = ap.parse_args(argv)
    oracle.build()
    rows = []
    w = inputs.single_sphere_64()
    dn = inputs.dn_to_f64(w.dn())
    E0 = inputs.plane_wave(w.n, w.n)
    dt = _time(lambda: oracle.bpm(dn, E0, w.d, w.d, w.d, w.lam, w.n0))
    rows.append(("sphere64: 64^3, plane wave, one n = 1.38 sphere of 2 um", w.n * w.n * w.nz, dt))
    w = inputs.light_sheet_256()
    dn = inputs.dn_to_f64(w.dn())

    def sheet():
        E0 = oracle.light_sheet(w.n, w.n, w.d, w.d, w.lam, w.n0, w.sheet_NA, w.sheet_zf())
        oracle.bpm(dn, E0, w.d, w.d, w.d, w.lam, w.n0)
    rows.append(("light_sheet256: 256^3, light sheet NA 0.15, 300 spheres", w.n * w.n * w.nz, _time(sheet)))
    if not args.skip_1024:
        w = inputs.multiplex_1024()
        dn16 = w.dn()
        f = w.foci()
        dn = inputs.dn_to_f64(dn16)
        del dn16

        def multiplex():
            E0 = oracle.multiplex_psf(w.n, w.n, w.d, w.d, w.lam, w.n0, f.ix, f.iy, f.phase, f.zf, f.NA)
            oracle.bpm(dn, E0, w.d, w.d, w.d, w.lam, w.n0)
        rows.append(("multiplex1024: 1024^3, 32x32 foci NA 0.6, 800 spheres (synthesis included)",
                     w.n * w.n * w.nz, _time(multiplex)))
    for name, vox, dt in rows:
        print(json.dumps({"workload": name, "seconds": dt, "voxel_steps_per_s": vox / dt,
                          "threads": oracle.num_threads(), "cpus": os.cpu_count(), "kind": "oracle (FP64, C, OpenMP)"}),
              flush=True)


if __name__ == "__main__":
    main()
