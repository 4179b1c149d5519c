"""Studies run on the engine (one GPU).

  python -m paper_2005_14454_gb300.study precision [--size 512] [--steps 2000] [--box 48]

precision: the same Minkowski run (a = 1, no damping; lambda0 = 2, e0 = 1, sigma = 1,
dx = 0.5, dt = 0.1, random-phase start) in the three precision modes -- float32,
float32 with compensated momenta, FP64 -- reporting per mode the energy drift
max|H_n - H_1|/H_1 over the measurements after the first (the start's Pi^{-1/2} = 0
offsets the n = 0 energy), the Gauss-law residual, and the field
error against the FP64 run on a 48^3 sub-box at checkpoints.  The dynamics is
chaotic, so field differences grow with time whatever the precision; energy and
Gauss residual are the conserved quantities.  (The comparison of the three modes
with the FP64 CPU oracle on a small lattice is a test.)  Prints one JSON object per
line.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import AHS_FIELD_ALL, AHS_FIELD_LOW, Lattice

PARAMS = dict(dx=0.5, dt=0.1, lambda0=2.0, e0=1.0, sigma=1.0, s=0.0)
MODES = ("fp32", "fp32c", "fp64")


def _errors(a, b):
    """Relative L2 differences of phi, Pi, E and of exp(-i theta)."""
    def rel(x, y):
        return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))
    return {"phi": rel(a[0:2], b[0:2]), "Pi": rel(a[2:4], b[2:4]), "E": rel(a[7:10], b[7:10]),
            "U": float(np.linalg.norm(np.exp(-1j * a[4:7]) - np.exp(-1j * b[4:7])) / np.sqrt(a[4:7].size))}


def _run(N, mode, steps, checkpoints, box, measure_every, seed):
    out = {"mode": mode, "N": N, "steps": steps}
    snaps = {}
    with Lattice(N, era=0, measure_every=measure_every, precision=mode, **PARAMS) as lat:
        lat.init(seed)
        t0 = time.perf_counter()
        n = 0
        for c in checkpoints:
            lat.step(c - n)
            n = c
            if box is None:
                F = lat.state().astype(np.float64)
                if mode == "fp32c":
                    lo = lat.field(AHS_FIELD_LOW).astype(np.float64)
                    F[2:4] += lo[0:2]
                    F[7:10] += lo[2:5]
            else:
                if mode == "fp64":
                    F = lat.state()[:, :box, :box, :box].astype(np.float64)
                else:
                    F = lat.box(AHS_FIELD_ALL, 0, 0, 0, box, box, box).astype(np.float64)
            snaps[c] = F
        out["seconds"] = time.perf_counter() - t0
        recs = lat.records()
        final = lat.measure()
    # the first measurement (n = 0) sees Pi^{-1/2} = 0 of the start and is skipped:
    # drift is taken from the measurement at n = measure_every on
    e = np.array([r["e_total"] for r in recs[1:]] + [final["e_total"]])
    out["energy_drift"] = float(np.abs(e - e[0]).max() / e[0])
    out["energy_final_rel"] = float((e[-1] - e[0]) / e[0])
    out["gauss_rms_final"] = final["gauss_rms"]
    out["gauss_max_final"] = final["gauss_max"]
    out["n_wind_final"] = final["n_wind"]
    return out, snaps


def precision(args):
    checkpoints = sorted({c for c in (10, 100, 500, 1000, args.steps) if c <= args.steps})
    # at full size: compare against the FP64 run on a sub-box
    big = {}
    for mode in MODES:
        res, snaps = _run(args.size, mode, args.steps, checkpoints, args.box, args.measure_every, args.seed)
        big[mode] = (res, snaps)
    for mode in MODES:
        res, snaps = big[mode]
        res["field_error_vs_fp64"] = {c: _errors(snaps[c], big["fp64"][1][c]) for c in checkpoints}
        res["reference"] = "fp64 run on the GPU, 48^3 sub-box"
        print(json.dumps(res), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2005_14454_gb300.study")
    sub = ap.add_subparsers(dest="cmd", required=True)
    pp = sub.add_parser("precision")
    pp.add_argument("--size", type=int, default=512)
    pp.add_argument("--steps", type=int, default=2000)
    pp.add_argument("--box", type=int, default=48)
    pp.add_argument("--measure-every", type=int, default=100)
    pp.add_argument("--seed", type=int, default=1)
    args = ap.parse_args(argv)
    if args.cmd == "precision":
        precision(args)
    return 0


if __name__ == "__main__":
    sys.exit(main())
