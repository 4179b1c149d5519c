"""Studies run on the engine (one GPU).

  python -m paper_2005_14454_gb300.study precision [--size 512] [--steps 2000] [--box 48]
  python -m paper_2005_14454_gb300.study table1 [--size 1024] [--eras 1 2] [--seeds 1-20] [--every 5]
  python -m paper_2005_14454_gb300.study table1-summary FILE...

table1: the scaling runs of Sec. 4 (Table 1): random-phase starts evolved with constant
comoving width (s = 0) to half a light-crossing time, diagnostics every `every` steps;
per run the slopes of xi_L(tau) and xi_W(tau) from a least-squares line over the fit
range (Table 1's [100.5, 255.5] at 1024^3, scaled with the box otherwise) and the means
of <v^2>_omega and <v^2>_phi over the same range; then the mean and the sample standard
deviation over the realisations of each era.  One JSON object per run and per era.
table1-summary aggregates the run lines of earlier invocations.

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


def fit_rate(tau, xi, lo, hi):
    """Slope of the least-squares line through (tau, xi) over lo <= tau <= hi
    (finite points only); NaN with fewer than three points."""
    tau, xi = np.asarray(tau, float), np.asarray(xi, float)
    m = (tau >= lo) & (tau <= hi) & np.isfinite(xi)
    if m.sum() < 3:
        return float("nan")
    t = tau[m] - tau[m].mean()
    return float(np.dot(t, xi[m] - xi[m].mean()) / np.dot(t, t))


def fit_range(N, dx=0.5, tau0=1.0):
    """Table 1's fit range [100.5, 255.5] of the 1024^3, dx = 0.5 runs (end of run at
    tau = 256), scaled to the end of a run on N^3."""
    end = 0.5 * dx * N
    return 100.5 / 256.0 * end, 255.5 / 256.0 * end


def table1_run(N, era, seed, every, lo, hi, chunk=250):
    """One realisation: (per-run summary, series of tau, xi_L, xi_W, v2_omega, v2_phi)."""
    steps = int(round((0.5 * PARAMS["dx"] * N - 1.0) / PARAMS["dt"]))
    recs = []
    t0 = time.perf_counter()
    with Lattice(N, era=era, measure_every=every, **PARAMS) as lat:
        lat.init(seed)
        done = 0
        while done <= steps:
            k = min(chunk, steps + 1 - done)
            lat.step(k)
            done += k
            recs += lat.records()
    secs = time.perf_counter() - t0
    ser = {k: np.array([r[k] for r in recs], float) for k in ("tau", "xi_l", "xi_w", "v2_omega", "v2_phi")}
    m = (ser["tau"] >= lo) & (ser["tau"] <= hi)
    out = {"study": "table1", "N": N, "era": era, "seed": seed, "steps": steps, "every": every,
           "fit": [lo, hi], "points": int(m.sum()),
           "xi_dot_L": fit_rate(ser["tau"], ser["xi_l"], lo, hi),
           "xi_dot_W": fit_rate(ser["tau"], ser["xi_w"], lo, hi),
           "v2_omega": float(np.mean(ser["v2_omega"][m])), "v2_phi": float(np.mean(ser["v2_phi"][m])),
           "xi_w_end": float(ser["xi_w"][-1]), "xi_l_end": float(ser["xi_l"][-1]),
           "n_wind_end": int(recs[-1]["n_wind"]), "seconds": secs}
    return out, ser


TABLE1_KEYS = ("xi_dot_L", "xi_dot_W", "v2_omega", "v2_phi")


def table1_summary(runs):
    """Mean and sample standard deviation over realisations, per (N, era)."""
    groups = {}
    for r in runs:
        groups.setdefault((r["N"], r["era"]), []).append(r)
    out = []
    for (N, era), rs in sorted(groups.items()):
        d = {"study": "table1-summary", "N": N, "era": era, "runs": len(rs),
             "seeds": sorted(r["seed"] for r in rs)}
        for k in TABLE1_KEYS:
            v = np.array([r[k] for r in rs], float)
            d[k] = [float(v.mean()), float(v.std(ddof=1)) if v.size > 1 else float("nan")]
        out.append(d)
    return out


def _seeds(spec):
    a, _, b = spec.partition("-")
    return list(range(int(a), int(b or a) + 1))


def table1(args):
    lo, hi = args.fit if args.fit else fit_range(args.size)
    runs = []
    for seed in _seeds(args.seeds):
        for era in args.eras:
            r, _ = table1_run(args.size, era, seed, args.every, lo, hi)
            runs.append(r)
            print(json.dumps(r), flush=True)
    for d in table1_summary(runs):
        print(json.dumps(d), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2005_14454_gb300.study")
    sub = ap.add_subparsers(dest="cmd", required=True)
    pp = sub.add_parser("precision")
    pp.add_argument("--size", type=int, default=512)
    pp.add_argument("--steps", type=int, default=2000)
    pp.add_argument("--box", type=int, default=48)
    pp.add_argument("--measure-every", type=int, default=100)
    pp.add_argument("--seed", type=int, default=1)
    tp = sub.add_parser("table1")
    tp.add_argument("--size", type=int, default=1024)
    tp.add_argument("--eras", type=int, nargs="+", default=[1, 2])
    tp.add_argument("--seeds", default="1-20", help="first-last realisation seed")
    tp.add_argument("--every", type=int, default=5)
    tp.add_argument("--fit", type=float, nargs=2, default=None, help="fit range in tau")
    sp = sub.add_parser("table1-summary")
    sp.add_argument("files", nargs="+")
    args = ap.parse_args(argv)
    if args.cmd == "precision":
        precision(args)
    elif args.cmd == "table1":
        table1(args)
    elif args.cmd == "table1-summary":
        runs = []
        for f in args.files:
            for line in open(f):
                line = line.strip()
                if line.startswith("{"):
                    d = json.loads(line)
                    if d.get("study") == "table1":
                        runs.append(d)
        for d in table1_summary(runs):
            print(json.dumps(d), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
