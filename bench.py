"""Throughput of the fused Abelian-Higgs leapfrog step on GB300.

Workload (default): 1024^3 periodic lattice, float32 fields, radiation era (a ~ eta),
s = 0, lambda0 = 2, e0 = 1, sigma = 1, dx = 0.5, dt = 0.1, random-phase initial
condition (Sec. 2).  One benchmark step = one measurement period: 10 leapfrog steps
(Eqs. 7-10) with the diagnostics of Eqs. diagxi / diagvel fused into the first of
them, i.e. one ahs_step(h, 10) call.  Metric: lattice site-updates per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--size N]

Under torchrun each rank advances an independent realisation (its own seed) on its
own GPU: weak scaling, no collective on the data path; rank 0 prints one JSON line.
The reference arm times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PERIOD = 10                     # leapfrog steps per benchmark step (measurement cadence)
BYTES_PER_SITE = 80             # float32: read phi, Pi, theta, E (40 B) + write them (40 B)
PARAMS = dict(dx=0.5, dt=0.1, lambda0=2.0, e0=1.0, sigma=1.0, s=0.0)
ERA = 1                         # radiation


def workload(N, inplace=False, precision="fp32", steps_per_pass=1):
    d = {"workload": f"abelian-higgs leapfrog {N}^3 {precision}, radiation era, s=0, lambda0=2, e0=1, "
                     f"sigma=1, dx=0.5, dt=0.1, random-phase init, diagnostics fused every {PERIOD} steps",
         "lattice": N, "leapfrog_steps_per_step": PERIOD, "era": "radiation", "s": 0.0,
         "l2": "inputs larger than L2 (state %.1f GB resident in HBM)" % (N ** 3 * BYTES_PER_SITE / 1e9),
         "parallelism": "replicas (one lattice per GPU)"}
    if inplace:
        d["storage"] = "Pi and E updated in place (60 B/site allocated); measuring steps as two launches"
    if steps_per_pass == 2:
        d["steps_per_pass"] = "pairs of plain steps as one two-step launch (temporal blocking)"
    return d


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Group:
    """The replicas of a multi-GPU run, one process per GPU, each advancing its own
    realisation (no collective on the data path): a barrier around the timed
    region and the maximum of the per-rank times.  Single process: no-ops.
    backend "nccl" on the GPU run, "gloo" for CPU tests of the same logic."""

    def __init__(self, backend: str = "nccl", device=None):
        import torch
        self.torch = torch
        self.ws, self.rank, self.local = dist_env()
        self.dist = None
        self.device = device if device is not None else ("cuda" if backend == "nccl" else "cpu")
        if self.ws > 1:
            import torch.distributed as dist
            kw = {"device_id": torch.device("cuda", self.local)} if backend == "nccl" else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()
        if self.device == "cuda":
            self.torch.cuda.synchronize()

    def max(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        t = self.torch.tensor([float(x)], dtype=self.torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def replica_seed(rank: int) -> int:
    """Seed of the realisation a rank advances (distinct per rank)."""
    return 1000 + rank


def aggregate_rate(ws: int, sites_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job site-updates per second: all ranks' work over the slowest rank's time."""
    return ws * sites_per_rank * steps / seconds


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------- helpers
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e datasheet figure
# Sec. 5: the 8192^3 lattice (20470 steps to half light-crossing) in 1990.51 s on 4096 GPUs
PAPER_8192_RATE = 8192 ** 3 * 20470 / 1990.51
STEP_KERNEL_SOURCES = ("ahs_step.cu", "ahs_stencil.cuh", "ahs_device.cuh", "ahs_internal.cuh")


def code_only(text):
    """C++/CUDA source without its comments and blank lines (edits to comments do not
    change the compiled kernel)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def kernel_hash():
    """Hash of the code (comments removed) of the sources the step kernel is
    compiled from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2005_14454_gb300", "csrc")
    for f in STEP_KERNEL_SOURCES:
        h.update(code_only(open(os.path.join(csrc, f)).read()).encode())
    return h.hexdigest()[:16]


def measured_traffic(N):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("kernel_hash") != kernel_hash():
        return None
    per_site = d.get("dram_bytes_per_site")
    return None if per_site is None else per_site * N ** 3


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def cpu_baseline(seconds=12.0, N=128):
    """The FP64 oracle as it stands, on this host's cores, over a bounded sample of
    the workload: an N^3 lattice with the same couplings and era, leapfrog steps
    until about `seconds` of CPU wall time have passed."""
    import oracle
    oracle.build()
    p = oracle.Params(N=N, era=ERA, **PARAMS)
    F = oracle.init(p, 1)
    oracle.run(p, 0, 1, F)                       # warm-up (page-in, thread spin-up)
    n, t0 = 1, time.perf_counter()
    while True:
        oracle.run(p, n, 1, F)
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    steps = n - 1
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": N ** 3 * steps / dt, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, {N}^3 lattice of the same workload, {steps} leapfrog steps in {dt:.1f} s"}


def cpu_baseline_one_core(seconds=5.0, N=64):
    """The same measurement on one core (a fresh interpreter with OMP_NUM_THREADS=1,
    which the oracle's OpenMP runtime reads when it starts)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_baseline(%r, %d)))" % (ROOT, seconds, N))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if out.returncode != 0:
        return {"error": out.stderr.strip().splitlines()[-1:] or ["failed"]}
    return json.loads(out.stdout.strip().splitlines()[-1])


# --------------------------------------------------------------------- ensemble
ENSEMBLE = [(128, 24), (192, 16), (256, 8)]     # (side, realisations), half radiation / half matter


def ensemble_members():
    members, seed = [], 1
    for N, count in ENSEMBLE:
        for j in range(count):
            members.append((N, 1 if j % 2 == 0 else 2, seed))
            seed += 1
    return members


def run_ensemble(torch):
    """Realisations/hour of the ensemble 24x128^3 + 16x192^3 + 8x256^3 (s = 0, half
    radiation, half matter, each evolved to half light-crossing with a measurement
    every 10 steps): one batch (persistent launch per step, graph-replayed
    measurement periods, autotuned z-chunks) against the same realisations run back
    to back as single lattices.  Both time the evolution on the device (CUDA events);
    the fields of the two runs are identical (same kernel, same coefficients)."""
    from paper_2005_14454_gb300 import Batch, Lattice, _abi
    members = ensemble_members()
    N, era, seed = zip(*members)
    sites = sum(n ** 3 * round((0.5 * PARAMS["dx"] * n - 1.0) / PARAMS["dt"]) for n in N)
    with Batch(N, era, seed, measure_every=PERIOD, **PARAMS) as b:
        b.init()
        b.autotune()
        _abi.ahs_batch_set_option(b.b, _abi.AHS_OPT_PROFILE, 1)
        _abi.ahs_batch_kernel_time(b.b, reset=True)
        t0 = time.perf_counter()
        b.run()
        wall_b = time.perf_counter() - t0
        ms_b, steps_b = _abi.ahs_batch_kernel_time(b.b)
        dz = sorted({(n, _abi.ahs_batch_member_zchunk(b.b, i)) for i, n in enumerate(N)})
        by = int(_abi.ahs_batch_get_option(b.b, _abi.AHS_OPT_TILE_Y))
    stream = torch.cuda.current_stream()
    ms_s = 0.0
    t0 = time.perf_counter()
    for n, e, sd in members:
        with Lattice(n, era=e, measure_every=PERIOD, stream=stream.cuda_stream, **PARAMS) as lat:
            lat.init(sd)
            steps = round((0.5 * PARAMS["dx"] * n - 1.0) / PARAMS["dt"])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(steps)
            e1.record(stream)
            e1.synchronize()
            ms_s += e0.elapsed_time(e1)
    wall_s = time.perf_counter() - t0
    R = len(members)
    return {
        "members": " + ".join(f"{c}x{n}^3" for n, c in ENSEMBLE) + ", half radiation / half matter, s=0, "
                   f"to half light-crossing, measurement every {PERIOD} steps",
        "batched_realisations_per_hour": R / (ms_b / 1e3) * 3600.0,
        "back_to_back_realisations_per_hour": R / (ms_s / 1e3) * 3600.0,
        "speedup": ms_s / ms_b,
        "batched_site_updates_per_s": sites / (ms_b / 1e3),
        "back_to_back_site_updates_per_s": sites / (ms_s / 1e3),
        "batched_device_s": ms_b / 1e3, "back_to_back_device_s": ms_s / 1e3,
        "batched_wall_s": wall_b, "back_to_back_wall_s_incl_init": wall_s,
        "batch_tile_y": by, "batch_zchunks": dz,
    }


# --------------------------------------------------------------------- reference arm
CAPACITY_N = 1536


def extra_leg(fn, *args):
    try:
        return fn(*args)
    except Exception as e:   # noqa: BLE001 -- any failure of an extra leg is reported in it
        return {"unavailable": f"{type(e).__name__}: {e}"}


def run_capacity(torch, N=CAPACITY_N, steps=3):
    """The same workload on N^3 with Pi and E updated in place (60 B/site allocated,
    217 GB at 1536^3, a lattice the default 80 B/site storage cannot hold beside the
    benchmark's other buffers): site-updates/s over `steps` periods of 10 leapfrog
    steps after one warm-up period, and the plain step's roofline."""
    from paper_2005_14454_gb300 import _abi
    stream = torch.cuda.current_stream()
    h = _abi.ahs_create(N, PARAMS["dx"], PARAMS["dt"], PARAMS["lambda0"], PARAMS["e0"], PARAMS["sigma"],
                        PARAMS["s"], ERA)
    try:
        _abi.ahs_set_stream(h, stream.cuda_stream)
        _abi.ahs_set_option(h, _abi.AHS_OPT_MOMENTA_IN_PLACE, 1)
        _abi.ahs_set_option(h, _abi.AHS_OPT_MEASURE_EVERY, PERIOD)
        _abi.ahs_init(h, 1)
        _abi.ahs_step(h, PERIOD)
        _abi.ahs_records(h)
        _abi.ahs_set_option(h, _abi.AHS_OPT_PROFILE, 1)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            _abi.ahs_step(h, PERIOD)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        k_ms, k_n = _abi.ahs_kernel_time(h, _abi.AHS_KERNEL_STEP)
        km_ms, km_n = _abi.ahs_kernel_time(h, _abi.AHS_KERNEL_STEP_MEASURE)
        nbytes = _abi.ahs_device_bytes(h)
    finally:
        _abi.ahs_destroy(h)
    pk, pk_kind = peaks()
    avg = k_ms / max(k_n, 1)
    achieved = BYTES_PER_SITE * N ** 3 / (avg / 1e3) / 1e9
    return {"lattice": N, "storage": "Pi and E updated in place", "device_bytes": nbytes,
            "value": N ** 3 * PERIOD * steps / (ms / 1e3), "unit": "site-updates/s", "ms_per_step": ms / steps,
            "plain_step_ms": avg, "measuring_step_ms": km_ms / max(km_n, 1),
            "roofline_frac": achieved / pk["hbm_gbs"], "achieved_gbs": achieved, "peak_kind": pk_kind}


def reference_config(Ns, N):
    """The configuration the reference arm actually runs: the FP64 oracle on an Ns^3
    lattice of the workload (same couplings, era, start and measurement cadence) in
    host memory.  Its rate is per site-update and flat in the lattice side (4.6e7,
    4.40e7 and 4.36e7 site-updates/s at 128^3, 256^3 and 512^3 on the 16 host
    cores), so it stands for the N^3 workload; N^3 itself (172 GB of FP64 state,
    ~24 s per leapfrog step) does not fit a bounded run."""
    d = workload(Ns, precision="fp64")
    d["l2"] = "FP64 oracle in host memory (state %.2f GB); no GPU" % (Ns ** 3 * 80 / 1e9)
    d["parallelism"] = "OpenMP over the host cores, rank 0 only"
    d["stands_for"] = f"the {N}^3 workload of the GPU arm, per site-update"
    d["rate_note"] = ("site-updates/s is a per-site rate; the oracle's rate is flat from 128^3 to 512^3 "
                      "(4.6e7, 4.40e7, 4.36e7 on 16 host cores), so the sample's rate stands for the full lattice")
    return d


def run_reference(args, N):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    Ns = args.ref_size
    p = oracle.Params(N=Ns, era=ERA, **PARAMS)
    F = oracle.init(p, 1)
    n = 0

    def one_step():
        nonlocal n
        oracle.measure(p, n, F)                 # fused-measurement cadence of the engine
        oracle.run(p, n, PERIOD, F)
        n += PERIOD

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    dt = time.perf_counter() - t0
    value = Ns ** 3 * PERIOD * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": reference_config(Ns, N),
        "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"FP64 oracle on a {Ns}^3 lattice of the same workload: each step = "
                                   f"one measurement + {PERIOD} leapfrog steps"},
        "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- our arm
def run_ours(args, N):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    group = Group("nccl")

    from paper_2005_14454_gb300 import _abi
    stream = torch.cuda.current_stream()
    h = _abi.ahs_create(N, PARAMS["dx"], PARAMS["dt"], PARAMS["lambda0"], PARAMS["e0"], PARAMS["sigma"],
                        PARAMS["s"], ERA)
    _abi.ahs_set_stream(h, stream.cuda_stream)
    if args.momenta_in_place:
        _abi.ahs_set_option(h, _abi.AHS_OPT_MOMENTA_IN_PLACE, 1)
    _abi.ahs_set_option(h, _abi.AHS_OPT_MEASURE_EVERY, PERIOD)
    _abi.ahs_set_option(h, _abi.AHS_OPT_TILE_Y, args.tile_y)
    _abi.ahs_set_option(h, _abi.AHS_OPT_MEASURE_TILE_Y, args.measure_tile_y)
    _abi.ahs_set_option(h, _abi.AHS_OPT_ZCHUNK, args.zchunk)
    _abi.ahs_set_option(h, _abi.AHS_OPT_STEPS_PER_PASS, args.steps_per_pass)
    _abi.ahs_init(h, replica_seed(rank))
    shape = {"tile": [32, int(_abi.ahs_get_option(h, _abi.AHS_OPT_TILE_Y))],
             "measure_tile": [32, int(_abi.ahs_get_option(h, _abi.AHS_OPT_MEASURE_TILE_Y))],
             "zchunk": int(_abi.ahs_get_option(h, _abi.AHS_OPT_ZCHUNK))}

    barrier = group.barrier

    for _ in range(args.warmup):
        _abi.ahs_step(h, PERIOD)
    _abi.ahs_records(h)

    # ---- device-timed region: inputs resident in HBM
    _abi.ahs_set_option(h, _abi.AHS_OPT_PROFILE, 1)
    for kind in (_abi.AHS_KERNEL_STEP, _abi.AHS_KERNEL_STEP_MEASURE, _abi.AHS_KERNEL_STEP_PAIR):
        _abi.ahs_kernel_time(h, kind, reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            _abi.ahs_step(h, PERIOD)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    k_ms, k_n = _abi.ahs_kernel_time(h, _abi.AHS_KERNEL_STEP)
    km_ms, km_n = _abi.ahs_kernel_time(h, _abi.AHS_KERNEL_STEP_MEASURE)
    kp_ms, kp_n = _abi.ahs_kernel_time(h, _abi.AHS_KERNEL_STEP_PAIR)
    _abi.ahs_set_option(h, _abi.AHS_OPT_PROFILE, 0)
    recs = _abi.ahs_records(h)
    nonfinite = any(r["nonfinite"] for r in recs)

    # ---- end-to-end through the C ABI with host buffers: the initial state comes
    # from pinned host memory, every step's measurement record goes back to the
    # host, and the final state is copied back at the end.
    e2e = None
    if not args.no_e2e:
        planes = 10
        host = torch.empty((planes, N, N, N), dtype=torch.float32, pin_memory=True)
        _abi.lib().ahs_fields(h, _abi.AHS_FIELD_ALL, host.data_ptr(), host.numel() * 4)
        state_bytes = host.numel() * 4
        barrier()
        t0 = time.perf_counter()
        _abi.check(_abi.lib().ahs_set_fields(h, _abi.AHS_FIELD_ALL, host.data_ptr(), state_bytes), "ahs_set_fields")
        rec_bytes = 0
        for _ in range(args.steps):
            _abi.ahs_step(h, PERIOD)
            rec_bytes += len(_abi.ahs_records(h)) * _abi.lib().ahs_sizeof_obs()
        _abi.check(_abi.lib().ahs_fields(h, _abi.AHS_FIELD_ALL, host.data_ptr(), state_bytes), "ahs_fields")
        barrier()
        e2e_s = group.max(time.perf_counter() - t0)
        e2e = {"value": aggregate_rate(ws, N ** 3, PERIOD * args.steps, e2e_s), "unit": "site-updates/s",
               "h2d_bytes_per_step": state_bytes / args.steps,
               "d2h_bytes_per_step": (state_bytes + rec_bytes) / args.steps,
               "note": "state uploaded from pinned host memory once, records read back every step, "
                       "state read back at the end; per-step bytes are the totals / steps"}
        del host

    _abi.ahs_destroy(h)

    ms = group.max(ms)
    if rank != 0:
        group.close()
        return 0

    value = aggregate_rate(ws, N ** 3, PERIOD * args.steps, ms / 1e3)
    pk, pk_kind = peaks()
    # the dominant kernel: the plain step, or with two steps per pass the two-step
    # launch (one read and one write of every field per launch, two site-updates)
    pair = kp_n > 0
    avg_ms = (kp_ms / kp_n) if pair else k_ms / max(k_n, 1)
    bytes_per_launch = BYTES_PER_SITE * N ** 3
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    traffic = None if pair else measured_traffic(N)
    kernel_name = ("step_two (two plain leapfrog steps per pass)" if pair
                   else "step_pair (plain leapfrog step, even N)")
    line = {
        "metric": "site-updates/s", "value": value, "unit": "site-updates/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": workload(N, args.momenta_in_place, steps_per_pass=args.steps_per_pass),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                     "kernel": kernel_name, "peak_kind": pk_kind,
                     "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
                     "site_updates_per_launch": N ** 3 * (2 if pair else 1),
                     "launches": kp_n if pair else k_n, "measure_kernel_avg_ms": km_ms / max(km_n, 1),
                     "launch_shape": shape, "frac_of_nominal": achieved / NOMINAL_HBM_GBS},
        # the paper's largest run, another machine's whole-run figure: context only
        "context": {"paper_8192_run": "8192^3, 20470 steps in 1990.51 s on 4096 P100 GPUs: "
                                      f"{PAPER_8192_RATE:.3g} site-updates/s, {PAPER_8192_RATE / 4096:.3g} per GPU",
                    "value_per_gpu_over_paper_per_gpu": value / ws / (PAPER_8192_RATE / 4096)},
        # the step launches the profiler counted, plus per period one reduction (and
        # the Gauss launch of a measuring step with in-place momenta)
        "gpu_launches": (kp_n + k_n + km_n) + args.steps * (2 if args.momenta_in_place else 1),
        "clocks": clocks.summary(),
        "e2e": e2e,
        "nonfinite": nonfinite,
    }
    # the additional legs report a failure (e.g. a GPU without room for the 217 GB
    # capacity lattice) in their own object instead of losing the benchmark line
    if not args.no_ensemble and ws == 1:
        line["ensemble"] = extra_leg(run_ensemble, torch)
    if not args.no_capacity and ws == 1 and not args.momenta_in_place:
        line["capacity"] = extra_leg(run_capacity, torch)
    if not args.no_cpu and ws == 1:       # the CPU baseline belongs to the one-GPU line
        cb = extra_leg(cpu_baseline)
        if "unavailable" not in cb:
            cb["one_core"] = extra_leg(cpu_baseline_one_core)
        line["cpu_baseline"] = cb
    group.close()
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--ref-size", type=int, default=128)
    ap.add_argument("--tile-y", type=int, default=0, help="step-kernel tile height (8, 16; 0 = auto)")
    ap.add_argument("--measure-tile-y", type=int, default=0, help="measuring-step tile height (4, 8, 16; 0 = auto)")
    ap.add_argument("--zchunk", type=int, default=0, help="z planes per CTA (0 = auto)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble leg")
    ap.add_argument("--no-capacity", action="store_true", help="skip the 1536^3 in-place-momenta leg")
    ap.add_argument("--steps-per-pass", type=int, default=1, choices=(1, 2),
                    help="2: pairs of plain steps as one two-step launch (temporal blocking)")
    ap.add_argument("--momenta-in-place", action="store_true",
                    help="store Pi and E once (60 B/site; lattices up to 1600^3)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warm-up must be at least 3 steps", file=sys.stderr)
        return 2
    if args.impl == "reference":
        return run_reference(args, args.size)
    return run_ours(args, args.size)


if __name__ == "__main__":
    sys.exit(main())
