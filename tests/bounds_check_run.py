"""Runs every step path of the engine on small and ragged lattices with the
bounds-check build of the library (path given as the first argument) and prints
one JSON line: the number of paths run, the out-of-range indices the kernels
counted (expected 0), and the count of the counter's self-test (one index per
kernel translation unit).  Run by tests/test_gpu_bounds.py in a process of its own,
so that only the checked library is loaded."""
import ctypes
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2005_14454_gb300 import _abi  # noqa: E402

_abi._lib = _abi.load(sys.argv[1])
import paper_2005_14454_gb300 as pkg  # noqa: E402

PARAMS = dict(dx=0.5, dt=0.1, lambda0=2.0, e0=1.0, sigma=1.0)
SIDES = (4, 5, 7, 65, 66)


def counted(reset=False):
    c = ctypes.c_int64()
    _abi.check(_abi.lib().ahs_bounds_check(1 if reset else 0, ctypes.byref(c)), "ahs_bounds_check")
    return c.value


def run_lattice(N, era, **opts):
    with pkg.Lattice(N, era=era, measure_every=opts.pop("measure_every", 3), **PARAMS,
                     **{k: opts.pop(k) for k in ("precision", "momenta_in_place", "steps_per_pass") if k in opts}) as lat:
        for key, v in opts.items():
            lat.set_option(getattr(_abi, key), v)
        lat.init(N)
        lat.step(7)
        lat.measure()
        return lat.state() if N <= 66 else None


def main():
    counted(reset=True)
    paths = 0
    for N in SIDES:
        era = 1 + N % 2
        for opts in ({}, {"AHS_OPT_TILE_Y": 16}, {"AHS_OPT_MEASURE_TILE_Y": 8}, {"AHS_OPT_MEASURE_TILE_Y": 16},
                     {"AHS_OPT_ZCHUNK": 3}, {"AHS_OPT_ZCHUNK": N},
                     {"momenta_in_place": True}, {"precision": "fp32c"}, {"precision": "fp64"},
                     {"steps_per_pass": 2}, {"steps_per_pass": 2, "AHS_OPT_ZCHUNK": 2}):
            run_lattice(N, era, **dict(opts))
            paths += 1
        with pkg.Lattice(N, era=era, measure_every=0, **PARAMS) as lat:
            lat.init(3)
            lat.step(2)
            lat.windings()
            state = lat.state()
        paths += 1
        # the allocation-free measurement on caller-owned device buffers
        import torch
        dev = torch.from_numpy(state).to("cuda")
        out = torch.zeros(ctypes.sizeof(_abi.ahs_obs_t), dtype=torch.uint8, device="cuda")
        _abi.check(_abi.lib().ahs_measure_noalloc(N, 0.5, 0.1, 2.0, 1.0, 1.0, 0.0, era, 2.0, 1.0, 2,
                                                  ctypes.c_void_p(dev.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                                  None), "ahs_measure_noalloc")
        torch.cuda.synchronize()
        paths += 1
    with pkg.Batch(list(SIDES), [1, 2, 1, 2, 1], [1, 2, 3, 4, 5], [9, 12, 7, 12, 10], measure_every=5,
                   **PARAMS) as b:
        b.init()
        b.run()
        b.measure(3)
    paths += 1
    errors = counted()
    c = ctypes.c_int64()
    _abi.check(_abi.lib().ahs_bounds_check(2, ctypes.byref(c)), "ahs_bounds_check")
    print(json.dumps({"paths": paths, "errors": errors, "selftest": c.value - errors}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
