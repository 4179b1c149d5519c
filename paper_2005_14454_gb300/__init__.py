"""GB300 engine for lattice Abelian-Higgs cosmic-string evolution.

Implements the data-parallel hot path of Correia & Martins, "Abelian-Higgs cosmic
string evolution with multiple GPUs" (arXiv:2005.14454): the staggered-leapfrog
step of Eqs. 7-10 for a complex scalar and compact U(1) links on a periodic
comoving lattice in an expanding background, with the string-winding, energy and
velocity diagnostics of Eqs. diagxi / diagvel fused into it.

The compute runs in hand-written sm_103a CUDA kernels behind the C ABI of
``include/ahs.h`` (``_ahs.so``); this package is its ctypes binding plus a small
object wrapper.  Build with ``paper_2005_14454_gb300.build.build()``.
"""
from __future__ import annotations

import numpy as np

from . import _abi
from ._abi import (AHS_FIELD_ALL, AHS_FIELD_E, AHS_FIELD_LOW, AHS_FIELD_PHI, AHS_FIELD_PI, AHS_FIELD_THETA,
                   AHS_MATTER, AHS_MINKOWSKI, AHS_PREC_FP32, AHS_PREC_FP32_COMPENSATED, AHS_PREC_FP64,
                   AHS_RADIATION, AHSError)

ERAS = {"minkowski": AHS_MINKOWSKI, "radiation": AHS_RADIATION, "matter": AHS_MATTER}
PRECISIONS = {"fp32": _abi.AHS_PREC_FP32, "fp32c": _abi.AHS_PREC_FP32_COMPENSATED, "fp64": _abi.AHS_PREC_FP64}


def stable_dt(dx: float, lambda0: float, e0: float, sigma: float, s: float, era: int, tau_end: float,
              tau0: float = 1.0, s_cg: float = 0.0, tau_cg: float = 0.0, safety: float = 0.9) -> float:
    """Largest leapfrog time step that stays stable up to conformal time tau_end,
    times `safety` (ahs_stable_dt of the C ABI: dt omega_max < 2, omega_max^2 =
    12/dx^2 + max(lambda0, 2 e0^2) sigma^2 c at the largest c = a^{2s} of the run,
    core-growth schedule included)."""
    return _abi.ahs_stable_dt(dx, lambda0, e0, sigma, s, era, tau0, tau_end, s_cg, tau_cg, safety)


class Lattice:
    """One N^3 lattice on the current CUDA device (owns its device memory)."""

    def __init__(self, N: int, dx: float = 0.5, dt: float = 0.1, lambda0: float = 2.0,
                 e0: float = 1.0, sigma: float = 1.0, s: float = 0.0, era=AHS_RADIATION,
                 measure_every: int = 10, stream: int | None = None, precision=None,
                 momenta_in_place: bool = False, core_growth=None, steps_per_pass: int = 1):
        era = ERAS.get(era, era) if isinstance(era, str) else era
        self.N = N
        self.params = dict(N=N, dx=dx, dt=dt, lambda0=lambda0, e0=e0, sigma=sigma, s=s, era=era)
        self.h = _abi.ahs_create(N, dx, dt, lambda0, e0, sigma, s, era)
        _abi.ahs_set_option(self.h, _abi.AHS_OPT_MEASURE_EVERY, measure_every)
        if precision is not None:
            precision = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
            _abi.ahs_set_option(self.h, _abi.AHS_OPT_PRECISION, precision)
        if momenta_in_place:
            _abi.ahs_set_option(self.h, _abi.AHS_OPT_MOMENTA_IN_PLACE, 1)
        if core_growth is not None:          # (s_cg, tau_cg)
            _abi.ahs_set_option(self.h, _abi.AHS_OPT_CORE_GROWTH_S, core_growth[0])
            _abi.ahs_set_option(self.h, _abi.AHS_OPT_CORE_GROWTH_TAU, core_growth[1])
        if steps_per_pass != 1:
            _abi.ahs_set_option(self.h, _abi.AHS_OPT_STEPS_PER_PASS, steps_per_pass)
        if stream is not None:
            _abi.ahs_set_stream(self.h, stream)

    # lifecycle ---------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            _abi.ahs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # evolution -----------------------------------------------------------------
    def init(self, seed: int):
        _abi.ahs_init(self.h, seed)

    def step(self, n: int = 1):
        _abi.ahs_step(self.h, n)

    def measure(self) -> dict:
        return _abi.ahs_measure(self.h)

    def records(self):
        return _abi.ahs_records(self.h)

    @property
    def n(self) -> int:
        return int(_abi.ahs_get_option(self.h, _abi.AHS_OPT_STEP))

    @n.setter
    def n(self, value: int):
        _abi.ahs_set_option(self.h, _abi.AHS_OPT_STEP, value)

    def set_option(self, key: int, value: float):
        _abi.ahs_set_option(self.h, key, value)

    # data movement -------------------------------------------------------------
    def state(self) -> np.ndarray:
        """All ten planes (Re phi, Im phi, Re Pi, Im Pi, theta_xyz, E_xyz) as float32
        of shape (10, N, N, N) indexed [plane, z, y, x]."""
        return _abi.ahs_fields(self.h, AHS_FIELD_ALL)

    def set_state(self, F: np.ndarray):
        _abi.ahs_set_fields(self.h, AHS_FIELD_ALL, F)

    def field(self, which: int) -> np.ndarray:
        return _abi.ahs_fields(self.h, which)

    def box(self, which: int, x0: int, y0: int, z0: int, nx: int, ny: int, nz: int) -> np.ndarray:
        return _abi.ahs_fields_box(self.h, which, x0, y0, z0, nx, ny, nz)

    def windings(self):
        return _abi.ahs_windings(self.h)

    def autotune(self):
        _abi.ahs_autotune(self.h)

    # checkpoint / restart ------------------------------------------------------
    _SAVED_OPTIONS = ("AHS_OPT_STEP", "AHS_OPT_ALPHA", "AHS_OPT_TAU0", "AHS_OPT_WRAP_THETA",
                      "AHS_OPT_MEASURE_EVERY", "AHS_OPT_PRECISION", "AHS_OPT_COOLING",
                      "AHS_OPT_MOMENTA_IN_PLACE", "AHS_OPT_CORE_GROWTH_S", "AHS_OPT_CORE_GROWTH_TAU",
                      "AHS_OPT_TILE_Y", "AHS_OPT_ZCHUNK", "AHS_OPT_STEPS_PER_PASS", "AHS_OPT_MEASURE_TILE_Y")

    def save(self, path: str):
        """Write a restart file (numpy .npz): the fields at the current time level in
        their storage precision (with the low words in compensated precision), the
        parameters of ahs_create and every option that shapes the evolution.  A run
        restored from it continues bit for bit (the measurement log is not saved)."""
        import json
        opts = {k: _abi.ahs_get_option(self.h, getattr(_abi, k)) for k in self._SAVED_OPTIONS}
        arrays = {"fields": self.state()}
        if int(opts["AHS_OPT_PRECISION"]) == _abi.AHS_PREC_FP32_COMPENSATED:
            arrays["low"] = self.field(AHS_FIELD_LOW)
        meta = json.dumps({"params": self.params, "options": opts})
        with open(path, "wb") as f:
            np.savez(f, meta=np.frombuffer(meta.encode(), dtype=np.uint8), **arrays)

    @classmethod
    def restore(cls, path: str, stream: int | None = None) -> "Lattice":
        """A new lattice with the parameters, options, time level and fields of a
        restart file written by save()."""
        import json
        with np.load(path) as z:
            meta = json.loads(bytes(z["meta"]).decode())
            fields = z["fields"]
            low = z["low"] if "low" in z.files else None
        lat = cls(measure_every=0, stream=stream, **meta["params"])
        opts = meta["options"]
        order = ["AHS_OPT_PRECISION", "AHS_OPT_MOMENTA_IN_PLACE"]   # these reallocate: first
        for k in order + [k for k in opts if k not in order]:
            _abi.ahs_set_option(lat.h, getattr(_abi, k), opts[k])
        lat.set_state(fields)
        if low is not None:
            _abi.ahs_set_fields(lat.h, AHS_FIELD_LOW, low)
        return lat


class Batch:
    """An ensemble of independent lattices advanced together (one persistent launch
    per step, each measurement period replayed as a CUDA graph)."""

    def __init__(self, N, era, seed, n_end=None, dx: float = 0.5, dt: float = 0.1, lambda0: float = 2.0,
                 e0: float = 1.0, sigma: float = 1.0, s: float = 0.0, measure_every: int = 10):
        era = [ERAS.get(e, e) if isinstance(e, str) else e for e in era]
        self.N = list(N)
        self.b = _abi.ahs_batch_create(self.N, era, seed, n_end, dx, dt, lambda0, e0, sigma, s)
        _abi.ahs_batch_set_option(self.b, _abi.AHS_OPT_MEASURE_EVERY, measure_every)

    def close(self):
        if getattr(self, "b", None):
            _abi.ahs_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self):
        _abi.ahs_batch_init(self.b)

    def run(self, max_steps: int = 1 << 30) -> int:
        return _abi.ahs_batch_run(self.b, max_steps)

    def records(self, m: int):
        return _abi.ahs_batch_records(self.b, m)

    def state(self, m: int) -> np.ndarray:
        return _abi.ahs_batch_fields(self.b, m, AHS_FIELD_ALL, self.N[m])

    def set_state(self, m: int, F: np.ndarray):
        _abi.ahs_batch_set_fields(self.b, m, AHS_FIELD_ALL, F)

    def step_info(self, m: int):
        return _abi.ahs_batch_step_info(self.b, m)

    def measure(self, m: int) -> dict:
        return _abi.ahs_batch_measure(self.b, m)

    def set_option(self, key: int, value: float):
        _abi.ahs_batch_set_option(self.b, key, value)

    def autotune(self):
        _abi.ahs_batch_autotune(self.b)


__all__ = ["Lattice", "Batch", "stable_dt", "AHSError", "ERAS", "PRECISIONS", "AHS_FIELD_ALL", "AHS_FIELD_E", "AHS_FIELD_LOW",
           "AHS_FIELD_PHI", "AHS_FIELD_PI", "AHS_FIELD_THETA", "AHS_MATTER", "AHS_MINKOWSKI", "AHS_RADIATION",
           "AHS_PREC_FP32", "AHS_PREC_FP32_COMPENSATED", "AHS_PREC_FP64"]
