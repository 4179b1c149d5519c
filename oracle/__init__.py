"""FP64 CPU oracle of the lattice Abelian-Higgs evolution (arXiv:2005.14454, Sec. 2).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The CUDA engine never imports it, and
it imports nothing from the engine.

The arithmetic lives in ``ahs_oracle.c`` (plain C, FP64, OpenMP over independent
site loops, built with ``-ffp-contract=off`` so x86 and Arm give identical bits).
This module only builds the shared object, marshals numpy arrays through ctypes and
converts the observable record into a dict.

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
property the paper and the mathematics fix (see tests/test_oracle_pins.py):
Gauss law, energy conservation, forces = -dH/dq, gauge invariance, time
reversal, linear dispersion, vacuum fixed point, hand-placed windings,
symmetries, and the step-count formula of Sec. 2.  Two conventions have no
value in the paper and are "parity unpinned" beyond their definition:
the tension mu = 2 pi sigma^2 inside xi_L and the weight W = L in <v^2>_omega.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ahs_oracle.c")
_LIB = os.path.join(_HERE, "_ahs_oracle.so")

# plane order of a state array of shape (10, N, N, N), [z][y][x] with x fastest
PHI_RE, PHI_IM, PI_RE, PI_IM, TH_X, TH_Y, TH_Z, E_X, E_Y, E_Z = range(10)
ERAS = {"minkowski": 0, "radiation": 1, "matter": 2}


def build(force: bool = False) -> str:
    """Compile ahs_oracle.c into _ahs_oracle.so next to it (gcc, no GPU needed)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-std=gnu11", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("e0", ctypes.c_double),
                ("sigma", ctypes.c_double), ("s", ctypes.c_double), ("era", ctypes.c_int),
                ("alpha", ctypes.c_double), ("tau0", ctypes.c_double), ("cool", ctypes.c_double),
                ("s_cg", ctypes.c_double), ("tau_cg", ctypes.c_double)]


class _Obs(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("tau", ctypes.c_double), ("a", ctypes.c_double),
                ("n_wind", ctypes.c_int64), ("string_length", ctypes.c_double),
                ("xi_w", ctypes.c_double), ("xi_l", ctypes.c_double),
                ("lagrangian", ctypes.c_double), ("v2_phi", ctypes.c_double),
                ("v2_omega", ctypes.c_double), ("e_kin", ctypes.c_double),
                ("e_grad", ctypes.c_double), ("e_pot", ctypes.c_double),
                ("e_elec", ctypes.c_double), ("e_mag", ctypes.c_double),
                ("e_total", ctypes.c_double), ("gauss_rms", ctypes.c_double),
                ("gauss_max", ctypes.c_double), ("nonfinite", ctypes.c_int64),
                ("sum_K", ctypes.c_double), ("sum_G", ctypes.c_double),
                ("sum_V", ctypes.c_double), ("sum_El", ctypes.c_double),
                ("sum_B", ctypes.c_double), ("sum_L", ctypes.c_double),
                ("sum_KL", ctypes.c_double), ("sum_GL", ctypes.c_double),
                ("sum_pL", ctypes.c_double), ("sum_rhoL", ctypes.c_double)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        _lib.orc_scalars.argtypes = [pp, ctypes.c_int64, dp]
        _lib.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        _lib.orc_uniform.restype = ctypes.c_double
        _lib.orc_init.argtypes = [pp, ctypes.c_uint64, dp]
        _lib.orc_forces.argtypes = [pp, ctypes.c_int64, dp, dp]
        _lib.orc_kick.argtypes = [pp, ctypes.c_int64, dp, dp]
        _lib.orc_drift.argtypes = [pp, dp]
        _lib.orc_kick_inplace.argtypes = [pp, ctypes.c_int64, dp, dp]
        _lib.orc_step.argtypes = [pp, ctypes.c_int64, dp, dp]
        _lib.orc_run.argtypes = [pp, ctypes.c_int64, ctypes.c_int64, dp, dp]
        _lib.orc_wrap.argtypes = [ctypes.c_double]
        _lib.orc_wrap.restype = ctypes.c_double
        _lib.orc_windings.argtypes = [pp, dp, ctypes.POINTER(ctypes.c_int8)]
        _lib.orc_windings.restype = ctypes.c_int64
        _lib.orc_gauss.argtypes = [pp, ctypes.c_int64, dp, dp, dp]
        _lib.orc_measure.argtypes = [pp, ctypes.c_int64, dp, dp, ctypes.POINTER(_Obs)]
        _lib.orc_hamiltonian.argtypes = [pp, ctypes.c_int64, dp, ctypes.c_int]
        _lib.orc_hamiltonian.restype = ctypes.c_double
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Params:
    """Run parameters (Sec. 2): lattice side N, spacing dx, time step dt, couplings
    lambda0, e0, vev sigma, width exponent s (lambda, e scale so a^{2s} multiplies
    the potential and the current), era p (a = (eta/eta0)^p), damping form alpha,
    initial conformal time tau0, cooling damping cool (> 0: a = 1, delta = omega = cool),
    core growth: the steps with eta < tau_cg use s_cg in place of s."""
    N: int
    dx: float = 0.5
    dt: float = 0.1
    lambda0: float = 2.0
    e0: float = 1.0
    sigma: float = 1.0
    s: float = 0.0
    era: int = 1
    alpha: float = 2.0
    tau0: float = 1.0
    cool: float = 0.0
    s_cg: float = 0.0
    tau_cg: float = 0.0

    def c(self) -> _Params:
        return _Params(self.N, self.dx, self.dt, self.lambda0, self.e0, self.sigma,
                       self.s, self.era, self.alpha, self.tau0, self.cool, self.s_cg, self.tau_cg)


def zeros(N: int) -> np.ndarray:
    return np.zeros((10, N, N, N), dtype=np.float64)


def scalars(p: Params, n: int) -> dict:
    out = np.zeros(5)
    _L().orc_scalars(ctypes.byref(p.c()), n, _dp(out))
    return dict(eta=out[0], a=out[1], delta=out[2], omega=out[3], c=out[4])


def uniform(seed: int, idx: int) -> float:
    return _L().orc_uniform(seed, idx)


def init(p: Params, seed: int) -> np.ndarray:
    F = zeros(p.N)
    _L().orc_init(ctypes.byref(p.c()), seed, _dp(F))
    return F


def forces(p: Params, n: int, F: np.ndarray) -> np.ndarray:
    out = np.zeros((5,) + F.shape[1:])
    _L().orc_forces(ctypes.byref(p.c()), n, _dp(F), _dp(out))
    return out


def kick(p: Params, n: int, F: np.ndarray) -> np.ndarray:
    """New momenta (Re Pi, Im Pi, E_x, E_y, E_z) at n+1/2; F unchanged."""
    out = np.zeros((5,) + F.shape[1:])
    _L().orc_kick(ctypes.byref(p.c()), n, _dp(F), _dp(out))
    return out


def kick_inplace(p: Params, n: int, F: np.ndarray) -> None:
    work = np.zeros((5,) + F.shape[1:])
    _L().orc_kick_inplace(ctypes.byref(p.c()), n, _dp(F), _dp(work))


def drift(p: Params, F: np.ndarray) -> None:
    _L().orc_drift(ctypes.byref(p.c()), _dp(F))


def run(p: Params, n0: int, steps: int, F: np.ndarray) -> None:
    """Advance F in place by `steps` leapfrog steps starting at integer time n0."""
    work = np.zeros((5,) + F.shape[1:])
    _L().orc_run(ctypes.byref(p.c()), n0, steps, _dp(F), _dp(work))


def wrap(a: float) -> float:
    return _L().orc_wrap(a)


def windings(p: Params, F: np.ndarray):
    """(W, n_wind): W int8 of shape (3, N, N, N) for the xy, xz, yz plaquettes."""
    W = np.zeros((3,) + F.shape[1:], dtype=np.int8)
    n = _L().orc_windings(ctypes.byref(p.c()), _dp(F), W.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
    return W, n


def gauss(p: Params, n: int, F: np.ndarray):
    """(G, rms, max): Gauss residual of the stored momenta (time n-1/2) with phi^n."""
    G = np.zeros(F.shape[1:])
    out = np.zeros(2)
    _L().orc_gauss(ctypes.byref(p.c()), n, _dp(F), _dp(G), _dp(out))
    return G, out[0], out[1]


def measure(p: Params, n: int, F: np.ndarray) -> dict:
    work = np.zeros((5,) + F.shape[1:])
    o = _Obs()
    _L().orc_measure(ctypes.byref(p.c()), n, _dp(F), _dp(work), ctypes.byref(o))
    return {k: getattr(o, k) for k, _ in _Obs._fields_}


def hamiltonian(p: Params, n: int, F: np.ndarray, kinetic: bool = True) -> float:
    return _L().orc_hamiltonian(ctypes.byref(p.c()), n, _dp(F), int(kinetic))


def steps_to(N: int, dx: float = 0.5, dt: float = 0.1, tau0: float = 1.0) -> int:
    """Run length of Sec. 2: evolve until eta_end = 0.5 * dx * N (half light-crossing)."""
    return int(round((0.5 * dx * N - tau0) / dt))
