"""ahs_measure_noalloc: the measurement for callers that cannot allocate device
memory (their device memory belongs to another allocator), fed caller-owned
device buffers and using only the library's static scratch array.

Checked through the C ABI against the regular ahs_measure of a handle holding the
same fields, with the tolerances of the parity tests, on two calls in a row with
different lattices (the second call reuses the scratch the first one wrote).
Collected last on purpose so that a stop-at-first-failure run has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PARAMS = dict(dx=0.5, dt=0.1, lambda0=2.0, e0=1.0, sigma=1.0)


def reference_and_fields(N, era, s, seed, steps):
    import paper_2005_14454_gb300 as pkg
    with pkg.Lattice(N, era=era, s=s, measure_every=0, **PARAMS) as lat:
        lat.init(seed)
        lat.step(steps)
        return lat.measure(), lat.state()


def noalloc(N, era, s, step, state):
    import torch
    from paper_2005_14454_gb300 import _abi
    L = _abi.lib()
    dev = torch.from_numpy(np.ascontiguousarray(state)).to("cuda")
    out = torch.zeros(ctypes.sizeof(_abi.ahs_obs_t), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    rc = L.ahs_measure_noalloc(N, PARAMS["dx"], PARAMS["dt"], PARAMS["lambda0"], PARAMS["e0"], PARAMS["sigma"],
                               s, era, 2.0, 1.0, step, ctypes.c_void_p(dev.data_ptr()),
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    _abi.check(rc, "ahs_measure_noalloc")
    stream.synchronize()
    raw = out.cpu().numpy().tobytes()
    return _abi.ahs_obs_t.from_buffer_copy(raw).as_dict()


SUMS = ("sum_K", "sum_G", "sum_V", "sum_El", "sum_B", "e_total")
SIGNED = ("lagrangian", "xi_l", "v2_phi", "v2_omega", "sum_KL", "sum_GL", "sum_pL", "sum_rhoL")


def same(a, b):
    assert a["step"] == b["step"] and a["tau"] == b["tau"] and a["a"] == b["a"]
    assert a["n_wind"] == b["n_wind"] and a["nonfinite"] == b["nonfinite"] == 0
    for k in SUMS:
        assert a[k] == pytest.approx(b[k], rel=2e-5), k
    for k in SIGNED:
        assert a[k] == pytest.approx(b[k], rel=2e-4), k
    assert a["gauss_max"] == pytest.approx(b["gauss_max"], rel=1e-3, abs=1e-6)


def test_noalloc_matches_measure_twice_in_a_row():
    cases = [(48, 1, 0.0, 7, 12), (40, 2, 0.0, 8, 9)]
    for N, era, s, seed, steps in cases:
        ref, state = reference_and_fields(N, era, s, seed, steps)
        got = noalloc(N, era, s, steps, state)
        same(got, ref)


def test_noalloc_rejects_bad_sizes():
    from paper_2005_14454_gb300 import _abi
    L = _abi.lib()
    for N in (3, 1601):
        rc = L.ahs_measure_noalloc(N, 0.5, 0.1, 2.0, 1.0, 1.0, 0.0, 1, 2.0, 1.0, 0,
                                   ctypes.c_void_p(1), ctypes.c_void_p(1), None)
        assert rc == _abi.AHS_EINVAL
        assert b"N outside" in L.ahs_last_error_message()
    rc = L.ahs_measure_noalloc(16, 0.5, 0.1, 2.0, 1.0, 1.0, 0.0, 1, 2.0, 1.0, 0, None, None, None)
    assert rc == _abi.AHS_EINVAL
