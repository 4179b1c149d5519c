"""In-place momenta (AHS_OPT_MOMENTA_IN_PLACE): Pi and E stored once, phi and theta
double-buffered, 60 instead of 80 bytes per site.  The arithmetic is the default
path's, so fields and records must be bit-identical to it; at 1536^3 (217 GB, a
size the default storage cannot hold next to nothing else) sampled sites are checked
against the oracle."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

PARAMS = dict(dx=0.5, dt=0.1, lambda0=2.0, e0=1.0, sigma=1.0)


@pytest.fixture(scope="module")
def eng():
    from paper_2005_14454_gb300 import _abi
    import paper_2005_14454_gb300 as pkg
    _abi.lib()
    return pkg


def run_pair(eng, N, steps, era=1, s=0.0, every=5, seed=3, start=None, shape=None):
    out = []
    for inplace in (False, True):
        with eng.Lattice(N, era=era, s=s, measure_every=every, momenta_in_place=inplace, **PARAMS) as lat:
            for k, v in (shape or {}).items():
                lat.set_option(k, v)
            if start is None:
                lat.init(seed)
            else:
                lat.set_state(start)
            lat.step(steps)
            out.append((lat.state(), lat.records(), lat.measure()))
    return out


@pytest.mark.parametrize("N,era,s,steps", [(36, 1, 0.0, 25), (64, 2, 0.0, 20), (20, 0, 0.0, 31), (24, 2, 1.0, 12),
                                         (5, 1, 0.0, 7)])
def test_fields_and_records_bit_identical_to_double_buffering(eng, N, era, s, steps):
    (F0, R0, M0), (F1, R1, M1) = run_pair(eng, N, steps, era=era, s=s)
    assert np.array_equal(F0, F1)
    assert len(R0) == len(R1) > 0
    for a, b in zip(R0 + [M0], R1 + [M1]):
        assert a == b


def test_perturbed_gauge_fields_and_launch_shapes(eng):
    from paper_2005_14454_gb300._abi import AHS_OPT_MEASURE_TILE_Y, AHS_OPT_TILE_Y, AHS_OPT_ZCHUNK
    N = 40
    F = inputs.to_f32(inputs.perturbed_state(N, seed=11))
    for shape in ({}, {AHS_OPT_TILE_Y: 16, AHS_OPT_ZCHUNK: 7}, {AHS_OPT_MEASURE_TILE_Y: 8, AHS_OPT_ZCHUNK: 5}):
        (F0, R0, _), (F1, R1, _) = run_pair(eng, N, 15, start=F, shape=shape)
        assert np.array_equal(F0, F1)
        assert R0 == R1


def test_storage_is_60_bytes_per_site_and_accessors_work(eng):
    from paper_2005_14454_gb300 import AHS_FIELD_ALL, AHS_FIELD_E, AHS_FIELD_THETA, _abi
    N = 32
    ref = {}
    for inplace in (False, True):
        with eng.Lattice(N, measure_every=0, momenta_in_place=inplace, **PARAMS) as lat:
            lat.init(8)
            lat.step(7)                      # odd: phi, theta live in the second buffer
            ref[inplace] = dict(state=lat.state(), W=lat.windings()[0],
                                box=lat.box(AHS_FIELD_ALL, 30, 1, 31, 5, 4, 3),
                                bytes=_abi.ahs_device_bytes(lat.h))
            # overwrite E and theta at the odd time level, continue
            E = lat.field(AHS_FIELD_E) * 0.5
            _abi.ahs_set_fields(lat.h, AHS_FIELD_E, E)
            _abi.ahs_set_fields(lat.h, AHS_FIELD_THETA, lat.field(AHS_FIELD_THETA) + 0.25)
            lat.step(4)
            ref[inplace]["after"] = lat.state()
    a, b = ref[False], ref[True]
    for k in ("state", "W", "box", "after"):
        assert np.array_equal(a[k], b[k]), k
    V = N ** 3
    assert a["bytes"] - b["bytes"] == 20 * V
    assert b["bytes"] >= 60 * V


def test_option_rules(eng):
    from paper_2005_14454_gb300 import AHSError, _abi
    with eng.Lattice(8, measure_every=0, **PARAMS) as lat:
        lat.init(1)
        lat.set_option(_abi.AHS_OPT_MOMENTA_IN_PLACE, 1)
        assert _abi.ahs_get_option(lat.h, _abi.AHS_OPT_MOMENTA_IN_PLACE) == 1
        with pytest.raises(AHSError):
            lat.step(1)                      # switching storage discards the fields
        lat.init(1)
        with pytest.raises(AHSError) as e:
            _abi.ahs_autotune(lat.h)
        assert e.value.status == _abi.AHS_ESTATE
        for prec in (_abi.AHS_PREC_FP32_COMPENSATED, _abi.AHS_PREC_FP64):
            with pytest.raises(AHSError):
                lat.set_option(_abi.AHS_OPT_PRECISION, prec)
        with pytest.raises(AHSError):
            lat.set_option(_abi.AHS_OPT_MOMENTA_IN_PLACE, 2)
        with pytest.raises(AHSError):
            lat.field(_abi.AHS_FIELD_LOW)
        lat.set_option(_abi.AHS_OPT_MOMENTA_IN_PLACE, 0)
        lat.set_option(_abi.AHS_OPT_PRECISION, _abi.AHS_PREC_FP64)
        with pytest.raises(AHSError):
            lat.set_option(_abi.AHS_OPT_MOMENTA_IN_PLACE, 1)


def test_1536_cubed_sampled_sites(eng, orc):
    """1536^3 with in-place momenta (217 GB): one step from a later state, checked
    at sampled sites against the oracle on the 5^3 periodic neighbourhood of each
    site, and a fused measurement with finite, positive energies."""
    from paper_2005_14454_gb300 import AHS_FIELD_ALL, _abi
    N = 1536
    rng = np.random.default_rng(1)
    sites = [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(10)]
    sites += [(0, 0, 0), (N - 1, N - 1, N - 1), (N - 1, 0, 767)]
    with eng.Lattice(N, measure_every=2, momenta_in_place=True, **PARAMS) as lat:
        assert _abi.ahs_device_bytes(lat.h) < 61 * N ** 3
        lat.init(2)
        lat.step(3)
        before = [lat.box(AHS_FIELD_ALL, x - 2, y - 2, z - 2, 5, 5, 5).astype(np.float64) for (x, y, z) in sites]
        lat.step(1)
        after = [lat.box(AHS_FIELD_ALL, x, y, z, 1, 1, 1).astype(np.float64)[:, 0, 0, 0] for (x, y, z) in sites]
        recs = lat.records()
    assert [r["step"] for r in recs] == [0, 2]
    for r in recs:
        assert r["nonfinite"] == 0 and r["e_total"] > 0 and r["n_wind"] > 0
    p = orc.Params(N=5, era=1, **PARAMS)
    for B, A in zip(before, after):
        ref = B.copy()
        orc.run(p, 3, 1, ref)
        assert np.allclose(A, ref[:, 2, 2, 2], rtol=2e-6, atol=2e-6), (A, ref[:, 2, 2, 2])


def test_largest_lattice_1600_cubed(eng, orc):
    """N = 1600, the largest side the 32-bit site offsets allow (N^3 < 2^32), with
    in-place momenta (246 GB): one step from the random-phase start checked at
    sampled sites against the oracle, corner sites included."""
    import torch
    from paper_2005_14454_gb300 import AHS_FIELD_ALL
    N = 1600
    free, _ = torch.cuda.mem_get_info()
    if free < 60 * N ** 3 + (4 << 30):
        pytest.skip(f"needs {60 * N ** 3 / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")
    sites = [(0, 0, 0), (N - 1, N - 1, N - 1), (N - 1, 0, N - 1), (0, N - 1, 800), (1234, 567, 1599)]
    with eng.Lattice(N, measure_every=0, momenta_in_place=True, **PARAMS) as lat:
        lat.init(3)
        lat.step(2)
        before = [lat.box(AHS_FIELD_ALL, x - 2, y - 2, z - 2, 5, 5, 5).astype(np.float64) for (x, y, z) in sites]
        lat.step(1)
        after = [lat.box(AHS_FIELD_ALL, x, y, z, 1, 1, 1).astype(np.float64)[:, 0, 0, 0] for (x, y, z) in sites]
    p = orc.Params(N=5, era=1, **PARAMS)
    for B, A in zip(before, after):
        ref = B.copy()
        orc.run(p, 2, 1, ref)
        assert np.allclose(A, ref[:, 2, 2, 2], rtol=2e-6, atol=2e-6), (A, ref[:, 2, 2, 2])
