"""Two leapfrog steps per pass (AHS_OPT_STEPS_PER_PASS = 2, temporal blocking of
the z-marching step) against the FP64 oracle and against single steps.

* Two steps from identical float32 states against two oracle steps (Eqs. 7-10),
  element by element: every site within the per-site bound of the parity tests,
  for even, odd and sub-tile sides and every era, s = 1, a perturbed state with
  gauge fields and wrapped link angles.
* Against the single-step path: each site-update runs the same arithmetic in the
  same order, so the fields are equal bit for bit, also when pairs, measuring
  steps and left-over single steps interleave, at several z-chunks; the records
  (measured by the single-step kernel) are equal too.
"""
import numpy as np
import pytest

import inputs
from parity import field_errors, site_errors, worst_site

pytestmark = pytest.mark.gpu

PARAMS = dict(dx=0.5, dt=0.1, lambda0=2.0, e0=1.0, sigma=1.0)
SITE_TOL = 5e-6


@pytest.fixture(scope="module")
def pkg():
    import paper_2005_14454_gb300 as p
    from paper_2005_14454_gb300 import _abi
    _abi.lib()
    return p


def lattice(pkg, N, era=1, s=0.0, measure_every=0, steps_per_pass=2, zchunk=0, wrap=0):
    from paper_2005_14454_gb300 import _abi
    lat = pkg.Lattice(N, era=era, s=s, measure_every=measure_every, **PARAMS)
    lat.set_option(_abi.AHS_OPT_STEPS_PER_PASS, steps_per_pass)
    lat.set_option(_abi.AHS_OPT_ZCHUNK, zchunk)
    lat.set_option(_abi.AHS_OPT_WRAP_THETA, wrap)
    return lat


def assert_close(got, ref):
    err = field_errors(got, ref)
    assert max(err.values()) < 1e-5, err
    se = site_errors(got, ref)
    bad = {k: (v, worst_site(got, ref, k)) for k, v in se.items() if not v < SITE_TOL}
    assert not bad, bad


@pytest.mark.parametrize("N,era,s", [(24, 1, 0.0), (65, 1, 0.0), (66, 2, 0.0), (4, 1, 0.0), (7, 2, 0.0),
                                     (40, 0, 0.0), (36, 2, 1.0), (20, 1, 1.0)])
def test_two_steps_match_oracle(pkg, orc, N, era, s):
    with lattice(pkg, N, era=era, s=s) as lat:
        lat.init(300 + N)
        lat.step(3)
        F0 = lat.state().astype(np.float64)
        lat.step(2)                          # one two-step launch
        assert lat.n == 5
        got = lat.state().astype(np.float64)
    ref = F0.copy()
    orc.run(orc.Params(N=N, era=era, s=s, **PARAMS), 3, 2, ref)
    assert_close(got, ref)


def test_ten_steps_as_five_passes_match_oracle(pkg, orc):
    N = 66
    with lattice(pkg, N, era=2) as lat:
        lat.init(9)
        F0 = lat.state().astype(np.float64)
        lat.step(10)
        got = lat.state().astype(np.float64)
    ref = F0.copy()
    orc.run(orc.Params(N=N, era=2, **PARAMS), 0, 10, ref)
    assert_close(got, ref)


def test_perturbed_gauge_fields_and_wrapped_angles(pkg, orc):
    N = 32
    F = inputs.perturbed_state(N, 23, amp_theta=3.0, amp_e=0.4)
    F0 = inputs.to_f32(F).astype(np.float64)
    with lattice(pkg, N, era=1, wrap=1) as lat:
        lat.set_state(F0)
        lat.n = 2
        lat.step(2)
        got = lat.state().astype(np.float64)
    with lattice(pkg, N, era=1, wrap=1, steps_per_pass=1) as lat:
        lat.set_state(F0)
        lat.n = 2
        lat.step(2)
        single = lat.state()
    assert np.array_equal(got.astype(np.float32), single)
    assert np.abs(got[4:7]).max() <= np.pi + 1e-6
    ref = F0.copy()
    orc.run(orc.Params(N=N, era=1, **PARAMS), 2, 2, ref)
    assert_close(got, ref)


@pytest.mark.parametrize("N,zchunk", [(24, 0), (65, 0), (66, 0), (66, 5), (40, 1), (33, 33), (5, 0)])
def test_pairs_equal_single_steps_bit_for_bit(pkg, N, zchunk):
    out = {}
    for spp in (1, 2):
        with lattice(pkg, N, era=1, measure_every=5, steps_per_pass=spp, zchunk=zchunk) as lat:
            lat.init(41)
            lat.step(7)      # measuring step 0, pairs (1,2) (3,4), measuring 5, single 6
            lat.step(6)      # pairs (7,8), single 9, measuring 10, pair (11,12)
            out[spp] = (lat.state(), lat.records(), lat.n)
    assert out[1][2] == out[2][2] == 13
    assert np.array_equal(out[1][0], out[2][0])
    assert out[1][1] == out[2][1] and [r["step"] for r in out[2][1]] == [0, 5, 10]


def test_kernel_time_counts_pair_launches(pkg):
    from paper_2005_14454_gb300 import _abi
    with lattice(pkg, 32, measure_every=10) as lat:
        lat.init(1)
        _abi.ahs_set_option(lat.h, _abi.AHS_OPT_PROFILE, 1)
        lat.step(10)
        _, n_pair = _abi.ahs_kernel_time(lat.h, _abi.AHS_KERNEL_STEP_PAIR)
        _, n_one = _abi.ahs_kernel_time(lat.h, _abi.AHS_KERNEL_STEP)
        _, n_meas = _abi.ahs_kernel_time(lat.h, _abi.AHS_KERNEL_STEP_MEASURE)
    assert (n_pair, n_one, n_meas) == (4, 1, 1)


def test_option_requires_fp32_double_buffered(pkg):
    from paper_2005_14454_gb300 import AHSError, _abi
    with pkg.Lattice(16, **PARAMS) as lat:
        _abi.ahs_set_option(lat.h, _abi.AHS_OPT_MOMENTA_IN_PLACE, 1)
        with pytest.raises(AHSError):
            _abi.ahs_set_option(lat.h, _abi.AHS_OPT_STEPS_PER_PASS, 2)
    with pkg.Lattice(16, precision="fp64", **PARAMS) as lat:
        with pytest.raises(AHSError):
            _abi.ahs_set_option(lat.h, _abi.AHS_OPT_STEPS_PER_PASS, 2)
    with pkg.Lattice(16, **PARAMS) as lat:
        _abi.ahs_set_option(lat.h, _abi.AHS_OPT_STEPS_PER_PASS, 2)
        with pytest.raises(AHSError):
            _abi.ahs_set_option(lat.h, _abi.AHS_OPT_PRECISION, _abi.AHS_PREC_FP32_COMPENSATED)
        with pytest.raises(AHSError):
            _abi.ahs_set_option(lat.h, _abi.AHS_OPT_MOMENTA_IN_PLACE, 1)
        with pytest.raises(AHSError):
            _abi.ahs_set_option(lat.h, _abi.AHS_OPT_STEPS_PER_PASS, 3)
        assert _abi.ahs_get_option(lat.h, _abi.AHS_OPT_STEPS_PER_PASS) == 2
