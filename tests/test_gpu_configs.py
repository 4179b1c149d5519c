"""Whole runs of the benchmark configurations against the oracle.

* 64^3, radiation, s = 0, tau 1 -> 16 (150 steps, Sec. 2 run length), measurements
  every 10 steps: every record's xi_W, xi_L, <v^2>_phi and <v^2>_omega within 1% of
  the oracle's, winding counts close (the float32 and FP64 trajectories separate
  only slowly over 150 steps of this damped run).
* matter era with s = 1 (the 256^3 benchmark configuration) is beyond the leapfrog
  stability bound dt^2 omega_max^2 < 4 from eta ~ 3.6 on: engine and
  oracle agree step by step until the energy blows up, and the blow-up happens at
  the same step.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PARAMS = dict(dx=0.5, dt=0.1, lambda0=2.0, e0=1.0, sigma=1.0)


@pytest.fixture(scope="module")
def pkg():
    import paper_2005_14454_gb300 as p
    from paper_2005_14454_gb300 import _abi
    _abi.lib()
    return p


def test_radiation_64_full_run_observables(pkg, orc):
    N, seed = 64, 2020
    steps = orc.steps_to(N) + 1     # 0..150 inclusive: tau 1 -> 16
    assert steps - 1 == 150
    with pkg.Lattice(N, era=1, measure_every=10, **PARAMS) as lat:
        lat.init(seed)
        F0 = lat.state().astype(np.float64)
        lat.step(steps)
        recs = lat.records()
    assert [r["step"] for r in recs] == list(range(0, steps, 10))
    p = orc.Params(N=N, era=1, **PARAMS)
    F = F0.copy()
    n = 0
    for r in recs:
        orc.run(p, n, r["step"] - n, F)
        n = r["step"]
        o = orc.measure(p, n, F)
        assert r["tau"] == pytest.approx(o["tau"])
        for k in ("xi_w", "xi_l", "v2_phi", "v2_omega"):
            if math.isfinite(o[k]):
                assert r[k] == pytest.approx(o[k], rel=0.01), (n, k, r[k], o[k])
        assert abs(r["n_wind"] - o["n_wind"]) <= max(4, 0.01 * o["n_wind"]), (n, r["n_wind"], o["n_wind"])


def test_matter_s1_instability_onset_matches_oracle(pkg, orc):
    from paper_2005_14454_gb300 import AHSError
    N, seed, max_steps = 32, 7, 60
    with pkg.Lattice(N, era=2, s=1.0, measure_every=1, **PARAMS) as lat:
        lat.init(seed)
        F0 = lat.state().astype(np.float64)
        try:
            lat.step(max_steps)
        except AHSError:
            pass
        recs = lat.records()
    p = orc.Params(N=N, era=2, s=1.0, **PARAMS)
    F = F0.copy()
    e_gpu = np.array([r["e_total"] for r in recs])
    e_orc = []
    for n in range(len(recs)):
        e_orc.append(orc.measure(p, n, F)["e_total"])
        orc.run(p, n, 1, F)
    e_orc = np.array(e_orc)

    def onset(e):
        bad = np.nonzero(~np.isfinite(e) | (e > 1e3 * e[1]))[0]
        return int(bad[0]) if bad.size else None

    n_gpu, n_orc = onset(e_gpu), onset(e_orc)
    assert n_orc is not None and n_gpu is not None, (n_gpu, n_orc)
    assert abs(n_gpu - n_orc) <= 2
    # before the blow-up the two runs agree
    stable = max(2, int(0.7 * min(n_gpu, n_orc)))
    assert np.allclose(e_gpu[:stable], e_orc[:stable], rtol=1e-4)
    # stability bound of the leapfrog: dt^2 w_max^2 < 4 with w_max^2 ~ 12/dx^2 + lambda0 a^2 sigma^2
    eta = 1.0 + 0.1 * n_orc
    assert eta > ((4 / 0.01 - 12 / 0.25) / 2.0) ** 0.25 * 0.8


def test_matter_s1_256_runs_to_the_monitor(pkg):
    """The 256^3 matter-era, s = 1 configuration on the GPU: the fused measurement
    reports non-finite sites (the step call returns AHS_ENONFINITE) well before
    tau = 64; the step it trips at is reported."""
    from paper_2005_14454_gb300 import AHSError
    from paper_2005_14454_gb300._abi import AHS_ENONFINITE
    with pkg.Lattice(256, era=2, s=1.0, measure_every=10, **PARAMS) as lat:
        lat.init(1)
        tripped = None
        for chunk in range(63):
            try:
                lat.step(10)
            except AHSError as e:
                assert e.status == AHS_ENONFINITE
                tripped = lat.n
                break
        recs = lat.records()
    assert tripped is not None and tripped < 630
    e = [r["e_total"] for r in recs]
    assert math.isfinite(e[0]) and e[1] > 0
    print(f"256^3 matter s=1: non-finite measurement at step {tripped} (tau = {1 + 0.1 * (tripped - 10):.1f})")
