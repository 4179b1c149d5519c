"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (float32 storage and arithmetic against FP64):
* fields after 10 leapfrog steps from identical float32 states: relative L2 error
  <= 1e-5 per field group (phi, Pi, theta via exp(-i theta), E), and at every
  single site an error <= 5e-6 of the group's RMS (tests/parity.py);
* windings on identical snapshots: bit-exact, per plaquette;
* observables on identical snapshots: sums of non-negative site terms to 2e-5
  relative; signed or ratio observables to 2e-4 relative (per-site float32
  rounding ~1e-7 amplified by cancellation between the Lagrangian's terms);
* Gauss residual: float32 rounding level on both sides (same snapshot).
"""
import math

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


def lattice(eng, N, era=1, s=0.0, measure_every=0, **kw):
    p = dict(PARAMS)
    p.update(kw)
    return eng.Lattice(N, era=era, s=s, measure_every=measure_every, **p)


def oparams(orc, N, era=1, s=0.0, **kw):
    p = dict(PARAMS)
    p.update(kw)
    return orc.Params(N=N, era=era, s=s, **p)


from parity import field_errors, rel, site_errors, worst_site  # noqa: E402

# Per-site bound of the 10-step field checks: the largest error at any single site,
# on the scale of the field group's RMS (see parity.site_errors).  Ten float32 steps
# leave errors of a few 1e-7 of that scale at a typical site (the L2 measure); the
# worst of up to 3e5 sites sits a few times above the typical one.
SITE_TOL = 5e-6


def assert_fields_match(got, ref):
    err = field_errors(got, ref)
    assert max(err.values()) < 1e-5, err
    se = site_errors(got, ref)
    bad = {k: (v, worst_site(got, ref, k)) for k, v in se.items() if not v < SITE_TOL}
    assert not bad, bad


# ------------------------------------------------------------------ init
@pytest.mark.parametrize("N", [4, 24, 40, 64])
def test_init_matches_oracle(eng, orc, N):
    with lattice(eng, N) as lat:
        lat.init(99)
        F = lat.state().astype(np.float64)
    ref = orc.init(oparams(orc, N), 99)
    ref32 = ref.astype(np.float32).astype(np.float64)
    assert not F[2:].any()
    diff = np.abs(F - ref32)
    # FP64 cos/sin of the GPU and of libm may differ in the last bit, which changes
    # the float32 rounding only next to a rounding boundary
    assert diff.max() <= 1.2e-7
    assert (diff > 0).sum() <= max(2, F.size // 100000)


# ------------------------------------------------------------------ evolution
CASES = [
    (4, 1, 0.0), (5, 1, 0.0), (7, 2, 0.0),                  # smaller than one tile, odd N
    (8, 1, 0.0), (24, 1, 0.0), (40, 1, 0.0), (64, 1, 0.0),   # radiation, several tiles, ragged
    (24, 2, 0.0), (24, 0, 0.0), (36, 2, 1.0), (20, 1, 1.0),  # matter, Minkowski, s = 1
    (6, 1, 0.0), (66, 2, 0.0), (65, 1, 0.0),                # paired step with a 2-site ragged tile; odd N > 64
]


@pytest.mark.parametrize("N,era,s", CASES)
def test_ten_steps_match_oracle(eng, orc, N, era, s):
    with lattice(eng, N, era=era, s=s) as lat:
        lat.init(2024 + N)
        F0 = lat.state().astype(np.float64)
        lat.step(10)
        got = lat.state().astype(np.float64)
        assert lat.n == 10
    ref = F0.copy()
    orc.run(oparams(orc, N, era=era, s=s), 0, 10, ref)
    assert_fields_match(got, ref)


@pytest.mark.parametrize("N", [20, 40, 64])
def test_launch_shapes_give_identical_fields(eng, N):
    # every link phase and plaquette is computed by the same arithmetic whatever the
    # tile heights (plain and measuring steps) and z-chunk, so the fields agree bit
    # for bit; the reductions differ only in grouping
    from paper_2005_14454_gb300._abi import AHS_OPT_MEASURE_TILE_Y, AHS_OPT_TILE_Y, AHS_OPT_ZCHUNK
    outs, recs = [], []
    for by, mby, dz in [(8, 0, 0), (16, 8, 0), (8, 16, 5), (16, 4, 3), (8, 8, N), (16, 4, 1), (8, 4, 2)]:
        with lattice(eng, N, measure_every=3) as lat:
            lat.set_option(AHS_OPT_TILE_Y, by)
            lat.set_option(AHS_OPT_MEASURE_TILE_Y, mby)
            lat.set_option(AHS_OPT_ZCHUNK, dz)
            lat.init(5)
            lat.step(7)
            outs.append(lat.state())
            recs.append(lat.records())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    for r in recs[1:]:
        for a, b in zip(r, recs[0]):
            assert a["n_wind"] == b["n_wind"]
            assert a["e_total"] == pytest.approx(b["e_total"], rel=1e-6)
            assert a["lagrangian"] == pytest.approx(b["lagrangian"], rel=1e-5)


def test_measure_tile_height_option(eng):
    """AHS_OPT_MEASURE_TILE_Y: 4-row tiles by default (8 in FP64 precision), 4, 8 or
    16 when set, anything else rejected; ahs_autotune picks one of the three."""
    from paper_2005_14454_gb300 import _abi
    L = _abi.lib()
    key = _abi.AHS_OPT_MEASURE_TILE_Y
    with lattice(eng, 24) as lat:
        assert int(_abi.ahs_get_option(lat.h, key)) == 4
        for bad in (1, 2, 12, 32, -4, 4.5):
            assert L.ahs_set_option(lat.h, key, bad) == _abi.AHS_EINVAL
        assert b"measure_tile_y" in L.ahs_last_error_message()
        for v in (16, 8, 4):
            lat.set_option(key, v)
            assert int(_abi.ahs_get_option(lat.h, key)) == v
        lat.init(3)
        lat.autotune()
        assert int(_abi.ahs_get_option(lat.h, key)) in (4, 8, 16)
        lat.set_option(_abi.AHS_OPT_PRECISION, _abi.AHS_PREC_FP64)
        assert int(_abi.ahs_get_option(lat.h, key)) == 8


def test_perturbed_state_with_gauge_fields(eng, orc):
    # nonzero theta, E, Pi from the start (all force terms active in step 1)
    N = 32
    F0 = inputs.to_f32(inputs.perturbed_state(N, 5, amp_theta=0.6, amp_e=0.4)).astype(np.float64)
    with lattice(eng, N, era=2) as lat:
        lat.set_state(F0)
        lat.n = 3
        lat.step(10)
        got = lat.state().astype(np.float64)
    ref = F0.copy()
    orc.run(oparams(orc, N, era=2), 3, 10, ref)
    assert_fields_match(got, ref)


@pytest.mark.parametrize("span", [3.0, 50.0, 9000.0])
def test_large_link_angles(eng, orc, span):
    # link angles over many turns, up to the large-argument range of the float32
    # sine and cosine: one step against the oracle
    N = 16
    F = inputs.perturbed_state(N, 31)
    rng = np.random.default_rng(5)
    F[4:7] = rng.uniform(-span, span, (3, N, N, N))
    F0 = inputs.to_f32(F).astype(np.float64)
    with lattice(eng, N) as lat:
        lat.set_state(F0)
        lat.step(1)
        got = lat.state().astype(np.float64)
    ref = F0.copy()
    orc.run(oparams(orc, N), 0, 1, ref)
    # theta itself carries float32 rounding of its magnitude: compare the kicks
    for sl in (slice(0, 2), slice(2, 4), slice(7, 10)):
        assert rel(got[sl], ref[sl]) < 2e-6 * max(1.0, span / 50.0)
    assert np.abs(got[4:7] - ref[4:7]).max() < 4e-7 * span + 1e-6


def test_vacuum_is_exact_fixed_point(eng):
    N = 16
    F = np.zeros((10, N, N, N), np.float32)
    F[0] = 1.0
    with lattice(eng, N, era=2) as lat:
        lat.set_state(F)
        lat.step(7)
        assert np.array_equal(lat.state(), F)


# ------------------------------------------------------------------ windings
@pytest.mark.parametrize("N,steps", [(24, 15), (64, 30)])
def test_windings_bit_exact_on_identical_snapshot(eng, orc, N, steps):
    with lattice(eng, N) as lat:
        lat.init(7)
        lat.step(steps)
        snap = lat.state().astype(np.float64)
        W, n = lat.windings()
        obs = lat.measure()
    Wo, no = orc.windings(oparams(orc, N), snap)
    assert no > 0
    assert np.array_equal(W, Wo)
    assert n == no == obs["n_wind"]


@pytest.mark.parametrize("N,eps", [(16, 2e-6), (40, 2e-6), (32, 5e-5)])
def test_windings_at_the_branch_cut(eng, orc, N, eps):
    """Every x and y link phase within 2 eps of +-pi.  With eps = 2e-6 all of them
    are flagged (|Im z| <= 1e-5 |Re z|) and their sites' windings come from FP64
    angles; with eps = 5e-5 most are decided by the sign of the float32 value in the
    margin the flag leaves.  Either way the windings must equal the oracle's FP64
    windings plaquette by plaquette."""
    F = inputs.to_f32(inputs.with_phase(inputs.branch_cut_phase(N, 3, eps=eps))).astype(np.float64)
    with lattice(eng, N) as lat:
        lat.set_state(F)
        W, n = lat.windings()
        obs = lat.measure()
    Wo, no = orc.windings(oparams(orc, N), F)
    assert no > N ** 3 // 10
    assert np.array_equal(W, Wo)
    assert n == no == obs["n_wind"]


def test_vortex_pair_windings(eng):
    N = 32
    F = inputs.with_phase(inputs.vortex_pair_phase(N))
    chi = inputs.gauge_function(N, 4)
    e = np.exp(1j * chi)
    phi = (F[0] + 1j * F[1]) * e
    F[0], F[1] = phi.real, phi.imag
    for i, ax in enumerate((2, 1, 0)):
        F[4 + i] = np.roll(chi, -1, axis=ax) - chi
    with lattice(eng, N) as lat:
        lat.set_state(F)
        W, n = lat.windings()
        obs = lat.measure()
    assert n == 2 * N and obs["n_wind"] == 2 * N
    (x1, y1), (x2, y2) = inputs.vortex_pair_cores(N)
    assert (W[0, :, y1, x1] == 1).all() and (W[0, :, y2, x2] == -1).all()


# ------------------------------------------------------------------ measurement
SUMS = ("sum_K", "sum_G", "sum_V", "sum_El", "sum_B", "e_total")
SIGNED = ("lagrangian", "xi_l", "v2_phi", "v2_omega", "sum_KL", "sum_GL", "sum_pL", "sum_rhoL")


@pytest.mark.parametrize("N,era,s,steps", [(32, 1, 0.0, 12), (48, 2, 0.0, 25), (24, 1, 1.0, 5)])
def test_measure_matches_oracle_on_identical_snapshot(eng, orc, N, era, s, steps):
    with lattice(eng, N, era=era, s=s) as lat:
        lat.init(31)
        lat.step(steps)
        snap = lat.state().astype(np.float64)
        obs = lat.measure()
        assert lat.n == steps
    o = orc.measure(oparams(orc, N, era=era, s=s), steps, snap)
    assert obs["step"] == steps and obs["tau"] == pytest.approx(o["tau"]) and obs["a"] == pytest.approx(o["a"])
    for k in SUMS:
        assert obs[k] == pytest.approx(o[k], rel=2e-5), k
    for k in SIGNED:
        assert obs[k] == pytest.approx(o[k], rel=2e-4), k
    assert obs["n_wind"] == o["n_wind"]
    assert obs["xi_w"] == pytest.approx(o["xi_w"], rel=1e-12)
    assert obs["nonfinite"] == 0
    # Gauss residual of a float32-evolved snapshot sits at float32 rounding; both
    # sides evaluate it on the same snapshot, the engine in float32
    scale = np.abs(snap[7:10]).max() / PARAMS["dx"] + np.abs(snap[2:4]).max() + 1.0
    assert o["gauss_max"] < 1e-5 * scale
    assert obs["gauss_max"] < 1e-5 * scale
    assert abs(obs["gauss_rms"] - o["gauss_rms"]) < 1e-6 * scale


def test_fused_records_equal_standalone_measure(eng):
    N = 32
    with lattice(eng, N, measure_every=10) as lat:
        lat.init(3)
        lat.step(10)
        standalone = lat.measure()
        lat.step(15)
        recs = lat.records()
    assert [r["step"] for r in recs] == [0, 10, 20]
    assert recs[1] == standalone


def test_step_zero_and_records_drain(eng):
    with lattice(eng, 16, measure_every=3) as lat:
        lat.init(1)
        lat.step(0)
        assert lat.records() == []
        lat.step(7)
        assert [r["step"] for r in lat.records()] == [0, 3, 6]
        assert lat.records() == []


def test_nonfinite_is_reported(eng):
    from paper_2005_14454_gb300 import AHSError
    from paper_2005_14454_gb300._abi import AHS_ENONFINITE
    N = 16
    F = inputs.to_f32(inputs.perturbed_state(N, 2))
    F[7, 3, 4, 5] = np.nan
    with lattice(eng, N, measure_every=1) as lat:
        lat.set_state(F)
        with pytest.raises(AHSError) as ei:
            lat.step(2)
        assert ei.value.status == AHS_ENONFINITE
        assert lat.n == 2
        assert lat.measure()["nonfinite"] > 0


# ------------------------------------------------------------------ data movement
def test_resume_is_bit_exact(eng):
    N = 24
    with lattice(eng, N) as a:
        a.init(77)
        a.step(20)
        full = a.state()
    with lattice(eng, N) as b:
        b.init(77)
        b.step(10)
        snap = b.state()
    with lattice(eng, N) as c:
        c.set_state(snap)
        c.n = 10
        c.step(10)
        assert np.array_equal(c.state(), full)


def test_fields_box_periodic(eng):
    N = 20
    F = inputs.to_f32(inputs.perturbed_state(N, 9))
    with lattice(eng, N) as lat:
        lat.set_state(F)
        from paper_2005_14454_gb300 import AHS_FIELD_ALL, AHS_FIELD_THETA
        B = lat.box(AHS_FIELD_ALL, 17, 3, 19, 6, 5, 4)
        T = lat.box(AHS_FIELD_THETA, -2, 0, 0, N, 1, 1)
    xs, ys, zs = (np.arange(17, 23) % N), (np.arange(3, 8) % N), (np.arange(19, 23) % N)
    want = F[:, zs][:, :, ys][:, :, :, xs]
    assert np.array_equal(B, want)
    assert np.array_equal(T[:, 0, 0, :], F[4:7, 0, 0, (np.arange(-2, N - 2) % N)])


def test_bad_buffers_rejected(eng):
    from paper_2005_14454_gb300 import AHSError, _abi
    with lattice(eng, 8) as lat:
        with pytest.raises(AHSError):
            lat.step(1)                                  # not initialised
        lat.init(1)
        with pytest.raises(AHSError):
            _abi.ahs_set_fields(lat.h, 0, np.zeros(10, np.float32))
        with pytest.raises(AHSError):
            _abi.ahs_set_option(lat.h, _abi.AHS_OPT_MEASURE_EVERY, -1)
        with pytest.raises(AHSError):
            lat.box(0, 0, 0, 0, 9, 1, 1)


# ------------------------------------------------------------------ full size
def sampled_sites(N, count, seed):
    rng = np.random.default_rng(seed)
    sites = [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(count)]
    # corners, and sites on both sides of the 192-plane z-chunk boundaries of 1024^3
    sites += [(0, 0, 0), (N - 1, N - 1, N - 1), (0, N - 1, 511), (N - 1, 0, 0)]
    sites += [(5, 77, 191), (64, 63, 192), (1023, 8, 383), (31, 7, 384), (700, 900, 767), (1, 1, 768)]
    return [(x % N, y % N, z % N) for (x, y, z) in sites]


def check_sites(orc, before, after, n):
    p = oparams(orc, 5)
    for B, A in zip(before, after):
        ref = B.copy()
        orc.run(p, n, 1, ref)
        r = ref[:, 2, 2, 2]
        assert np.allclose(A, r, rtol=2e-6, atol=2e-6), (A, r)


def test_full_size_sampled_sites(eng, orc):
    """1024^3 in the launch configuration the benchmark times: a plain step (the
    paired kernel) and a measuring step (the fused measurement kernel, 32 x 4 tiles,
    192-plane z-chunks, 49152 rows of partial sums), each checked at sampled sites
    against the oracle run on the 5^3 periodic neighbourhood of each site (the update
    of a site reads only its nearest and next-nearest neighbours).  The record of the
    measuring step is checked by properties that hold at any size: it equals
    ahs_measure at the same launch shape bit for bit, its winding count equals the
    sum of |W| of the separate winding kernel, and measurements at another z-chunk
    (64 planes, 131072 rows) and with 8-row tiles (24576 rows) agree up to the
    grouping of the sums."""
    N = 1024
    sites = sampled_sites(N, 12, 0)
    from paper_2005_14454_gb300 import AHS_FIELD_ALL
    from paper_2005_14454_gb300._abi import AHS_OPT_MEASURE_TILE_Y, AHS_OPT_ZCHUNK

    def boxes(lat, w):
        o = -(w // 2)
        return [lat.box(AHS_FIELD_ALL, x + o, y + o, z + o, w, w, w).astype(np.float64) for (x, y, z) in sites]

    with lattice(eng, N, measure_every=10) as lat:
        assert int(lat.n) == 0
        lat.init(1)
        lat.step(3)
        before = boxes(lat, 5)
        lat.step(1)                                # n = 3: plain step
        check_sites(orc, before, [b[:, 0, 0, 0] for b in boxes(lat, 1)], 3)
        lat.step(6)
        assert lat.n == 10
        get = __import__("paper_2005_14454_gb300")._abi.ahs_get_option
        assert int(get(lat.h, AHS_OPT_ZCHUNK)) == 192 and int(get(lat.h, AHS_OPT_MEASURE_TILE_Y)) == 4
        lat.records()
        before = boxes(lat, 5)
        standalone = lat.measure()
        W, n_wind = lat.windings()
        del W
        lat.set_option(AHS_OPT_ZCHUNK, 64)
        other = lat.measure()
        lat.set_option(AHS_OPT_ZCHUNK, 0)
        lat.set_option(AHS_OPT_MEASURE_TILE_Y, 8)
        rows8 = lat.measure()
        lat.set_option(AHS_OPT_MEASURE_TILE_Y, 0)
        lat.step(1)                                # n = 10: measuring step
        rec = lat.records()
        check_sites(orc, before, [b[:, 0, 0, 0] for b in boxes(lat, 1)], 10)
    assert [r["step"] for r in rec] == [10]
    assert rec[0] == standalone
    assert rec[0]["n_wind"] == n_wind == other["n_wind"] == rows8["n_wind"] > 0
    assert rec[0]["gauss_max"] == other["gauss_max"] == rows8["gauss_max"]
    assert rec[0]["nonfinite"] == 0
    for alt in (other, rows8):
        for k in SUMS:
            assert rec[0][k] == pytest.approx(alt[k], rel=1e-5), k
        for k in SIGNED:
            assert rec[0][k] == pytest.approx(alt[k], rel=2e-4), k


def test_measure_at_benchmark_zchunk_matches_oracle(eng, orc):
    """The fused measurement at the z-chunk the 1024^3 benchmark uses (192 planes),
    on a 640^3 lattice (three full chunks and a ragged one of 64; 32 x 4 tiles,
    12800 rows of partial sums) against the oracle's measurement of the same snapshot: windings
    bit-exact, sums and ratios to the tolerances of the identical-snapshot test."""
    from paper_2005_14454_gb300._abi import AHS_OPT_ZCHUNK
    N, steps = 640, 10
    with lattice(eng, N, era=1) as lat:
        lat.init(11)
        lat.step(steps)
        lat.set_option(AHS_OPT_ZCHUNK, 192)
        obs = lat.measure()
        snap = lat.state()
    o = orc.measure(oparams(orc, N), steps, snap.astype(np.float64))
    del snap
    assert obs["n_wind"] == o["n_wind"] > 0
    assert obs["nonfinite"] == o["nonfinite"] == 0
    for k in SUMS:
        assert obs[k] == pytest.approx(o[k], rel=2e-5), k
    for k in SIGNED:
        assert obs[k] == pytest.approx(o[k], rel=2e-4), k
    assert abs(obs["gauss_rms"] - o["gauss_rms"]) < 1e-6 * (1.0 + abs(o["gauss_rms"]))


# ------------------------------------------------------------------ core growth
@pytest.mark.parametrize("era", [1, 2])
def test_core_growth_matches_oracle(eng, orc, era):
    """s = -1 until eta = 2.05, then s = 1 with c continuous (Sec. 2 core growth):
    fields after the switch and every record of the run against the oracle."""
    N = 24
    with lattice(eng, N, era=era, s=1.0, measure_every=4, core_growth=(-1.0, 2.05)) as lat:
        lat.init(31)
        F0 = lat.state().astype(np.float64)
        lat.step(18)
        got = lat.state().astype(np.float64)
        recs = lat.records()
    p = oparams(orc, N, era=era, s=1.0, s_cg=-1.0, tau_cg=2.05)
    ref = F0.copy()
    n = 0
    for r in recs:
        orc.run(p, n, r["step"] - n, ref)
        n = r["step"]
        o = orc.measure(p, n, ref)
        # two trajectories (float32 engine, FP64 oracle) from the same start: the
        # total to 2e-5, the small magnetic and potential parts to 1e-4
        assert r["e_total"] == pytest.approx(o["e_total"], rel=2e-5), n
        for k in ("e_pot", "e_mag"):
            assert r[k] == pytest.approx(o[k], rel=1e-4), (n, k)
        assert r["gauss_max"] == pytest.approx(o["gauss_max"], rel=2e-2, abs=5e-6), n
    orc.run(p, n, 18 - n, ref)
    err = field_errors(got, ref)
    assert max(err.values()) < 1e-5, err
    # 18 steps through the switch of c: every site within 1e-5 of its field's RMS
    se = site_errors(got, ref)
    assert max(se.values()) < 1e-5, se


# ------------------------------------------------------------------ cooling, straight strings
def test_cooled_vortex_pair_matches_oracle(eng, orc):
    """Straight vortex-antivortex pair along z relaxed by 200 cooling steps (a = 1,
    delta = omega = 0.5): windings exactly +-1 at the cores on every z-layer and
    2N in total at every measurement, fields equal to the oracle's."""
    from paper_2005_14454_gb300._abi import AHS_OPT_COOLING
    N = 32
    F0 = inputs.to_f32(inputs.with_phase(inputs.vortex_pair_phase(N))).astype(np.float64)
    with lattice(eng, N, measure_every=20) as lat:
        lat.set_option(AHS_OPT_COOLING, 0.5)
        lat.set_state(F0)
        lat.step(200)
        recs = lat.records()
        got = lat.state().astype(np.float64)
        W, n = lat.windings()
    assert [r["n_wind"] for r in recs] == [2 * N] * 10
    e = [r["e_total"] for r in recs]
    assert all(b < a for a, b in zip(e, e[1:]))
    (x1, y1), (x2, y2) = inputs.vortex_pair_cores(N)
    assert n == 2 * N and (W[0, :, y1, x1] == 1).all() and (W[0, :, y2, x2] == -1).all()
    ref = F0.copy()
    orc.run(oparams(orc, N, cool=0.5), 0, 200, ref)
    err = field_errors(got, ref)
    assert err["phi"] < 1e-5 and err["theta"] < 1e-5, err
    se = site_errors(got, ref)
    assert se["phi"] < 1e-5 and se["theta"] < 1e-5, se
    # the momenta are damped towards zero: compare them on the scale of phi
    scale = np.linalg.norm(ref[0:2])
    assert np.linalg.norm(got[2:4] - ref[2:4]) / scale < 1e-5
    assert np.linalg.norm(got[7:10] - ref[7:10]) / scale < 1e-5
