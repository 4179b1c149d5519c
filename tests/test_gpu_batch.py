"""Batched ensembles: members of uneven sizes and eras advanced by one persistent
launch per step (graph-replayed measurement periods) equal single-lattice runs of
the same seeds bit for bit, stop at their own last step, and match the oracle."""
import numpy as np
import pytest

from parity import field_errors, site_errors

pytestmark = pytest.mark.gpu

PARAMS = dict(dx=0.5, dt=0.1, lambda0=2.0, e0=1.0, sigma=1.0)
MEMBERS = [  # (N, era, seed, n_end)
    (16, 1, 11, 25), (24, 2, 12, 17), (20, 0, 13, 30), (36, 1, 14, 22), (8, 2, 15, 9),
]
# odd and even sides: a plain step runs the paired launch and the one-site launch
MIXED = [(15, 1, 21, 19), (16, 2, 22, 23), (21, 0, 23, 12), (66, 1, 24, 16), (5, 2, 25, 21), (33, 1, 26, 14)]


@pytest.fixture(scope="module")
def pkg():
    import paper_2005_14454_gb300 as p
    from paper_2005_14454_gb300 import _abi
    _abi.lib()
    return p


def single(pkg, N, era, seed, steps, measure_every=5):
    with pkg.Lattice(N, era=era, measure_every=measure_every, **PARAMS) as lat:
        lat.init(seed)
        lat.step(steps)
        return lat.state(), lat.records()


def make_batch(pkg, members=MEMBERS, measure_every=5):
    N, era, seed, end = zip(*members)
    return pkg.Batch(N, era, seed, list(end), measure_every=measure_every, **PARAMS)


@pytest.mark.parametrize("graph,members", [(1, MEMBERS), (0, MEMBERS), (1, MIXED), (0, MIXED)])
def test_batch_equals_single_runs(pkg, graph, members):
    from paper_2005_14454_gb300._abi import AHS_OPT_GRAPH
    with make_batch(pkg, members=members) as b:
        b.set_option(AHS_OPT_GRAPH, graph)
        b.init()
        done = b.run()
        assert done == max(m[3] for m in members)
        assert b.run() == 0
        for i, (N, era, seed, end) in enumerate(members):
            n, n_end = b.step_info(i)
            assert n == n_end == end
            F, rec = single(pkg, N, era, seed, end)
            assert np.array_equal(b.state(i), F), i
            got = b.records(i)
            assert [r["step"] for r in got] == [r["step"] for r in rec] == list(range(0, end, 5))
            assert got == rec


def test_batch_measuring_tile_height(pkg):
    """Measuring steps on 4-row tiles (the default) or 8- and 16-row ones: the fields
    are the same bit for bit, the records those of single lattices of the same
    measuring height, and other heights are rejected."""
    from paper_2005_14454_gb300 import _abi
    key = _abi.AHS_OPT_MEASURE_TILE_Y
    members = MIXED[:4]
    with make_batch(pkg, members=members) as a:
        assert int(_abi.ahs_batch_get_option(a.b, key)) == 4
        for bad in (2, 12, -1, 4.5):
            assert _abi.lib().ahs_batch_set_option(a.b, key, bad) == _abi.AHS_EINVAL
        a.init()
        a.run()
        ref = [a.state(i) for i in range(len(members))]
    for mby in (8, 16):
        with make_batch(pkg, members=members) as b:
            b.set_option(key, mby)
            assert int(_abi.ahs_batch_get_option(b.b, key)) == mby
            b.init()
            b.run()
            for i, (N, era, seed, end) in enumerate(members):
                assert np.array_equal(b.state(i), ref[i]), (mby, i)
                with pkg.Lattice(N, era=era, measure_every=5, **PARAMS) as lat:
                    lat.set_option(key, mby)
                    lat.init(seed)
                    lat.step(end)
                    assert b.records(i) == lat.records(), (mby, i)


def test_batch_runs_in_pieces(pkg):
    # uneven run lengths: graph periods and single steps interleave
    with make_batch(pkg) as b1, make_batch(pkg) as b2:
        b1.init()
        b2.init()
        b1.run()
        for chunk in (3, 7, 1, 12, 100):
            b2.run(chunk)
        for i in range(len(MEMBERS)):
            assert np.array_equal(b1.state(i), b2.state(i))
            assert b1.records(i) == b2.records(i)


def test_batch_member_matches_oracle(pkg, orc):
    with make_batch(pkg, members=[(24, 1, 3, 10), (32, 2, 4, 10)]) as b:
        b.init()
        F0 = [b.state(i).astype(np.float64) for i in range(2)]
        b.run()
        for i, (N, era) in enumerate([(24, 1), (32, 2)]):
            ref = F0[i].copy()
            orc.run(orc.Params(N=N, era=era, **PARAMS), 0, 10, ref)
            got = b.state(i).astype(np.float64)
            err = field_errors(got, ref)
            assert max(err.values()) < 1e-5, err
            se = site_errors(got, ref)
            assert max(se.values()) < 5e-6, se


@pytest.mark.parametrize("members", [MEMBERS, MIXED])
def test_batch_autotune_keeps_results(pkg, members):
    from paper_2005_14454_gb300._abi import AHS_OPT_TILE_Y, ahs_batch_get_option, ahs_batch_member_zchunk
    with make_batch(pkg, members=members) as a, make_batch(pkg, members=members) as b:
        a.init()
        b.init()
        b.autotune()
        by = int(ahs_batch_get_option(b.b, AHS_OPT_TILE_Y))
        # the tile height only shapes the one-site plain tiles of odd sides
        assert by in ((8, 16) if any(m[0] % 2 for m in members) else (8,))
        assert all(ahs_batch_member_zchunk(b.b, i) >= 1 for i in range(len(members)))
        a.run()
        b.run()
        for i in range(len(members)):
            assert np.array_equal(a.state(i), b.state(i))
            assert a.records(i)[-1]["n_wind"] == b.records(i)[-1]["n_wind"]


def test_batch_set_fields_and_nonfinite(pkg):
    from paper_2005_14454_gb300 import AHSError
    from paper_2005_14454_gb300._abi import AHS_ENONFINITE
    with make_batch(pkg, members=[(16, 1, 1, 20), (12, 1, 2, 20)]) as b:
        b.init()
        F = b.state(1)
        F[8, 2, 3, 4] = np.inf
        b.set_state(1, F)
        with pytest.raises(AHSError) as ei:
            b.run(6)
        assert ei.value.status == AHS_ENONFINITE
        assert b.step_info(0)[0] == 6


def test_batch_bad_arguments(pkg):
    from paper_2005_14454_gb300 import AHSError
    with pytest.raises(AHSError):
        pkg.Batch([16, 3], [1, 1], [1, 2])
    with pytest.raises(AHSError):
        pkg.Batch([16], [5], [1])
    with make_batch(pkg) as b:
        with pytest.raises(AHSError):
            b.run(1)          # not initialised
        b.init()
        from paper_2005_14454_gb300 import _abi
        with pytest.raises(AHSError):
            _abi.ahs_batch_fields(b.b, 99, _abi.AHS_FIELD_ALL, 16)


def test_batch_core_growth_equals_single_runs(pkg):
    from paper_2005_14454_gb300._abi import AHS_OPT_CORE_GROWTH_S, AHS_OPT_CORE_GROWTH_TAU
    members = [(16, 1, 21, 30), (20, 2, 22, 26)]
    N, era, seed, end = zip(*members)
    with pkg.Batch(N, era, seed, list(end), measure_every=5, s=1.0, **PARAMS) as b:
        b.set_option(AHS_OPT_CORE_GROWTH_S, -1.0)
        b.set_option(AHS_OPT_CORE_GROWTH_TAU, 2.05)
        b.init()
        b.run()
        for i, (n, e, sd, ne) in enumerate(members):
            with pkg.Lattice(n, era=e, s=1.0, measure_every=5, core_growth=(-1.0, 2.05), **PARAMS) as lat:
                lat.init(sd)
                lat.step(ne)
                assert np.array_equal(b.state(i), lat.state()), i
                for rb, rs in zip(b.records(i), lat.records()):
                    assert rb == rs, {k: (rb[k], rs[k]) for k in rb if rb[k] != rs[k]}


def test_ensemble_means_match_oracle(pkg, orc):
    """The ensemble comparison of the benchmark's batched run, scaled down: four
    64^3 realisations (two radiation, two matter, s = 0) batched to half
    light-crossing (150 steps); the ensemble means of xi_W / tau, xi_L / tau,
    <v^2>_omega and <v^2>_phi at every measurement after the first agree with the
    oracle's run of the same starts within 1%."""
    members = [(64, 1, 41, 151), (64, 1, 42, 151), (64, 2, 43, 151), (64, 2, 44, 151)]
    N, era, seed, end = zip(*members)
    with pkg.Batch(N, era, seed, list(end), measure_every=10, **PARAMS) as b:
        b.init()
        starts = [b.state(i).astype(np.float64) for i in range(len(members))]
        b.run()
        recs = [b.records(i) for i in range(len(members))]
    keys = ("xi_w", "xi_l", "v2_omega", "v2_phi")
    for eras in ((0, 1), (2, 3)):
        gpu = {k: [] for k in keys}
        ref = {k: [] for k in keys}
        for i in eras:
            p = orc.Params(N=64, era=members[i][1], **PARAMS)
            F = starts[i].copy()
            n = 0
            rows_g, rows_o = [], []
            for r in recs[i][1:]:
                orc.run(p, n, r["step"] - n, F)
                n = r["step"]
                o = orc.measure(p, n, F)
                rows_g.append([r["xi_w"] / r["tau"], r["xi_l"] / r["tau"], r["v2_omega"], r["v2_phi"]])
                rows_o.append([o["xi_w"] / o["tau"], o["xi_l"] / o["tau"], o["v2_omega"], o["v2_phi"]])
            for j, k in enumerate(keys):
                gpu[k].append([row[j] for row in rows_g])
                ref[k].append([row[j] for row in rows_o])
        for k in keys:
            g, o = np.mean(gpu[k], axis=0), np.mean(ref[k], axis=0)
            assert np.allclose(g, o, rtol=0.01), (eras, k, g, o)


def test_benchmark_ensemble_128_members_match_oracle(pkg, orc):
    """The first four 128^3 realisations of the benchmark's ensemble (seeds 1-4,
    radiation and matter alternating, s = 0, 310 steps to half light-crossing,
    measurement every 10 steps) run as one batch: ensemble means of xi_W / tau and
    of both velocity estimators at every measurement after the first within 1% of
    the oracle's runs from the same starts."""
    members = [(128, 1, 1, 311), (128, 2, 2, 311), (128, 1, 3, 311), (128, 2, 4, 311)]
    N, era, seed, end = zip(*members)
    with pkg.Batch(N, era, seed, list(end), measure_every=10, **PARAMS) as b:
        b.init()
        starts = [b.state(i).astype(np.float64) for i in range(len(members))]
        b.run()
        recs = [b.records(i) for i in range(len(members))]
    keys = ("xi_w", "v2_omega", "v2_phi")
    gpu, ref = [], []
    for i, (n, e, sd, ne) in enumerate(members):
        p = orc.Params(N=n, era=e, **PARAMS)
        F = starts[i]
        k = 0
        rg, ro = [], []
        for r in recs[i][1:]:
            orc.run(p, k, r["step"] - k, F)
            k = r["step"]
            o = orc.measure(p, k, F)
            rg.append([r["xi_w"] / r["tau"], r["v2_omega"], r["v2_phi"]])
            ro.append([o["xi_w"] / o["tau"], o["v2_omega"], o["v2_phi"]])
        gpu.append(rg)
        ref.append(ro)
    g, o = np.mean(gpu, axis=0), np.mean(ref, axis=0)
    for j, k in enumerate(keys):
        assert np.allclose(g[:, j], o[:, j], rtol=0.01), (k, g[:, j], o[:, j])


def test_batch_measure_equals_single_lattice_measure(pkg):
    """ahs_batch_measure: a member measured at its current time (mid-run, and after
    it stopped) gives the record ahs_measure gives for the same state and launch
    shape, and leaves the batch unchanged."""
    from paper_2005_14454_gb300._abi import AHS_OPT_TILE_Y, AHS_OPT_ZCHUNK, ahs_batch_member_zchunk
    members = [(24, 1, 31, 9), (20, 2, 32, 14)]
    N, era, seed, end = zip(*members)
    with pkg.Batch(N, era, seed, list(end), measure_every=5, **PARAMS) as b:
        b.init()
        b.run(6)
        got = [b.measure(i) for i in range(2)]
        before = [b.state(i) for i in range(2)]
        again = [b.measure(i) for i in range(2)]
        assert got == again and all(np.array_equal(b.state(i), before[i]) for i in range(2))
        b.run()
        final = b.measure(0)
        for i, (n, e, sd, ne) in enumerate(members):
            with pkg.Lattice(n, era=e, measure_every=0, **PARAMS) as lat:
                lat.set_option(AHS_OPT_TILE_Y, 8)
                lat.set_option(AHS_OPT_ZCHUNK, ahs_batch_member_zchunk(b.b, i))
                lat.init(sd)
                lat.step(6)
                assert lat.measure() == got[i], i
                if i == 0:
                    lat.step(ne - 6)
                    assert lat.measure() == final
    assert got[0]["step"] == 6 and final["step"] == 9
