"""Restart files (Lattice.save / Lattice.restore): a run continued from a file
written mid-run equals the uninterrupted run bit for bit, in every precision and
storage mode, with the options that shape the evolution carried over."""
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


@pytest.mark.parametrize("kw", [dict(), dict(precision="fp32c"), dict(precision="fp64"),
                                dict(momenta_in_place=True), dict(core_growth=(-1.0, 1.75), s=1.0)])
def test_restart_continues_bit_for_bit(pkg, tmp_path, kw):
    from paper_2005_14454_gb300 import Lattice, _abi
    kw = dict(kw)
    s = kw.pop("s", 0.0)
    N, first, second = 20, 7, 9
    with Lattice(N, era=2, s=s, measure_every=4, **PARAMS, **kw) as a:
        a.set_option(_abi.AHS_OPT_ALPHA, 1.5)
        a.init(12)
        a.step(first)
        a.save(str(tmp_path / "ck.npz"))
        a.step(second)
        want, want_recs = a.state(), a.records()
    with Lattice.restore(str(tmp_path / "ck.npz")) as b:
        assert b.n == first and _abi.ahs_get_option(b.h, _abi.AHS_OPT_ALPHA) == 1.5
        b.step(second)
        got, got_recs = b.state(), b.records()
    assert np.array_equal(got, want)
    assert got_recs == [r for r in want_recs if r["step"] >= first]
