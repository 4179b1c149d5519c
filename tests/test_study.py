"""The scaling study of Sec. 4 (Table 1): the rate fit and the aggregation on the
host, and one small realisation on the GPU."""
import math

import numpy as np
import pytest


def test_fit_rate_recovers_a_line_and_ignores_points_outside_the_range():
    from paper_2005_14454_gb300.study import fit_rate
    tau = np.arange(1.0, 256.1, 0.5)
    xi = 0.27 * tau + 4.0
    xi[tau < 100] = 1e3                    # outside the fit range: must not matter
    xi[5] = np.nan
    assert fit_rate(tau, xi, 100.5, 255.5) == pytest.approx(0.27, rel=1e-12)
    assert math.isnan(fit_rate(tau, xi, 300.0, 400.0))


def test_fit_range_is_table1s_at_1024_and_scales_with_the_box():
    from paper_2005_14454_gb300.study import fit_range
    assert fit_range(1024) == pytest.approx((100.5, 255.5))
    lo, hi = fit_range(512)
    assert (lo, hi) == pytest.approx((100.5 / 2, 255.5 / 2))


def test_summary_mean_and_sample_std_per_era():
    from paper_2005_14454_gb300.study import table1_summary
    runs = [{"N": 64, "era": e, "seed": s, "xi_dot_L": v, "xi_dot_W": v, "v2_omega": 0.3, "v2_phi": 0.2}
            for e, vals in ((1, (0.2, 0.3, 0.4)), (2, (0.5,))) for s, v in enumerate(vals)]
    out = {d["era"]: d for d in table1_summary(runs)}
    assert out[1]["runs"] == 3 and out[1]["xi_dot_L"] == pytest.approx([0.3, 0.1])
    assert out[2]["runs"] == 1 and math.isnan(out[2]["xi_dot_W"][1])


@pytest.mark.gpu
def test_small_realisation_gives_growing_string_separation():
    from paper_2005_14454_gb300.study import fit_range, table1_run
    N = 64
    lo, hi = fit_range(N)
    r, ser = table1_run(N, 1, 5, 5, lo, hi)
    assert r["steps"] == 150 and ser["tau"][0] == pytest.approx(1.0) and ser["tau"][-1] == pytest.approx(16.0)
    assert r["points"] >= 15
    # the network coarsens: both length scales grow over the fit range (the
    # velocity estimators are not yet in their scaling range on so small a box:
    # R = sum KL / sum GL can be negative there)
    assert r["xi_dot_W"] > 0 and r["xi_dot_L"] > 0
    assert np.isfinite(r["v2_phi"]) and np.isfinite(r["v2_omega"])
