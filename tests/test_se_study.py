"""The standard-error study driver (Sections 3.3-3.4): the range of the design on
the CPU, and a short run of the study through ce_se_map against the oracle."""
import math

import numpy as np
import pytest

import oracle
import workloads
from paper_2109_11044_gb300 import se_study


@pytest.mark.parametrize("nu", [0.5, 1.5])
@pytest.mark.parametrize("dist", [20.0, 45.0, 70.0])
def test_range_gives_five_percent_correlation(nu, dist):
    theta = se_study.range_for_5pct(dist, nu)
    assert oracle.matern(dist, 1.0, theta, nu) == pytest.approx(0.05, rel=1e-10)
    if nu == 0.5:   # the values Table 1 prints
        assert round(theta, 2) == {20.0: 6.68, 45.0: 15.02, 70.0: 23.37}[dist]


@pytest.mark.gpu
def test_study_on_the_gpu_matches_the_oracle():
    rows = se_study.run(configs=2, nu=0.5, orders=(1, 2))
    assert len(rows) == 9
    for r in rows:
        fr = {1: [], 2: []}
        for c in range(2):
            sites = workloads.se_study_sites(c)
            prob = oracle.Problem(61, 0.0, 0.0, 1.0, 1.0, r["theta"], 0.5, r["tau"] ** 2)
            se_e = oracle.se_exact(prob, sites)
            for p in (1, 2):
                oracle.setup_local(prob, sites, np.zeros(len(sites)), p)
                fr[p].append(oracle.sig_fig_fraction(oracle.se_approx(prob), se_e))
        for p in (1, 2):
            assert abs(r[f"np{p}"]["sig3_mean"] - float(np.mean(fr[p]))) < 0.01
            assert 0.0 <= r[f"np{p}"]["p95_abs_pct_error"] < 5.0
        assert math.isfinite(r["np2"]["sig3_sd"])
