"""Closed-form standard errors (ce_se_map) against the oracle's se_exact and
se_approx: the paper's numerical design (Section 3.3), the 512 x 512 grid with
local Kriging (independent and joint grid-box draws), and NN Kriging.

Bar: the variances agree within 1e-5 sigma^2 at every node compared (the
products with the stored inverse are FP32 with compensated sums; the score of
Section 3.4 needs three significant figures of the standard error)."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VAR_TOL = 1e-5


@pytest.fixture(scope="module")
def ce():
    from paper_2109_11044_gb300.build import build
    build()
    import paper_2109_11044_gb300 as mod
    mod.load_library()
    return mod


def _var_err(se, ref, sigma2):
    se = np.asarray(se, dtype=np.float64)
    return float(np.abs(se * se - ref * ref).max() / sigma2)


@pytest.mark.parametrize("theta,tau", [(6.68, 0.1), (23.37, 0.3)])
def test_se_map_on_the_papers_design(ce, theta, tau):
    """61 x 61 grid on [0,60]^2, 35 uniform sites, exponential covariance, n_p = 1..4."""
    for config in (0, 1):
        sites = workloads.se_study_sites(config)
        prob = oracle.Problem(61, 0.0, 0.0, 1.0, 1.0, theta, 0.5, tau * tau)
        ref_e = oracle.se_exact(prob, sites)
        for np_ in (1, 2, 3, 4):
            ctx = ce.Context(61, 0.0, 0.0, 1.0, 1.0, theta, 0.5, tau * tau).krige_weights(sites, "local", np_=np_)
            se_e, se_l = ctx.se_map()
            se_e, se_l = se_e.cpu().numpy().reshape(-1), se_l.cpu().numpy().reshape(-1)
            oracle.setup_local(prob, sites, np.zeros(len(sites)), np_)
            ref_l = oracle.se_approx(prob)
            assert _var_err(se_e, ref_e, 1.0) < VAR_TOL
            assert _var_err(se_l, ref_l, 1.0) < VAR_TOL
            # the study's score from the GPU's standard errors matches the oracle's
            assert abs(oracle.sig_fig_fraction(se_l, se_e) - oracle.sig_fig_fraction(ref_l, ref_e)) < 0.01
            ctx.close()


@pytest.mark.parametrize("name,n,joint", [("shakemap512", 300, False), ("plain64", 600, True)])
def test_se_map_local(ce, name, n, joint):
    """512 x 512 grid, Matern 3/2, 300 clustered sites (6 x 6 windows); 64 x 64 grid with 600
    uniform sites drawn jointly in their 32 shared grid boxes.  Every node on the GPU; 2000
    sampled nodes (all of them at 64^2) plus the windows of the first sites against the oracle."""
    wl = workloads.workload(name).scaled(n=n)
    sites = workloads.make_sites(wl)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_)
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    oracle.setup_local(prob, sites, np.zeros(len(sites)), wl.np_, joint_boxes=joint)
    if joint:
        assert ctx.set_box_joint(True) == len(prob.boxes) == 32
    se_e, se_l = ctx.se_map()
    rng = np.random.default_rng(9)
    M = wl.m * wl.m
    nodes = np.arange(M) if M <= 4096 else np.concatenate([rng.choice(M, 2000, replace=False),
                                                            np.unique(prob.idx[:20].reshape(-1))])
    ge = se_e.view(-1)[torch.tensor(nodes, device="cuda")].cpu().numpy()
    gl = se_l.view(-1)[torch.tensor(nodes, device="cuda")].cpu().numpy()
    s2 = wl.sigma ** 2
    err_e = _var_err(ge, oracle.se_exact(prob, sites, nodes), s2)
    err_l = _var_err(gl, oracle.se_approx(prob, nodes), s2)
    print(f"se_map {name} n={n} joint={joint}: variance errors {err_e:.2e} (exact), {err_l:.2e} (approximate)")
    assert err_e < VAR_TOL and err_l < VAR_TOL
    assert bool(torch.isfinite(se_e).all()) and bool(torch.isfinite(se_l).all())
    ctx.close()


def test_se_map_nn_and_errors(ce):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl, n=50)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "nn", k=wl.k_nn)
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    oracle.setup_nn(prob, sites, np.zeros(len(sites)), wl.k_nn)
    _, se_n = ctx.se_map(exact=False)
    assert _var_err(se_n.cpu().numpy().reshape(-1), oracle.se_approx(prob), wl.sigma ** 2) < VAR_TOL
    with pytest.raises(ce.CEError) as e:
        ctx.se_map(exact=True, approx=False)
    assert e.value.status == ce.CE_ERR_STATE
    loc = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=2).set_trend(0)
    with pytest.raises(ce.CEError) as e:
        loc.se_map()
    assert e.value.status == ce.CE_ERR_STATE
    # the approximate standard errors describe the draws: a Monte Carlo check on the same context
    loc.set_trend(-1)
    _, se_l = loc.se_map(exact=False)
    z = torch.zeros(len(sites), dtype=torch.float32, device="cuda")
    v = loc.condsim(z, 4000, 3)
    sd = v.std(dim=0, unbiased=True).cpu().numpy()
    ratio = sd / se_l.cpu().numpy()
    assert abs(float(np.median(ratio)) - 1.0) < 0.01 and float(np.abs(ratio - 1).max()) < 0.08
