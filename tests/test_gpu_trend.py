"""The linear mean model (GLS coefficients, universal Kriging predictor in the
conditional draw) on the GPU against the oracle's condsim_trend."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32, TOL_F16 = 1e-5, 1e-4


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def ce():
    from paper_2109_11044_gb300.build import build
    build()
    import paper_2109_11044_gb300 as mod
    mod.load_library()
    return mod


def _dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float32, device="cuda")


def _data_with_trend(wl, sites):
    # data with a clear mean: a plane in the coordinates plus the field and nugget
    return workloads.make_data(wl, sites) + 2.0 + 1.5 * sites[:, 0] - 0.8 * sites[:, 1]


@pytest.mark.parametrize("degree", [0, 1])
def test_trend_plain64(ce, degree):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl)
    z = _data_with_trend(wl, sites)
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    oracle.setup_local(prob, sites, z, wl.np_)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_).set_trend(degree)
    v = ctx.condsim(_dev(z), wl.R, wl.sim_seed).cpu().numpy()
    ref = oracle.condsim_trend(prob, degree, wl.sim_seed, 0, wl.R)
    assert rel(v, ref) < TOL32
    # the model changes the draws, and switching it off restores the zero-mean ones
    plain = oracle.condsim(prob, wl.sim_seed, 0, wl.R)
    assert rel(ref, plain) > 1e-3
    ctx.set_trend(-1)
    assert rel(ctx.condsim(_dev(z), wl.R, wl.sim_seed).cpu().numpy(), plain) < TOL32


@pytest.mark.parametrize("prec,tol", [("fp32", TOL32), ("f16x3", TOL_F16)])
def test_trend_shakemap512_sampled(ce, prec, tol):
    wl = workloads.workload("shakemap512")
    sites = workloads.make_sites(wl)
    z = _data_with_trend(wl, sites)
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    oracle.setup_local(prob, sites, z, wl.np_)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_, prec=prec).set_trend(1)
    v = ctx.condsim(_dev(z), wl.R, wl.sim_seed).view(wl.R, -1)
    ctx.sync()
    rng = np.random.default_rng(9)
    nodes = rng.choice(wl.m * wl.m, 2000, replace=False)
    reals = [0, 1, wl.R - 1]
    ref = np.concatenate([oracle.condsim_trend(prob, 1, wl.sim_seed, r - r % 2, 2, nodes=nodes)[r % 2:r % 2 + 1]
                          for r in reals])
    got = v[torch.tensor(reals, device="cuda")][:, torch.tensor(nodes, device="cuda")].cpu().numpy()
    assert rel(got, ref) < tol


def test_trend_reset_by_new_sites_and_rejected_by_gradient(ce):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl, n=60)
    z = _data_with_trend(wl, sites)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=2).set_trend(1)
    with pytest.raises(ce.CEError) as e:
        ctx.condsim_grad(_dev(z), 4, 3, (10, 30, 10, 30))
    assert e.value.status == ce.CE_ERR_STATE
    ctx.krige_weights(sites, "local", np_=2)   # new sites: the model is reset
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    oracle.setup_local(prob, sites, z, 2)
    assert rel(ctx.condsim(_dev(z), 4, 3).cpu().numpy(), oracle.condsim(prob, 3, 0, 4)) < TOL32
    ctx_nn = ce.Context.from_workload(wl).krige_weights(sites, "nn", k=4)
    with pytest.raises(ce.CEError) as e:
        ctx_nn.set_trend(0)
    assert e.value.status == ce.CE_ERR_STATE
