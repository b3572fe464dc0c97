"""Geometric anisotropy (ce_set_anisotropy) on the GPU against the oracle run
with the same map: the embedding, the unconditional fields, local and NN
conditional draws (direct and circulant corrections, FP32 and f16x3), the
closed-form standard errors, and the return to the isotropic model."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32, TOL_F16 = 1e-5, 1e-4
AN = (0.45, 0.7)   # range * 0.45 across the direction 0.7 rad from the x axis


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


def _prob(wl, an=AN):
    return oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2, aniso=an)


def test_embedding_and_unconditional(ce):
    wl = workloads.workload("plain64")
    prob = _prob(wl)
    ctx = ce.Context.from_workload(wl).set_anisotropy(*AN)
    assert ctx.info()["P"] == prob.P
    sq = ctx.array("sqrt_lambda")
    assert rel(sq, np.sqrt(prob.lam / prob.P ** 2)) < TOL32
    y = ctx.unconditional(6, seed=21, r_offset=2).cpu().numpy()
    assert rel(y, oracle.ce_unconditional(prob.lam, wl.m, 21, 2, 6)) < TOL32


@pytest.mark.parametrize("prec,tol", [("fp32", TOL32), ("f16x3", TOL_F16), ("bf16x3", 1e-3), ("fp64", TOL32)])
def test_condsim_local_plain64(ce, prec, tol):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    prob = _prob(wl)
    oracle.setup_local(prob, sites, z, wl.np_)
    ctx = ce.Context.from_workload(wl).set_anisotropy(*AN).krige_weights(sites, "local", np_=wl.np_, prec=prec)
    v = ctx.condsim(_dev(z), wl.R, wl.sim_seed).cpu().numpy()
    ref = oracle.condsim(prob, wl.sim_seed, 0, wl.R)
    err = rel(v, ref)
    print(f"anisotropic plain64 {prec}: {err:.2e}")
    assert err < tol
    # and it is not the isotropic answer
    iso = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    oracle.setup_local(iso, sites, z, wl.np_)
    assert rel(v, oracle.condsim(iso, wl.sim_seed, 0, wl.R)) > 100 * tol


@pytest.mark.parametrize("prec,tol", [("fp32", TOL32), ("f16x3", TOL_F16)])
def test_condsim_local_shakemap512_sampled(ce, prec, tol):
    wl = workloads.workload("shakemap512")
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    an = (0.5, 0.6)
    prob = _prob(wl, an)
    oracle.setup_local(prob, sites, z, wl.np_)
    ctx = ce.Context.from_workload(wl).set_anisotropy(*an).krige_weights(sites, "local", np_=wl.np_, prec=prec)
    assert ctx.info()["P"] == prob.P
    v = ctx.condsim(_dev(z), wl.R, wl.sim_seed).view(wl.R, -1)
    ctx.sync()
    rng = np.random.default_rng(12)
    nodes = np.concatenate([rng.choice(wl.m * wl.m, 1500, replace=False), prob.idx[:40].reshape(-1)])
    reals = [0, wl.R - 1]
    ref, _ = oracle.condsim_at(prob, wl.sim_seed, 0, reals, nodes)
    got = v[torch.tensor(reals, device="cuda")][:, torch.tensor(nodes, device="cuda")].cpu().numpy()
    err = rel(got, ref)
    print(f"anisotropic shakemap512 {prec}: {err:.2e}")
    assert err < tol


@pytest.mark.parametrize("method", ["direct", "circulant"])
def test_condsim_nn_plain64(ce, method):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl, n=50)
    z = workloads.make_data(wl, sites)
    prob = _prob(wl)
    oracle.setup_nn(prob, sites, z, wl.k_nn)
    ctx = ce.Context.from_workload(wl).set_anisotropy(*AN).krige_weights(sites, "nn", k=wl.k_nn)
    assert np.array_equal(ctx.array("J"), prob.J.astype(np.int32))
    ctx.set_nn_correction(method)
    R = 6
    v = ctx.condsim(_dev(z), R, wl.sim_seed).cpu().numpy().reshape(R, -1)
    if method == "direct":
        ref = oracle.condsim(prob, wl.sim_seed, 0, R).reshape(R, -1)
    else:
        y = oracle.ce_unconditional(prob.lam, wl.m, wl.sim_seed, 0, R)
        B = oracle.solve_B(prob, oracle.residuals(prob, y, wl.sim_seed, 0))
        ref = oracle.correction_circulant(prob, y, B)
    assert rel(v, ref) < TOL32


def test_se_map(ce):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl, n=120)
    prob = _prob(wl)
    oracle.setup_local(prob, sites, np.zeros(len(sites)), wl.np_)
    ctx = ce.Context.from_workload(wl).set_anisotropy(*AN).krige_weights(sites, "local", np_=wl.np_)
    se_e, se_l = ctx.se_map()
    e = se_e.cpu().numpy().reshape(-1).astype(np.float64)
    a = se_l.cpu().numpy().reshape(-1).astype(np.float64)
    assert np.abs(e * e - oracle.se_exact(prob, sites) ** 2).max() < 1e-5
    assert np.abs(a * a - oracle.se_approx(prob) ** 2).max() < 1e-5


def test_back_to_isotropic_and_errors(ce):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl, n=40)
    z = _dev(workloads.make_data(wl, sites))
    ctx = ce.Context.from_workload(wl).set_anisotropy(*AN)
    # the off-grid set-up is discarded by the change
    ctx.krige_weights(sites, "local", np_=2)
    ctx.set_anisotropy(1.0, 0.0)
    with pytest.raises(ce.CEError) as e:
        ctx.condsim(z, 2, 1)
    assert e.value.status == ce.CE_ERR_STATE
    ctx.krige_weights(sites, "local", np_=2)
    a = ctx.condsim(z, 4, 9).cpu().numpy()
    b = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=2).condsim(z, 4, 9).cpu().numpy()
    assert np.array_equal(a, b)
    with pytest.raises(ce.CEError) as e:
        ctx.set_anisotropy(0.0, 0.3)
    assert e.value.status == ce.CE_ERR_ARG
    ctx.set_anisotropy(*AN).krige_weights(sites, "local", np_=2)
    with pytest.raises(ce.CEError) as e:
        ctx.condsim_grad(z, 2, 1, (0, 8, 0, 8))
    assert e.value.status == ce.CE_ERR_STATE


def test_failed_anisotropy_keeps_the_previous_covariance(ce):
    # Matern 3/2 with range 0.6 on the unit square: three times that across the major direction
    # leaves the embedding indefinite after growth (the oracle's embedding fails too)
    wl = workloads.workload("plain64").scaled(range=0.6, nu=1.5)
    sites = workloads.make_sites(wl, n=30)
    z = _dev(workloads.make_data(wl, sites))
    with pytest.raises(RuntimeError):
        oracle.ce_eigenvalues(wl.m, wl.h, wl.sigma, wl.range, wl.nu, max_growth=3, aniso=(3.0, 0.3))
    ctx = ce.Context.from_workload(wl).set_anisotropy(0.5, 0.3)
    P = ctx.info()["P"]
    with pytest.raises(ce.CEError) as e:
        ctx.set_anisotropy(3.0, 0.3)
    assert e.value.status == ce.CE_ERR_EMBED
    assert ctx.info()["P"] == P
    ctx.krige_weights(sites, "local", np_=2)
    a = ctx.condsim(z, 4, 3).cpu().numpy()
    b = ce.Context.from_workload(wl).set_anisotropy(0.5, 0.3).krige_weights(sites, "local", np_=2)
    assert np.array_equal(a, b.condsim(z, 4, 3).cpu().numpy())
