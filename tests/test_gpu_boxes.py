"""Joint draws of the sites that share a grid box (the multivariate form of step
(b) of local Kriging, Section 2.1; the Cholesky blocks of Section 3.6) on the GPU
against the oracle's setup_local(joint_boxes=True)."""
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


def _problem(wl, sites, z, joint):
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    return oracle.setup_local(prob, sites, z, wl.np_, joint_boxes=joint)


@pytest.fixture(scope="module")
def dense64(ce):
    # 600 uniform sites on the 64 x 64 grid: 32 boxes hold two or three sites
    wl = workloads.workload("plain64").scaled(n=600, R=6)
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    return wl, sites, z, _problem(wl, sites, z, True)


def test_residuals_with_joint_boxes(ce, dense64):
    wl, sites, z, prob = dense64
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_)
    assert ctx.set_box_joint(True) == len(prob.boxes) == 32
    R = 6
    y = oracle.ce_unconditional(prob.lam, wl.m, 9, 4, R).astype(np.float32)
    E = ctx.residuals(_dev(y), _dev(z), R, seed=9, r_offset=4).cpu().numpy()
    ref = oracle.residuals(prob, y.astype(np.float64), 9, 4)
    ref_z32 = ref + (z.astype(np.float32).astype(np.float64) - z)[None, :]
    assert rel(E, ref_z32) < TOL32
    # the sites of shared boxes after the first really take the joint noise
    shared = np.concatenate([b[1:] for b in prob.boxes])
    ind = _problem(wl, sites, z, False)
    e_ind = oracle.residuals(ind, y.astype(np.float64), 9, 4)
    assert np.abs(e_ind[:, shared] - ref[:, shared]).max() > 100 * TOL32 * np.abs(ref).max()
    ctx.close()


def test_condsim_with_joint_boxes_plain64(ce, dense64):
    wl, sites, z, prob = dense64
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_)
    plain = ctx.condsim(_dev(z), wl.R, wl.sim_seed).cpu().numpy()
    ctx.set_box_joint(True)
    v = ctx.condsim(_dev(z), wl.R, wl.sim_seed).cpu().numpy()
    ref = oracle.condsim(prob, wl.sim_seed, 0, wl.R)
    assert rel(v, ref) < TOL32
    # switched off again: the independent draws, bit for bit
    assert ctx.set_box_joint(False) == 0
    again = ctx.condsim(_dev(z), wl.R, wl.sim_seed).cpu().numpy()
    assert np.array_equal(again, plain)
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp32", TOL32), ("f16x3", TOL_F16)])
def test_condsim_with_joint_boxes_shakemap512(ce, prec, tol):
    """512 x 512, Matern 3/2, 2000 clustered sites (34 boxes hold two or three), R = 100,
    sampled against the oracle."""
    wl = workloads.workload("shakemap512")
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    prob = _problem(wl, sites, z, True)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_, prec=prec)
    assert ctx.set_box_joint(True) == len(prob.boxes) == 34
    v = ctx.condsim(_dev(z), wl.R, wl.sim_seed).view(wl.R, -1)
    ctx.sync()
    # nodes near the shared boxes, where the joint draw matters, and random ones
    rng = np.random.default_rng(8)
    near = np.unique(prob.idx[np.concatenate(prob.boxes)].reshape(-1))
    nodes = np.concatenate([rng.choice(wl.m * wl.m, 1500, replace=False), near[:500]])
    reals = [0, 1, wl.R - 1]
    ref, _ = oracle.condsim_at(prob, wl.sim_seed, 0, reals, nodes)
    got = v[torch.tensor(reals, device="cuda")][:, torch.tensor(nodes, device="cuda")].cpu().numpy()
    assert rel(got, ref) < tol
    ctx.close()


def test_box_joint_errors(ce):
    wl = workloads.workload("plain64")
    h = wl.h
    # nine sites in box (10, 20): more than can be drawn jointly
    crowd = np.array([[(20 + 0.1 + 0.1 * a) * h, (10 + 0.05 + 0.1 * a) * h] for a in range(9)])
    sites = np.concatenate([workloads.make_sites(wl, n=30), crowd])
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=2)
    with pytest.raises(ce.CEError) as e:
        ctx.set_box_joint(True)
    assert e.value.status == ce.CE_ERR_ARG
    # eight are accepted
    ctx = ce.Context.from_workload(wl).krige_weights(sites[:-1], "local", np_=2)
    assert ctx.set_box_joint(True) >= 1
    # the gradient does not cover the joint draw
    with pytest.raises(ce.CEError) as e:
        ctx.condsim_grad(_dev(workloads.make_data(wl, sites[:-1])), 2, 1, (0, 8, 0, 8))
    assert e.value.status == ce.CE_ERR_STATE
    # NN mode has no grid boxes of sites
    nn = ce.Context.from_workload(wl).krige_weights(sites[:30], "nn", k=4)
    with pytest.raises(ce.CEError) as e:
        nn.set_box_joint(True)
    assert e.value.status == ce.CE_ERR_STATE
    # a new set-up resets the choice
    ctx.krige_weights(sites[:30], "local", np_=2)
    z = workloads.make_data(wl, sites[:30])
    a = ctx.condsim(_dev(z), 2, 5).cpu().numpy()
    b = ce.Context.from_workload(wl).krige_weights(sites[:30], "local", np_=2).condsim(_dev(z), 2, 5).cpu().numpy()
    assert np.array_equal(a, b)
