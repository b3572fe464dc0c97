"""Edge cases of the whole draw against the oracle: a single site, sites exactly
on grid nodes and on the far boundary of the grid (the window shifted inward),
and the largest R one call accepts."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


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


def _run(ce, wl, sites, z, mode, R, seed, **kw):
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    if mode == "local":
        oracle.setup_local(prob, sites, z, kw["np_"])
        ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=kw["np_"])
    else:
        oracle.setup_nn(prob, sites, z, kw["k"])
        ctx = ce.Context.from_workload(wl).krige_weights(sites, "nn", k=kw["k"])
    v = ctx.condsim(_dev(z), R, seed).cpu().numpy()
    ctx.close()
    return v, oracle.condsim(prob, seed, 0, R)


@pytest.mark.parametrize("mode", ["local", "nn"])
def test_single_site(ce, mode):
    wl = workloads.workload("plain64")
    sites = np.array([[0.37, 0.61]])
    v, ref = _run(ce, wl, sites, np.array([0.8]), mode, 3, 5, np_=2, k=4)
    assert rel(v, ref) < TOL32


@pytest.mark.parametrize("mode", ["local", "nn"])
def test_sites_on_nodes_and_on_the_far_boundary(ce, mode):
    wl = workloads.workload("plain64")
    h = wl.h
    sites = np.array([[0.0, 0.0], [1.0, 1.0], [0.5, 1.0], [1.0, 0.25], [3 * h, 5 * h], [0.2, 0.7]])
    z = np.array([0.4, -0.3, 1.1, 0.2, -0.7, 0.05])
    v, ref = _run(ce, wl, sites, z, mode, 4, 9, np_=2, k=4)
    assert rel(v, ref) < TOL32


def test_largest_R(ce):
    # R = 4096, the most one call takes, on a small grid: every realization against the oracle
    wl = workloads.workload("plain64").scaled(m=12)
    sites = workloads.make_sites(wl, n=5)
    z = workloads.make_data(wl, sites)
    v, ref = _run(ce, wl, sites, z, "local", 4096, 13, np_=2)
    assert v.shape == (4096, 12, 12)
    assert rel(v, ref) < TOL32
