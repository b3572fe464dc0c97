"""Pathwise gradient of the window loss plus the log-likelihood (ce_condsim_grad)
against FP64 central finite differences of the oracle's loss at fixed noise."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ce():
    from paper_2109_11044_gb300.build import build
    build()
    import paper_2109_11044_gb300 as mod
    mod.load_library()
    return mod


CASES = [
    dict(m=48, nu=0.5, sigma=0.8, range=0.15, tau2=0.06, n=40, R=6, window=(10, 30, 12, 36), seed=31),
    dict(m=40, nu=1.5, sigma=1.1, range=0.12, tau2=0.08, n=30, R=5, window=(5, 25, 8, 30), seed=47),
]


@pytest.mark.parametrize("case", CASES)
def test_gradient_matches_oracle_finite_differences(ce, case):
    wl = workloads.workload("plain64").scaled(m=case["m"], nu=case["nu"], sigma=case["sigma"], range=case["range"],
                                              tau2=case["tau2"], n=case["n"], R=case["R"], site_seed=9)
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    np_, R, win, seed = 2, case["R"], case["window"], case["seed"]
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=np_)
    zd = torch.tensor(z, dtype=torch.float32, device="cuda")
    v, gt, gz, L = ctx.condsim_grad(zd, R, seed, win)
    gz = gz.cpu().numpy().astype(np.float64)
    z32 = z.astype(np.float32).astype(np.float64)

    def loss(sigma=wl.sigma, theta=wl.range, tau2=wl.tau2, zz=z32):
        return oracle.diff_loss(wl.m, wl.x0, wl.y0, wl.h, sigma, theta, wl.nu, tau2, sites, zz, np_, seed, 0, R, win)

    L0 = loss()
    assert abs(L - L0) <= 1e-5 * max(1.0, abs(L0))
    fd = []
    for name, val in (("sigma", wl.sigma), ("theta", wl.range), ("tau2", wl.tau2)):
        hstep = 1e-4 * val
        up = loss(**{name: val + hstep})
        dn = loss(**{name: val - hstep})
        fd.append((up - dn) / (2 * hstep))
    fd = np.array(fd)
    assert np.allclose(gt, fd, rtol=2e-3, atol=2e-4 * np.abs(fd).max()), (gt, fd)
    fdz = np.empty_like(z32)
    for i in range(z32.size):
        e = np.zeros_like(z32)
        e[i] = 1e-4
        fdz[i] = (loss(zz=z32 + e) - loss(zz=z32 - e)) / 2e-4
    assert np.abs(gz - fdz).max() <= 2e-3 * np.abs(fdz).max()


def test_gradient_rejects_nn_mode_and_bad_window(ce):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl, n=20)
    zd = torch.tensor(workloads.make_data(wl, sites), dtype=torch.float32, device="cuda")
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=2)
    with pytest.raises(ce.CEError) as e:
        ctx.condsim_grad(zd, 4, 1, (10, 5, 0, 8))
    assert e.value.status == ce.CE_ERR_ARG
    nn = ce.Context.from_workload(wl).krige_weights(sites, "nn", k=4)
    with pytest.raises(ce.CEError) as e:
        nn.condsim_grad(zd, 4, 1, (0, 8, 0, 8))
    assert e.value.status == ce.CE_ERR_STATE


def test_autograd_function_returns_the_adjoint_gradients(ce):
    wl = workloads.workload("plain64").scaled(m=40, nu=1.5, sigma=0.9, range=0.14, tau2=0.07, n=25, site_seed=5)
    sites = workloads.make_sites(wl)
    z = torch.tensor(workloads.make_data(wl, sites), dtype=torch.float32, device="cuda")
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=2)
    win = (4, 30, 6, 33)
    _, gt, gz, L = ctx.condsim_grad(z, 4, 19, win)
    theta = torch.tensor([wl.sigma, wl.range, wl.tau2], dtype=torch.float64, requires_grad=True)
    zz = z.clone().requires_grad_(True)
    loss = ce.condsim_loss(ctx, theta, zz, 4, 19, win)
    # the adjoint sums with atomics, so two calls agree to rounding, not bit for bit
    assert loss.item() == pytest.approx(L, rel=1e-6)
    (2.0 * loss).backward()
    assert torch.allclose(theta.grad, 2.0 * torch.tensor(gt, dtype=torch.float64), rtol=1e-4, atol=0)
    assert torch.allclose(zz.grad, 2.0 * gz, rtol=1e-4, atol=1e-5 * float(gz.abs().max()))
    # at another theta the set-up is redone there: the same loss and gradients as a context built at it
    th2 = [0.8 * wl.sigma, 1.3 * wl.range, 1.5 * wl.tau2]
    theta2 = torch.tensor(th2, dtype=torch.float64, requires_grad=True)
    z2 = z.clone().requires_grad_(True)
    loss2 = ce.condsim_loss(ctx, theta2, z2, 4, 19, win)
    loss2.backward()
    ref = ce.Context(wl.m, wl.x0, wl.y0, wl.h, th2[0], th2[1], wl.nu, th2[2]).krige_weights(sites, "local", np_=2)
    _, gt2, gz2, L2 = ref.condsim_grad(z, 4, 19, win)
    assert loss2.item() == pytest.approx(L2, rel=1e-6) and abs(L2 - L) > 1e-3 * abs(L)
    assert torch.allclose(theta2.grad, torch.tensor(gt2, dtype=torch.float64), rtol=1e-4, atol=0)
    assert torch.allclose(z2.grad, gz2, rtol=1e-4, atol=1e-5 * float(gz2.abs().max()))


@pytest.mark.parametrize("name,n", [("plain64", 200), ("diff1024", 3000)])
def test_loglik_matches_oracle(ce, name, n):
    """ce_loglik against the oracle's Gaussian log-likelihood (Eq. (condmvn)'s model) on the same
    float32 data, at the differentiation workload's full size (1024^2 grid, 3000 clustered sites)."""
    wl = workloads.workload(name)
    sites = workloads.make_sites(wl, n=n)
    z32 = workloads.make_data(wl, sites).astype(np.float32)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_)
    got = ctx.loglik(torch.tensor(z32, device="cuda"))
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    prob.sites = sites
    prob.zeff = z32.astype(np.float64)
    prob.L = oracle.cholesky(prob.cov(sites, sites) + wl.tau2 * np.eye(n))
    ref = oracle.log_likelihood(prob)
    assert got == pytest.approx(ref, rel=1e-9, abs=1e-9 * n)
    nn = ce.Context.from_workload(wl).krige_weights(sites[:50], "nn", k=4)
    with pytest.raises(ce.CEError) as e:
        nn.loglik(torch.tensor(z32[:50], device="cuda"))
    assert e.value.status == ce.CE_ERR_STATE
