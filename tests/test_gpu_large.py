"""Parity at the large sizes: the generic shared-memory FFT at P = 512 ... 4096,
the 2048 x 2048, n = 10000, R = 256 workload in all three precision forms on
sampled realizations and nodes, and nearest-neighbour Kriging on the 512 x 512
grid.  Tolerances as in test_gpu_parity.py: 1e-5 for the FP32 form also on the
ill-conditioned 2048 x 2048 workload, whose correction sum cancels by about a
thousand (the compensated solve keeps B within a few roundings)."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32, TOL_F16, TOL_BF16 = 1e-5, 1e-4, 1e-3
TOL = {"fp32": TOL32, "f16x3": TOL_F16, "tf32x3": TOL_F16, "bf16x3": TOL_BF16}


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


def _dev(x, dtype=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("m,nu,rng_,R,r_offset", [
    (200, 0.5, 0.1, 4, 2),      # P = 512
    (700, 0.5, 0.05, 2, 0),     # P = 2048 (grid side not a power of two)
    (1024, 1.5, 0.12, 2, 62),   # P = 2048, the differentiation grid
    (2048, 0.5, 0.08, 2, 254),  # P = 4096, the precision grid
    (1500, 1.5, 0.1, 3, 4),     # P = 4096 with m < 2048 and an odd R (the last imaginary part dropped)
])
def test_unconditional_generic_fft_sizes(ce, m, nu, rng_, R, r_offset):
    wl = workloads.workload("plain64").scaled(m=m, nu=nu, range=rng_)
    ctx = ce.Context.from_workload(wl)
    lam, P, _ = oracle.ce_eigenvalues(wl.m, wl.h, wl.sigma, wl.range, wl.nu)
    assert ctx.info()["P"] == P
    y = ctx.unconditional(R, seed=77, r_offset=r_offset).cpu().numpy()
    assert rel(y, oracle.ce_unconditional(lam, wl.m, 77, r_offset, R)) < TOL32


@pytest.fixture(scope="module")
def precision2048():
    wl = workloads.workload("precision2048")
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    oracle.setup_local(prob, sites, z, wl.np_)
    rng = np.random.default_rng(4)
    nodes = np.concatenate([rng.choice(wl.m * wl.m, 2000, replace=False), np.arange(wl.m - 300, wl.m)])
    reals = [0, wl.R - 1]
    ref, kappa = [], 0.0
    C = oracle.cov_matrix(prob.grid()[nodes], sites, wl.sigma, wl.range, wl.nu)
    for r in reals:
        base = r - r % 2
        y = oracle.ce_unconditional(prob.lam, wl.m, wl.sim_seed, base, 2)[r % 2:r % 2 + 1]
        B = oracle.solve_B(prob, oracle.residuals(prob, y, wl.sim_seed, r))
        ref.append(oracle.correction(prob, y, B, nodes)[0])
        kappa = max(kappa, float((np.abs(C) @ np.abs(B[:, 0])).max()))
    ref = np.stack(ref)
    # cancellation of the correction sum: the largest sum of |C B| over the largest |v|
    kappa /= float(np.abs(ref).max())
    return wl, sites, z, nodes, reals, ref, kappa


@pytest.mark.parametrize("prec", ["fp32", "f16x3", "bf16x3", "tf32x3"])
def test_condsim_precision2048_sampled(ce, precision2048, prec):
    """2048 x 2048 grid (P = 4096), 10000 sites (3 dense clusters), R = 256, in the
    launch configuration of a full call; sampled against the oracle."""
    wl, sites, z, nodes, reals, ref, kappa = precision2048
    assert 500 < kappa < 3000   # the dense clusters make this the ill-conditioned case
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_, prec=prec)
    out = torch.empty((wl.R, wl.m, wl.m), dtype=torch.float32, device="cuda")
    ctx.condsim(_dev(z), wl.R, wl.sim_seed, out=out)
    ctx.sync()
    flat = out.view(wl.R, -1)
    got = flat[torch.tensor(reals, device="cuda")][:, torch.tensor(nodes, device="cuda")].cpu().numpy()
    tol = TOL[prec]
    err = rel(got, ref)
    print(f"precision2048 {prec}: max rel error {err:.3e}, cancellation {kappa:.0f}, tolerance {tol:.2e}")
    assert err < tol
    assert bool(torch.isfinite(flat).all())
    ctx.close()
    del out


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_condsim_nn_shakemap512_grid(ce, prec):
    """Nearest-neighbour Kriging (k = 8) on the 512 x 512 Matern-3/2 grid with 300
    clustered sites, R = 100, sampled against the oracle."""
    wl = workloads.workload("shakemap512").scaled(n=300)
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "nn", k=wl.k_nn, prec=prec)
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    oracle.setup_nn(prob, sites, z, wl.k_nn)
    assert np.array_equal(ctx.array("J"), prob.J.astype(np.int32))
    v = ctx.condsim(_dev(z), wl.R, wl.sim_seed).view(wl.R, -1)
    ctx.sync()
    rng = np.random.default_rng(6)
    nodes = np.concatenate([rng.choice(wl.m * wl.m, 2000, replace=False), prob.J[:200]])
    reals = [0, 1, wl.R - 1]
    ref, _ = oracle.condsim_at(prob, wl.sim_seed, 0, reals, nodes)
    got = v[torch.tensor(reals, device="cuda")][:, torch.tensor(nodes, device="cuda")].cpu().numpy()
    assert rel(got, ref) < TOL[prec]


@pytest.mark.parametrize("name,n,R", [("plain64", 50, 6), ("shakemap512", 300, 100)])
def test_condsim_nn_circulant_correction(ce, name, n, R):
    """NN Kriging with the correction formed as a circulant convolution on the
    torus (surrogate nodes lie on the grid), against the oracle's direct sum."""
    wl = workloads.workload(name).scaled(n=n)
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "nn", k=wl.k_nn).set_nn_correction("circulant")
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    oracle.setup_nn(prob, sites, z, wl.k_nn)
    v = ctx.condsim(_dev(z), R, wl.sim_seed).view(R, -1)
    ctx.sync()
    rng = np.random.default_rng(7)
    nodes = np.concatenate([rng.choice(wl.m * wl.m, min(2000, wl.m * wl.m), replace=False), prob.J[:200]])
    reals = sorted({0, 1, R - 1})
    ref, direct = [], []
    for r in reals:
        base = r - r % 2
        y = oracle.ce_unconditional(prob.lam, wl.m, wl.sim_seed, base, 2)[r % 2:r % 2 + 1]
        B = oracle.solve_B(prob, oracle.residuals(prob, y, wl.sim_seed, r))
        ref.append(oracle.correction_circulant(prob, y, B, nodes)[0])
        direct.append(oracle.correction(prob, y, B, nodes)[0])
    ref, direct = np.stack(ref), np.stack(direct)
    got = v[torch.tensor(reals, device="cuda")][:, torch.tensor(nodes, device="cuda")].cpu().numpy()
    print(f"{name} NN circulant: max rel error {rel(got, ref):.3e} against the oracle's circulant form, "
          f"{rel(got, direct):.3e} against the direct sum (the clipped part of the spectrum)")
    assert rel(got, ref) < TOL32


def test_nn_correction_setter_rejects_local_mode(ce):
    wl = workloads.workload("plain64")
    ctx = ce.Context.from_workload(wl).krige_weights(workloads.make_sites(wl, n=20), "local", np_=2)
    with pytest.raises(ce.CEError) as e:
        ctx.set_nn_correction("circulant")
    assert e.value.status == ce.CE_ERR_STATE


def test_condsim_precision2048_fp64(ce, precision2048):
    """The FP64 correction form on the same 2048 x 2048 workload, 16 realizations (FP64
    runs far below FP32 on this part), realization 0 against the oracle: the draw's
    remaining error is that of the FP32 ensemble, residuals and solve."""
    wl, sites, z, nodes, reals, ref, kappa = precision2048
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_, prec="fp64")
    out = torch.empty((16, wl.m, wl.m), dtype=torch.float32, device="cuda")
    ctx.condsim(_dev(z), 16, wl.sim_seed, out=out)
    ctx.sync()
    got = out.view(16, -1)[0][torch.tensor(nodes, device="cuda")].cpu().numpy()
    err = rel(got[None], ref[:1])
    print(f"precision2048 fp64 (realization 0): max rel error {err:.3e}, cancellation {kappa:.0f}")
    assert err < TOL32
    ctx.close()


@pytest.fixture(scope="module")
def solve4500(ce):
    wl = workloads.workload("plain64").scaled(m=160)
    sites = workloads.make_sites(wl, n=4500)
    z = workloads.make_data(wl, sites)
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    oracle.setup_local(prob, sites, z, wl.np_)
    return wl, sites, z, prob


@pytest.mark.parametrize("R", [1, 77, 130])
def test_solve_on_tensor_cores(ce, solve4500, R):
    """The solve B = A^-1 E in both forms for 4500 sites against the oracle's FP64 solve:
    the default compensated FP32 products at the FP32 bar, and the tensor-core form (f16
    hi/lo operands of A^-1 and E, K split over several work items and joined in order) at
    its stated 1e-6 level; one realization, a ragged 77, and 130 (two launches of up to
    128)."""
    wl, sites, z, prob = solve4500
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_, prec="f16x3")
    assert ctx.info()["solve_tc"] == 0      # the compensated FP32 form by default
    E = np.random.default_rng(5 + R).standard_normal((R, len(sites))).astype(np.float32)
    ref = oracle.solve_B(prob, E.astype(np.float64)).T
    B32 = ctx.solve(_dev(E)).cpu().numpy()
    ctx.sync()
    ctx.set_solve_form("tensor")
    assert ctx.info()["solve_tc"] == 1
    B = ctx.solve(_dev(E)).cpu().numpy()
    ctx.sync()
    again = ctx.solve(_dev(E)).cpu().numpy()
    ctx.sync()
    assert np.array_equal(B, again)          # the K parts are joined in a fixed order
    err, err32 = rel(B, ref), rel(B32, ref)
    print(f"solve, 4500 sites, R = {R}: tensor cores {err:.2e}, CUDA cores {err32:.2e}")
    assert err < 1e-5                       # the form's stated accuracy: about 1e-6
    assert err32 < TOL32
