"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: integer work (Philox words, window indices, surrogate nodes) is
bit-exact.  Floating-point stages are compared as max |gpu - oracle| divided by
max |oracle| of the same tensor, against 1e-5 for the FP32 path.  Stages are
fed the oracle's own inputs rounded to FP32, so each stage is checked alone;
the whole path is checked end to end as well.
"""
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


def _oracle_problem(wl, sites, z, mode="local", np_=None, k=None):
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    if mode == "local":
        oracle.setup_local(prob, sites, z, wl.np_ if np_ is None else np_)
    else:
        oracle.setup_nn(prob, sites, z, wl.k_nn if k is None else k)
    return prob


def _dev(x, dtype=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


# ----------------------------------------------------------------------------- noise
def test_philox_words_bit_exact(ce):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4099, 4), dtype=np.uint64)
    ctr[:3] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4]]
    seed = 0x1234_5678_9ABC_DEF0
    out = ce.philox(_dev(ctr.astype(np.uint32).view(np.int32), torch.int32), seed).cpu().numpy().view(np.uint32)
    ref = oracle.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], seed & 0xFFFFFFFF, seed >> 32)
    assert np.array_equal(out, np.stack(ref, axis=1))


def test_normals_match_box_muller(ce):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(20000, 4), dtype=np.uint64)
    seed = 77
    out = ce.normals(_dev(ctr.astype(np.uint32).view(np.int32), torch.int32), seed).cpu().numpy()
    w = oracle.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], seed, 0)
    a = oracle.box_muller(w[0], w[1])
    b = oracle.box_muller(w[2], w[3])
    ref = np.stack([a[0], a[1], b[0], b[1]], axis=1)
    assert np.abs(out - ref).max() < 1e-5
    # words at the ends of the uniform range
    ext = np.array([[0, 0, 0, 0], [0xFFFFFFFF, 0, 0xFFFFFFFE, 0x80000000]], dtype=np.uint64)
    o2 = ce.normals(_dev(ext.astype(np.uint32).view(np.int32), torch.int32), seed).cpu().numpy()
    assert np.all(np.isfinite(o2))


# ----------------------------------------------------------------------------- embedding + CE
@pytest.mark.parametrize("name,m", [("plain64", 64), ("plain64", 100), ("shakemap512", 96)])
def test_spectral_weights(ce, name, m):
    wl = workloads.workload(name).scaled(m=m)
    ctx = ce.Context.from_workload(wl)
    info = ctx.info()
    lam, P, oinfo = oracle.ce_eigenvalues(wl.m, wl.h, wl.sigma, wl.range, wl.nu)
    assert info["P"] == P
    got = ctx.array("sqrt_lambda")
    ref = np.sqrt(lam / P ** 2)
    assert rel(got, ref) < 1e-6
    # eigenvalues within rounding of zero may land on either side of it
    assert abs(info["clipped"] - oinfo["clipped"]) <= max(2, oinfo["clipped"] // 50)
    assert info["lambda_max"] == pytest.approx(oinfo["lambda_max"], rel=1e-10)


@pytest.mark.parametrize("m,R,r_offset", [(64, 10, 0), (100, 7, 4), (8, 3, 0), (33, 2, 2)])
def test_unconditional_fields(ce, m, R, r_offset):
    wl = workloads.workload("plain64").scaled(m=m)
    ctx = ce.Context.from_workload(wl)
    y = ctx.unconditional(R, seed=123, r_offset=r_offset).cpu().numpy()
    lam, P, _ = oracle.ce_eigenvalues(wl.m, wl.h, wl.sigma, wl.range, wl.nu)
    ref = oracle.ce_unconditional(lam, wl.m, 123, r_offset, R)
    assert rel(y, ref) < TOL32


def test_unconditional_matern32_growth(ce):
    # smooth covariance on a small grid: the embedding must grow beyond 2m
    wl = workloads.workload("plain64").scaled(m=32, nu=1.5, range=0.3)
    ctx = ce.Context.from_workload(wl)
    lam, P, _ = oracle.ce_eigenvalues(wl.m, wl.h, wl.sigma, wl.range, wl.nu)
    assert ctx.info()["P"] == P and P > 64
    y = ctx.unconditional(6, seed=5).cpu().numpy()
    assert rel(y, oracle.ce_unconditional(lam, wl.m, 5, 0, 6)) < TOL32


# ----------------------------------------------------------------------------- off-grid set-up
def test_local_weights_and_windows(ce):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl)
    sites[:4] = [[0.0, 0.0], [1.0, 1.0], [1.0, 0.0], [wl.h * 5, wl.h * 7]]   # corners and a node
    z = workloads.make_data(wl, sites)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_)
    prob = _oracle_problem(wl, sites, z)
    assert np.array_equal(ctx.array("idx"), prob.idx.astype(np.int32))
    assert np.abs(ctx.array("W") - prob.W).max() < 1e-5 * np.abs(prob.W).max()
    assert rel(ctx.array("phi"), prob.phi) < 1e-6


def test_nn_surrogates(ce):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl, n=40)
    z = workloads.make_data(wl, sites)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "nn", k=8)
    prob = _oracle_problem(wl, sites, z, "nn", k=8)
    assert np.array_equal(ctx.array("J"), prob.J.astype(np.int32))
    assert rel(ctx.array("phi"), prob.phi) < 1e-6


# ----------------------------------------------------------------------------- stages
@pytest.fixture(scope="module")
def plain_case(ce):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    prob = _oracle_problem(wl, sites, z)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_)
    return wl, sites, z, prob, ctx


def test_residual_stage(plain_case):
    wl, sites, z, prob, ctx = plain_case
    R = 10
    y = oracle.ce_unconditional(prob.lam, wl.m, 9, 0, R).astype(np.float32)
    E = ctx.residuals(_dev(y), _dev(z), R, seed=9).cpu().numpy()
    ref = oracle.residuals(prob, y.astype(np.float64), 9, 0)
    ref_z32 = ref + (z.astype(np.float32).astype(np.float64) - z)[None, :]
    assert rel(E, ref_z32) < TOL32


def test_solve_stage(plain_case):
    wl, sites, z, prob, ctx = plain_case
    E = np.random.default_rng(3).standard_normal((13, len(sites))).astype(np.float32)
    B = ctx.solve(_dev(E)).cpu().numpy()
    ref = oracle.solve_B(prob, E.astype(np.float64)).T
    assert rel(B, ref) < TOL32


def test_correction_stage(plain_case):
    wl, sites, z, prob, ctx = plain_case
    R = 5
    rng = np.random.default_rng(4)
    y = rng.standard_normal((R, wl.m, wl.m)).astype(np.float32)
    B = rng.standard_normal((R, len(sites))).astype(np.float32)
    v = ctx.correct(_dev(B), _dev(y)).cpu().numpy()
    ref = oracle.correction(prob, y.astype(np.float64), B.T.astype(np.float64)).reshape(R, wl.m, wl.m)
    assert rel(v, ref) < TOL32


# FP64 form: products and sums in FP64, only the field's FP32 storage rounds (a few
# 1e-8 of max |v|), so its bar is far below the FP32 one
TOL64_STAGE = 2e-7


@pytest.mark.parametrize("m,n,R,mode,aniso", [(64, 200, 5, "local", False), (77, 150, 70, "local", True),
                                               (64, 50, 3, "nn", False)])
def test_correction_stage_fp64(ce, m, n, R, mode, aniso):
    """The FP64 correction on ragged tiles (m = 77, R = 70 over two realization tiles),
    anisotropic, and on NN surrogate nodes, against the oracle's FP64 correction."""
    wl = workloads.workload("plain64").scaled(m=m, nu=1.5 if m % 2 else 0.5)
    sites = workloads.make_sites(wl, n=n)
    z = workloads.make_data(wl, sites)
    an = (0.45, 0.7) if aniso else None
    ctx = ce.Context.from_workload(wl)
    if aniso:
        ctx.set_anisotropy(*an)
    ctx.krige_weights(sites, mode, np_=wl.np_, k=8, prec="fp64")
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2, aniso=an)
    if mode == "local":
        oracle.setup_local(prob, sites, z, wl.np_)
    else:
        oracle.setup_nn(prob, sites, z, 8)
    rng = np.random.default_rng(m + R)
    y = rng.standard_normal((R, wl.m, wl.m)).astype(np.float32)
    nrow = ctx.info()["n_obs"]
    B = rng.standard_normal((R, nrow)).astype(np.float32)
    v = ctx.correct(_dev(B), _dev(y)).cpu().numpy()
    ctx.sync()
    ref = oracle.correction(prob, y.astype(np.float64), B.T.astype(np.float64)).reshape(R, wl.m, wl.m)
    err = rel(v, ref)
    print(f"FP64 correction m={m} n={n} R={R} {mode}{' aniso' if aniso else ''}: {err:.2e}")
    assert err < TOL64_STAGE


def test_condsim_plain64_fp64(plain_case):
    wl, sites, z, prob, ctx = plain_case
    ctx.set_precision("fp64")
    try:
        v = ctx.condsim(_dev(z), 10, wl.sim_seed).cpu().numpy()
        ctx.sync()
    finally:
        ctx.set_precision("fp32")
    err = rel(v, oracle.condsim(prob, wl.sim_seed, 0, 10))
    print(f"plain64 fp64 draw: {err:.2e}")
    assert err < TOL32


# ----------------------------------------------------------------------------- whole path
@pytest.mark.parametrize("R,r_offset", [(10, 0), (1, 0), (5, 6)])
def test_condsim_plain64(plain_case, R, r_offset):
    wl, sites, z, prob, ctx = plain_case
    v = ctx.condsim(_dev(z), R, wl.sim_seed, r_offset).cpu().numpy()
    ref = oracle.condsim(prob, wl.sim_seed, r_offset, R)
    assert rel(v, ref) < TOL32


def test_condsim_pieces_concatenate_exactly(plain_case):
    wl, sites, z, prob, ctx = plain_case
    zd = _dev(z)
    full = ctx.condsim(zd, 8, 5, 0).cpu().numpy()
    tail = ctx.condsim(zd, 4, 5, 4).cpu().numpy()
    assert np.array_equal(full[4:], tail)


def test_condsim_ragged_grid_and_np1(ce):
    wl = workloads.workload("plain64").scaled(m=77, nu=1.5, range=0.2)
    sites = workloads.make_sites(wl, n=150)
    z = workloads.make_data(wl, sites)
    for np_ in (1, 4):
        ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=np_)
        prob = _oracle_problem(wl, sites, z, np_=np_)
        v = ctx.condsim(_dev(z), 3, 11).cpu().numpy()
        assert rel(v, oracle.condsim(prob, 11, 0, 3)) < TOL32


def test_condsim_nn_mode(ce):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl, n=50)
    z = workloads.make_data(wl, sites)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "nn", k=8)
    prob = _oracle_problem(wl, sites, z, "nn", k=8)
    v = ctx.condsim(_dev(z), 6, 21).cpu().numpy()
    assert rel(v, oracle.condsim(prob, 21, 0, 6)) < TOL32


def test_condsim_host_buffers(plain_case):
    wl, sites, z, prob, ctx = plain_case
    zh = torch.tensor(z, dtype=torch.float32).pin_memory()
    out = ctx.condsim_host(zh, 4, wl.sim_seed).numpy()
    ref = ctx.condsim(_dev(z), 4, wl.sim_seed).cpu().numpy()
    assert np.array_equal(out, ref)


# ----------------------------------------------------------------------------- full size
def test_condsim_shakemap512_sampled(ce):
    """The 512 x 512, n = 2000, R = 100 workload in the launch configuration of the
    benchmark, checked on sampled realizations and grid nodes."""
    wl = workloads.workload("shakemap512")
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_)
    v = ctx.condsim(_dev(z), wl.R, wl.sim_seed).cpu().numpy().reshape(wl.R, -1)
    prob = _oracle_problem(wl, sites, z)
    rng = np.random.default_rng(0)
    nodes = np.concatenate([rng.choice(wl.m * wl.m, 3000, replace=False), np.arange(wl.m * wl.m - 512, wl.m * wl.m)])
    reals = [0, 1, 98, 99]
    ref, _ = oracle.condsim_at(prob, wl.sim_seed, 0, reals, nodes)
    assert rel(v[reals][:, nodes], ref) < TOL32
    # every realization is finite and has the right scale
    assert np.all(np.isfinite(v))
    assert 0.2 < float(v.std()) < 2.0


# ----------------------------------------------------------------------------- errors
def test_error_statuses(ce):
    wl = workloads.workload("plain64")
    ctx = ce.Context.from_workload(wl)
    z = _dev(np.zeros(3))
    with pytest.raises(ce.CEError) as e:
        ctx.condsim(z, 2, 0)
    assert e.value.status == ce.CE_ERR_STATE
    with pytest.raises(ce.CEError) as e:
        ctx.krige_weights(np.array([[0.5, 0.5], [1.5, 0.2]]))
    assert e.value.status == ce.CE_ERR_ARG
    ctx.krige_weights(np.array([[0.5, 0.5], [0.2, 0.2], [0.7, 0.1]]))
    with pytest.raises(ce.CEError) as e:
        ctx.condsim(z, 2, 0, r_offset=1)
    assert e.value.status == ce.CE_ERR_ARG
    with pytest.raises(ce.CEError) as e:
        ce.Context(32, 0, 0, 1 / 31, 1.0, 0.3, 1.5, 0.05, max_growth=0)
    assert e.value.status == ce.CE_ERR_EMBED
    dup = ce.Context(16, 0, 0, 1 / 15, 1.0, 0.2, 0.5, 0.0)
    with pytest.raises(ce.CEError) as e:
        dup.krige_weights(np.array([[0.3, 0.3], [0.3, 0.3]]))
    assert e.value.status == ce.CE_ERR_NOT_SPD
    lib = ce.load_library()
    assert lib.ce_set_solve_form(ctx._ctx, 2) == ce.CE_ERR_ARG       # forms are 0 (FP32) and 1 (tensor)
    assert lib.ce_set_precision(ctx._ctx, 5) == ce.CE_ERR_ARG        # forms 0 .. 4
    assert lib.ce_set_solve_form(ctx._ctx, 1) == ce.CE_OK
    assert ctx.info()["solve_tc"] == 1


# ----------------------------------------------------------------------------- tensor-core correction
TOL_BF16 = 1e-3
TOL_F16 = 1e-4


@pytest.mark.parametrize("prec", ["bf16x3", "f16x3", "tf32x3"])
@pytest.mark.parametrize("m,n,R", [(64, 200, 5), (77, 150, 1), (40, 70, 300), (130, 333, 37), (96, 1100, 20)])
def test_correction_stage_tensor(ce, m, n, R, prec):
    """Tensor-core correction (hi/lo splits, one refinement pass) on ragged tiles
    (m not a multiple of 128), R = 1, R above one launch's 128 columns, and sites over
    several 512-site accumulation units (n = 1100)."""
    wl = workloads.workload("plain64").scaled(m=m, nu=1.5 if m % 2 else 0.5)
    sites = workloads.make_sites(wl, n=n)
    z = workloads.make_data(wl, sites)
    prob = _oracle_problem(wl, sites, z)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_, prec=prec)
    rng = np.random.default_rng(m)
    y = rng.standard_normal((R, m, m)).astype(np.float32)
    B = rng.standard_normal((R, n)).astype(np.float32)
    v = ctx.correct(_dev(B), _dev(y)).cpu().numpy()
    ctx.sync()
    ref = oracle.correction(prob, y.astype(np.float64), B.T.astype(np.float64)).reshape(R, m, m)
    assert rel(v, ref) < (TOL_BF16 if prec == "bf16x3" else TOL_F16)


def test_condsim_plain64_bf16x3(plain_case):
    wl, sites, z, prob, ctx = plain_case
    ctx.set_precision("bf16x3")
    try:
        v = ctx.condsim(_dev(z), 10, wl.sim_seed).cpu().numpy()
        ctx.sync()
    finally:
        ctx.set_precision("fp32")
    assert rel(v, oracle.condsim(prob, wl.sim_seed, 0, 10)) < TOL_BF16


@pytest.mark.parametrize("prec", ["bf16x3", "f16x3", "tf32x3"])
def test_condsim_shakemap512_tensor_sampled(ce, prec):
    wl = workloads.workload("shakemap512")
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_, prec=prec)
    v = ctx.condsim(_dev(z), wl.R, wl.sim_seed).cpu().numpy().reshape(wl.R, -1)
    ctx.sync()
    prob = _oracle_problem(wl, sites, z)
    rng = np.random.default_rng(1)
    nodes = rng.choice(wl.m * wl.m, 3000, replace=False)
    reals = [0, 57, 99]
    ref, _ = oracle.condsim_at(prob, wl.sim_seed, 0, reals, nodes)
    # f16x3, the benchmarked form, is held to the FP32 bar on this workload; tf32x3 (about
    # 1.1e-5 here) to the reduced-precision bar of 1e-4, bf16x3 to 1e-3
    tol = {"bf16x3": TOL_BF16, "f16x3": TOL32, "tf32x3": TOL_F16}[prec]
    assert rel(v[reals][:, nodes], ref) < tol


def test_condsim_host_async_pipelined(plain_case):
    """Pipelined host-buffer calls: three calls in flight on two staging buffers, each
    equal bit for bit to the device-buffer call with the same seed and offset."""
    wl, sites, z, prob, ctx = plain_case
    zh = torch.tensor(z, dtype=torch.float32).pin_memory()
    runs = [(5, 17, 0), (4, 23, 6), (5, 17, 10)]
    outs = [torch.empty((R, wl.m, wl.m), dtype=torch.float32).pin_memory() for R, _, _ in runs]
    for (R, seed, off), o in zip(runs, outs):
        ctx.condsim_host_async(zh, R, seed, off, o)
    ctx.host_wait()
    for (R, seed, off), o in zip(runs, outs):
        ref = ctx.condsim(_dev(z), R, seed, off).cpu()
        assert torch.equal(o, ref)
