"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, a library routine for a special case,
brute force on tiny inputs, or Monte Carlo against a closed-form covariance.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    for row in _rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = oracle.philox4x32_10(v[0], v[1], v[2], v[3], v[4], v[5])
        assert [int(o) for o in out] == v[6:10]


def test_philox_vectorised_matches_scalar():
    ctr = np.arange(17, dtype=np.uint64) * 977
    vec = oracle.philox4x32_10(ctr, 5, 1, 3, 0x1234, 0x9876)
    for i, c in enumerate(ctr):
        sc = oracle.philox4x32_10(int(c), 5, 1, 3, 0x1234, 0x9876)
        assert [int(a[i]) for a in vec] == [int(s) for s in sc]


def test_uniform_open_interval_and_box_muller_special_values():
    assert oracle.uniform01(0) == 2.0 ** -33
    assert oracle.uniform01(0xFFFFFFFF) == 1.0 - 2.0 ** -33
    # u1 = exp(-1/2) gives radius 1; u2 = 1/4 gives angle pi/2.
    x1 = int(round(math.exp(-0.5) * 2 ** 32 - 0.5))
    x2 = int(round(0.25 * 2 ** 32 - 0.5))
    z0, z1 = oracle.box_muller(np.array([x1]), np.array([x2]))
    assert abs(z0[0]) < 1e-8 and abs(z1[0] - 1.0) < 1e-8


def test_normals_are_standard_normal():
    from scipy import stats
    e1, e2 = oracle.ce_noise(7, 3, 256)
    z = np.concatenate([e1.ravel(), e2.ravel()])
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # eps1 and eps2 are uncorrelated
    assert abs(np.mean(e1 * e2)) < 5 / math.sqrt(e1.size)
    nug = oracle.nugget_noise(7, 11, 100001)
    assert stats.kstest(nug, "norm").pvalue > 1e-4


def test_noise_streams_are_distinct():
    a1, _ = oracle.ce_noise(1, 0, 16)
    b1, _ = oracle.ce_noise(1, 1, 16)
    c1, _ = oracle.ce_noise(2, 0, 16)
    assert not np.allclose(a1, b1) and not np.allclose(a1, c1)
    assert not np.allclose(oracle.nugget_noise(1, 0, 8), oracle.nugget_noise(1, 1, 8))


# ----------------------------------------------------------------------------- Matern
@pytest.mark.parametrize("nu", [0.5, 1.5])
def test_matern_closed_form_matches_bessel_form(nu):
    d = np.linspace(0.0, 3.0, 301)
    a = oracle.matern(d, 0.7, 0.4, nu)
    b = oracle.matern_bessel(d, 0.7, 0.4, nu)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-14)
    assert a[0] == pytest.approx(0.49)


def test_matern_paper_ranges_give_five_percent():
    for dist, theta, nu in _rows("matern_5pct_ranges.txt"):
        c = oracle.matern(float(dist), 1.0, float(theta), float(nu))
        # theta printed to 2 decimals: 0.005 relative change in theta moves C by < 0.05 * 3 * 0.005/theta*d
        assert abs(c - 0.05) < 0.05 * float(dist) * 0.005 / float(theta) ** 2 * float(theta) + 1e-3
        assert float(theta) == pytest.approx(float(dist) / math.log(20.0), abs=0.005)


# ----------------------------------------------------------------------------- FFT
@pytest.mark.parametrize("P", [2, 4, 8, 32, 64])
def test_fft_matches_direct_dft(P):
    rng = np.random.default_rng(P)
    x = rng.standard_normal((3, P)) + 1j * rng.standard_normal((3, P))
    assert np.allclose(oracle.fft(x), oracle.dft_direct(x), atol=1e-11 * P)


def test_fft_against_library_parseval_and_delta():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((4, 256)) + 1j * rng.standard_normal((4, 256))
    X = oracle.fft(x)
    assert np.allclose(X, np.fft.fft(x), atol=1e-10)
    assert np.allclose((np.abs(X) ** 2).sum(axis=1), 256 * (np.abs(x) ** 2).sum(axis=1))
    d = np.zeros(64, complex)
    d[5] = 1.0
    assert np.allclose(oracle.fft(d), np.exp(-2j * np.pi * 5 * np.arange(64) / 64))
    y = rng.standard_normal((16, 32))
    assert np.allclose(oracle.fft2(y), np.fft.fft2(y), atol=1e-10)


# ----------------------------------------------------------------------------- embedding
def test_eigenvalues_equal_direct_dft_of_embedded_row():
    m, P = 8, 16
    c = oracle.embed_row(m, 0.1, P, 1.3, 0.25, 0.5)
    assert np.allclose(c, c.T) and np.allclose(c[1:, :], c[:0:-1, :])
    direct = oracle.dft_direct(oracle.dft_direct(c.astype(complex)).T).T
    lam, P_out, info = oracle.ce_eigenvalues(m, 0.1, 1.3, 0.25, 0.5, P=P, max_growth=0)
    assert P_out == P
    assert np.abs(direct.imag).max() < 1e-10
    assert np.allclose(np.where(direct.real < 0, 0, direct.real), lam, atol=1e-10)
    assert lam.sum() / P ** 2 == pytest.approx(1.3 ** 2, rel=1e-12)  # c[0] = sigma^2


def test_embedding_growth():
    # a smooth covariance that is indefinite at P = 2m must grow
    lam, P, info = oracle.ce_eigenvalues(32, 1 / 31, 1.0, 0.3, 1.5)
    assert P > 64 and info["lambda_min"] >= -1e-6 * info["lambda_max"]
    with pytest.raises(RuntimeError):
        oracle.ce_eigenvalues(32, 1 / 31, 1.0, 0.3, 1.5, max_growth=0)


def _ce_linear_map(lam, m):
    """Columns of the linear maps eps1 -> y and eps2 -> y of the CE sampler, obtained by
    pushing unit noise vectors through the oracle's own FFT pipeline."""
    P = lam.shape[0]
    scale = np.sqrt(lam / P ** 2)
    cols = []
    for k in range(P * P):
        e = np.zeros(P * P)
        e[k] = 1.0
        w = oracle.fft2(scale * e.reshape(P, P))
        cols.append(w[:m, :m].reshape(-1))
    F = np.array(cols).T          # M x N complex: y_{2p} = Re(F eps1 + i F eps2)
    return F


def test_ce_field_covariance_is_exactly_matern():
    m, h, sig, th, nu = 6, 0.2, 1.1, 0.5, 0.5
    lam, P, _ = oracle.ce_eigenvalues(m, h, sig, th, nu)
    F = _ce_linear_map(lam, m)
    # Re w = Re(F) eps1 - Im(F) eps2; Im w = Im(F) eps1 + Re(F) eps2
    cov_re = F.real @ F.real.T + F.imag @ F.imag.T
    cross = F.real @ F.imag.T - F.imag @ F.real.T
    K = oracle.cov_matrix(oracle.grid_xy(m, 0, 0, h), oracle.grid_xy(m, 0, 0, h), sig, th, nu)
    assert np.allclose(cov_re, K, atol=1e-12)
    # the two realizations of a pair (Re w, Im w) are uncorrelated: lambda is even
    assert np.abs(cross).max() < 1e-12


def test_ce_sampler_monte_carlo_matches_matern_and_cholesky_sampler():
    m, h, sig, th, nu = 4, 0.25, 1.0, 0.3, 1.5
    lam, P, _ = oracle.ce_eigenvalues(m, h, sig, th, nu)
    R = 40000
    y = oracle.ce_unconditional(lam, m, seed=99, r_offset=0, R=R).reshape(R, -1)
    emp = y.T @ y / R
    K = oracle.cov_matrix(oracle.grid_xy(m, 0, 0, h), oracle.grid_xy(m, 0, 0, h), sig, th, nu)
    se = np.sqrt((K ** 2 + np.outer(np.diag(K), np.diag(K))) / R)
    assert np.max(np.abs(emp - K) / se) < 5.0
    # a Cholesky sampler of the same law, with an independent generator, agrees too
    L = oracle.cholesky(K)
    yc = (L @ np.random.default_rng(3).standard_normal((K.shape[0], R))).T
    emp_c = yc.T @ yc / R
    assert np.max(np.abs(emp - emp_c) / (np.sqrt(2) * se)) < 5.0


# ----------------------------------------------------------------------------- off-grid weights
def test_local_weights_site_on_node_is_selection():
    m, h = 16, 1 / 15
    sites = np.array([[5 * h, 7 * h], [0.0, 0.0], [15 * h, 15 * h], [3 * h, 14 * h]])
    for np_ in (1, 2, 3):
        idx, W, gamma = oracle.local_weights(sites, m, 0.0, 0.0, h, 1.0, 0.2, 1.5, np_)
        node = np.array([7 * m + 5, 0, 15 * m + 15, 14 * m + 3])
        for s in range(len(sites)):
            k = int(np.where(idx[s] == node[s])[0][0])
            e = np.zeros(idx.shape[1])
            e[k] = 1.0
            assert np.allclose(W[s], e, atol=1e-9)
        assert np.allclose(gamma, 0.0, atol=1e-9)


def test_local_weights_against_library_solve_and_bounds():
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl)
    idx, W, gamma = oracle.local_weights(sites, wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.np_)
    g = oracle.grid_xy(wl.m, wl.x0, wl.y0, wl.h)
    for s in (0, 17, 199):
        nodes = g[idx[s]]
        K11 = oracle.cov_matrix(nodes, nodes, wl.sigma, wl.range, wl.nu)
        k21 = oracle.cov_matrix(sites[s:s + 1], nodes, wl.sigma, wl.range, wl.nu)[0]
        w = np.linalg.solve(K11, k21)
        assert np.allclose(W[s], w, atol=1e-10)
        assert gamma[s] == pytest.approx(wl.sigma ** 2 - k21 @ w, abs=1e-12)
        # window is inside the grid and surrounds the site when away from the edge
        assert nodes[:, 0].min() <= sites[s, 0] <= nodes[:, 0].max()
        assert nodes[:, 1].min() <= sites[s, 1] <= nodes[:, 1].max()
    assert np.all(gamma >= -1e-12) and np.all(gamma <= wl.sigma ** 2)
    assert idx.min() >= 0 and idx.max() < wl.m ** 2


def test_sites_outside_grid_are_rejected():
    with pytest.raises(ValueError):
        oracle.local_weights(np.array([[1.2, 0.5]]), 8, 0, 0, 1 / 7, 1, 0.2, 0.5, 1)


def test_nn_nodes_brute_force():
    m, h = 12, 1 / 11
    rng = np.random.default_rng(5)
    sites = np.concatenate([rng.uniform(0, 1, (40, 2)),
                            np.array([[0.5 * h, 0.5 * h], [h, h], [1.0, 1.0], [0.0, 0.5]])])
    got = oracle.nn_nodes(sites, m, 0.0, 0.0, h, 8)
    g = oracle.grid_xy(m, 0.0, 0.0, h)
    for s in range(len(sites)):
        dx = sites[s, 0] - g[:, 0]
        dy = sites[s, 1] - g[:, 1]
        d2 = dx * dx + dy * dy
        order = np.lexsort((np.arange(m * m), d2))
        assert list(got[s]) == list(order[:8])


# ----------------------------------------------------------------------------- linear algebra
def test_cholesky_and_solves():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((30, 30))
    A = X @ X.T + 30 * np.eye(30)
    L = oracle.cholesky(A)
    assert np.allclose(L @ L.T, A) and np.allclose(L, np.linalg.cholesky(A))
    B = rng.standard_normal((30, 4))
    assert np.allclose(oracle.chol_solve(L, B), np.linalg.solve(A, B))
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky(A - 100 * np.eye(30))


# ----------------------------------------------------------------------------- the method
def _small_problem(m=8, sigma=1.0, theta=0.3, nu=0.5, tau2=0.1):
    h = 1.0 / (m - 1)
    return oracle.Problem(m, 0.0, 0.0, h, sigma, theta, nu, tau2)


def test_kriging_reproduces_data_without_nugget():
    prob = _small_problem(tau2=0.0)
    h = prob.h
    sites = np.array([[1 * h, 2 * h], [5 * h, 5 * h], [6 * h, 1 * h], [3 * h, 6 * h]])
    z = np.array([0.3, -1.2, 0.8, 2.0])
    oracle.setup_local(prob, sites, z, 1)
    B = oracle.solve_B(prob, z[None, :])
    nodes = np.array([2 * 8 + 1, 5 * 8 + 5, 1 * 8 + 6, 6 * 8 + 3])
    pred = oracle.correction(prob, np.zeros((1, 8, 8)), B, nodes)[0]
    assert np.allclose(pred, z, atol=1e-10)


def test_on_grid_sites_give_the_exact_conditional_law():
    prob = _small_problem()
    h = prob.h
    sites = np.array([[1 * h, 2 * h], [5 * h, 5 * h], [6 * h, 1 * h], [3 * h, 6 * h]])
    oracle.setup_local(prob, sites, np.zeros(4), 1)
    assert np.allclose(prob.gamma, 0.0, atol=1e-12)
    assert np.allclose(oracle.local_approx_cov(prob), oracle.exact_conditional_cov(prob, sites), atol=1e-10)


@pytest.mark.parametrize("mode", ["local", "nn"])
def test_condsim_ensemble_matches_closed_form_covariance_and_mean(mode):
    prob = _small_problem(m=6, theta=0.4, nu=1.5, tau2=0.05)
    rng = np.random.default_rng(11)
    sites = rng.uniform(0.05, 0.95, (5, 2))
    z = rng.standard_normal(5)
    if mode == "local":
        oracle.setup_local(prob, sites, z, 1)
    else:
        oracle.setup_nn(prob, sites, z, 2)
    R = 20000
    v = oracle.condsim(prob, seed=5, r_offset=0, R=R).reshape(R, -1)
    # E[v] = K_go A^-1 z_eff (the synthetic data have mean zero)
    mean = oracle.correction(prob, np.zeros((1, prob.m, prob.m)), oracle.solve_B(prob, prob.zeff[None, :]))[0]
    C = oracle.local_approx_cov(prob)
    sd = np.sqrt(np.diag(C))
    assert np.max(np.abs(v.mean(0) - mean) / (sd / math.sqrt(R))) < 5.0
    dv = v - mean
    emp = dv.T @ dv / R
    se = np.sqrt((C ** 2 + np.outer(np.diag(C), np.diag(C))) / R)
    assert np.max(np.abs(emp - C) / np.maximum(se, 1e-12)) < 5.5


def test_nn_surrogate_variance_on_grid_sites():
    prob = _small_problem(tau2=0.07)
    h = prob.h
    sites = np.array([[2 * h, 3 * h], [5 * h, 1 * h], [4 * h, 6 * h]])
    oracle.setup_nn(prob, sites, np.array([1.0, -0.5, 0.2]), 1)
    assert list(prob.J) == sorted([3 * 8 + 2, 1 * 8 + 5, 6 * 8 + 4])
    # each surrogate node coincides with its site: sigma_N^2 is the Kriging variance there
    A = oracle.cov_matrix(sites, sites, 1.0, 0.3, 0.5) + 0.07 * np.eye(3)
    order = np.argsort([3 * 8 + 2, 1 * 8 + 5, 6 * 8 + 4])
    K = oracle.cov_matrix(sites, sites, 1.0, 0.3, 0.5)
    kv = 1.0 - np.diag(K @ np.linalg.solve(A, K))
    assert np.allclose(prob.sigN2, kv[order], atol=1e-12)


def test_r_offset_concatenation():
    prob = _small_problem()
    rng = np.random.default_rng(2)
    sites = rng.uniform(0, 1, (6, 2))
    oracle.setup_local(prob, sites, rng.standard_normal(6), 1)
    full = oracle.condsim(prob, 3, 0, 6)
    part = oracle.condsim(prob, 3, 2, 4)
    assert np.allclose(full[2:], part)
    vs, ys = oracle.condsim_at(prob, 3, 0, [1, 4], np.array([0, 9, 63]))
    assert np.allclose(vs, full.reshape(6, -1)[[1, 4]][:, [0, 9, 63]])


def test_log_likelihood_matches_library_gaussian():
    from scipy.stats import multivariate_normal
    prob = _small_problem(m=8, tau2=0.07)
    rng = np.random.default_rng(8)
    sites = rng.uniform(0.02, 0.98, (7, 2))
    z = rng.standard_normal(7)
    oracle.setup_local(prob, sites, z, 1)
    A = oracle.cov_matrix(sites, sites, prob.sigma, prob.theta, prob.nu) + 0.07 * np.eye(7)
    assert oracle.log_likelihood(prob) == pytest.approx(multivariate_normal(np.zeros(7), A).logpdf(z), rel=1e-12)


def test_window_loss_definition():
    v = np.zeros((3, 6, 6))
    v[:, 1:3, 2:5] = 2.0
    v[1, 1, 2] = 4.0
    # window rows 1..2, columns 2..4: 6 nodes, values 2 except one 4 in realization 1
    expected = ((4.0 * 6) + (4.0 * 5 + 16.0) + (4.0 * 6)) / 6 / 3
    assert oracle.window_loss(v, (1, 3, 2, 5)) == pytest.approx(expected)


def test_circulant_correction_equals_direct_sum_without_clipping():
    # exponential covariance: the embedding is nonnegative definite, nothing is
    # clipped, and the torus convolution must reproduce the direct sum K_gN B
    prob = _small_problem(m=12, theta=0.2, nu=0.5, tau2=0.05)
    assert prob.lam.min() >= 0.0
    rng = np.random.default_rng(12)
    sites = rng.uniform(0.05, 0.95, (7, 2))
    oracle.setup_nn(prob, sites, rng.standard_normal(7), 3)
    B = rng.standard_normal((prob.J.size, 3))
    y = rng.standard_normal((3, 12, 12))
    assert np.allclose(oracle.correction_circulant(prob, y, B), oracle.correction(prob, y, B), rtol=0, atol=1e-12)
    with pytest.raises(ValueError):
        prob_local = _small_problem()
        oracle.setup_local(prob_local, sites, np.zeros(7), 1)
        oracle.correction_circulant(prob_local, y, B)


def test_gls_beta_against_whitened_library_least_squares():
    prob = _small_problem(m=10, theta=0.25, nu=1.5, tau2=0.1)
    rng = np.random.default_rng(21)
    sites = rng.uniform(0.0, 1.0, (15, 2))
    oracle.setup_local(prob, sites, rng.standard_normal(15), 2)
    X = oracle.trend_basis(sites, 10, 0.0, 0.0, prob.h, 1)
    W = rng.standard_normal((15, 4))
    A = oracle.cov_matrix(sites, sites, 1.0, 0.25, 1.5) + 0.1 * np.eye(15)
    Li = np.linalg.inv(np.linalg.cholesky(A))
    ref = np.linalg.lstsq(Li @ X, Li @ W, rcond=None)[0]
    assert np.allclose(oracle.gls_beta(prob, X, W), ref, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("degree", [0, 1])
def test_trend_model_reproduces_a_mean_added_to_the_data(degree):
    # the universal Kriging predictor is exact for the trend: adding a mean in the span
    # of the regressors to the data adds the same mean to every conditional draw
    prob = _small_problem(m=12, theta=0.2, nu=0.5, tau2=0.08)
    rng = np.random.default_rng(5 + degree)
    sites = rng.uniform(0.0, 1.0, (14, 2))
    z = rng.standard_normal(14)
    coef = np.array([1.7]) if degree == 0 else np.array([1.7, -0.9, 2.3])
    Xs = oracle.trend_basis(sites, 12, 0.0, 0.0, prob.h, degree)
    Xg = oracle.trend_basis(prob.grid(), 12, 0.0, 0.0, prob.h, degree)
    oracle.setup_local(prob, sites, z, 2)
    v0 = oracle.condsim_trend(prob, degree, 31, 0, 4)
    plain = oracle.condsim(prob, 31, 0, 4)
    oracle.setup_local(prob, sites, z + Xs @ coef, 2)
    v1 = oracle.condsim_trend(prob, degree, 31, 0, 4)
    assert np.allclose(v1 - v0, (Xg @ coef).reshape(12, 12)[None], rtol=0, atol=1e-9)
    # on the same data the trend draws differ from the zero-mean ones (the mean is estimated)
    assert not np.allclose(v0, plain, atol=1e-6)


# ----------------------------------------------------------------------------- sites sharing a grid box
def _box_sites(h, box, offsets):
    """Sites at (box corner + offset) * h, offsets inside [0, 1)^2 (grid units)."""
    i0, j0 = box
    return np.array([[(j0 + a) * h, (i0 + b) * h] for a, b in offsets])


def test_joint_box_with_the_whole_grid_as_window_is_the_exact_conditional_law():
    # m = 4 and np = 2: every window is the whole grid, so W_1 and Gamma_b are the exact
    # conditional law of the sites given the grid; drawn jointly (Section 2.1, Section 3.6)
    # the synthetic data have the exact joint law and the draws the exact conditional covariance
    for nu in (0.5, 1.5):
        prob = _small_problem(m=4, theta=0.5, nu=nu, tau2=0.1)
        sites = _box_sites(prob.h, (1, 1), [(0.2, 0.3), (0.7, 0.4), (0.5, 0.9), (0.1, 0.8)])
        oracle.setup_local(prob, sites, np.zeros(4), 2, joint_boxes=True)
        assert [list(b) for b in prob.boxes] == [[0, 1, 2, 3]]
        exact = oracle.exact_conditional_cov(prob, sites)
        assert np.allclose(oracle.local_approx_cov(prob), exact, rtol=0, atol=1e-10)
        # drawn one by one (the algorithm the paper studies) they are not exact
        oracle.setup_local(prob, sites, np.zeros(4), 2)
        assert np.abs(oracle.local_approx_cov(prob) - exact).max() > 1e-4


def test_box_factor_is_the_inverse_of_the_precision_block():
    # Gamma_b is the Schur complement of the window block; equivalently the inverse of the
    # sites' block of the inverse joint covariance (a library inverse, another route)
    prob = _small_problem(m=16, theta=0.25, nu=1.5, tau2=0.06)
    h = prob.h
    sites = np.concatenate([_box_sites(h, (5, 7), [(0.1, 0.2), (0.8, 0.7), (0.45, 0.5)]),
                            _box_sites(h, (0, 14), [(0.3, 0.3), (0.6, 0.9)]),
                            _box_sites(h, (9, 2), [(0.5, 0.5)])])
    oracle.setup_local(prob, sites, np.zeros(len(sites)), 2, joint_boxes=True)
    assert [list(b) for b in prob.boxes] == [[3, 4], [0, 1, 2]]     # by box key i0*m + j0
    gxy = prob.grid()
    for mem, Lb in zip(prob.boxes, prob.box_L):
        pts = np.concatenate([sites[mem], gxy[prob.idx[mem[0]]]])
        S = oracle.cov_matrix(pts, pts, prob.sigma, prob.theta, prob.nu)
        k = mem.size
        gam = np.linalg.inv(np.linalg.inv(S)[:k, :k])
        assert np.allclose(Lb @ Lb.T, gam + prob.tau2 * np.eye(k), rtol=1e-8, atol=1e-10)
        assert np.allclose(np.diag(Lb @ Lb.T), prob.phi[mem] ** 2, rtol=1e-10)
        assert np.allclose(Lb, np.tril(Lb))


def test_singleton_boxes_keep_the_independent_draws():
    prob = _small_problem(m=16, theta=0.25, nu=0.5, tau2=0.06)
    h = prob.h
    sites = np.concatenate([_box_sites(h, (5, 7), [(0.1, 0.2), (0.8, 0.7)]),
                            _box_sites(h, (1, 1), [(0.5, 0.5)]),
                            _box_sites(h, (12, 3), [(0.25, 0.75)])])
    z = np.array([0.3, -0.2, 1.1, 0.4])
    y = oracle.ce_unconditional(prob.lam, prob.m, 9, 0, 3)
    oracle.setup_local(prob, sites, z, 2)
    e_ind = oracle.residuals(prob, y, 9, 0)
    oracle.setup_local(prob, sites, z, 2, joint_boxes=True)
    e_joint = oracle.residuals(prob, y, 9, 0)
    assert np.array_equal(e_ind[:, 2:], e_joint[:, 2:])
    # first site of the shared box: L_00 = phi_0, so its draw is unchanged as well
    assert np.allclose(e_ind[:, 0], e_joint[:, 0], rtol=1e-13, atol=1e-13)
    assert np.abs(e_ind[:, 1] - e_joint[:, 1]).max() > 1e-3


def test_joint_box_ensemble_matches_its_closed_form_covariance():
    # Monte Carlo of the drawing code (L_b eps) against the covariance formula (L_b L_b^T)
    prob = _small_problem(m=6, theta=0.4, nu=1.5, tau2=0.02)
    h = prob.h
    sites = np.concatenate([_box_sites(h, (2, 2), [(0.15, 0.2), (0.85, 0.3), (0.5, 0.9)]),
                            _box_sites(h, (0, 4), [(0.4, 0.6)])])
    rng = np.random.default_rng(12)
    z = rng.standard_normal(4)
    oracle.setup_local(prob, sites, z, 1, joint_boxes=True)
    R = 20000
    v = oracle.condsim(prob, seed=8, r_offset=0, R=R).reshape(R, -1)
    mean = oracle.correction(prob, np.zeros((1, prob.m, prob.m)), oracle.solve_B(prob, prob.zeff[None, :]))[0]
    C = oracle.local_approx_cov(prob)
    dv = v - mean
    emp = dv.T @ dv / R
    se = np.sqrt((C ** 2 + np.outer(np.diag(C), np.diag(C))) / R)
    assert np.max(np.abs(emp - C) / np.maximum(se, 1e-12)) < 5.5
    # and the independent-draw formula is rejected by the same ensemble
    oracle.setup_local(prob, sites, z, 1)
    C_ind = oracle.local_approx_cov(prob)
    assert np.max(np.abs(emp - C_ind) / np.maximum(se, 1e-12)) > 8.0


# ----------------------------------------------------------------------------- standard errors (Section 3.4)
@pytest.mark.parametrize("mode", ["local", "local_joint", "nn"])
def test_standard_errors_are_the_closed_form_diagonals(mode):
    prob = _small_problem(m=9, theta=0.3, nu=1.5, tau2=0.05)
    rng = np.random.default_rng(21)
    sites = np.concatenate([rng.uniform(0.0, 1.0, (7, 2)), _box_sites(prob.h, (2, 2), [(0.2, 0.3), (0.6, 0.7)])])
    if mode == "nn":
        oracle.setup_nn(prob, sites, np.zeros(len(sites)), 3)
    else:
        oracle.setup_local(prob, sites, np.zeros(len(sites)), 2, joint_boxes=mode == "local_joint")
    full = np.sqrt(np.diag(oracle.local_approx_cov(prob)))
    assert np.allclose(oracle.se_approx(prob), full, rtol=0, atol=1e-12)
    nodes = np.array([0, 17, 40, 80])
    assert np.allclose(oracle.se_approx(prob, nodes), full[nodes], rtol=0, atol=1e-12)
    exact = np.sqrt(np.diag(oracle.exact_conditional_cov(prob, sites)))
    assert np.allclose(oracle.se_exact(prob, sites), exact, rtol=0, atol=1e-12)
    assert np.allclose(oracle.se_exact(prob, sites, nodes), exact[nodes], rtol=0, atol=1e-12)


def test_significant_figures():
    # (values chosen away from ties: 9.995 is stored as 9.99499... and rounds to 9.99)
    x = np.array([0.12345, 0.0012345, 9.9951, 9.995, -0.4567, 123456.0, 0.0, 0.12351])
    assert np.allclose(oracle.signif(x, 3), [0.123, 0.00123, 10.0, 9.99, -0.457, 123000.0, 0.0, 0.124], rtol=1e-12)
    a = np.array([0.4561, 0.4564, 0.4566, 0.9994, 0.5])
    b = np.array([0.4559, 0.4556, 0.4566, 0.99951, 0.5004])
    # 0.456|0.456, 0.456|0.456, equal, 0.999|1.00, 0.500|0.500
    assert oracle.sig_fig_fraction(a, b) == pytest.approx(4 / 5)
    assert np.allclose(oracle.relative_pct_error([1.01, 0.5], [1.0, 0.4]), [1.0, 25.0])


def test_local_standard_errors_reproduce_table_1():
    """The paper's numerical design (Section 3.3): exponential covariance, 61 x 61 grid on [0,60]^2,
    35 uniform sites.  Six configurations per case.  The reproduced fractions of standard errors
    correct to three significant figures lie within 0.025 of Table 1's means at n_p = 1 and n_p = 3
    (about one printed sd; the mean over six configurations has sd 0.015 at n_p = 1).  At n_p = 2
    they sit below the table by a gap of 0.025 to 0.08, one-sided and in every case (the reading
    of the window, R5, is the likely cause: the (2 n_p)^2 nodes nearest each site reproduce that
    column, the box-anchored square of Section 3.6 does not).  The pattern holds: rising with the
    neighbourhood order, n_p = 2 rising with the range and the nugget, n_p = 1 falling with the range."""
    table = {(float(r[0]), float(r[1])): [float(v) for v in r[2:]] for r in _rows("se_sigfig_table1.txt")}
    got = {}
    for theta, tau in [(6.68, 0.1), (6.68, 0.3), (23.37, 0.1), (23.37, 0.3)]:
        fr = {1: [], 2: [], 3: []}
        for c in range(6):
            sites = workloads.se_study_sites(c)
            prob = oracle.Problem(61, 0.0, 0.0, 1.0, 1.0, theta, 0.5, tau * tau)
            se_e = oracle.se_exact(prob, sites)
            for np_ in (1, 2, 3):
                oracle.setup_local(prob, sites, np.zeros(len(sites)), np_)
                fr[np_].append(oracle.sig_fig_fraction(oracle.se_approx(prob), se_e))
        got[(theta, tau)] = [float(np.mean(fr[k])) for k in (1, 2, 3)]
        printed = table[(theta, tau)]
        d1, d2, d3 = (got[(theta, tau)][k] - printed[2 * k] for k in range(3))
        assert abs(d1) < 0.025, (theta, tau, 1, got[(theta, tau)][0])
        assert abs(d3) < 0.02, (theta, tau, 3, got[(theta, tau)][2])
        assert -0.08 < d2 < -0.025, (theta, tau, 2, got[(theta, tau)][1])
        assert got[(theta, tau)][0] < got[(theta, tau)][1] < got[(theta, tau)][2]
    assert got[(23.37, 0.1)][1] > got[(6.68, 0.1)][1] and got[(23.37, 0.3)][1] > got[(23.37, 0.1)][1]
    assert got[(6.68, 0.1)][0] > got[(23.37, 0.1)][0]


# ----------------------------------------------------------------------------- anisotropy (Section 5, R18)
def test_anisotropic_distance_closed_forms():
    dx, dy = np.array([0.3, -0.2, 0.0]), np.array([0.1, 0.4, -0.5])
    # no anisotropy at ratio 1, whatever the angle
    assert np.allclose(oracle.lag_distance(dx, dy, (1.0, 0.7)), np.hypot(dx, dy), rtol=1e-14)
    # angle 0: the range is theta along x and theta * ratio along y
    assert np.allclose(oracle.lag_distance(dx, dy, (0.5, 0.0)), np.sqrt(dx ** 2 + (dy / 0.5) ** 2), rtol=1e-14)
    # a quarter turn swaps the axes
    assert np.allclose(oracle.lag_distance(dx, dy, (0.5, math.pi / 2)), np.sqrt(dy ** 2 + (dx / 0.5) ** 2), rtol=1e-14)
    # along the major direction the length is Euclidean, across it divided by the ratio
    ang = 0.6
    u = np.array([math.cos(ang), math.sin(ang)])
    assert oracle.lag_distance(0.7 * u[0], 0.7 * u[1], (0.3, ang)) == pytest.approx(0.7, rel=1e-14)
    assert oracle.lag_distance(-0.7 * u[1], 0.7 * u[0], (0.3, ang)) == pytest.approx(0.7 / 0.3, rel=1e-14)
    with pytest.raises(ValueError):
        oracle.aniso_map((0.0, 0.1))


def test_anisotropic_embedding_is_even_and_reduces_to_isotropic():
    m, P, h = 8, 16, 0.1
    iso = oracle.embed_row(m, h, P, 1.3, 0.25, 0.5)
    assert np.allclose(oracle.embed_row(m, h, P, 1.3, 0.25, 0.5, (1.0, 0.4)), iso, rtol=1e-14, atol=0)
    c = oracle.embed_row(m, h, P, 1.3, 0.25, 0.5, (0.4, 0.5))
    a = np.arange(P)
    assert np.array_equal(c, c[(-a) % P][:, (-a) % P])          # even on the torus: lambda is real
    assert not np.allclose(c, c.T)                               # but not symmetric under a transpose
    direct = oracle.dft_direct(oracle.dft_direct(c.astype(complex)).T).T
    assert np.abs(direct.imag).max() < 1e-10
    # lags inside the grid keep the covariance of the offset
    gx = oracle.grid_xy(m, 0, 0, h)
    K = oracle.cov_matrix(gx[:1], gx, 1.3, 0.25, 0.5, (0.4, 0.5)).reshape(m, m)
    assert np.allclose(c[:m, :m], K, rtol=1e-14)


@pytest.mark.parametrize("nu", [0.5, 1.5])
def test_anisotropic_ce_field_covariance_is_exact(nu):
    m, h, sig, th, an = 6, 0.2, 1.1, 0.6, (0.45, 0.7)
    lam, P, info = oracle.ce_eigenvalues(m, h, sig, th, nu, aniso=an)
    assert info["clipped"] == 0 and info["imag_max"] < 1e-10
    F = _ce_linear_map(lam, m)
    cov_re = F.real @ F.real.T + F.imag @ F.imag.T
    gx = oracle.grid_xy(m, 0, 0, h)
    K = oracle.cov_matrix(gx, gx, sig, th, nu, an)
    assert np.allclose(cov_re, K, atol=1e-12)
    # and it is not the isotropic covariance
    assert np.abs(K - oracle.cov_matrix(gx, gx, sig, th, nu)).max() > 0.05


@pytest.mark.parametrize("mode", ["local", "nn"])
def test_anisotropic_condsim_ensemble_matches_closed_form(mode):
    prob = oracle.Problem(6, 0.0, 0.0, 0.2, 1.0, 0.5, 1.5, 0.05, aniso=(0.5, 0.4))
    rng = np.random.default_rng(13)
    sites = rng.uniform(0.05, 0.95, (5, 2))
    z = rng.standard_normal(5)
    if mode == "local":
        oracle.setup_local(prob, sites, z, 1)
        # a site on a node keeps the exact law: unit weight, gamma = 0
        idx, W, gamma = oracle.local_weights(np.array([[0.4, 0.6]]), 6, 0.0, 0.0, 0.2, 1.0, 0.5, 1.5, 1, prob.aniso)
        assert np.allclose(np.sort(W[0]), [0, 0, 0, 1], atol=1e-12) and abs(gamma[0]) < 1e-12
    else:
        oracle.setup_nn(prob, sites, z, 2)
    R = 20000
    v = oracle.condsim(prob, seed=7, r_offset=0, R=R).reshape(R, -1)
    mean = oracle.correction(prob, np.zeros((1, prob.m, prob.m)), oracle.solve_B(prob, prob.zeff[None, :]))[0]
    C = oracle.local_approx_cov(prob)
    dv = v - mean
    emp = dv.T @ dv / R
    se = np.sqrt((C ** 2 + np.outer(np.diag(C), np.diag(C))) / R)
    assert np.max(np.abs(emp - C) / np.maximum(se, 1e-12)) < 5.5


def test_anisotropic_circulant_correction_equals_direct_sum():
    # the circulant identity holds for any stationary covariance whose embedding needs no clipping
    prob = oracle.Problem(12, 0.0, 0.0, 1.0 / 11, 1.0, 0.2, 0.5, 0.05, aniso=(0.4, 0.9))
    assert prob.eig_info["clipped"] == 0
    rng = np.random.default_rng(31)
    sites = rng.uniform(0.0, 1.0, (7, 2))
    oracle.setup_nn(prob, sites, rng.standard_normal(7), 3)
    y = oracle.ce_unconditional(prob.lam, prob.m, 4, 0, 3)
    B = oracle.solve_B(prob, oracle.residuals(prob, y, 4, 0))
    assert np.allclose(oracle.correction_circulant(prob, y, B), oracle.correction(prob, y, B), rtol=0, atol=1e-12)


def test_joint_box_whole_grid_window_exact_with_anisotropy():
    prob = oracle.Problem(4, 0.0, 0.0, 1.0 / 3, 1.0, 0.5, 1.5, 0.1, aniso=(0.5, 0.8))
    sites = _box_sites(prob.h, (1, 2), [(0.2, 0.3), (0.7, 0.4), (0.5, 0.9)])
    oracle.setup_local(prob, sites, np.zeros(3), 2, joint_boxes=True)
    assert np.allclose(oracle.local_approx_cov(prob), oracle.exact_conditional_cov(prob, sites), rtol=0, atol=1e-10)


def test_exact_standard_error_vanishes_at_noise_free_data():
    prob = _small_problem(m=10, theta=0.3, nu=1.5, tau2=0.0)
    h = prob.h
    sites = np.array([[3 * h, 4 * h], [7 * h, 2 * h], [0.55, 0.81]])
    se = oracle.se_exact(prob, sites)
    assert se[4 * 10 + 3] < 1e-6 and se[2 * 10 + 7] < 1e-6
    assert se.max() <= prob.sigma + 1e-12 and se.min() >= 0.0


def test_table_2_against_the_readings_of_section_3_2():
    """Table 2 (NN Kriging) is not reproduced by any reading of Section 3.2 tried
    (oracle/table2_readings.py; the means over six configurations are recorded with the
    readings).  Pinned here on two configurations of (theta, tau) = (6.68, 0.1), where the table
    prints 0.896 (sd 0.003) at n_p = 2: the library's reading R7, the same with nearest nodes,
    noise-free surrogate variances, no nugget in the prediction matrix and the full surrogate
    error covariance all score below 0.05, because surrogate errors taken as independent make the
    ensemble over-confident where surrogates cluster; the NN predictor's mean-squared error (not
    an ensemble spread) has the table's shape but scores 0.95.  The means of the table's
    (15.02, 0.3) row are Table 1's means of that row."""
    from oracle import table2_readings as t2
    t1 = {(float(r[0]), float(r[1])): [float(v) for v in r[2:]] for r in _rows("se_sigfig_table1.txt")}
    t2rows = {(float(r[0]), float(r[1])): [float(v) for v in r[2:]] for r in _rows("se_sigfig_table2.txt")}
    assert t2rows[(15.02, 0.3)][0::2] == t1[(15.02, 0.3)][0::2]     # the means; the sds differ
    acc = {}
    for c in range(2):
        for key, v in t2.fractions(6.68, 0.1, c, orders=(2,)).items():
            acc.setdefault(key[0], []).append(v)
    mean = {k: float(np.mean(v)) for k, v in acc.items()}
    printed = t2rows[(6.68, 0.1)][2]
    for reading in ("r7", "r7_knn", "noise_free", "no_tau", "full_sigma"):
        assert mean[reading] < 0.05, (reading, mean[reading])
    assert 0.9 < mean["mse"] < 1.0 and mean["mse"] - printed > 0.03


def test_diff_loss_window_path_equals_the_whole_draw():
    """diff_loss evaluates step 5 on the window's nodes only; on a small problem it equals the
    window loss of the whole conditional draw plus the log-likelihood, and a library Cholesky
    passed as `factor` gives the same value."""
    m, h = 12, 1.0 / 11
    rng = np.random.default_rng(5)
    sites = rng.uniform(0.0, 1.0, (9, 2))
    z = rng.standard_normal(9)
    win = (3, 9, 2, 8)
    got = oracle.diff_loss(m, 0.0, 0.0, h, 0.9, 0.2, 1.5, 0.07, sites, z, 2, 17, 4, 3, win)
    prob = oracle.Problem(m, 0.0, 0.0, h, 0.9, 0.2, 1.5, 0.07)
    oracle.setup_local(prob, sites, z, 2)
    v = oracle.condsim(prob, 17, 4, 3)
    ref = oracle.window_loss(v, win) + oracle.log_likelihood(prob)
    assert got == pytest.approx(ref, rel=1e-13, abs=1e-13)
    lib = oracle.diff_loss(m, 0.0, 0.0, h, 0.9, 0.2, 1.5, 0.07, sites, z, 2, 17, 4, 3, win, factor=np.linalg.cholesky)
    assert lib == pytest.approx(ref, rel=1e-12, abs=1e-12)
