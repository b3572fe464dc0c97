"""FP64 CPU oracle: a plain, slow restatement of the method of Bailey,
Bandyopadhyay & Nychka, "Adapting conditional simulation using circulant
embedding for irregularly spaced spatial data" (arXiv 2109.11044).

TEST INFRASTRUCTURE ONLY.  Imported by the tests, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``; nothing in the CUDA library uses
it, and it shares no code, table or constant generator with that library.

Everything is float64 numpy.  The FFT, the direct DFT, the Cholesky factor and
the triangular solves are written out here; numpy supplies only elementwise
math, reductions and matrix products.  Each function names the passage of
the paper it follows.  Readings of passages that are silent, garbled or
inconsistent are stated where they are used:

* R1 Grid: node (i, j) sits at (x0 + j h, y0 + i h); flat index g = i*m + j.
* R2 Embedding: P = the smallest power of two >= 2m to start; c[a,b] = C(h * sqrt(min(a,P-a)^2 + min(b,P-b)^2)).
  If the smallest eigenvalue is below -1e-6 * lambda_max, P doubles (at most
  ``max_growth`` times); remaining negatives are clipped to 0 and their count
  and mass are reported (the 512 x 512, Matern 3/2, range 0.15 workload is
  specified with a 1024 x 1024 embedding, whose negative part is 2e-6 of the
  trace, so the growth threshold admits it).
* R3 Fourier convention: unnormalised forward DFT (sign -1); the spectral
  weights are sqrt(lambda / N), N = P^2.
* R4 Noise: Philox4x32-10 keyed by the 64-bit seed.  The field of realization
  pair p uses counter (a P + b, p, 0, event) for torus rows a < P/2, whose four
  words give (eps1, eps2) at element (a, b) and at element (a + P/2, b) of the
  same column; the nugget of realization r uses counter (site group, r, 1,
  event); uniforms are (x + 0.5) 2^-32, normals by Box-Muller (cos, sin).
* R5 Local Kriging window: box corner (i0, j0) = floor of the site's grid
  coordinates; window rows/columns [i0-np+1, i0+np], shifted inward to lie in
  [0, m-1] when the site is near the edge (same shape, true offsets).
* R6 Prediction weights use A = K_oo + tau^2 I (the transpose and the tau in
  the printed W_2 of Section 3.1 are read as K_go (K_oo + tau^2 I)^-1, as in
  Eq. (condmvn)).
* R7 NN Kriging: the k nearest grid nodes of each site by Euclidean distance
  (ties to the smaller flat index), union sorted and deduplicated; surrogate
  data J_N K_go A^-1 z; surrogate error variances
  diag J_N (K_gg - K_go A^-1 K_og) J_N^T; prediction with
  K_NN + tau^2 I + Sigma_N (Section 3.2, with the dimensions made consistent).
* R16 Sites sharing a grid box (optional, ``joint_boxes``): the box's noise is
  L_b eps_b, L_b = chol(Gamma_b + tau^2 I) over the box's sites in ascending
  caller order, eps_b their own nugget draws (reading R4); a site alone in its
  box keeps phi_i eps_i.
* R18 Anisotropy (optional): geometric, C(|A (dx, dy)|) with A = diag(1, 1/ratio)
  Rot(-angle); the embedding row is made even at the torus lag P/2 (mean of the
  entry and its mirror); nearest nodes stay Euclidean in grid units.
* R17 The score of standard errors correct to three significant figures (Tables
  1-2): both standard errors rounded to three significant figures are equal.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "PHILOX_M0", "PHILOX_M1", "PHILOX_W0", "PHILOX_W1",
    "philox4x32_10", "uniform01", "box_muller", "ce_noise", "nugget_noise",
    "matern", "aniso_map", "lag_distance", "matern_bessel", "fft", "dft_direct", "fft2", "embed_row",
    "ce_eigenvalues", "ce_unconditional", "grid_xy", "local_window",
    "local_weights", "nn_nodes", "box_nodes", "cholesky", "solve_lower", "solve_upper",
    "chol_solve", "cov_matrix", "Problem", "setup_local", "box_noise_factors", "setup_nn",
    "offgrid_local", "offgrid_nn", "residuals", "solve_B", "correction", "correction_circulant",
    "trend_basis", "gls_beta", "condsim_trend",
    "condsim", "condsim_at", "exact_conditional_cov", "local_approx_cov",
    "se_exact", "se_approx", "relative_pct_error", "signif", "sig_fig_fraction",
    "log_likelihood", "window_loss", "diff_loss",
]

MASK32 = 0xFFFFFFFF

# ---------------------------------------------------------------------------
# Counter-based generator (the paper draws its noise with R's generator; the
# GPU path needs a stream both sides can reproduce, so both implement
# Philox4x32-10 from Salmon, Moraes, Dror & Shaw, "Parallel random numbers:
# as easy as 1, 2, 3", SC'11, Section 4.2: multipliers, Weyl key increments,
# ten rounds).
# ---------------------------------------------------------------------------
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit counters; returns 4 uint32 arrays.

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0));
    the key advances by (W0, W1) between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK32 for v in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & MASK32)
    k1 = np.uint64(int(k1) & MASK32)
    m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
    for rnd in range(10):
        if rnd:
            k0 = np.uint64((int(k0) + PHILOX_W0) & MASK32)
            k1 = np.uint64((int(k1) + PHILOX_W1) & MASK32)
        p0 = m0 * c0
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK32)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(v.astype(np.uint32) for v in (c0, c1, c2, c3))


def uniform01(x):
    """uint32 -> (x + 1/2) 2^-32, strictly inside (0, 1)."""
    return (np.asarray(x, dtype=np.float64) + 0.5) * 2.0 ** -32


def box_muller(xa, xb):
    """Two uint32 words -> two independent N(0,1) values (Box & Muller 1958)."""
    u1 = uniform01(xa)
    u2 = uniform01(xb)
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * math.pi * u2
    return rad * np.cos(ang), rad * np.sin(ang)


def _key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & MASK32, seed >> 32


def ce_noise(seed: int, pair: int, P: int, event: int = 0):
    """Complex white noise eps1 + i eps2 on the P x P torus for realization pair `pair`.

    Counter (a P + b, pair, 0, event) for a < P/2 gives the normals
    eps1[a, b], eps2[a, b] (words 0, 1) and eps1[a + P/2, b], eps2[a + P/2, b]
    (words 2, 3) (reading R4).
    """
    k0, k1 = _key(seed)
    g = np.arange(P * P // 2, dtype=np.uint64)          # g = a P + b, a < P/2
    x0, x1, x2, x3 = philox4x32_10(g, pair, 0, event, k0, k1)
    a0, a1 = box_muller(x0, x1)
    b0, b1 = box_muller(x2, x3)
    h = P // 2
    e1 = np.concatenate([a0.reshape(h, P), b0.reshape(h, P)], axis=0)
    e2 = np.concatenate([a1.reshape(h, P), b1.reshape(h, P)], axis=0)
    return e1, e2


def nugget_noise(seed: int, r: int, n: int, event: int = 0):
    """N(0,1) nugget draws eps*_r for sites 0..n-1 of realization r (reading R4)."""
    k0, k1 = _key(seed)
    q = np.arange((n + 3) // 4, dtype=np.uint64)
    x0, x1, x2, x3 = philox4x32_10(q, r, 1, event, k0, k1)
    z0, z1 = box_muller(x0, x1)
    z2, z3 = box_muller(x2, x3)
    return np.stack([z0, z1, z2, z3], axis=1).reshape(-1)[:n]


# ---------------------------------------------------------------------------
# Covariance model, Section 3.3: Matern family, closed forms for nu = 1/2, 3/2.
# ---------------------------------------------------------------------------
def matern(d, sigma: float, theta: float, nu: float):
    """C_nu(d) = sigma^2 2^(1-nu)/Gamma(nu) (sqrt(2 nu) d/theta)^nu K_nu(sqrt(2 nu) d/theta),
    in the closed forms nu = 1/2: sigma^2 exp(-d/theta) and
    nu = 3/2: sigma^2 (1 + sqrt(3) d/theta) exp(-sqrt(3) d/theta)."""
    d = np.asarray(d, dtype=np.float64)
    if nu == 0.5:
        return sigma * sigma * np.exp(-d / theta)
    if nu == 1.5:
        t = math.sqrt(3.0) * d / theta
        return sigma * sigma * (1.0 + t) * np.exp(-t)
    raise ValueError("only nu = 0.5 and nu = 1.5 have closed forms here")


def aniso_map(aniso):
    """Geometric anisotropy (reading R18): aniso = (ratio, angle) gives the 2 x 2 map
    A = diag(1, 1/ratio) Rot(-angle), and the covariance of an offset (dx, dy) is
    C(|A (dx, dy)|): range theta along the direction at `angle` from the x axis,
    theta * ratio across it.  None is the isotropic model (A = I)."""
    if aniso is None:
        return None
    ratio, angle = float(aniso[0]), float(aniso[1])
    if not ratio > 0.0:
        raise ValueError("anisotropy ratio must be positive")
    c, s = math.cos(angle), math.sin(angle)
    return np.array([[c, s], [-s / ratio, c / ratio]])


def lag_distance(dx, dy, aniso=None):
    """|A (dx, dy)|: the Euclidean length of the offset, or its anisotropic length (R18)."""
    dx = np.asarray(dx, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    A = aniso_map(aniso)
    if A is None:
        return np.sqrt(dx * dx + dy * dy)
    u = A[0, 0] * dx + A[0, 1] * dy
    v = A[1, 0] * dx + A[1, 1] * dy
    return np.sqrt(u * u + v * v)


def matern_bessel(d, sigma: float, theta: float, nu: float):
    """The general Matern form of Section 3.3 through scipy's Bessel K (used only as a pin)."""
    from scipy.special import gamma, kv
    d = np.asarray(d, dtype=np.float64)
    t = math.sqrt(2.0 * nu) * d / theta
    out = np.full(d.shape, sigma * sigma)
    pos = t > 0
    out[pos] = sigma * sigma * 2.0 ** (1.0 - nu) / gamma(nu) * t[pos] ** nu * kv(nu, t[pos])
    return out


# ---------------------------------------------------------------------------
# Discrete Fourier transforms (own code; numpy's FFT is not used).
# ---------------------------------------------------------------------------
def dft_direct(x):
    """Forward DFT along the last axis by the O(P^2) sum X[k] = sum_j x[j] e^{-2 pi i jk/P}."""
    x = np.asarray(x, dtype=np.complex128)
    P = x.shape[-1]
    jk = np.outer(np.arange(P), np.arange(P)) % P
    W = np.exp(-2j * math.pi * jk / P)
    return x @ W.T


def fft(x):
    """Forward DFT along the last axis by iterative radix-2 decimation in time
    (Cooley & Tukey 1965): bit-reversed reordering, then log2 P stages that
    merge pairs of half-length transforms E, O into E + w^k O and E - w^k O."""
    x = np.asarray(x, dtype=np.complex128)
    P = x.shape[-1]
    if P & (P - 1):
        raise ValueError("length must be a power of two")
    bits = P.bit_length() - 1
    rev = np.zeros(P, dtype=np.int64)
    for b in range(bits):
        rev |= ((np.arange(P) >> b) & 1) << (bits - 1 - b)
    lead = x.shape[:-1]
    y = x[..., rev]
    half = 1
    while half < P:
        y = y.reshape(*lead, P // (2 * half), 2, half)
        w = np.exp(-2j * math.pi * np.arange(half) / (2 * half))
        even = y[..., 0, :]
        odd = y[..., 1, :] * w
        y = np.concatenate([even + odd, even - odd], axis=-1).reshape(*lead, P)
        half *= 2
    return y


def fft2(x):
    """2-D forward DFT over the last two axes (rows, then columns)."""
    y = fft(x)
    return np.swapaxes(fft(np.swapaxes(y, -1, -2)), -1, -2)


# ---------------------------------------------------------------------------
# Circulant embedding (Section 1; Wood & Chan 1994; Section 2.1 step (a)).
# ---------------------------------------------------------------------------
def embed_row(m: int, h: float, P: int, sigma: float, theta: float, nu: float, aniso=None):
    """First row of the block-circulant covariance on the P x P torus (reading R2):
    c[a, b] = C of the torus lag (row lag a, column lag b), each taken in (-P/2, P/2].
    With anisotropy (R18) C(a, b) = C(-a, -b) but not C(a, -b), so the entries whose
    lag is P/2 are replaced by their mean with the mirrored entry, which makes c even
    on the torus (lambda real); the grid never uses a lag of P/2 or more."""
    a = np.arange(P)
    lag = np.where(a <= P // 2, a, a - P).astype(np.float64)
    d = lag_distance(h * lag[None, :], h * lag[:, None], aniso)
    c = matern(d, sigma, theta, nu)
    if aniso is not None:
        c = 0.5 * (c + c[(-a) % P][:, (-a) % P])
    return c


def ce_eigenvalues(m: int, h: float, sigma: float, theta: float, nu: float,
                   max_growth: int = 3, P: int | None = None, neg_tol: float = 1e-6, aniso=None):
    """Eigenvalues lambda = DFT2(c) of the circulant embedding, with growth and clipping.

    Returns (lam, P, info) where lam is P x P float64 with negatives clipped
    to 0 and info holds lambda_min before clipping, lambda_max and the count
    and mass of clipped values.  Raises if the embedding stays indefinite.
    """
    if P is None:
        P = 1
        while P < 2 * m:
            P *= 2
    for _ in range(max_growth + 1):
        c = embed_row(m, h, P, sigma, theta, nu, aniso)
        lam_c = fft2(c.astype(np.complex128))
        lam = lam_c.real
        lmax = float(lam.max())
        lmin = float(lam.min())
        if lmin >= -neg_tol * lmax:
            neg = lam < 0
            info = dict(lambda_min=lmin, lambda_max=lmax, clipped=int(neg.sum()),
                        clipped_mass=float(-lam[neg].sum()), imag_max=float(np.abs(lam_c.imag).max()))
            return np.where(neg, 0.0, lam), P, info
        P *= 2
    raise RuntimeError("circulant embedding is not nonnegative definite after growth")


def ce_unconditional(lam, m: int, seed: int, r_offset: int, R: int, event: int = 0):
    """R unconditional grid fields y_r (R x m x m), realizations r_offset .. r_offset+R-1.

    For the pair p = r/2: w = DFT2(sqrt(lam/N) (eps1 + i eps2)); realization 2p
    is Re w, realization 2p+1 is Im w, both cropped to [0, m)^2.  Each part has
    covariance c exactly: Cov(Re w_k, Re w_k') = sum_a (lam_a/N) cos(2 pi <a, k-k'>/P).
    """
    if r_offset % 2:
        raise ValueError("r_offset must be even")
    P = lam.shape[0]
    scale = np.sqrt(lam / (P * P))
    out = np.empty((R, m, m))
    for loc in range(0, R, 2):
        p = (r_offset + loc) // 2
        e1, e2 = ce_noise(seed, p, P, event)
        w = fft2(scale * (e1 + 1j * e2))
        out[loc] = w.real[:m, :m]
        if loc + 1 < R:
            out[loc + 1] = w.imag[:m, :m]
    return out


# ---------------------------------------------------------------------------
# Grid and off-grid neighbourhoods (Section 2.1, Section 3.6).
# ---------------------------------------------------------------------------
def grid_xy(m: int, x0: float, y0: float, h: float):
    """Coordinates of all M = m^2 grid nodes, flat index g = i*m + j (reading R1)."""
    i, j = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    return np.stack([x0 + j.reshape(-1) * h, y0 + i.reshape(-1) * h], axis=1)


def _box(sites, m, x0, y0, h):
    """Grid box (i0, j0) of every site: the floor of its grid coordinates (Section 3.6:
    finding neighbours on a regular grid is rounding real numbers to integers)."""
    sites = np.asarray(sites, dtype=np.float64)
    u = (sites[:, 0] - x0) / h
    v = (sites[:, 1] - y0) / h
    if np.any(u < 0) or np.any(v < 0) or np.any(u > m - 1) or np.any(v > m - 1):
        raise ValueError("site outside the grid's bounding box")
    return np.floor(v).astype(np.int64), np.floor(u).astype(np.int64)


def local_window(sites, m, x0, y0, h, np_: int):
    """Top-left node (is, js) of the (2 np)^2 window of every site (reading R5)."""
    if 2 * np_ > m:
        raise ValueError("neighbourhood wider than the grid")
    i0, j0 = _box(sites, m, x0, y0, h)
    is_ = np.clip(i0 - np_ + 1, 0, m - 2 * np_)
    js_ = np.clip(j0 - np_ + 1, 0, m - 2 * np_)
    return is_, js_


def local_weights(sites, m, x0, y0, h, sigma, theta, nu, np_: int, aniso=None):
    """Local-Kriging weights of Section 2.1 (b)-(c) and Section 3.1.

    For site s_i with window nodes S_i: W_1^i = K_21^i (K_11)^-1 and
    gamma_i = sigma^2 - K_21^i (K_11)^-1 K_12^i.  K_11 is the same for every
    site (stationarity, Section 3.6), so it is factored once.
    Returns idx (n x K int64 flat node indices), W (n x K), gamma (n).
    """
    sites = np.asarray(sites, dtype=np.float64)
    w = 2 * np_
    a, b = np.meshgrid(np.arange(w), np.arange(w), indexing="ij")
    a, b = a.reshape(-1), b.reshape(-1)
    dk = lag_distance(h * (b[:, None] - b[None, :]), h * (a[:, None] - a[None, :]), aniso)
    L11 = cholesky(matern(dk, sigma, theta, nu))
    is_, js_ = local_window(sites, m, x0, y0, h, np_)
    rows = is_[:, None] + a[None, :]
    cols = js_[:, None] + b[None, :]
    idx = rows * m + cols
    dx = sites[:, 0:1] - (x0 + cols * h)
    dy = sites[:, 1:2] - (y0 + rows * h)
    K21 = matern(lag_distance(dx, dy, aniso), sigma, theta, nu)      # n x K
    W = chol_solve(L11, K21.T).T                                      # K21 K11^-1
    gamma = sigma * sigma - np.sum(W * K21, axis=1)
    return idx, W, gamma


def nn_nodes(sites, m, x0, y0, h, k: int):
    """The k nearest grid nodes of every site (reading R7): candidates are the
    nodes of the 6 x 6 block around the site's box, clipped to the grid; the
    squared distance is (sx - x)^2 + (sy - y)^2 in float64 with no fused
    multiply-add, ties go to the smaller flat index.  Returns n x k flat indices."""
    sites = np.asarray(sites, dtype=np.float64)
    i0, j0 = _box(sites, m, x0, y0, h)
    off = np.arange(-2, 4)
    out = np.empty((sites.shape[0], k), dtype=np.int64)
    for s in range(sites.shape[0]):
        ii = i0[s] + off
        jj = j0[s] + off
        ii = ii[(ii >= 0) & (ii < m)]
        jj = jj[(jj >= 0) & (jj < m)]
        I, J = np.meshgrid(ii, jj, indexing="ij")
        I, J = I.reshape(-1), J.reshape(-1)
        dx = sites[s, 0] - (x0 + J * h)
        dy = sites[s, 1] - (y0 + I * h)
        d2 = dx * dx + dy * dy
        flat = I * m + J
        order = np.lexsort((flat, d2))
        out[s] = flat[order[:k]]
    return out


# ---------------------------------------------------------------------------
# Dense linear algebra (own code): Cholesky and triangular solves.
# ---------------------------------------------------------------------------
def cholesky(A):
    """Lower-triangular L with L L^T = A, column by column (Cholesky-Banachiewicz, left-looking)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    L = np.zeros((n, n))
    for j in range(n):
        s = A[j, j] - L[j, :j] @ L[j, :j]
        if not s > 0.0:
            raise np.linalg.LinAlgError("matrix is not positive definite")
        L[j, j] = math.sqrt(s)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def solve_lower(L, B):
    """X with L X = B by forward substitution (B may have several columns)."""
    X = np.array(B, dtype=np.float64, copy=True)
    for i in range(L.shape[0]):
        X[i] = (X[i] - L[i, :i] @ X[:i]) / L[i, i]
    return X


def solve_upper(U, B):
    """X with U X = B by back substitution."""
    X = np.array(B, dtype=np.float64, copy=True)
    n = U.shape[0]
    for i in range(n - 1, -1, -1):
        X[i] = (X[i] - U[i, i + 1:] @ X[i + 1:]) / U[i, i]
    return X


def chol_solve(L, B):
    """A^-1 B for A = L L^T."""
    return solve_upper(L.T, solve_lower(L, B))


def cov_matrix(p, q, sigma, theta, nu, aniso=None):
    """Cross-covariance C(||p_a - q_b||) between two point sets (Section 3, Eq. covmatrices);
    with anisotropy the length of the offset is |A (p_a - q_b)| (R18)."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    dx = p[:, 0:1] - q[None, :, 0]
    dy = p[:, 1:2] - q[None, :, 1]
    return matern(lag_distance(dx, dy, aniso), sigma, theta, nu)


# ---------------------------------------------------------------------------
# The conditional simulation algorithm (Section 2, steps 1-5) with the local
# Kriging (Section 2.1) and nearest-neighbour Kriging (Section 2.2) off-grid steps.
# ---------------------------------------------------------------------------
class Problem:
    """Everything computed once per covariance model and site set."""

    def __init__(self, m, x0, y0, h, sigma, theta, nu, tau2, max_growth=3, aniso=None):
        self.m, self.x0, self.y0, self.h = int(m), float(x0), float(y0), float(h)
        self.sigma, self.theta, self.nu, self.tau2 = float(sigma), float(theta), float(nu), float(tau2)
        self.aniso = None if aniso is None else (float(aniso[0]), float(aniso[1]))
        self.lam, self.P, self.eig_info = ce_eigenvalues(self.m, self.h, self.sigma, self.theta, self.nu,
                                                         max_growth, aniso=self.aniso)
        self.mode = None

    def cov(self, p, q):
        return cov_matrix(p, q, self.sigma, self.theta, self.nu, self.aniso)

    def grid(self):
        return grid_xy(self.m, self.x0, self.y0, self.h)


def setup_local(prob: Problem, sites, z, np_: int, joint_boxes: bool = False, factor=None):
    """Local Kriging set-up (Section 2.1 (b)-(d), Section 3.6): sparse W_1, gamma,
    the synthetic-data nugget sd phi_i = sqrt(tau^2 + gamma_i), and the factor of
    A = K_oo + tau^2 I used for prediction with tau^2 alone (reading R6).

    joint_boxes: sites that share a grid box are drawn jointly given the box's
    window (the multivariate variant of step (b), Section 2.1 and Section 3.6);
    see box_noise_factors.
    factor: the Cholesky routine for A (this module's `cholesky` by default; tests of
    thousands of sites may pass a library routine, which returns the same factor)."""
    sites = np.asarray(sites, dtype=np.float64)
    prob.mode = "local"
    prob.sites = sites
    prob.obs_xy = sites
    prob.zeff = np.asarray(z, dtype=np.float64)
    prob.idx, prob.W, prob.gamma = local_weights(sites, prob.m, prob.x0, prob.y0, prob.h,
                                                 prob.sigma, prob.theta, prob.nu, np_, prob.aniso)
    prob.phi = np.sqrt(prob.tau2 + prob.gamma)
    prob.boxes, prob.box_L = box_noise_factors(prob) if joint_boxes else ([], [])
    A = prob.cov(sites, sites) + prob.tau2 * np.eye(sites.shape[0])
    prob.L = (factor or cholesky)(A)
    return prob


def box_noise_factors(prob: Problem):
    """Noise factors of the grid boxes that hold more than one site (reading R16).

    Sites in one box share the box's window S_b (the window depends only on the
    box corner, reading R5), so their off-grid values are drawn together from the
    conditional law of y(s_b) given y(S_b): mean W_1 y as before, covariance
    Gamma_b = K(s_b, s_b) - K(s_b, S_b) K_11^-1 K(S_b, s_b), whose diagonal is the
    gamma_i of the single-site draw.  Adding the nugget, the synthetic observations
    of the box carry noise of covariance Gamma_b + tau^2 I, drawn as L_b eps_b with
    L_b its Cholesky factor (Section 3.6: diagonal blocks holding the Cholesky
    factor of the conditional covariance, phi_i for a site alone in its box).
    Returns (boxes, factors): caller indices of each such box in ascending order,
    and L_b in that order."""
    i0, j0 = _box(prob.sites, prob.m, prob.x0, prob.y0, prob.h)
    key = i0 * prob.m + j0
    gxy = prob.grid()
    boxes, factors = [], []
    for b in np.unique(key):
        mem = np.flatnonzero(key == b)
        if mem.size < 2:
            continue
        K21 = prob.cov(prob.sites[mem], gxy[prob.idx[mem[0]]])         # k x (2 np)^2
        gam = prob.cov(prob.sites[mem], prob.sites[mem]) - prob.W[mem] @ K21.T
        boxes.append(mem)
        factors.append(cholesky(gam + prob.tau2 * np.eye(mem.size)))
    return boxes, factors


def box_nodes(sites, m, x0, y0, h, np_: int):
    """Every site's (2 np)^2 window nodes (reading R5) as an n x (2 np)^2 array of
    flat indices: the n_p-order neighbourhood from which Section 3.2 takes the
    surrogate nodes of NN Kriging (n_N = n (2 n_p)^2 without overlaps)."""
    is_, js_ = local_window(sites, m, x0, y0, h, np_)
    w = 2 * np_
    a, b = np.meshgrid(np.arange(w), np.arange(w), indexing="ij")
    return (is_[:, None] + a.reshape(-1)[None, :]) * m + js_[:, None] + b.reshape(-1)[None, :]


def setup_nn(prob: Problem, sites, z, k: int, nodes=None, factor=None):
    """Nearest-neighbour Kriging set-up (Section 2.2, Section 3.2, reading R7).

    Surrogate nodes J_N: union of the k nearest grid nodes of every site, or of
    the per-site node lists `nodes` (n x K flat indices, e.g. box_nodes) when given.
    factor: the Cholesky routine (as in setup_local).
    Surrogate data: J_N K_go A^-1 z with A = K_oo + tau^2 I.
    Surrogate error variances sigma_N^2 = diag J_N (K_gg - K_go A^-1 K_og) J_N^T.
    Synthetic data nugget sd phi = sqrt(sigma_N^2 + tau^2); prediction matrix
    A_N = K_NN + tau^2 I + diag(sigma_N^2).
    """
    sites = np.asarray(sites, dtype=np.float64)
    prob.mode = "nn"
    prob.sites = sites
    prob.boxes, prob.box_L = [], []
    if nodes is None:
        nodes = nn_nodes(sites, prob.m, prob.x0, prob.y0, prob.h, k)
    J = np.unique(np.asarray(nodes).reshape(-1))
    prob.J = J
    gxy = prob.grid()[J]
    A = prob.cov(sites, sites) + prob.tau2 * np.eye(sites.shape[0])
    La = (factor or cholesky)(A)
    KoN = prob.cov(sites, gxy)                                # n x nN
    prob.zeff = KoN.T @ chol_solve(La, np.asarray(z, dtype=np.float64))
    V = solve_lower(La, KoN)                                  # L^-1 K_oN
    prob.sigN2 = prob.sigma ** 2 - np.sum(V * V, axis=0)
    prob.phi = np.sqrt(prob.sigN2 + prob.tau2)
    prob.obs_xy = gxy
    AN = prob.cov(gxy, gxy) + np.diag(prob.tau2 + prob.sigN2)
    prob.L = (factor or cholesky)(AN)
    return prob


def offgrid_local(prob: Problem, y):
    """y*_r(s_i) = sum_k W_1[i,k] y_r[idx[i,k]]: one sparse product per realization (Section 3.6)."""
    yf = y.reshape(y.shape[0], -1)
    return np.einsum("ik,rik->ri", prob.W, yf[:, prob.idx])


def offgrid_nn(prob: Problem, y):
    """J_N y_r: the grid values at the surrogate nodes (Section 3.2)."""
    return y.reshape(y.shape[0], -1)[:, prob.J]


def residuals(prob: Problem, y, seed: int, r_offset: int, event: int = 0):
    """Step 3 and the data side of step 4: e_r = z - z*_r, z*_r = y*_r + phi * eps*_r (R x n)."""
    ystar = offgrid_local(prob, y) if prob.mode == "local" else offgrid_nn(prob, y)
    n = ystar.shape[1]
    eps = np.stack([nugget_noise(seed, r_offset + r, n, event) for r in range(y.shape[0])])
    noise = prob.phi[None, :] * eps
    for mem, Lb in zip(getattr(prob, "boxes", []), getattr(prob, "box_L", [])):
        noise[:, mem] = eps[:, mem] @ Lb.T            # L_b eps_b per realization (reading R16)
    zstar = ystar + noise
    return prob.zeff[None, :] - zstar


def solve_B(prob: Problem, E):
    """B = A^-1 E^T (n x R), the Kriging weights of the residuals (Eq. condmvn)."""
    return chol_solve(prob.L, np.asarray(E, dtype=np.float64).T)


def correction(prob: Problem, y, B, nodes=None, tile: int = 4096):
    """Step 5: v_r = y_r + K_go B[:, r] at every grid node (or at `nodes` only).

    K_go B[:, r] = K_go A^-1 (z - z*_r) = y_hat - y_tilde_r, so v_r = y_hat + (y_r - y_tilde_r).
    """
    gxy = prob.grid()
    R = B.shape[1]
    yf = y.reshape(R, -1)
    nodes = np.arange(gxy.shape[0]) if nodes is None else np.asarray(nodes)
    out = np.empty((R, nodes.size))
    for t0 in range(0, nodes.size, tile):
        sel = nodes[t0:t0 + tile]
        out[:, t0:t0 + tile] = yf[:, sel] + (prob.cov(gxy[sel], prob.obs_xy) @ B).T
    return out


def correction_circulant(prob: Problem, y, B, nodes=None):
    """Step 5 in NN mode as a circulant convolution (Section 2.1 (a), Section 2.2):
    the surrogate nodes J_N lie on the grid, so K_gN B[:, r] is the 2-D circular
    convolution, on the P x P torus, of the embedding row c with B[:, r] placed at
    the nodes, restricted to the grid (every lag inside the grid is below P/2).
    With lambda = DFT2(c) as used for the unconditional fields (negative values
    clipped to zero), the convolution is IDFT2(lambda * DFT2(b)), the inverse
    taken as conj(DFT2(conj(.))) / N.  Equals `correction` up to the clipped part
    of the spectrum."""
    if prob.mode != "nn":
        raise ValueError("the circulant correction needs surrogate nodes on the grid (NN mode)")
    P = prob.lam.shape[0]
    m = prob.m
    R = B.shape[1]
    yf = np.asarray(y, dtype=np.float64).reshape(R, -1)
    nodes = np.arange(m * m) if nodes is None else np.asarray(nodes)
    out = np.empty((R, nodes.size))
    gi, gj = prob.J // m, prob.J % m
    for r in range(R):
        b = np.zeros((P, P))
        b[gi, gj] = B[:, r]
        u = np.conj(fft2(np.conj(prob.lam * fft2(b)))).real / (P * P)
        out[r] = yf[r, nodes] + u[:m, :m].reshape(-1)[nodes]
    return out


def trend_basis(xy, m: int, x0: float, y0: float, h: float, degree: int):
    """Regressors of the linear mean mu(s) = x(s)^T beta (Section 2, the standard
    geostatistical model): x(s) = [1] for degree 0, [1, u, v] for degree 1, with
    u = ((x - x0)/h - (m - 1)/2) / m and v likewise in y (centred, scaled grid units)."""
    xy = np.asarray(xy, dtype=np.float64)
    c = (m - 1) / 2.0
    u = ((xy[:, 0] - x0) / h - c) / m
    v = ((xy[:, 1] - y0) / h - c) / m
    cols = [np.ones(len(xy))] if degree == 0 else [np.ones(len(xy)), u, v]
    return np.stack(cols, axis=1)


def gls_beta(prob: Problem, X, W):
    """Generalized least squares (Section 2): beta = (X^T A^-1 X)^-1 X^T A^-1 W for
    each column of W (n x R), A the prediction matrix of `prob` (factor prob.L)."""
    AinvX = chol_solve(prob.L, X)
    S = X.T @ AinvX
    return chol_solve(cholesky(S), AinvX.T @ np.asarray(W, dtype=np.float64))


def condsim_trend(prob: Problem, degree: int, seed: int, r_offset: int, R: int, event: int = 0, nodes=None):
    """Conditional simulation with a linear mean estimated by GLS (Section 2):
    v = yhat(z) + y - yhat(z*) = y + yhat(z - z*), with the universal Kriging
    predictor yhat(w) = X_g beta(w) + K_go A^-1 (w - X beta(w)) and
    beta(w) = gls_beta(w).  Local Kriging only.  R x m x m, or R x len(nodes)."""
    if prob.mode != "local":
        raise ValueError("the trend model is built for local Kriging")
    y = ce_unconditional(prob.lam, prob.m, seed, r_offset, R, event)
    E = residuals(prob, y, seed, r_offset, event)                  # R x n: z - z*
    X = trend_basis(prob.sites, prob.m, prob.x0, prob.y0, prob.h, degree)
    beta = gls_beta(prob, X, E.T)                                   # p x R
    B = chol_solve(prob.L, E.T - X @ beta)                          # A^-1 (w - X beta)
    nodes = np.arange(prob.m * prob.m) if nodes is None else np.asarray(nodes)
    Xg = trend_basis(prob.grid()[nodes], prob.m, prob.x0, prob.y0, prob.h, degree)
    v = correction(prob, y, B, nodes) + (Xg @ beta).T
    return v.reshape(R, prob.m, prob.m) if v.shape[1] == prob.m * prob.m else v


def condsim(prob: Problem, seed: int, r_offset: int, R: int, event: int = 0, stages: bool = False):
    """The whole conditional simulation for R realizations: R x m x m float64."""
    y = ce_unconditional(prob.lam, prob.m, seed, r_offset, R, event)
    E = residuals(prob, y, seed, r_offset, event)
    B = solve_B(prob, E)
    v = correction(prob, y, B).reshape(R, prob.m, prob.m)
    if stages:
        return v, dict(y=y, E=E, B=B)
    return v


def condsim_at(prob: Problem, seed: int, r_offset: int, reals, nodes, event: int = 0):
    """v at selected realizations (absolute indices relative to r_offset) and grid nodes.

    Computes only the realization pairs that contain the selected realizations,
    so it stays cheap at full problem size.  Returns (v[len(reals), len(nodes)], y of those).
    """
    reals = list(reals)
    vs, ys = [], []
    for r in reals:
        base = r - (r % 2)
        y2 = ce_unconditional(prob.lam, prob.m, seed, r_offset + base, 2, event)
        y = y2[r % 2:r % 2 + 1]
        E = residuals(prob, y, seed, r_offset + r, event)
        B = solve_B(prob, E)
        vs.append(correction(prob, y, B, nodes)[0])
        ys.append(y[0])
    return np.stack(vs), np.stack(ys)


# ---------------------------------------------------------------------------
# Closed-form covariances (pins): Eq. (condmvn) and the Section 3.1 / 3.2 forms.
# ---------------------------------------------------------------------------
def exact_conditional_cov(prob: Problem, sites):
    """K_gg - K_go (K_oo + tau^2 I)^-1 K_og, the conditional covariance of Eq. (condmvn)."""
    gxy = prob.grid()
    Kgo = prob.cov(gxy, sites)
    L = cholesky(prob.cov(sites, sites) + prob.tau2 * np.eye(len(sites)))
    V = solve_lower(L, Kgo.T)
    return prob.cov(gxy, gxy) - V.T @ V


def local_approx_cov(prob: Problem):
    """Covariance of the approximate draws v = y_hat + (Lambda - I)... of Section 3.1 /
    Section 3.2, written as Cov((I - W_2 S) y) + W_2 diag(phi^2) W_2^T, where S is W_1
    (local) or J_N (NN), W_2 = K_go A^-1 with the prediction matrix A of the mode, and
    y has the grid covariance K_gg.  Valid for any mode set up on `prob`."""
    gxy = prob.grid()
    M = gxy.shape[0]
    Kgg = prob.cov(gxy, gxy)
    W2 = chol_solve(prob.L, prob.cov(prob.obs_xy, gxy)).T          # M x n
    S = np.zeros((prob.obs_xy.shape[0], M))
    if prob.mode == "local":
        np.add.at(S, (np.repeat(np.arange(S.shape[0]), prob.idx.shape[1]), prob.idx.reshape(-1)),
                  prob.W.reshape(-1))
    else:
        S[np.arange(prob.J.size), prob.J] = 1.0
    T = np.eye(M) - W2 @ S
    out = T @ Kgg @ T.T + (W2 * prob.phi ** 2) @ W2.T
    # jointly drawn boxes: the noise covariance block is L_b L_b^T instead of diag(phi^2)
    for mem, Lb in zip(getattr(prob, "boxes", []), getattr(prob, "box_L", [])):
        Wb = W2[:, mem]
        out += Wb @ (Lb @ Lb.T - np.diag(prob.phi[mem] ** 2)) @ Wb.T
    return out


def se_exact(prob: Problem, sites=None, nodes=None):
    """Exact prediction standard errors at the grid nodes (all, or `nodes`): the
    square roots of the diagonal of Eq. (condmvn)'s conditional covariance
    (Section 3.4's SE_E), sigma^2 - k_g^T (K_oo + tau^2 I)^-1 k_g, k_g = K(sites, g)."""
    sites = prob.sites if sites is None else np.asarray(sites, dtype=np.float64)
    gxy = prob.grid() if nodes is None else prob.grid()[np.asarray(nodes)]
    Kgo = prob.cov(gxy, sites)
    L = cholesky(prob.cov(sites, sites) + prob.tau2 * np.eye(len(sites)))
    V = solve_lower(L, Kgo.T)
    return np.sqrt(prob.sigma ** 2 - np.sum(V * V, axis=0))


def se_approx(prob: Problem, nodes=None):
    """Standard errors of the approximate draws at the grid nodes (Section 3.4's
    SE_L in local mode, SE_N in NN mode): the square roots of the diagonal of
    local_approx_cov, formed node by node.  With W_2 = K_go A^-1, U = S K_gg and
    Q = S K_gg S^T + D (D the noise covariance of the synthetic data),
    diag = sigma^2 - 2 rowsum(W_2 . U^T) + rowsum((W_2 Q) . W_2)."""
    grid = prob.grid()
    gxy = grid if nodes is None else grid[np.asarray(nodes)]
    n = prob.obs_xy.shape[0]
    W2 = chol_solve(prob.L, prob.cov(prob.obs_xy, gxy)).T           # nodes x n
    if prob.mode == "local":
        U = np.stack([prob.W[i] @ prob.cov(grid[prob.idx[i]], gxy) for i in range(n)])   # W_1^i K(S_i, g)
        win = grid[prob.idx.reshape(-1)]                              # every site's window, n K points
        Q = np.zeros((n, n))
        for j in range(n):                                            # Q[i, j] = W_1^i K(S_i, S_j) W_1^j^T
            Cj = prob.cov(win, grid[prob.idx[j]]) @ prob.W[j]
            Q[:, j] = np.sum(Cj.reshape(n, -1) * prob.W, axis=1)
    else:
        U = prob.cov(prob.obs_xy, gxy)                                # S = J_N
        Q = prob.cov(prob.obs_xy, prob.obs_xy)
    Q = Q + np.diag(prob.phi ** 2)
    for mem, Lb in zip(getattr(prob, "boxes", []), getattr(prob, "box_L", [])):
        Q[np.ix_(mem, mem)] += Lb @ Lb.T - np.diag(prob.phi[mem] ** 2)
    var = prob.sigma ** 2 - 2.0 * np.sum(W2 * U.T, axis=1) + np.sum((W2 @ Q) * W2, axis=1)
    return np.sqrt(var)


def relative_pct_error(se, se_ref):
    """100 (SE - SE_E) / SE_E per node (Section 3.4, E_L and E_N)."""
    return 100.0 * (np.asarray(se) - np.asarray(se_ref)) / np.asarray(se_ref)


def signif(x, digits: int):
    """x rounded to `digits` significant figures (half away from zero, on the decimal value)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = x != 0
    e = np.floor(np.log10(np.abs(x[nz]))) - (digits - 1)
    scale = 10.0 ** e
    q = np.abs(x[nz]) / scale
    out[nz] = np.sign(x[nz]) * np.floor(q + 0.5) * scale
    return out


def sig_fig_fraction(se, se_ref, digits: int = 3):
    """Fraction of nodes whose SE rounded to `digits` significant figures equals the
    exact SE so rounded (Section 3.4, Tables 1-2; reading R17)."""
    return float(np.mean(signif(se, digits) == signif(se_ref, digits)))


# ---------------------------------------------------------------------------
# Loss for the differentiation workload: the mean over realizations of the
# squared field in a window of the grid, plus the Gaussian log-likelihood of the
# data under A = K_oo + tau^2 I (the law of z in Eq. (condmvn)'s model).
# ---------------------------------------------------------------------------
def log_likelihood(prob: Problem):
    """l = -1/2 z^T A^-1 z - 1/2 log det A - n/2 log(2 pi) with A = K_oo + tau^2 I (local mode)."""
    z = prob.zeff
    alpha = chol_solve(prob.L, z)
    return float(-0.5 * z @ alpha - np.sum(np.log(np.diag(prob.L))) - 0.5 * z.size * math.log(2.0 * math.pi))


def window_loss(v, window):
    """(1/R) sum_r mean over the window of v_r^2; window = (i0, i1, j0, j1), half-open."""
    i0, i1, j0, j1 = window
    return float(np.mean(v[:, i0:i1, j0:j1] ** 2, axis=(1, 2)).mean())


def diff_loss(m, x0, y0, h, sigma, theta, nu, tau2, sites, z, np_, seed, r_offset, R, window, factor=None):
    """L(sigma, theta, tau^2, z) at fixed noise: window loss of the conditional draws plus the
    log-likelihood of the data.  Used for finite-difference gradients.  The draws are the
    five steps of `condsim`, with step 5 evaluated on the window's nodes only (the loss
    reads nothing else)."""
    prob = Problem(m, x0, y0, h, sigma, theta, nu, tau2, max_growth=3)
    setup_local(prob, sites, z, np_, factor=factor)
    y = ce_unconditional(prob.lam, prob.m, seed, r_offset, R)
    B = solve_B(prob, residuals(prob, y, seed, r_offset))
    i0, i1, j0, j1 = window
    ii, jj = np.meshgrid(np.arange(i0, i1), np.arange(j0, j1), indexing="ij")
    v = correction(prob, y, B, nodes=(ii * prob.m + jj).reshape(-1))
    return window_loss(v.reshape(R, i1 - i0, j1 - j0), (0, i1 - i0, 0, j1 - j0)) + log_likelihood(prob)
