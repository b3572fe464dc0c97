"""Named synthetic workloads and their seeded generators.

Every workload lives on the unit square [0,1]^2 with an m x m grid of nodes at
spacing h = 1/(m-1) (the paper's 61 nodes on [0,60], Section 3.3, rescaled).
Sites are uniform or ShakeMap-like clustered; the data at the sites are a
smooth stationary random field plus an independent nugget.

The field is drawn with random Fourier features of the Matern spectral
density (a sum of cosines with random frequencies), not with the circulant
embedding or Kriging machinery that the method itself uses, so this module
shares no arithmetic with either implementation of the method.  Only the
statistics of the inputs matter for the method's timings; parity is checked on
whatever inputs these generators produce.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    m: int                 # grid side; M = m*m nodes
    sigma: float           # marginal standard deviation (sill sigma^2)
    range: float           # Matern range theta
    nu: float              # smoothness, 0.5 or 1.5
    tau2: float            # nugget variance
    n: int                 # number of observation sites
    layout: str            # "uniform", "cluster70" or "uniform+3clusters"
    np_: int               # local-Kriging neighbourhood order; (2 np)^2 nodes
    k_nn: int              # nearest-neighbour count for NN Kriging
    R: int                 # realizations per call
    site_seed: int         # seed of the site and data generators
    sim_seed: int          # Philox key of the conditional simulation

    @property
    def x0(self) -> float:
        return 0.0

    @property
    def y0(self) -> float:
        return 0.0

    @property
    def h(self) -> float:
        return 1.0 / (self.m - 1)

    def scaled(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


WORKLOADS = {
    # 64x64 grid, exponential covariance, 200 uniform sites, 4x4 neighbourhood, R=10.
    "plain64": Workload("plain64", 64, 1.0, 0.1, 0.5, 0.05, 200, "uniform", 2, 8, 10, 0, 1001),
    # 512x512 grid, Matern 3/2, 2000 stations (70% clustered), 6x6 neighbourhood / 8-NN, R=100.
    "shakemap512": Workload("shakemap512", 512, 0.6, 0.15, 1.5, 0.1, 2000, "cluster70", 3, 8, 100, 1, 1002),
    # 2048x2048 grid, exponential covariance, 7000 uniform + 3 x 1000 clustered sites, R=256.
    "precision2048": Workload("precision2048", 2048, 1.0, 0.08, 0.5, 0.05, 10000, "uniform+3clusters",
                              4, 8, 256, 3, 1004),
    # 1024x1024 grid, Matern 3/2, 3000 clustered sites, R=64.
    "diff1024": Workload("diff1024", 1024, 1.0, 0.12, 1.5, 0.08, 3000, "cluster70", 4, 8, 64, 4, 1005),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def _clustered(rng: np.random.Generator, count: int, centre: np.ndarray, sd: float) -> np.ndarray:
    """`count` points from N(centre, sd^2 I), redrawn until they fall inside [0,1]^2."""
    out = np.empty((0, 2))
    while out.shape[0] < count:
        pts = centre + sd * rng.standard_normal((2 * (count - out.shape[0]) + 8, 2))
        keep = np.all((pts >= 0.0) & (pts <= 1.0), axis=1)
        out = np.concatenate([out, pts[keep]], axis=0)
    return out[:count]


def make_sites(wl: Workload, n: int | None = None, seed: int | None = None) -> np.ndarray:
    """Observation sites as an (n, 2) float64 array of (x, y) in [0,1]^2."""
    n = wl.n if n is None else n
    rng = np.random.default_rng(wl.site_seed if seed is None else seed)
    if wl.layout == "uniform":
        return rng.uniform(0.0, 1.0, size=(n, 2))
    if wl.layout == "cluster70":
        n_c = int(round(0.7 * n))
        epi = rng.uniform(0.2, 0.8, size=2)
        pts = np.concatenate([_clustered(rng, n_c, epi, 0.1),
                              rng.uniform(0.0, 1.0, size=(n - n_c, 2))], axis=0)
        return pts[rng.permutation(n)]
    if wl.layout == "uniform+3clusters":
        n_c = (3 * n) // 10
        per = [n_c // 3, n_c // 3, n_c - 2 * (n_c // 3)]
        parts = [rng.uniform(0.0, 1.0, size=(n - n_c, 2))]
        for cnt in per:
            parts.append(_clustered(rng, cnt, rng.uniform(0.2, 0.8, size=2), 0.03))
        pts = np.concatenate(parts, axis=0)
        return pts[rng.permutation(n)]
    raise ValueError(f"unknown layout {wl.layout!r}")


def se_study_sites(config: int, n: int = 35, extent: float = 60.0, seed: int = 7) -> np.ndarray:
    """Sites of configuration `config` of the standard-error study's design (Section 3.3:
    35 sites with both coordinates uniform on [0, 60], a 61 x 61 grid of unit spacing)."""
    rng = np.random.default_rng([seed, config])
    return rng.uniform(0.0, extent, size=(n, 2))


def _spectral_frequencies(rng: np.random.Generator, count: int, rng_range: float, nu: float) -> np.ndarray:
    """Frequencies with density proportional to (2 nu / theta^2 + |w|^2)^-(nu+1) in 2-D.

    That density is a bivariate Student-t with 2 nu degrees of freedom and
    scale 1/theta, sampled as Z / (theta sqrt(W / (2 nu))), W ~ chi^2_{2 nu}.
    """
    z = rng.standard_normal((count, 2))
    w = rng.chisquare(2.0 * nu, size=(count, 1))
    return z / (rng_range * np.sqrt(w / (2.0 * nu)))


def make_data(wl: Workload, sites: np.ndarray, seed: int | None = None, n_features: int = 4096) -> np.ndarray:
    """Data z at the sites: a random-Fourier-feature field plus N(0, tau^2) nugget."""
    rng = np.random.default_rng(10_000 + (wl.site_seed if seed is None else seed))
    omega = _spectral_frequencies(rng, n_features, wl.range, wl.nu)
    phase = rng.uniform(0.0, 2.0 * math.pi, size=n_features)
    field = wl.sigma * math.sqrt(2.0 / n_features) * np.cos(sites @ omega.T + phase).sum(axis=1)
    return field + math.sqrt(wl.tau2) * rng.standard_normal(sites.shape[0])


def batch_events(count: int = 64, seed: int = 2, R: int = 32):
    """Uneven independent events for the batched workload: grid side uniform in
    {128, 192, 256, 384, 512, 768, 1024}, n log-uniform in [100, 5000], Matern
    nu in {1/2, 3/2}, range uniform in [0.05, 0.3], nugget uniform in
    [0.02, 0.2], sigma = 1, local neighbourhood np = 4, R realizations each,
    uniform sites."""
    rng = np.random.default_rng(seed)
    sides = [128, 192, 256, 384, 512, 768, 1024]
    out = []
    for e in range(count):
        m = int(rng.choice(sides))
        n = int(round(math.exp(rng.uniform(math.log(100), math.log(5000)))))
        nu = float(rng.choice([0.5, 1.5]))
        out.append(Workload(f"event{e}", m, 1.0, float(rng.uniform(0.05, 0.3)), nu, float(rng.uniform(0.02, 0.2)), n,
                            "uniform", 4, 8, R, 100 + e, 5000 + e))
    return out
