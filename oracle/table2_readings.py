"""Readings of nearest-neighbour Kriging (Section 3.2) tried against Table 2.

TEST INFRASTRUCTURE ONLY (a study on the oracle's side; the CUDA library never
runs it).  Section 3.2 prints its NN formulas with inconsistent dimensions, so
the surrogate model can be read several ways.  This script computes, on the
paper's design (Section 3.3: 61 x 61 grid of unit spacing on [0, 60]^2, 35
uniform sites, exponential covariance, sigma^2 = 1), the fraction of grid nodes
whose NN standard error equals the exact one after rounding both to three
significant figures (reading R17), for each candidate reading and
neighbourhood order, next to what Table 2 prints.

Candidates (every one takes surrogate data at the grid nodes J_N and the
exact standard error SE_E of Eq. (condmvn) as the reference):
  r7          the library's reading: sigma_N^2 = diag J_N (K_gg - K_go A^-1 K_og) J_N^T
              with A = K_oo + tau^2 I, prediction matrix K_NN + tau^2 I + diag(sigma_N^2),
              SE_N^2 = sigma^2 - k_g^T (K_NN + tau^2 I + Sigma_N)^-1 k_g;
  r7_knn      the same with each site's (2 n_p)^2 nearest nodes instead of its box window;
  noise_free  sigma_N^2 from Kriging with noise-free data (K_oo^-1, the printed K_22^-1);
  no_tau      prediction matrix K_NN + Sigma_N (the printed tau^2 left out);
  full_sigma  the full error covariance J_N (K_gg - K_go A^-1 K_og) J_N^T + tau^2 I
              in place of its diagonal;
  mse         not an ensemble spread: the root mean-squared error of the NN
              predictor k_g^T (K_NN + tau^2 I + Sigma_N)^-1 zhat_N against the
              field, under the true joint law of the surrogate data
              zhat_N = J_N K_go A^-1 z.
n_p = "full" takes every grid node as a surrogate.  Dense solves use LAPACK
through numpy (a library primitive; the design is 3721 nodes).

    python -m oracle.table2_readings [--configs 6]
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import ce_oracle as o  # noqa: E402
import workloads  # noqa: E402

M_SIDE = 61
READINGS = ("r7", "r7_knn", "noise_free", "no_tau", "full_sigma", "mse")
ORDERS = (1, 2, 3, "full")


def _solve_spd(S, B):
    L = np.linalg.cholesky(S)
    return np.linalg.solve(L.T, np.linalg.solve(L, B))


def _knn_nodes(sites, k):
    """The k nearest grid nodes of every site by distance (ties to the smaller flat index)."""
    g = o.grid_xy(M_SIDE, 0.0, 0.0, 1.0)
    out = np.empty((len(sites), k), dtype=np.int64)
    flat = np.arange(g.shape[0])
    for s, p in enumerate(sites):
        d2 = (g[:, 0] - p[0]) ** 2 + (g[:, 1] - p[1]) ** 2
        out[s] = flat[np.lexsort((flat, d2))[:k]]
    return out


def fractions(theta: float, tau: float, config: int, readings=READINGS, orders=ORDERS) -> dict:
    """{(reading, order): fraction} for one configuration of the design."""
    tau2 = tau * tau
    prob = o.Problem(M_SIDE, 0.0, 0.0, 1.0, 1.0, theta, 0.5, tau2)
    sites = workloads.se_study_sites(config)
    g = prob.grid()
    Kgg = prob.cov(g, g)
    Kgo = prob.cov(g, sites)
    Koo = prob.cov(sites, sites)
    se_e = o.se_exact(prob, sites)
    Q = Kgo @ _solve_spd(Koo + tau2 * np.eye(len(sites)), Kgo.T)       # K_go A^-1 K_og
    P_t = Kgg - Q
    P_0 = Kgg - Kgo @ np.linalg.solve(Koo, Kgo.T)                      # noise-free data
    out = {}
    for order in orders:
        sets = {}
        if order == "full":
            sets["box"] = np.arange(M_SIDE * M_SIDE)
            sets["knn"] = sets["box"]
        else:
            sets["box"] = np.unique(o.box_nodes(sites, M_SIDE, 0.0, 0.0, 1.0, order))
            sets["knn"] = np.unique(_knn_nodes(sites, (2 * order) ** 2))
        for reading in readings:
            J = sets["knn" if reading == "r7_knn" else "box"]
            KgN, KNN = Kgg[:, J], Kgg[np.ix_(J, J)]
            if reading == "noise_free":
                D = np.diag(np.diag(P_0)[J] + tau2)
            elif reading == "no_tau":
                D = np.diag(np.diag(P_t)[J])
            elif reading == "full_sigma":
                D = P_t[np.ix_(J, J)] + tau2 * np.eye(J.size)
            else:
                D = np.diag(np.diag(P_t)[J] + tau2)
            Wt = _solve_spd(KNN + D, KgN.T)                                # (K_NN + D)^-1 k_g, columns
            if reading == "mse":
                QN = Q[np.ix_(J, J)]
                var = 1.0 - 2.0 * np.sum(Wt * Q[:, J].T, axis=0) + np.sum(Wt * (QN @ Wt), axis=0)
            else:
                var = 1.0 - np.sum(Wt * KgN.T, axis=0)
            se = np.sqrt(np.maximum(var, 0.0))
            out[(reading, order)] = o.sig_fig_fraction(se, se_e)
    return out


def table2() -> dict:
    """Table 2 as printed: {(theta, tau): [np1, np2, np3, full] means}."""
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                        "se_sigfig_table2.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return {(float(r[0]), float(r[1])): [float(r[k]) for k in (2, 4, 6, 8)] for r in rows}


def run(configs: int, cases=((6.68, 0.1), (15.02, 0.2), (23.37, 0.3))):
    printed = table2()
    res = {}
    for theta, tau in cases:
        acc = {}
        for c in range(configs):
            for key, v in fractions(theta, tau, c).items():
                acc.setdefault(key, []).append(v)
        res[(theta, tau)] = {k: float(np.mean(v)) for k, v in acc.items()}
    return res, printed


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--configs", type=int, default=6)
    args = ap.parse_args()
    res, printed = run(args.configs)
    for (theta, tau), r in res.items():
        tab = printed[(theta, tau)]
        print(f"theta {theta} tau {tau}   Table 2: " + "  ".join(f"{v:.3f}" for v in tab))
        for reading in READINGS:
            print(f"  {reading:<11}" + "  ".join(f"{r[(reading, od)]:.3f}" for od in ORDERS))


if __name__ == "__main__":
    main()
