"""The standard-error study of Sections 3.3-3.4 on the GPU (ce_se_map).

Design: a 61 x 61 grid of unit spacing on [0, 60]^2, sigma^2 = 1, 35 sites with
both coordinates uniform on [0, 60] per configuration; Matern smoothness 1/2 or
3/2, the range set so that the correlation falls to 5% at 20, 45 or 70 units,
nugget sd tau = 0.1, 0.2, 0.3; local Kriging with neighbourhood orders
n_p = 1..4.  Per case it reports, over the configurations, the mean and sd of
the fraction of nodes whose local-Kriging standard error equals the exact one
after rounding both to three significant figures (Tables 1-2), and the mean
95th percentile over the nodes of |E_L| = 100 |SE_L - SE_E| / SE_E (Fig. 2).

    python -m paper_2109_11044_gb300.se_study --configs 50 --nu 0.5 [--json out.json]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

DISTANCES = (20.0, 45.0, 70.0)
TAUS = (0.1, 0.2, 0.3)


def range_for_5pct(distance: float, nu: float) -> float:
    """Range theta with C(distance) = 0.05 sigma^2 for the closed-form Matern covariances."""
    if nu == 0.5:
        return distance / math.log(20.0)
    # nu = 3/2: (1 + x) exp(-x) = 0.05 with x = sqrt(3) d / theta, by bisection on x
    lo, hi = 1.0, 20.0
    for _ in range(200):
        x = 0.5 * (lo + hi)
        if (1.0 + x) * math.exp(-x) > 0.05:
            lo = x
        else:
            hi = x
    return math.sqrt(3.0) * distance / (0.5 * (lo + hi))


def _signif3(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    e = np.floor(np.log10(np.abs(x))) - 2.0
    return np.floor(x / 10.0 ** e + 0.5) * 10.0 ** e


def run(configs: int, nu: float, orders=(1, 2, 3, 4), seed: int = 7):
    import torch  # noqa: F401  (device buffers)
    import paper_2109_11044_gb300 as ce
    import workloads
    out = []
    for dist in DISTANCES:
        theta = range_for_5pct(dist, nu)
        for tau in TAUS:
            frac = {p: [] for p in orders}
            p95 = {p: [] for p in orders}
            for c in range(configs):
                sites = workloads.se_study_sites(c, seed=seed)
                se_e = None
                for p in orders:
                    ctx = ce.Context(61, 0.0, 0.0, 1.0, 1.0, theta, nu, tau * tau).krige_weights(sites, "local", np_=p)
                    e, a = ctx.se_map(exact=se_e is None)
                    if se_e is None:
                        se_e = e.cpu().numpy().astype(np.float64).reshape(-1)
                    se_l = a.cpu().numpy().astype(np.float64).reshape(-1)
                    ctx.close()
                    frac[p].append(float(np.mean(_signif3(se_l) == _signif3(se_e))))
                    p95[p].append(float(np.percentile(np.abs(100.0 * (se_l - se_e) / se_e), 95)))
            row = {"nu": nu, "distance_5pct": dist, "theta": theta, "tau": tau, "configs": configs}
            for p in orders:
                row[f"np{p}"] = {"sig3_mean": float(np.mean(frac[p])), "sig3_sd": float(np.std(frac[p], ddof=1))
                                 if configs > 1 else 0.0, "p95_abs_pct_error": float(np.mean(p95[p]))}
            out.append(row)
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--configs", type=int, default=50)
    ap.add_argument("--nu", type=float, default=0.5, choices=[0.5, 1.5])
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    rows = run(args.configs, args.nu)
    hdr = f"{'theta':>6} {'tau':>4} " + " ".join(f"{'np' + str(p) + ' mean/sd':>16} {'p95%':>6}" for p in (1, 2, 3, 4))
    print(hdr)
    for r in rows:
        cells = " ".join(f"{r[f'np{p}']['sig3_mean']:>8.3f}/{r[f'np{p}']['sig3_sd']:<7.3f} {r[f'np{p}']['p95_abs_pct_error']:>6.3f}"
                         for p in (1, 2, 3, 4))
        print(f"{r['theta']:>6.2f} {r['tau']:>4.1f} {cells}")
    if args.json:
        with open(args.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
