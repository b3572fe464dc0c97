"""Ensemble moments (ce_ensemble_moments, ce_ensemble_stats) of the GPU's own
draws against FP64 sums of the same floats (the kernel sums in compensated
FP32 within a call: bar 2e-7 of the sum of magnitudes), accumulation over
calls, and the statistics against the closed-form standard errors (ce_se_map)."""
import numpy as np
import pytest

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


def test_moments_and_stats(ce):
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl, n=60)
    z = torch.tensor(workloads.make_data(wl, sites), dtype=torch.float32, device="cuda")
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=2)
    v = ctx.condsim(z, 10, 5)
    s, q = ctx.moments(v, 10)
    vn = v.cpu().numpy().astype(np.float64)
    # compensated FP32 sums within a call: within a few FP32 units of the sum of magnitudes
    scale = np.abs(vn).sum(axis=0)
    assert np.all(np.abs(s.cpu().numpy() - vn.sum(axis=0)) <= 2e-7 * scale + 1e-30)
    assert np.allclose(q.cpu().numpy(), (vn * vn).sum(axis=0), rtol=2e-7, atol=0)
    # two calls (realizations 0-5 and 6-9, pair-aligned offsets) accumulate to the one call
    a = ctx.condsim(z, 6, 5, r_offset=0)
    b = ctx.condsim(z, 4, 5, r_offset=6)
    sums = ctx.moments(a, 6)
    ctx.moments(b, 4, sums=sums)
    assert np.all(np.abs(sums[0].cpu().numpy() - s.cpu().numpy()) <= 4e-7 * scale + 1e-30)
    assert np.allclose(sums[1].cpu().numpy(), q.cpu().numpy(), rtol=4e-7, atol=0)
    mean, sd = ctx.ensemble_stats((s, q), 10)
    assert np.allclose(mean.cpu().numpy(), vn.mean(axis=0), rtol=1e-6, atol=1e-6)
    assert np.allclose(sd.cpu().numpy(), vn.std(axis=0, ddof=1), rtol=1e-5, atol=1e-6)


def test_ensemble_sd_matches_closed_form_standard_errors(ce):
    # 4000 draws with zero data: their spread is the approximate draws' standard error
    wl = workloads.workload("plain64")
    sites = workloads.make_sites(wl, n=60)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=2)
    z = torch.zeros(len(sites), dtype=torch.float32, device="cuda")
    sums = None
    for k in range(4):
        v = ctx.condsim(z, 1000, 11, r_offset=1000 * k)
        sums = ctx.moments(v, 1000, sums=sums)
    _, sd = ctx.ensemble_stats(sums, 4000)
    _, se = ctx.se_map(exact=False)
    ratio = (sd / se).cpu().numpy()
    assert abs(float(np.median(ratio)) - 1.0) < 0.01 and float(np.abs(ratio - 1).max()) < 0.08


def test_moments_odd_node_count(ce):
    # m = 61: an odd number of nodes
    sites = workloads.se_study_sites(0)
    ctx = ce.Context(61, 0.0, 0.0, 1.0, 1.0, 6.68, 0.5, 0.01).krige_weights(sites, "local", np_=2)
    z = torch.ones(len(sites), dtype=torch.float32, device="cuda")
    v = ctx.condsim(z, 7, 3)
    s, q = ctx.moments(v, 7)
    vn = v.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(s.cpu().numpy() - vn.sum(axis=0)) <= 2e-7 * np.abs(vn).sum(axis=0) + 1e-30)
    assert np.allclose(q.cpu().numpy(), (vn * vn).sum(axis=0), rtol=2e-7, atol=0)
