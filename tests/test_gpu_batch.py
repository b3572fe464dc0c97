"""Batched events (many contexts in one call, or one captured graph) against
single calls and the oracle, and the autotuner."""
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


def _events():
    base = workloads.workload("plain64")
    specs = [dict(m=40, n=60, nu=0.5, range=0.2, R=3), dict(m=64, n=150, nu=1.5, range=0.12, R=8),
             dict(m=96, n=90, nu=0.5, range=0.08, R=5), dict(m=130, n=260, nu=1.5, range=0.1, R=2)]
    out = []
    for i, sp in enumerate(specs):
        wl = base.scaled(m=sp["m"], n=sp["n"], nu=sp["nu"], range=sp["range"], R=sp["R"], site_seed=40 + i,
                         sim_seed=700 + i)
        sites = workloads.make_sites(wl)
        out.append((wl, sites, workloads.make_data(wl, sites)))
    return out


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_batch_equals_single_calls_and_graph_replay(ce, prec):
    evs = _events()
    ctxs = [ce.Context.from_workload(wl).krige_weights(s, "local", np_=2, prec=prec) for wl, s, _ in evs]
    zs = [torch.tensor(z, dtype=torch.float32, device="cuda") for _, _, z in evs]
    Rs = [wl.R for wl, _, _ in evs]
    seeds = [wl.sim_seed for wl, _, _ in evs]
    offs = [0, 2, 0, 4]
    single = [c.condsim(z, R, sd, o).clone() for c, z, R, sd, o in zip(ctxs, zs, Rs, seeds, offs)]
    outs = [torch.full_like(x, float("nan")) for x in single]
    ce.condsim_batch(ctxs, zs, Rs, seeds, offs, outs, nstreams=3)
    torch.cuda.synchronize()
    for a, b in zip(outs, single):
        assert torch.equal(a, b)
    outs2 = [torch.full_like(x, float("nan")) for x in single]
    batch = ce.Batch(ctxs, zs, Rs, seeds, offs, outs2, nstreams=4)
    for _ in range(2):
        batch.launch()
        torch.cuda.synchronize()
        for a, b in zip(outs2, single):
            assert torch.equal(a, b)
    batch.close()


def test_batch_event_matches_oracle(ce):
    wl, sites, z = _events()[1]
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=2)
    out = torch.empty((wl.R, wl.m, wl.m), device="cuda")
    other = _events()[0]
    ctx2 = ce.Context.from_workload(other[0]).krige_weights(other[1], "local", np_=2)
    out2 = torch.empty((other[0].R, other[0].m, other[0].m), device="cuda")
    ce.condsim_batch([ctx, ctx2], [torch.tensor(z, dtype=torch.float32, device="cuda"),
                                   torch.tensor(other[2], dtype=torch.float32, device="cuda")],
                     [wl.R, other[0].R], [wl.sim_seed, 3], [0, 0], [out, out2], nstreams=2)
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    oracle.setup_local(prob, sites, z, 2)
    ref = oracle.condsim(prob, wl.sim_seed, 0, wl.R)
    v = out.cpu().numpy()
    assert np.abs(v - ref).max() / np.abs(ref).max() < 1e-5


def test_batch_rejects_repeated_context(ce):
    wl, sites, z = _events()[0]
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=2)
    zd = torch.tensor(z, dtype=torch.float32, device="cuda")
    o = torch.empty((wl.R, wl.m, wl.m), device="cuda")
    with pytest.raises(ce.CEError) as e:
        ce.condsim_batch([ctx, ctx], [zd, zd], [wl.R, wl.R], [1, 2], [0, 0], [o, o])
    assert e.value.status == ce.CE_ERR_ARG


def test_autotune_keeps_results(ce):
    wl = workloads.workload("plain64").scaled(m=160, n=300)
    sites = workloads.make_sites(wl)
    z = torch.tensor(workloads.make_data(wl, sites), dtype=torch.float32, device="cuda")
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=3, prec="f16x3")
    a = ctx.condsim(z, 12, 5).clone()
    ctx.autotune(12)
    b = ctx.condsim(z, 12, 5)
    torch.cuda.synchronize()
    assert float((a - b).abs().max() / a.abs().max()) < 1e-4
