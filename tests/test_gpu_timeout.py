"""A bounded device wait that runs out.

The tensor-core correction's epilogue waits (bounded) for each accumulator.  With
the bound set to zero try_wait rounds (ce_set_wait_limit) the first such wait gives
up at once: the launch records CE_ERR_TIMEOUT, lets its bulk copies and tensor-core
work finish, frees its tensor memory and returns.  The host reads the status through
ce_sync_status, and the context stays usable: with the bound restored the next call
draws the same fields as a fresh context.  Nothing here faults or hangs the GPU: the
wait that expires is the last in its role's loop and the drain waits keep their own
bounds."""
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


def _setup(ce, wl, n, prec="f16x3"):
    sites = workloads.make_sites(wl, n=n)
    z = torch.tensor(workloads.make_data(wl, sites), dtype=torch.float32, device="cuda")
    return ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_, prec=prec), z


@pytest.mark.parametrize("prec", ["f16x3", "tf32x3"])
def test_expired_wait_reports_timeout_and_context_recovers(ce, prec):
    wl = workloads.workload("plain64").scaled(m=96)
    ctx, z = _setup(ce, wl, 300, prec)
    ref = ctx.condsim(z, 12, wl.sim_seed).clone()
    ctx.sync()
    ctx.set_wait_limit(0)
    ctx.condsim(z, 12, wl.sim_seed)
    with pytest.raises(ce.CEError) as e:
        ctx.sync()
    assert e.value.status == ce.CE_ERR_TIMEOUT
    ctx.sync()                                   # the status was reported once
    ctx.set_wait_limit(1 << 22)
    again = ctx.condsim(z, 12, wl.sim_seed)
    ctx.sync()
    assert torch.equal(again, ref)


def test_expired_wait_in_a_batched_launch(ce):
    """The same in the persistent launch that serves several events: the first event's
    context carries the bound and the status."""
    evs = [workloads.workload("plain64").scaled(m=m, site_seed=40 + i) for i, m in enumerate((64, 96, 128))]
    ctxs, zs, outs = [], [], []
    for wl in evs:
        c, z = _setup(ce, wl, 150)
        ctxs.append(c)
        zs.append(z)
        outs.append(torch.empty((8, wl.m, wl.m), dtype=torch.float32, device="cuda"))
    ce.condsim_batch(ctxs, zs, [8] * 3, [wl.sim_seed for wl in evs], [0] * 3, outs, nstreams=3)
    for c in ctxs:
        c.sync()
    refs = [o.clone() for o in outs]
    ctxs[0].set_wait_limit(0)
    ce.condsim_batch(ctxs, zs, [8] * 3, [wl.sim_seed for wl in evs], [0] * 3, outs, nstreams=3)
    with pytest.raises(ce.CEError) as e:
        ctxs[0].sync()
    assert e.value.status == ce.CE_ERR_TIMEOUT
    ctxs[0].set_wait_limit(1 << 22)
    ce.condsim_batch(ctxs, zs, [8] * 3, [wl.sim_seed for wl in evs], [0] * 3, outs, nstreams=3)
    for c, o, r in zip(ctxs, outs, refs):
        c.sync()
        assert torch.equal(o, r)
    assert all(np.isfinite(o.cpu().numpy()).all() for o in outs)
