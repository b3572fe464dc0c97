"""Benchmark: conditional realizations per second of CE conditional simulation
on the 512 x 512 grid, n = 2000 stations (70% clustered), Matern 3/2,
local Kriging with a 6 x 6 neighbourhood, R = 100 realizations per call.

One step = one ce_condsim call: unconditional CE fields, off-grid values and
residuals, the solve, and the Kriging correction on every grid node, for R
realizations, with the data already on the device.  L2 is flushed (a 256 MB
write) between timed steps; each step is timed with CUDA events on the
launching stream.  Prints one JSON line, which also carries: the same call
through the host-buffer entry points (e2e), the plain FP32 form of the
correction, the accuracy of both forms against the FP64 oracle on sampled
realizations and nodes, nearest-neighbour Kriging, variants (joint grid boxes,
GLS plane mean, anisotropy), the closed-form standard errors, ensemble moments,
set-up times, and three other workloads: the 2048 x 2048 grid with 10000 sites
and R = 256 in every precision form of the correction, 64 uneven events in one
graph, and the pathwise gradient on the 1024 x 1024 grid.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec f16x3|bf16x3|fp32]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOAD = "shakemap512"
METRIC = "conditional realizations/s at 512^2 grid, n=2000 obs, R=100"
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the f16x3 tensor-core
# correction on the 512^2 x 2000-site x R=100 workload (profiles/correct_tc_shakemap512.md);
# None while the kernel has changed since the last capture
CORRECT_TC_DRAM_BYTES = None   # last capture (150.6 MB) predates the double-buffered cross accumulator
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# Warp instructions of the two P = 1024 ensemble passes per realization pair
# (smsp__inst_executed.sum of one launch of each pass over its pairs;
# profiles/fft1024_colnoise_shakemap512.md, fft1024_rowout_shakemap512.md): column
# pass with the noise, row pass
FFT1024_WARP_INSTR_PER_PAIR = (44.190568e6 / 13, 9.220123e6 / 13)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def config_dict(wl, prec):
    return {"workload": WORKLOAD, "grid": f"{wl.m}x{wl.m}", "n_obs": wl.n, "R": wl.R, "nu": wl.nu,
            "range": wl.range, "tau2": wl.tau2, "offgrid": f"local np={wl.np_}", "precision": prec,
            "l2": "flushed between timed steps (256 MB write)"}


class ClockSampler:
    """SM clock and clock-event (throttle) reasons during a timed region.

    Polls NVML (read-only queries: the current and maximum SM clock and the active
    clock-event reasons) every 2 ms from a thread, so that a region of a few tens of
    milliseconds still gets several samples; falls back to `nvidia-smi -lms 200` where
    the NVML library cannot be loaded.  Only samples taken between __enter__ and
    __exit__ count."""

    # clock-event reason bits of the NVML API
    REASON_BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                   0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index: int, period_s: float = 0.002):
        self.index = index
        self.period = period_s
        self.samples = []      # (sm_mhz, max_mhz, reasons)
        self.source = None
        self.proc = None
        self.stop = threading.Event()
        self.thread = None

    def _nvml(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
            lib.nvmlShutdown()
            raise OSError("no NVML handle")
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h, get_reasons

    def _poll(self, lib, h, get_reasons):
        import ctypes
        clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 and
                    get_reasons(h, ctypes.byref(rs)) == 0):
                self.samples.append((float(clk.value), float(mx.value),
                                     [nm for bit, nm in self.REASON_BITS.items() if rs.value & bit]))
            time.sleep(self.period)
        lib.nvmlShutdown()

    def _read_smi(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.proc.stdout:
            parts = [p.strip() for p in ln.strip().split(",")]
            if len(parts) < 7:
                continue
            try:
                self.samples.append((float(parts[0]), float(parts[1]),
                                     [nm for nm, val in zip(names, parts[3:7]) if val.lower() == "active"]))
            except ValueError:
                continue

    def __enter__(self):
        try:
            lib, h, get_reasons = self._nvml()
            self.source = "nvml, 2 ms"
            self.thread = threading.Thread(target=self._poll, args=(lib, h, get_reasons), daemon=True)
            self.thread.start()
            return self
        except (OSError, AttributeError):
            pass
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi, 200 ms"
            self.thread = threading.Thread(target=self._read_smi, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.stop.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        samples = list(self.samples)
        if not samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        reasons = sorted({r for _, _, rs in samples for r in rs})
        return {"sm_mhz": statistics.median(s[0] for s in samples), "sm_max_mhz": max(s[1] for s in samples),
                "reasons": reasons, "samples": len(samples), "source": self.source}


def cpu_reference(wl, steps, warmup, node_fraction=1):
    """The FP64 oracle as it stands, on a bounded sample: each step simulates one
    realization pair of the workload (FFT, residuals, solve) and the correction
    on 1/node_fraction of the grid nodes (every node by default); a partial
    correction's time is scaled to the whole grid.  Returns realizations/s, the
    threads used, the sample description and the mean wall time of a step (s)."""
    import oracle
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
    oracle.setup_local(prob, sites, z, wl.np_)
    M = wl.m * wl.m
    nodes = np.arange(0, M, node_fraction)
    times, walls = [], []
    for s in range(warmup + steps):
        t0 = time.perf_counter()
        y = oracle.ce_unconditional(prob.lam, wl.m, wl.sim_seed, 2 * s, 2)
        E = oracle.residuals(prob, y, wl.sim_seed, 2 * s)
        B = oracle.solve_B(prob, E)
        t1 = time.perf_counter()
        oracle.correction(prob, y, B, nodes)
        t2 = time.perf_counter()
        if s >= warmup:
            times.append((t1 - t0) + (t2 - t1) * M / nodes.size)
            walls.append(t2 - t0)
    per_pair = statistics.mean(times)
    try:
        from threadpoolctl import threadpool_info
        cores = max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    if node_fraction == 1:
        sample = f"{steps} realization pair(s) of {WORKLOAD} in full (CE FFT, residuals, solve, correction on every node)"
    else:
        sample = (f"{steps} realization pairs of {WORKLOAD} (CE FFT, residuals, solve in full; correction on 1/"
                  f"{node_fraction} of the nodes, scaled to the grid)")
    return 2.0 / per_pair, cores, sample, statistics.mean(walls)


def oracle_errors(samples):
    """Max and RMS relative errors of GPU draws against the FP64 oracle at sampled
    realizations and nodes, per workload and precision form.  samples: {workload name:
    (reals, nodes, {form: array len(reals) x len(nodes)})}.  Runs the oracle (the
    CPU-baseline leg of this benchmark)."""
    import oracle
    out = {}
    for name, (reals, nodes, forms) in samples.items():
        wl = workloads.workload(name)
        sites = workloads.make_sites(wl)
        z = workloads.make_data(wl, sites).astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        prob = oracle.Problem(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2)
        oracle.setup_local(prob, sites, z, wl.np_)
        ref, _ = oracle.condsim_at(prob, wl.sim_seed, 0, reals, nodes)
        den = float(np.abs(ref).max())
        res = {"sample": f"realizations {list(reals)} at {len(nodes)} random nodes; relative to max |oracle|",
               "oracle_s": time.perf_counter() - t0}
        for form, got in forms.items():
            got = np.asarray(got, dtype=np.float64)
            d = got - ref[:got.shape[0]]   # a form may hold the first realizations only
            res[form] = {"max_rel": float(np.abs(d).max() / den), "rms_rel": float(np.sqrt(np.mean(d * d)) / den)}
        out[name] = res
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = workloads.workload(WORKLOAD)
    t0 = time.perf_counter()
    value, cores, sample, wall = cpu_reference(wl, args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "realizations/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3,
            "step": "one realization pair of the workload, every stage in full",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(wl, "fp64"),
            "cpu_baseline": {"value": value, "unit": "realizations/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "realizations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def cufft_comparison(wl, P, R, dev, flush, stream, ours_ms):
    """A library FFT of the same ensemble, for comparison only (not on the product path):
    torch.fft.fft2 (cuFFT) of the (R + 1) / 2 complex P x P fields of one call, from fields
    already in memory (the noise is not generated, the transform not pruned), then the
    crop of the m x m corner into the real and imaginary realizations."""
    import torch
    pairs = (R + 1) // 2
    x = torch.randn((pairs, P, P), dtype=torch.complex64, device=dev)
    y = torch.empty((2 * pairs, wl.m, wl.m), dtype=torch.float32, device=dev)

    def step():
        w = torch.fft.fft2(x)
        y[0::2].copy_(w.real[:, :wl.m, :wl.m])
        y[1::2].copy_(w.imag[:, :wl.m, :wl.m])

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    fft_only = []
    for k, (a, b) in enumerate(evs):
        flush.fill_(float(k))
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    t_all = statistics.mean(a.elapsed_time(b) for a, b in evs)
    for k, (a, b) in enumerate(evs):
        flush.fill_(float(k))
        a.record(stream)
        torch.fft.fft2(x)
        b.record(stream)
    torch.cuda.synchronize()
    fft_only = statistics.mean(a.elapsed_time(b) for a, b in evs)
    del x, y
    torch.cuda.empty_cache()
    return {"library": "cuFFT through torch.fft.fft2 (complex64)", "pairs": pairs, "P": P,
            "ms_fft_and_crop": t_all, "ms_fft_only": fft_only, "ours_ms": ours_ms,
            "note": "the library timing starts from noise fields already in memory and transforms all P x P "
                    "outputs; ours generates the noise in the column pass and keeps only the m x m corner"}


def sample_device(out, reals, nodes):
    """out[reals][:, nodes] of an R x m x m device tensor, as a host array."""
    import torch
    flat = out.view(out.shape[0], -1)
    idx_r = torch.tensor(reals, device=out.device)
    idx_n = torch.tensor(nodes, device=out.device)
    return flat[idx_r][:, idx_n].cpu().numpy().astype(np.float64)


def sample_nodes(wl, count, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(wl.m * wl.m, count, replace=False))


PREC_FORMS = ("fp32", "f16x3", "bf16x3", "tf32x3")


def precision_leg(dev, flush, stream, world):
    """The 2048 x 2048 grid (P = 4096), exponential covariance, 10000 sites (7000
    uniform + 3 dense clusters), R = 256 per call, in every precision form of the
    correction: ms per call and per stage, and the draws at sampled realizations and
    nodes (compared with the oracle in the CPU-baseline leg)."""
    import torch
    import paper_2109_11044_gb300 as ce
    from paper_2109_11044_gb300 import shard
    wl = workloads.workload("precision2048")
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    zd = torch.tensor(z, dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_, prec="f16x3")
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    out = torch.empty((wl.R, wl.m, wl.m), dtype=torch.float32, device=dev)
    reals, nodes = [0, wl.R - 1], sample_nodes(wl, 2000, 11)
    res = {"workload": "precision2048", "grid": f"{wl.m}x{wl.m}", "P": ctx.info()["P"], "n_obs": wl.n, "R": wl.R,
           "setup_s": setup_s, "forms": {}}
    samples = {}
    for form in PREC_FORMS:
        ctx.set_precision(form)
        ctx.condsim(zd, wl.R, wl.sim_seed, 0, out=out)   # warm-up
        torch.cuda.synchronize()
        count = 2 if form == "fp32" else 3
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(count)]
        ctx.profile(True)
        for k in range(count):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            ctx.condsim(zd, wl.R, wl.sim_seed, 0, out=out)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        st, calls = ctx.profile_read()
        ctx.profile(False)
        ms = shard.max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in evs), dev)
        res["forms"][form] = {"ms_per_call": ms, "value": world * wl.R / (ms / 1e3), "unit": "realizations/s",
                              "stages_ms": {k: v / calls for k, v in st.items()}}
        samples[form] = sample_device(out, reals, nodes)
    # the FP64 form at 16 realizations per call (FP64 runs far below FP32 on this part):
    # realizations/s from that call, and its realization 0 compared with the oracle
    r64 = 16
    out64 = out[:r64]
    ctx.set_precision("fp64")
    ctx.profile(True)
    flush.fill_(0.0)
    e64 = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    e64[0].record(stream)
    ctx.condsim(zd, r64, wl.sim_seed, 0, out=out64)
    e64[1].record(stream)
    torch.cuda.synchronize()
    st, calls = ctx.profile_read()
    ctx.profile(False)
    ms = shard.max_over_ranks(e64[0].elapsed_time(e64[1]), dev)
    res["forms"]["fp64"] = {"ms_per_call": ms, "R": r64, "value": world * r64 / (ms / 1e3), "unit": "realizations/s",
                            "stages_ms": {k: v / calls for k, v in st.items()},
                            "note": "16 realizations per call; error on realization 0"}
    samples["fp64"] = sample_device(out64, reals[:1], nodes)
    ctx.close()
    del out, out64
    torch.cuda.empty_cache()
    return res, ("precision2048", (reals, nodes, samples))


def batch_leg(dev, flush, stream, world, rank, warmup, steps, prec):
    """64 uneven events (grid side 128-1024, 100-5000 sites, Matern 1/2 or 3/2), R = 32
    each: one captured graph of per-event calls on 8 parallel streams (autotuned
    correction), against the same calls one after another on one stream."""
    import torch
    import paper_2109_11044_gb300 as ce
    from paper_2109_11044_gb300 import shard
    evs = workloads.batch_events()
    t0 = time.perf_counter()
    ctxs, zs, outs = [], [], []
    for wl in evs:
        sites = workloads.make_sites(wl)
        ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_, prec=prec)
        ctx.prepare(wl.R)
        if prec != "fp32":
            ctx.autotune(wl.R)
        ctxs.append(ctx)
        zs.append(torch.tensor(workloads.make_data(wl, sites), dtype=torch.float32, device=dev))
        outs.append(torch.empty((wl.R, wl.m, wl.m), dtype=torch.float32, device=dev))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    Rs = [wl.R for wl in evs]
    seeds = [wl.sim_seed + 7919 * rank for wl in evs]
    offs = [0] * len(evs)
    batch = ce.Batch(ctxs, zs, Rs, seeds, offs, outs, nstreams=8)

    def timed(fn, count):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(count)]
        for k in range(count):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev)

    def serial():
        for c, z, R, sd, o, out in zip(ctxs, zs, Rs, seeds, offs, outs):
            c.condsim(z, R, sd, o, out=out)

    for _ in range(warmup):
        batch.launch()
        serial()
    torch.cuda.synchronize()
    ms = shard.max_over_ranks(timed(batch.launch, steps), dev)
    ms_serial = shard.max_over_ranks(timed(serial, max(3, steps // 2)), dev)
    real = sum(Rs)
    res = {"metric": "conditional realizations/s, 64 uneven events (grid 128-1024, n 100-5000), R=32 each",
           "value": world * real / (ms / 1e3), "unit": "realizations/s", "ms_per_step": ms,
           "events_per_s": world * len(evs) / (ms / 1e3), "setup_s": setup_s, "precision": prec,
           "schedule": "one CUDA graph: per-event steps on 8 parallel streams, then one persistent tensor-core "
                       "correction launch over all events' tiles (device work queue)",
           "grid_points_x_realizations_per_s": world * sum(wl.R * wl.m * wl.m for wl in evs) / (ms / 1e3),
           "serial_form": {"ms_per_step": ms_serial, "value": world * real / (ms_serial / 1e3),
                           "schedule": "the same calls one after another on one stream"}}
    batch.close()
    for c in ctxs:
        c.close()
    del outs
    torch.cuda.empty_cache()
    return res


def diff_leg(dev, flush, world, rank, steps):
    """Forward draws plus the pathwise gradient of the window loss plus the
    log-likelihood on the 1024 x 1024 grid, Matern 3/2, 3000 clustered sites,
    R = 64 (window rows and columns [412, 612)): one synchronous ce_condsim_grad
    call per step."""
    import torch
    import paper_2109_11044_gb300 as ce
    from paper_2109_11044_gb300 import shard
    wl = workloads.workload("diff1024")
    sites = workloads.make_sites(wl)
    zd = torch.tensor(workloads.make_data(wl, sites), dtype=torch.float32, device=dev)
    win = (412, 612, 412, 612)
    seed = wl.sim_seed + 7919 * rank
    t0 = time.perf_counter()
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_)
    out = torch.empty((wl.R, wl.m, wl.m), dtype=torch.float32, device=dev)
    ctx.condsim_grad(zd, wl.R, seed, win, out=out)   # also sets up the derivatives
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    ctx.condsim_grad(zd, wl.R, seed, win, out=out)
    times = []
    for k in range(steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, gt, gz, L = ctx.condsim_grad(zd, wl.R, seed, win, out=out)   # synchronous
        times.append(time.perf_counter() - t1)
    ms = shard.max_over_ranks(statistics.mean(times) * 1e3, dev)
    ll = ctx.loglik(zd)
    ctx.close()
    del out
    torch.cuda.empty_cache()
    return {"metric": "gradient steps/s (forward R=64 draws + dL/d(sigma, range, tau2, z)), 1024^2 grid, n=3000",
            "value": world / (ms / 1e3), "unit": "steps/s", "ms_per_step": ms, "R": wl.R, "window": list(win),
            "realizations_per_s_with_gradient": world * wl.R / (ms / 1e3), "setup_s": setup_s, "loss": L,
            "log_likelihood": ll, "grad_theta": gt, "api": "ce_condsim_grad (synchronous), ce_loglik"}



def init_ranks(rank, world, local):
    """Build the library (rank 0 first), join the NCCL group for N > 1 and
    select this rank's GPU; returns the device and a barrier function."""
    import torch
    from paper_2109_11044_gb300.build import build
    if rank == 0:
        build()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
        if rank != 0:
            build()
    torch.cuda.set_device(local)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
    return torch.device("cuda", local), barrier


def run_batch(args, rank, world, local):
    """64 uneven independent events (grid side 128-1024, 100-5000 sites, Matern
    1/2 or 3/2), R = 32 each: one captured graph of per-event calls on parallel
    streams, against the same calls issued one after another on one stream."""
    import torch
    import paper_2109_11044_gb300 as ce
    from paper_2109_11044_gb300 import shard
    dev, barrier = init_ranks(rank, world, local)
    evs = workloads.batch_events()
    t0 = time.perf_counter()
    ctxs, zs, outs = [], [], []
    for wl in evs:
        sites = workloads.make_sites(wl)
        ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_, prec=args.prec)
        ctx.prepare(wl.R)
        if args.prec != "fp32":
            ctx.autotune(wl.R)
        ctxs.append(ctx)
        zs.append(torch.tensor(workloads.make_data(wl, sites), dtype=torch.float32, device=dev))
        outs.append(torch.empty((wl.R, wl.m, wl.m), dtype=torch.float32, device=dev))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    Rs = [wl.R for wl in evs]
    seeds = [wl.sim_seed + 7919 * rank for wl in evs]
    offs = [0] * len(evs)
    batch = ce.Batch(ctxs, zs, Rs, seeds, offs, outs, nstreams=8)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for s in range(steps):
            flush.fill_(float(s))
            ev[s][0].record(stream)
            fn()
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev)

    def serial():
        for c, z, R, sd, o, out in zip(ctxs, zs, Rs, seeds, offs, outs):
            c.condsim(z, R, sd, o, out=out)

    for _ in range(args.warmup):
        batch.launch()
        serial()
    torch.cuda.synchronize()
    barrier()
    with ClockSampler(local) as clk:
        ms = timed(batch.launch, args.steps)
        barrier()
    ms_serial = timed(serial, max(3, args.steps // 2))
    ms = shard.max_over_ranks(ms, dev)
    real = sum(Rs)
    line = {"metric": "conditional realizations/s, 64 uneven events (grid 128-1024, n 100-5000), R=32 each",
            "value": world * real / (ms / 1e3), "unit": "realizations/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else f"f32+{args.prec}", "data": "synthetic",
            "config": {"workload": "batch64", "events": len(evs), "R_each": 32, "precision": args.prec,
                       "schedule": "one CUDA graph: per-event steps on 8 parallel streams, then one persistent tensor-core "
                       "correction launch over all events' tiles (device work queue)",
                       "l2": "flushed between timed steps (256 MB write)"},
            "serial_form": {"ms_per_step": ms_serial, "value": real / (ms_serial / 1e3),
                            "schedule": "the same calls one after another on one stream"},
            "events_per_s": world * len(evs) / (ms / 1e3), "setup_s": setup_s,
            "grid_points_x_realizations_per_s": world * sum(wl.R * wl.m * wl.m for wl in evs) / (ms / 1e3),
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_diff(args, rank, world, local):
    """Forward draws plus the pathwise gradient of the window loss plus the
    log-likelihood on the 1024 x 1024 grid, Matern 3/2, 3000 clustered sites,
    R = 64 (window rows and columns [412, 612)).  Also checks the gradient
    against central differences of the same GPU loss (relative step 1e-3)."""
    import torch
    import paper_2109_11044_gb300 as ce
    from paper_2109_11044_gb300 import shard
    dev, barrier = init_ranks(rank, world, local)
    wl = workloads.workload("diff1024")
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    zd = torch.tensor(z, dtype=torch.float32, device=dev)
    win = (412, 612, 412, 612)
    seed = wl.sim_seed + 7919 * rank
    t0 = time.perf_counter()
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_)
    out = torch.empty((wl.R, wl.m, wl.m), dtype=torch.float32, device=dev)
    ctx.condsim_grad(zd, wl.R, seed, win, out=out)   # also sets up the derivatives
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ctx.condsim_grad(zd, wl.R, seed, win, out=out)
    times = []
    torch.cuda.synchronize()
    barrier()
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            flush.fill_(float(s))
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, gt, gz, L = ctx.condsim_grad(zd, wl.R, seed, win, out=out)   # synchronous
            times.append(time.perf_counter() - t1)
    barrier()
    ms = shard.max_over_ranks(statistics.mean(times) * 1e3, dev)
    # central differences of the GPU loss, relative step 1e-3
    fd = []
    for name in ("sigma", "range", "tau2"):
        val = getattr(wl, name)
        hs = 1e-3 * val
        ls = []
        for sgn in (1, -1):
            c2 = ce.Context.from_workload(wl.scaled(**{name: val + sgn * hs})).krige_weights(sites, "local", np_=wl.np_)
            ls.append(c2.condsim_grad(zd, wl.R, seed, win, out=out)[3])
            c2.close()
        fd.append((ls[0] - ls[1]) / (2 * hs))
    line = {"metric": "gradient steps/s (forward R=64 draws + dL/d(sigma, range, tau2, z)), 1024^2 grid, n=3000",
            "value": world / (ms / 1e3), "unit": "steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "diff1024", "grid": "1024x1024", "n_obs": wl.n, "R": wl.R, "nu": wl.nu,
                       "window": list(win), "l2": "flushed between timed steps (256 MB write)"},
            "realizations_per_s_with_gradient": world * wl.R / (ms / 1e3), "setup_s": setup_s, "loss": L,
            "grad_theta": gt, "grad_theta_gpu_central_diff": fd,
            "grad_theta_rel_diff": [abs(a - b) / max(abs(b), 1e-30) for a, b in zip(gt, fd)],
            "grad_z_norm": float(gz.norm().item()), "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="f16x3", choices=["fp32", "f16x3", "bf16x3", "tf32x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-nn", action="store_true", help="skip the nearest-neighbour Kriging leg")
    ap.add_argument("--no-se", action="store_true", help="skip the closed-form standard-error leg")
    ap.add_argument("--no-aniso", action="store_true", help="skip the anisotropic-covariance leg")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the 2048^2 precision, 64-event batch and 1024^2 gradient legs")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "batch64", "diff1024"])
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch64":
        return run_batch(args, rank, world, local)
    if args.workload == "diff1024":
        return run_diff(args, rank, world, local)

    import torch
    import paper_2109_11044_gb300 as ce
    from paper_2109_11044_gb300 import shard
    dev, barrier = init_ranks(rank, world, local)

    wl = workloads.workload(WORKLOAD)
    sites = workloads.make_sites(wl)
    z = workloads.make_data(wl, sites)
    ctx = ce.Context.from_workload(wl).krige_weights(sites, "local", np_=wl.np_, prec=args.prec)
    R = wl.R
    ctx.prepare(R)
    if args.prec != "fp32":
        ctx.autotune(R)   # producer configuration of the tensor-core correction
    zd = torch.tensor(z, dtype=torch.float32, device=dev)
    out = torch.empty((R, wl.m, wl.m), dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()
    r_base = shard.weak_offset(R, rank)   # weak scaling: every rank draws its own R realizations

    for s in range(args.warmup):
        ctx.condsim(zd, R, wl.sim_seed, r_base, out=out)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    ctx.profile(True)   # events between the stages of every timed call
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        for s in range(args.steps):
            flush.fill_(float(s))
            ev[s][0].record(stream)
            ctx.condsim(zd, R, wl.sim_seed, r_base, out=out)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        t_wall = time.perf_counter() - t_wall0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(step_ms)
    # the timed call's draws at sampled realizations and nodes, for the accuracy check
    acc_reals, acc_nodes = [0, 1], sample_nodes(wl, 4096, 7)
    samples_main = {args.prec: sample_device(out, acc_reals, acc_nodes)}
    launches = ctx.info()["launches"]
    ms = shard.max_over_ranks(ms, dev)
    value = world * R / (ms / 1e3)

    stages, calls = ctx.profile_read()
    ctx.profile(False)
    stage_ms = {k: v / calls for k, v in stages.items()}

    # end to end through the host-buffer entry points: pinned z in, every step's fields
    # copied back to pinned host memory.  The pipelined call overlaps one step's copy-back
    # with the next step's computation; the L2 flush runs between steps inside the timing.
    zh = torch.tensor(z, dtype=torch.float32).pin_memory()
    oh = [torch.empty((R, wl.m, wl.m), dtype=torch.float32).pin_memory() for _ in range(2)]
    for k in range(2):
        ctx.condsim_host_async(zh, R, wl.sim_seed, r_base, oh[k])
    ctx.host_wait()
    barrier()
    t0 = time.perf_counter()
    for s in range(args.steps):
        flush.fill_(float(s))
        ctx.condsim_host_async(zh, R, wl.sim_seed, r_base, oh[s % 2])
    ctx.host_wait()
    e2e_ms = shard.max_over_ranks((time.perf_counter() - t0) / args.steps * 1e3, dev)
    # the synchronous call (returns after its copy-back), for reference
    sync_times = []
    for s in range(max(3, args.steps // 2)):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ctx.condsim_host(zh, R, wl.sim_seed, r_base, oh[0])
        sync_times.append(time.perf_counter() - t1)
    e2e_sync_ms = statistics.mean(sync_times) * 1e3

    # the plain FP32 form of the correction, same call, for comparison
    plain = None
    if args.prec != "fp32":
        ctx.set_precision("fp32")
        ctx.profile(True)
        for s in range(max(3, args.steps // 2)):
            flush.fill_(float(s))
            ctx.condsim(zd, R, wl.sim_seed, r_base, out=out)
        st2, c2 = ctx.profile_read()
        ctx.profile(False)
        samples_main["fp32"] = sample_device(out, acc_reals, acc_nodes)
        ctx.set_precision(args.prec)
        tot = sum(st2.values()) / c2
        plain = {"ms_per_step": tot, "value": R / (tot / 1e3), "correct_ms": st2["correct"] / c2}

    # the same workload with nearest-neighbour Kriging (k = 8 nearest nodes per site)
    nn = None
    if not args.no_nn:
        t0 = time.perf_counter()
        cnn = ce.Context.from_workload(wl).krige_weights(sites, "nn", k=wl.k_nn, prec=args.prec)
        cnn.prepare(R)
        if args.prec != "fp32":
            cnn.autotune(R)
        torch.cuda.synchronize()
        nn_setup = time.perf_counter() - t0
        for s in range(2):
            cnn.condsim(zd, R, wl.sim_seed, r_base, out=out)
        torch.cuda.synchronize()
        nsteps = max(3, args.steps // 2)
        evn = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        cnn.profile(True)
        for s in range(nsteps):
            flush.fill_(float(s))
            evn[s][0].record(stream)
            cnn.condsim(zd, R, wl.sim_seed, r_base, out=out)
            evn[s][1].record(stream)
        torch.cuda.synchronize()
        st3, c3 = cnn.profile_read()
        cnn.profile(False)
        nn_ms = shard.max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in evn), dev)
        nn = {"value": world * R / (nn_ms / 1e3), "unit": "realizations/s", "ms_per_step": nn_ms,
              "surrogate_nodes": cnn.info()["n_obs"], "setup_s": nn_setup, "precision": args.prec,
              "stages_ms": {k: v / c3 for k, v in st3.items()}}
        # the same draws with the correction as a circulant convolution on the torus
        cnn.set_nn_correction("circulant")
        cnn.prepare(R)
        for s in range(2):
            cnn.condsim(zd, R, wl.sim_seed, r_base, out=out)
        torch.cuda.synchronize()
        cnn.profile(True)
        for s in range(nsteps):
            flush.fill_(float(s))
            evn[s][0].record(stream)
            cnn.condsim(zd, R, wl.sim_seed, r_base, out=out)
            evn[s][1].record(stream)
        torch.cuda.synchronize()
        st4, c4 = cnn.profile_read()
        cnn.profile(False)
        circ_ms = shard.max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in evn), dev)
        nn["circulant_correction"] = {"value": world * R / (circ_ms / 1e3), "ms_per_step": circ_ms,
                                      "stages_ms": {k: v / c4 for k, v in st4.items()}}
        # the same call with the solve on the tensor cores (ce_set_solve_form): a faster
        # solve whose B error (about 1e-6) the correction's cancellation turns into a draw
        # accurate to about 1e-3 (the parity tests hold it to that bar)
        cnn.set_nn_correction("direct")
        cnn.set_solve_form("tensor")
        for s in range(2):
            cnn.condsim(zd, R, wl.sim_seed, r_base, out=out)
        torch.cuda.synchronize()
        cnn.profile(True)
        for s in range(nsteps):
            flush.fill_(float(s))
            evn[s][0].record(stream)
            cnn.condsim(zd, R, wl.sim_seed, r_base, out=out)
            evn[s][1].record(stream)
        torch.cuda.synchronize()
        st5, c5 = cnn.profile_read()
        cnn.profile(False)
        tcs_ms = shard.max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in evn), dev)
        nn["tensor_core_solve"] = {"value": world * R / (tcs_ms / 1e3), "ms_per_step": tcs_ms,
                                   "stages_ms": {k: v / c5 for k, v in st5.items()},
                                   "accuracy": "draws within 1e-3 of the oracle (B within about 1e-6)"}
        # both: the circulant correction with the tensor-core solve
        cnn.set_nn_correction("circulant")
        for s in range(2):
            cnn.condsim(zd, R, wl.sim_seed, r_base, out=out)
        torch.cuda.synchronize()
        cnn.profile(True)
        for s in range(nsteps):
            flush.fill_(float(s))
            evn[s][0].record(stream)
            cnn.condsim(zd, R, wl.sim_seed, r_base, out=out)
            evn[s][1].record(stream)
        torch.cuda.synchronize()
        st6, c6 = cnn.profile_read()
        cnn.profile(False)
        both_ms = shard.max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in evn), dev)
        nn["circulant_and_tensor_core_solve"] = {"value": world * R / (both_ms / 1e3), "ms_per_step": both_ms,
                                                 "stages_ms": {k: v / c6 for k, v in st6.items()}}
        cnn.close()

    # special-function and FP32 FMA throughput of this GPU, measured live: the peaks of the
    # correction (one reciprocal square root and one exp2 per Matern evaluation) and of the
    # FP32 products
    units = ce.unit_rates(stream)
    fp32_peak = 2.0 * units["fma"] / 1e12

    # ensemble moments of the timed call's draws (per-node FP64 sums): an HBM-bound pass
    mom_times = []
    sums = ctx.moments(out, R, stream=stream)
    for s in range(3):
        flush.fill_(float(s))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.moments(out, R, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        mom_times.append(a.elapsed_time(b))
    mom_ms = shard.max_over_ranks(statistics.mean(mom_times), dev)
    mom_bytes = 4.0 * R * wl.m * wl.m + 16.0 * wl.m * wl.m
    del sums

    # set-up, timed on a fresh context after everything is warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx2 = ce.Context.from_workload(wl)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ctx2.krige_weights(sites, "local", np_=wl.np_, prec=args.prec)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    ctx2.close()
    setup = {"ce_setup_s": t1 - t0, "ce_krige_weights_s": t2 - t1}

    # the same call with the variants that change one stage: sites sharing a grid box drawn
    # jointly (the residual step), and a GLS plane as the mean (solve and correction steps)
    def time_calls(c, count):
        for s in range(2):
            c.condsim(zd, R, wl.sim_seed, r_base, out=out)
        torch.cuda.synchronize()
        evv = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(count)]
        c.profile(True)
        for s in range(count):
            flush.fill_(float(s))
            evv[s][0].record(stream)
            c.condsim(zd, R, wl.sim_seed, r_base, out=out)
            evv[s][1].record(stream)
        torch.cuda.synchronize()
        stv, cn = c.profile_read()
        c.profile(False)
        t = shard.max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in evv), dev)
        return {"value": world * R / (t / 1e3), "unit": "realizations/s", "ms_per_step": t,
                "stages_ms": {k: v / cn for k, v in stv.items()}}
    variants = {}
    nb = ctx.set_box_joint(True)
    variants["joint_grid_boxes"] = dict(time_calls(ctx, max(3, args.steps // 2)), shared_boxes=nb)
    ctx.set_box_joint(False)
    ctx.set_trend(1)
    variants["gls_plane_mean"] = time_calls(ctx, max(3, args.steps // 2))
    ctx.set_trend(-1)

    # the same call with a geometric anisotropy (range * 0.5 across the direction 0.6 rad):
    # the anisotropic tensor-core correction maps each site's offset once per chunk
    aniso = None
    if not args.no_aniso:
        ca = ce.Context.from_workload(wl).set_anisotropy(0.5, 0.6).krige_weights(sites, "local", np_=wl.np_,
                                                                                  prec=args.prec)
        ca.prepare(R)
        for s in range(2):
            ca.condsim(zd, R, wl.sim_seed, r_base, out=out)
        torch.cuda.synchronize()
        na = max(3, args.steps // 2)
        eva = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(na)]
        ca.profile(True)
        for s in range(na):
            flush.fill_(float(s))
            eva[s][0].record(stream)
            ca.condsim(zd, R, wl.sim_seed, r_base, out=out)
            eva[s][1].record(stream)
        torch.cuda.synchronize()
        sta, ca_n = ca.profile_read()
        ca.profile(False)
        an_ms = shard.max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in eva), dev)
        aniso = {"value": world * R / (an_ms / 1e3), "unit": "realizations/s", "ms_per_step": an_ms,
                 "anisotropy": {"ratio": 0.5, "angle_rad": 0.6}, "P": ca.info()["P"],
                 "stages_ms": {k: v / ca_n for k, v in sta.items()}}
        ca.close()

    # closed-form standard errors at every node (exact, and of the approximate draws), no draws
    se = None
    if not args.no_se:
        ctx.se_map(stream=stream)
        se_times = []
        for s in range(2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.se_map(stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            se_times.append(a.elapsed_time(b))
        se_ms = shard.max_over_ranks(statistics.mean(se_times), dev)
        Mn = wl.m * wl.m
        # two products of the M x n covariance rows with n x n matrices (A^-1, then Q)
        se_flops = 2 * 2.0 * Mn * wl.n * wl.n
        se = {"api": "ce_se_map (exact and approximate)", "ms": se_ms, "nodes_per_s": world * Mn / (se_ms / 1e3),
              "useful_tflops": se_flops / (se_ms / 1e3) / 1e12, "peak_fp32_tflops": fp32_peak,
              "peak_source": "measured FP32 FMA rate (ce_unit_rates)",
              "frac": se_flops / (se_ms / 1e3) / 1e12 / fp32_peak,
              "note": "FP32 CUDA-core products with the hi/lo pair issue 2x the useful flops; "
                      "includes the per-call work-buffer allocation"}

    # the other workloads: the precision forms at 2048^2, the 64-event batch, the gradient at 1024^2
    legs, samples_p2048 = {}, None
    if not args.no_legs:
        legs["precision2048"], samples_p2048 = precision_leg(dev, flush, stream, world)
        legs["batch64"] = batch_leg(dev, flush, stream, world, rank, 2, max(3, args.steps // 4), args.prec)
        legs["diff1024"] = diff_leg(dev, flush, world, rank, 5)

    pk, pk_kind = peaks()
    M, n = wl.m * wl.m, wl.n
    flops = 2.0 * M * n * R
    corr_s = stage_ms["correct"] / 1e3
    # The correction evaluates M x n covariances (2 special-function operations
    # each) and contracts them with R weights; the evaluations bound it.
    roof = {"kernel": "Kriging correction (" + ("FP32 CUDA cores" if args.prec == "fp32" else
                                                "tcgen05 " + args.prec) + "), 512^2 x 2000 sites x R=100",
            "bound": "alu", "achieved": M * n / corr_s / 1e12, "peak": units["matern_evals"] / 1e12,
            "unit": "Teval/s (Matern evaluations)",
            "peak_source": "measured on this GPU (ce_unit_rates: chained ex2(-sqrt(d2)) on every SM; "
                           f"ex2 {units['ex2'] / 1e12:.2f} T/s, sqrt {units['sqrt'] / 1e12:.2f} T/s)",
            "traffic": CORRECT_TC_DRAM_BYTES if args.prec == "f16x3" else None}
    if args.prec == "f16x3":
        roof["traffic_unit"] = "bytes per launch (dram read + write, one ncu capture of this kernel)"
        roof["algorithmic_bytes"] = 2.0 * R * M * 4
    roof["frac"] = roof["achieved"] / roof["peak"]
    if args.prec == "fp32":
        roof["fma"] = {"achieved_tflops": flops / corr_s / 1e12, "peak_tflops": fp32_peak,
                       "peak_source": "measured FP32 FMA rate (ce_unit_rates)",
                       "frac": flops / corr_s / 1e12 / fp32_peak}
    else:
        roof["tensor"] = {"achieved_tflops": flops / corr_s / 1e12, "peak_tflops": pk["bf16_tflops"],
                          "peak_source": f"{pk_kind} dense bf16 (f16 same rate)",
                          "frac": flops / corr_s / 1e12 / pk["bf16_tflops"],
                          "note": "useful 2*M*n*R flops; the hi/lo refinement issues 3x as many"}
    fft_bytes = (R + 1) // 2 * (10 * 2 ** 20) * (wl.m / 512) ** 2
    # without pruning or in-register noise: the P x P noise field written and read, and both
    # full P x P passes through memory (about 40 MiB per pair at P = 1024)
    fft_bytes_unpruned = (R + 1) // 2 * 40 * 2 ** 20 * (wl.m / 512) ** 2
    line = {
        "metric": METRIC, "value": value, "unit": "realizations/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else f"f32+{args.prec}",
        "data": "synthetic", "config": config_dict(wl, args.prec),
        "grid_points_x_realizations_per_s": value * M,
        "roofline": roof,
        "stages_ms": stage_ms,
        "fft_hbm": {"algorithmic_bytes": fft_bytes, "unpruned_bytes": fft_bytes_unpruned,
                    "achieved_gbs": fft_bytes / (stage_ms["unconditional"] / 1e3) / 1e9,
                    "peak_gbs": pk["hbm_gbs"], "peak_source": pk_kind},
        "e2e": {"value": world * R / (e2e_ms / 1e3), "unit": "realizations/s", "h2d_bytes_per_step": 4 * n,
                "d2h_bytes_per_step": 4 * R * M, "api": "ce_condsim_host_async (pipelined) + ce_host_wait",
                "synchronous_call": {"value": world * R / (e2e_sync_ms / 1e3), "api": "ce_condsim_host"}},
        "gpu_launches": launches * args.steps,
        "gpu_launches_per_step": launches,
        "wall_s_timed": t_wall,
    }
    line["fft_hbm"]["frac"] = line["fft_hbm"]["achieved_gbs"] / line["fft_hbm"]["peak_gbs"]
    # the bytes that must reach DRAM are only the fields written (the intermediate stays in L2),
    # so the stage is bound by instruction issue: its warp instructions against the issue peak
    pairs = (R + 1) // 2
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_peak = sm_count * 4 * pk.get("sm_max_mhz", 2070.0) * 1e6   # one warp instruction per scheduler per clock
    if ctx.info()["P"] == 1024:
        winstr = pairs * sum(FFT1024_WARP_INSTR_PER_PAIR)
        line["fft_hbm"]["output_bytes"] = pairs * 2 * 4 * M
        line["fft_hbm"]["issue"] = {
            "warp_instructions_per_call": winstr, "achieved_per_s": winstr / (stage_ms["unconditional"] / 1e3),
            "peak_per_s": issue_peak, "frac": winstr / (stage_ms["unconditional"] / 1e3) / issue_peak,
            "peak_source": f"{sm_count} SMs x 4 schedulers x {pk.get('sm_max_mhz', 2070.0):.0f} MHz",
            "count_source": "ncu smsp__inst_executed.sum per pair of the two passes"}
    if plain is not None:
        line["plain_fp32"] = plain
    line.update(legs)
    if nn is not None:
        line["nn_kriging"] = nn
    if se is not None:
        line["standard_errors"] = se
    if aniso is not None:
        line["anisotropic"] = aniso
    line.update(variants)
    line["cufft_comparison"] = cufft_comparison(wl, ctx.info()["P"], R, dev, flush, stream, stage_ms["unconditional"])
    line["ensemble_moments"] = {"api": "ce_ensemble_moments", "ms": mom_ms, "bytes": mom_bytes,
                                "achieved_gbs": mom_bytes / (mom_ms / 1e3) / 1e9, "peak_gbs": pk["hbm_gbs"],
                                "frac": mom_bytes / (mom_ms / 1e3) / 1e9 / pk["hbm_gbs"]}
    line["setup"] = dict(setup, incl_setup_value=R / (setup["ce_setup_s"] + setup["ce_krige_weights_s"] + ms / 1e3),
                         note="one call of R realizations including a fresh ce_setup and ce_krige_weights")
    line["clocks"] = clk.summary()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, _ = cpu_reference(wl, steps=1, warmup=0)
        line["cpu_baseline"] = {"value": v, "unit": "realizations/s", "cores": cores, "kind": "oracle", "sample": sample}
        # accuracy of the timed draws (and of the other forms) against the oracle
        todo = {WORKLOAD: (acc_reals, acc_nodes, samples_main)}
        if samples_p2048 is not None:
            todo[samples_p2048[0]] = samples_p2048[1]
        errs = oracle_errors(todo)
        line["accuracy"] = dict(errs[WORKLOAD], tolerance_fp32_paths=1e-5)
        if plain is not None:
            a, b = errs[WORKLOAD][args.prec]["max_rel"], errs[WORKLOAD]["fp32"]["max_rel"]
            line["plain_fp32"]["max_rel_error"] = b
            line["plain_fp32"]["same_error"] = (
                f"both forms within the 1e-5 FP32 tolerance on the same sample: {args.prec} {a:.2e}, fp32 {b:.2e}"
                if max(a, b) < 1e-5 else f"not the same error class: {args.prec} {a:.2e}, fp32 {b:.2e}")
        if "precision2048" in errs:
            for form, e in errs["precision2048"].items():
                if form in line["precision2048"]["forms"]:
                    line["precision2048"]["forms"][form]["error"] = e
            line["precision2048"]["error_sample"] = errs["precision2048"]["sample"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
