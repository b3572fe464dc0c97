"""Python binding of the CE conditional-simulation library (C ABI in
``include/ce_condsim.h``).  Argument marshalling only: every step of the
computation runs in the CUDA kernels of ``libce_condsim.so``.  PyTorch supplies
device memory and streams.  There is no CPU fallback: loading fails loudly if
the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libce_condsim.so")

CE_OK, CE_ERR_ARG, CE_ERR_EMBED, CE_ERR_NOT_SPD, CE_ERR_CUDA, CE_ERR_TIMEOUT, CE_ERR_OOM, CE_ERR_STATE = range(8)
CE_LOCAL, CE_NN = 0, 1
PRECISIONS = {"fp32": 0, "f16x3": 1, "bf16x3": 2, "tf32x3": 3, "fp64": 4}
SOLVE_FORMS = {"fp32": 0, "tensor": 1}
ARRAYS = {"sqrt_lambda": 0, "idx": 1, "W": 2, "phi": 3, "J": 4}

# Every symbol the header declares; tests check that the library exports them.
EXPORTS = (
    "ce_setup", "ce_krige_weights", "ce_set_precision", "ce_condsim", "ce_condsim_host",
    "ce_unconditional", "ce_residuals", "ce_solve", "ce_correct", "ce_philox", "ce_normals",
    "ce_get_info", "ce_copy_array", "ce_sync_status", "ce_last_error", "ce_destroy",
    "ce_profile", "ce_profile_read", "ce_unconditional_static", "ce_condsim_prepare",
    "ce_condsim_batch", "ce_batch_create", "ce_batch_launch", "ce_batch_destroy", "ce_autotune",
    "ce_condsim_grad", "ce_condsim_host_async", "ce_host_wait", "ce_set_nn_correction", "ce_set_trend",
    "ce_set_box_joint", "ce_se_map", "ce_unit_rates", "ce_ensemble_moments", "ce_ensemble_stats",
    "ce_set_anisotropy", "ce_loglik", "ce_set_wait_limit", "ce_set_solve_form",
)
STAGES = ("unconditional", "residuals", "solve", "correct")


def unit_rates(stream=None) -> dict:
    """ce_unit_rates: measured special-function and FP32 FMA throughput of the current GPU (per second)."""
    e, r, m, f = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load_library().ce_unit_rates(ctypes.byref(e), ctypes.byref(r), ctypes.byref(m), ctypes.byref(f),
                                        _stream(stream)), None)
    return {"ex2": e.value, "sqrt": r.value, "matern_evals": m.value, "fma": f.value}


class CEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[status {status}] {msg}")
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("h", ctypes.c_double)]


class _Cov(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("range", ctypes.c_double), ("nu", ctypes.c_double), ("tau2", ctypes.c_double)]


class _Nbhd(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("np", ctypes.c_int), ("k", ctypes.c_int), ("prec", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("P", ctypes.c_int), ("n", ctypes.c_int), ("n_obs", ctypes.c_int),
                ("K", ctypes.c_int), ("growth", ctypes.c_int), ("clipped", ctypes.c_longlong),
                ("lambda_min", ctypes.c_double), ("lambda_max", ctypes.c_double),
                ("clipped_mass", ctypes.c_double), ("logdet", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("launches", ctypes.c_int), ("solve_tc", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load (once) and type the shared library; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing (run paper_2109_11044_gb300.build.build())")
    lib = ctypes.CDLL(path)
    P, I, U64, D, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t
    sig = {
        "ce_setup": (I, [ctypes.POINTER(P), ctypes.POINTER(_Grid), ctypes.POINTER(_Cov), I, P]),
        "ce_krige_weights": (I, [P, P, I, ctypes.POINTER(_Nbhd)]),
        "ce_set_precision": (I, [P, I]),
        "ce_set_nn_correction": (I, [P, I]),
        "ce_set_trend": (I, [P, I]),
        "ce_set_anisotropy": (I, [P, D, D, P]),
        "ce_set_box_joint": (I, [P, I, P]),
        "ce_se_map": (I, [P, P, P, P]),
        "ce_unit_rates": (I, [ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D), P]),
        "ce_ensemble_moments": (I, [P, P, I, P, P, I, P]),
        "ce_ensemble_stats": (I, [P, P, P, D, P, P, P]),
        "ce_condsim": (I, [P, P, I, U64, U64, P, P]),
        "ce_condsim_host": (I, [P, P, I, U64, U64, P, P]),
        "ce_condsim_host_async": (I, [P, P, I, U64, U64, P, P]),
        "ce_host_wait": (I, [P]),
        "ce_unconditional": (I, [P, I, U64, U64, P, P]),
        "ce_residuals": (I, [P, P, P, I, U64, U64, P, P]),
        "ce_solve": (I, [P, P, I, P, P]),
        "ce_correct": (I, [P, P, I, P, P]),
        "ce_philox": (I, [P, I, U64, P, P]),
        "ce_normals": (I, [P, I, U64, P, P]),
        "ce_get_info": (I, [P, ctypes.POINTER(_Info)]),
        "ce_copy_array": (I, [P, I, P, SZ]),
        "ce_sync_status": (I, [P]),
        "ce_last_error": (ctypes.c_char_p, [P]),
        "ce_destroy": (None, [P]),
        "ce_profile": (I, [P, I]),
        "ce_unconditional_static": (I, [P, I, U64, U64, P, P]),
        "ce_condsim_prepare": (I, [P, I]),
        "ce_condsim_batch": (I, [P, P, P, P, P, P, I, I, P]),
        "ce_batch_create": (I, [ctypes.POINTER(P), P, P, P, P, P, P, I, I]),
        "ce_batch_launch": (I, [P, P]),
        "ce_batch_destroy": (None, [P]),
        "ce_autotune": (I, [P, I, P]),
        "ce_condsim_grad": (I, [P, P, I, U64, U64, ctypes.POINTER(ctypes.c_int), P, ctypes.POINTER(ctypes.c_double), P,
                                ctypes.POINTER(ctypes.c_double), P]),
        "ce_profile_read": (I, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
        "ce_loglik": (I, [P, P, ctypes.POINTER(ctypes.c_double), P]),
        "ce_set_wait_limit": (I, [P, ctypes.c_uint]),
        "ce_set_solve_form": (I, [P, I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, ctx=None):
    if status != CE_OK:
        msg = load_library().ce_last_error(ctx).decode(errors="replace")
        raise CEError(status, msg)


def _stream(stream=None) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _dev_ptr(t, dtype=None) -> int:
    import torch
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    return t.data_ptr()


class Context:
    """One covariance model on one grid (``ce_setup``) plus, after
    :meth:`krige_weights`, one set of observation sites."""

    def __init__(self, m: int, x0: float, y0: float, h: float, sigma: float, range: float, nu: float,
                 tau2: float, max_growth: int = 3, stream=None):
        lib = load_library()
        self._ctx = ctypes.c_void_p()
        g = _Grid(m, x0, y0, h)
        c = _Cov(sigma, range, nu, tau2)
        _check(lib.ce_setup(ctypes.byref(self._ctx), ctypes.byref(g), ctypes.byref(c), max_growth, _stream(stream)))
        self.m = m
        self.theta = (float(sigma), float(range), float(tau2))
        self._grid = (m, x0, y0, h, float(nu), max_growth)
        self._sites = None

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(wl.m, wl.x0, wl.y0, wl.h, wl.sigma, wl.range, wl.nu, wl.tau2, **kw)

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            load_library().ce_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def krige_weights(self, sites, mode: str = "local", np_: int = 3, k: int = 8, prec: str = "fp32"):
        xy = np.ascontiguousarray(np.asarray(sites, dtype=np.float64).reshape(-1, 2))
        nb = _Nbhd(CE_LOCAL if mode == "local" else CE_NN, np_, k, PRECISIONS[prec])
        _check(load_library().ce_krige_weights(self._ctx, xy.ctypes.data, xy.shape[0], ctypes.byref(nb)), self._ctx)
        self.n = xy.shape[0]
        self._sites = (xy.copy(), mode, np_, k, prec)
        return self

    def with_theta(self, sigma: float, range: float, tau2: float) -> "Context":
        """A new context on the same grid, smoothness and sites with the covariance
        parameters (sigma, range, tau^2) replaced (ce_setup + ce_krige_weights again)."""
        m, x0, y0, h, nu, growth = self._grid
        ctx = Context(m, x0, y0, h, sigma, range, nu, tau2, max_growth=growth)
        if self._sites is not None:
            xy, mode, np_, k, prec = self._sites
            ctx.krige_weights(xy, mode, np_=np_, k=k, prec=prec)
        return ctx

    def set_precision(self, prec: str):
        _check(load_library().ce_set_precision(self._ctx, PRECISIONS[prec]), self._ctx)

    def set_solve_form(self, form: str):
        """ce_set_solve_form: "fp32" (compensated FP32 products, the default) or "tensor"
        (tcgen05 f16 hi/lo split; B within about 1e-6 of the FP64 solve)."""
        _check(load_library().ce_set_solve_form(self._ctx, SOLVE_FORMS[form]), self._ctx)

    def set_wait_limit(self, iterations: int):
        """ce_set_wait_limit: bound (try_wait rounds) on the tensor-core correction's
        accumulator waits; 0 makes them give up at once (the call reports CE_ERR_TIMEOUT)."""
        _check(load_library().ce_set_wait_limit(self._ctx, int(iterations)), self._ctx)
        return self

    def set_nn_correction(self, method: str):
        """ce_set_nn_correction: "direct" (covariance tiles) or "circulant" (FFT convolution)."""
        _check(load_library().ce_set_nn_correction(self._ctx, {"direct": 0, "circulant": 1}[method]), self._ctx)
        return self

    def set_anisotropy(self, ratio: float, angle: float, stream=None):
        """ce_set_anisotropy: range * ratio across the direction at `angle` (radians); the
        off-grid set-up is discarded (call krige_weights again)."""
        _check(load_library().ce_set_anisotropy(self._ctx, float(ratio), float(angle), _stream(stream)), self._ctx)
        return self

    def set_trend(self, degree: int):
        """ce_set_trend: -1 zero mean, 0 constant, 1 plane (GLS mean, universal Kriging)."""
        _check(load_library().ce_set_trend(self._ctx, int(degree)), self._ctx)
        return self

    def set_box_joint(self, on: bool = True) -> int:
        """ce_set_box_joint: draw the sites that share a grid box jointly; returns the
        number of boxes holding more than one site."""
        nb = ctypes.c_int(0)
        _check(load_library().ce_set_box_joint(self._ctx, 1 if on else 0, ctypes.byref(nb)), self._ctx)
        return nb.value

    def se_map(self, exact: bool = True, approx: bool = True, stream=None):
        """ce_se_map: closed-form standard errors at every node, (se_exact, se_approx) as
        m x m float32 device tensors (None where not requested)."""
        import torch
        e = torch.empty((self.m, self.m), dtype=torch.float32, device="cuda") if exact else None
        a = torch.empty((self.m, self.m), dtype=torch.float32, device="cuda") if approx else None
        _check(load_library().ce_se_map(self._ctx, _dev_ptr(e, torch.float32) if exact else None,
                                        _dev_ptr(a, torch.float32) if approx else None, _stream(stream)), self._ctx)
        return e, a

    def moments(self, v, R: int, sums=None, stream=None):
        """ce_ensemble_moments: per-node FP64 (sum, sum of squares) over the R realizations of v
        (R x m x m float32, device); added to `sums` when given (a pair from an earlier call)."""
        import torch
        acc = sums is not None
        if sums is None:
            sums = (torch.empty((self.m, self.m), dtype=torch.float64, device=v.device),
                    torch.empty((self.m, self.m), dtype=torch.float64, device=v.device))
        _check(load_library().ce_ensemble_moments(self._ctx, _dev_ptr(v, torch.float32), int(R),
                                                  _dev_ptr(sums[0], torch.float64), _dev_ptr(sums[1], torch.float64),
                                                  1 if acc else 0, _stream(stream)), self._ctx)
        return sums

    def ensemble_stats(self, sums, count: float, stream=None):
        """ce_ensemble_stats: (mean, sd) maps, m x m float32, from moments over `count` draws."""
        import torch
        mean = torch.empty((self.m, self.m), dtype=torch.float32, device=sums[0].device)
        sd = torch.empty_like(mean)
        _check(load_library().ce_ensemble_stats(self._ctx, _dev_ptr(sums[0], torch.float64),
                                                _dev_ptr(sums[1], torch.float64), float(count),
                                                _dev_ptr(mean, torch.float32), _dev_ptr(sd, torch.float32),
                                                _stream(stream)), self._ctx)
        return mean, sd

    def info(self) -> dict:
        inf = _Info()
        _check(load_library().ce_get_info(self._ctx, ctypes.byref(inf)), self._ctx)
        return {f: getattr(inf, f) for f, _ in _Info._fields_}

    def array(self, name: str) -> np.ndarray:
        inf = self.info()
        which = ARRAYS[name]
        if name == "sqrt_lambda":
            out = np.empty((inf["P"], inf["P"]), np.float32)
        elif name in ("idx", "W"):
            out = np.empty((inf["n_obs"], inf["K"]), np.int32 if name == "idx" else np.float32)
        else:
            out = np.empty(inf["n_obs"], np.int32 if name == "J" else np.float32)
        _check(load_library().ce_copy_array(self._ctx, which, out.ctypes.data, out.nbytes), self._ctx)
        return out

    # --- the hot path -----------------------------------------------------
    def condsim(self, z, R: int, seed: int, r_offset: int = 0, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((R, self.m, self.m), dtype=torch.float32, device=z.device)
        _check(load_library().ce_condsim(self._ctx, _dev_ptr(z, torch.float32), R, seed, r_offset,
                                         _dev_ptr(out, torch.float32), _stream(stream)), self._ctx)
        return out

    def condsim_host(self, z_host, R: int, seed: int, r_offset: int = 0, out_host=None, stream=None):
        import torch
        if out_host is None:
            out_host = torch.empty((R, self.m, self.m), dtype=torch.float32, pin_memory=True)
        if z_host.dtype != torch.float32 or z_host.is_cuda or out_host.is_cuda:
            raise ValueError("condsim_host takes float32 host tensors")
        _check(load_library().ce_condsim_host(self._ctx, z_host.data_ptr(), R, seed, r_offset, out_host.data_ptr(),
                                              _stream(stream)), self._ctx)
        return out_host

    def condsim_host_async(self, z_host, R: int, seed: int, r_offset: int = 0, out_host=None, stream=None):
        """ce_condsim_host_async: queue the draws with host buffers and return at once; the
        fields are in out_host after host_wait().  Keep z_host and out_host alive until then."""
        import torch
        if out_host is None:
            out_host = torch.empty((R, self.m, self.m), dtype=torch.float32, pin_memory=True)
        if z_host.dtype != torch.float32 or z_host.is_cuda or out_host.is_cuda:
            raise ValueError("condsim_host_async takes float32 host tensors")
        _check(load_library().ce_condsim_host_async(self._ctx, z_host.data_ptr(), R, seed, r_offset,
                                                    out_host.data_ptr(), _stream(stream)), self._ctx)
        return out_host

    def host_wait(self):
        _check(load_library().ce_host_wait(self._ctx), self._ctx)

    # --- single steps -----------------------------------------------------
    def unconditional(self, R: int, seed: int, r_offset: int = 0, out=None, device="cuda", stream=None):
        import torch
        if out is None:
            out = torch.empty((R, self.m, self.m), dtype=torch.float32, device=device)
        _check(load_library().ce_unconditional(self._ctx, R, seed, r_offset, _dev_ptr(out, torch.float32),
                                               _stream(stream)), self._ctx)
        return out

    def unconditional_static(self, R: int, seed: int, r_offset: int = 0, out=None, device="cuda", stream=None):
        """ce_unconditional_static: the same fields with no device allocation inside the call
        (the FFT intermediate sits in the library's fixed device buffer)."""
        import torch
        if out is None:
            out = torch.empty((R, self.m, self.m), dtype=torch.float32, device=device)
        _check(load_library().ce_unconditional_static(self._ctx, R, seed, r_offset, _dev_ptr(out, torch.float32),
                                                      _stream(stream)), self._ctx)
        return out

    def residuals(self, y, z, R: int, seed: int, r_offset: int = 0, stream=None):
        import torch
        E = torch.empty((R, self.info()["n_obs"]), dtype=torch.float32, device=y.device)
        _check(load_library().ce_residuals(self._ctx, _dev_ptr(y, torch.float32), _dev_ptr(z, torch.float32), R,
                                           seed, r_offset, _dev_ptr(E), _stream(stream)), self._ctx)
        return E

    def solve(self, E, stream=None):
        import torch
        B = torch.empty_like(E)
        _check(load_library().ce_solve(self._ctx, _dev_ptr(E, torch.float32), E.shape[0], _dev_ptr(B),
                                       _stream(stream)), self._ctx)
        return B

    def correct(self, B, y, stream=None):
        import torch
        _check(load_library().ce_correct(self._ctx, _dev_ptr(B, torch.float32), B.shape[0],
                                         _dev_ptr(y, torch.float32), _stream(stream)), self._ctx)
        return y

    def profile(self, enable: bool):
        _check(load_library().ce_profile(self._ctx, 1 if enable else 0), self._ctx)

    def profile_read(self):
        """Summed per-stage milliseconds of the profiled ce_condsim calls, and their count."""
        ms = (ctypes.c_double * len(STAGES))()
        calls = ctypes.c_int()
        _check(load_library().ce_profile_read(self._ctx, ms, ctypes.byref(calls)), self._ctx)
        return dict(zip(STAGES, list(ms))), calls.value

    def condsim_grad(self, z, R: int, seed: int, window, r_offset: int = 0, out=None, stream=None):
        """Forward draws plus dL/d(sigma, range, tau^2) and dL/dz for the window loss plus the
        log-likelihood (ce_condsim_grad).  Returns (v, grad_theta[3], grad_z, L)."""
        import torch
        if out is None:
            out = torch.empty((R, self.m, self.m), dtype=torch.float32, device=z.device)
        gz = torch.empty_like(z)
        win = (ctypes.c_int * 4)(*[int(x) for x in window])
        gt = (ctypes.c_double * 3)()
        loss = ctypes.c_double()
        _check(load_library().ce_condsim_grad(self._ctx, _dev_ptr(z, torch.float32), R, seed, r_offset, win,
                                              _dev_ptr(out, torch.float32), gt, _dev_ptr(gz, torch.float32),
                                              ctypes.byref(loss), _stream(stream)), self._ctx)
        return out, list(gt), gz, loss.value

    def loglik(self, z, stream=None) -> float:
        """ce_loglik: Gaussian log-likelihood of the data z (device float32, n) under
        A = K_oo + tau^2 I (Eq. (condmvn)'s model)."""
        import torch
        out = ctypes.c_double()
        _check(load_library().ce_loglik(self._ctx, _dev_ptr(z, torch.float32), ctypes.byref(out), _stream(stream)),
               self._ctx)
        return out.value

    def prepare(self, R: int):
        _check(load_library().ce_condsim_prepare(self._ctx, R), self._ctx)

    def autotune(self, R: int, stream=None):
        _check(load_library().ce_autotune(self._ctx, R, _stream(stream)), self._ctx)

    def sync(self):
        _check(load_library().ce_sync_status(self._ctx), self._ctx)


def _batch_arrays(ctxs, zs, Rs, seeds, r_offsets, outs):
    import torch
    count = len(ctxs)
    if not (len(zs) == len(Rs) == len(seeds) == len(r_offsets) == len(outs) == count):
        raise ValueError("batch arrays must have one entry per event")
    arr = dict(
        ctx=(ctypes.c_void_p * count)(*[c._ctx.value for c in ctxs]),
        z=(ctypes.c_void_p * count)(*[_dev_ptr(z, torch.float32) for z in zs]),
        R=(ctypes.c_int * count)(*Rs),
        seed=(ctypes.c_uint64 * count)(*seeds),
        off=(ctypes.c_uint64 * count)(*r_offsets),
        out=(ctypes.c_void_p * count)(*[_dev_ptr(o, torch.float32) for o in outs]),
    )
    return count, arr


def condsim_batch(ctxs, zs, Rs, seeds, r_offsets, outs, nstreams: int = 8, stream=None):
    """ce_condsim for many independent events (distinct contexts) on parallel internal streams."""
    count, a = _batch_arrays(ctxs, zs, Rs, seeds, r_offsets, outs)
    _check(load_library().ce_condsim_batch(a["ctx"], a["z"], a["R"], a["seed"], a["off"], a["out"], count, nstreams,
                                           _stream(stream)))
    return outs


class Batch:
    """A batch schedule captured once into a CUDA graph (ce_batch_create); launch() replays it."""

    def __init__(self, ctxs, zs, Rs, seeds, r_offsets, outs, nstreams: int = 8):
        count, a = _batch_arrays(ctxs, zs, Rs, seeds, r_offsets, outs)
        self._keep = (ctxs, zs, outs)
        self._b = ctypes.c_void_p()
        _check(load_library().ce_batch_create(ctypes.byref(self._b), a["ctx"], a["z"], a["R"], a["seed"], a["off"],
                                              a["out"], count, nstreams))

    def launch(self, stream=None):
        _check(load_library().ce_batch_launch(self._b, _stream(stream)))

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            load_library().ce_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def philox(ctr, seed: int, stream=None):
    """Raw Philox4x32-10 words for an (count, 4) int32 CUDA tensor of counters."""
    import torch
    out = torch.empty_like(ctr)
    _check(load_library().ce_philox(_dev_ptr(ctr, torch.int32), ctr.shape[0], seed, _dev_ptr(out), _stream(stream)))
    return out


def normals(ctr, seed: int, stream=None):
    """Box-Muller normals (count, 4) float32 from the same counters."""
    import torch
    out = torch.empty(ctr.shape, dtype=torch.float32, device=ctr.device)
    _check(load_library().ce_normals(_dev_ptr(ctr, torch.int32), ctr.shape[0], seed, _dev_ptr(out), _stream(stream)))
    return out


_LOSS_FN = None


def _loss_function():
    """torch.autograd.Function over ce_condsim_grad: the forward runs the draws
    and the adjoint in one call and keeps the gradients; the backward scales them."""
    global _LOSS_FN
    if _LOSS_FN is None:
        import torch

        class CondsimLoss(torch.autograd.Function):
            @staticmethod
            def forward(fctx, ctx, theta, z, R, seed, window, r_offset):
                want = [float(x) for x in theta.detach().cpu().tolist()]
                if len(want) != 3:
                    raise ValueError("theta holds (sigma, range, tau2)")
                run = ctx
                if any(abs(a - b) > 1e-12 * max(1.0, abs(b)) for a, b in zip(want, ctx.theta)):
                    run = ctx.with_theta(*want)     # the set-up depends on theta: redo it there
                try:
                    _, gt, gz, L = run.condsim_grad(z.detach(), R, seed, window, r_offset)
                finally:
                    if run is not ctx:
                        run.close()
                fctx.save_for_backward(torch.tensor(gt, dtype=theta.dtype, device=theta.device), gz)
                return torch.tensor(L, dtype=torch.float64, device=z.device)

            @staticmethod
            def backward(fctx, grad):
                gt, gz = fctx.saved_tensors
                return (None, grad.to(gt.device, gt.dtype) * gt, grad.to(gz.device, gz.dtype) * gz,
                        None, None, None, None)

        _LOSS_FN = CondsimLoss
    return _LOSS_FN


def condsim_loss(ctx: Context, theta, z, R: int, seed: int, window, r_offset: int = 0):
    """The loss of ce_condsim_grad, L = (1/R) sum_r mean_window v_r^2 + log-likelihood,
    as a differentiable torch scalar (float64).  `theta` is a 3-element tensor
    (sigma, range, tau^2); where it differs from the context's own parameters the
    set-up is redone at theta on the context's grid and sites.  Gradients flow to
    `theta` and to the data `z` (device float32, n) through the library's adjoint,
    at the fixed noise of (seed, r_offset)."""
    return _loss_function().apply(ctx, theta, z, R, seed, tuple(int(x) for x in window), r_offset)
