"""Thin Python binding of the C ABI (include/smc.h) over torch CUDA tensors.

Every function checks dtypes / devices / shapes, passes ``data_ptr()`` and
the current CUDA stream, and raises :class:`SmcError` on a non-zero status.
All arithmetic happens in the CUDA kernels of libsmc.so; nothing here
computes any part of the method.
"""
from __future__ import annotations

import ctypes as C
import functools
import os
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L


class SmcError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = L.load().smc_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


def _chk(st: int, where: str):
    if st != 0:
        raise SmcError(st, where)


_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(stream=None):
    """The CUDA stream handle to launch on: the given torch stream, else the
    current stream of the current device (read without building a Stream
    object: this runs once per call)."""
    if stream is not None:
        return stream.cuda_stream
    if _raw_stream is not None:
        return _raw_stream(torch.cuda.current_device())
    return torch.cuda.current_stream().cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


def _need(t, dtype, name, shape=None):
    if t is None:
        return
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and t.shape != shape:
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


# ------------------------------------------------------------------ context
class Context:
    """Owns an smc_ctx (status word, scratch, launch overrides) on one device.
    Calls on one context share its scratch and must follow one another on
    the GPU (one stream, or streams ordered by events); work meant to
    overlap on several streams takes one context per stream."""

    def __init__(self, device: int | None = None):
        self._lib = L.load()
        dev = torch.cuda.current_device() if device is None else int(device)
        h = C.c_void_p()
        _chk(self._lib.smc_create(C.byref(h), dev), "smc_create")
        self.handle = h
        self.device = dev

    def close(self):
        if self.handle:
            self._lib.smc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, max_particles: int, max_pops: int = 0):
        _chk(self._lib.smc_reserve(self.handle, int(max_particles), int(max_pops)), "smc_reserve")

    def check(self, stream=None):
        """Synchronise the stream and raise the first device-latched error."""
        _chk(self._lib.smc_ctx_check(self.handle, _stream(stream)), "device status")

    def set_launch(self, op: int, lanes: int, threads: int = 256):
        _chk(self._lib.smc_set_launch(self.handle, op, lanes, threads), "smc_set_launch")

    def set_wait_limit(self, polls: int):
        """Polls of the first bounded wait on a bulk data copy (a test hook:
        0 makes every such wait give up and report SMC_ERR_TIMEOUT)."""
        _chk(self._lib.smc_set_wait_limit(self.handle, int(polls)), "smc_set_wait_limit")

    def get_launch(self, op: int, M: int, N: int, K: int):
        l, t = C.c_int32(), C.c_int32()
        _chk(self._lib.smc_get_launch(self.handle, op, M, N, K, C.byref(l), C.byref(t)),
             "smc_get_launch")
        return l.value, t.value


# ------------------------------------------------------------------ models
@dataclass
class GMM:
    """Gaussian mixture with known weights and sigma (Section 4.1), prior box."""
    K: int
    sigma: float
    log_w: np.ndarray = None
    lo: float = -10.0
    hi: float = 10.0
    d: int = 1
    precision: int = L.PREC_FP32
    _w: object = field(default=None, repr=False)

    def __post_init__(self):
        if self.log_w is None:
            self.log_w = np.full(self.K, -np.log(self.K))
        self.log_w = np.asarray(self.log_w, np.float64)
        self._w = (C.c_float * self.K)(*[float(v) for v in self.log_w])

    def __setattr__(self, name, value):
        # the C struct is built once per set of field values
        super().__setattr__(name, value)
        if name != "_c":
            self.__dict__.pop("_c", None)
            if name == "log_w" and "_w" in self.__dict__ and value is not None:
                w = np.asarray(value, np.float64)
                super().__setattr__("_w", (C.c_float * w.size)(*[float(v) for v in w]))

    def cstruct(self) -> L.SmcGmm:
        c = self.__dict__.get("_c")
        if c is None:
            c = self._build()
            self.__dict__["_c"] = c
        return c

    def _build(self) -> L.SmcGmm:
        return L.SmcGmm(L.GMM_1D, self.K, 1, L.PREC_FP32, self._w, self.sigma, self.lo, self.hi)


@dataclass
class DiagGMM(GMM):
    """d-dimensional mixture with N(mu_k, sigma^2 I_d) components."""

    def _build(self) -> L.SmcGmm:
        return L.SmcGmm(L.GMM_DIAG, self.K, self.d, self.precision, self._w, self.sigma,
                        self.lo, self.hi)


@dataclass
class PFModel:
    """State-space model for pf_step: MSV (Section 4.2 family), linear-Gaussian,
    or the factor stochastic volatility model of Section 4.2 (kind PF_FSV:
    state = factors' log-variances, loadings B [m][d], variances psi [m])."""
    kind: int
    phi: np.ndarray
    chol: np.ndarray
    beta: float = 1.0
    B: np.ndarray = None
    psi: np.ndarray = None

    def cstruct_cached(self) -> L.SmcPfModel:
        """The C struct, built once (the model's fields are not meant to change)."""
        c = self.__dict__.get("_c")
        if c is None:
            c = self.cstruct()
            self.__dict__["_c"] = c
        return c

    @property
    def state_dim(self) -> int:
        return np.asarray(self.phi).size  # FSV: the factors' log-variances

    @property
    def obs_dim(self) -> int:
        return np.asarray(self.B).shape[0] if self.kind == L.PF_FSV else np.asarray(self.phi).size

    def cstruct(self) -> L.SmcPfModel:
        phi = np.asarray(self.phi, np.float64)
        ch = np.asarray(self.chol, np.float64)
        d = phi.size
        m = L.SmcPfModel()
        m.kind = self.kind
        m.d = d
        for i in range(d):
            m.phi[i] = float(phi[i])
            for j in range(d):
                m.chol[i * d + j] = float(ch[i, j])
        m.beta = float(self.beta)
        if self.kind == L.PF_FSV:
            B = np.asarray(self.B, np.float64)
            psi = np.asarray(self.psi, np.float64)
            if B.ndim != 2 or B.shape[1] != d or psi.shape != (B.shape[0],):
                raise ValueError("FSV model: B must be [m][d] and psi [m]")
            m.m = B.shape[0]
            for i in range(m.m):
                m.psi[i] = float(psi[i])
                for k in range(d):
                    m.B[i * d + k] = float(B[i, k])
        return m


# ------------------------------------------------------------------ calls
def _match_model(model, y, theta, name="theta"):
    """The tensors' layout must be the model's (the C ABI takes bare pointers
    and sizes, so a tensor smaller than the model implies would be read past
    its end): 1-D y float[N], theta float[K][M]; diagonal y float[N][d],
    theta float[M][K][d]."""
    if isinstance(model, DiagGMM):
        ok = theta.dim() == 3 and theta.shape[1] == model.K and theta.shape[2] == model.d
        want = f"[M, {model.K}, {model.d}]"
        if y.dim() != 2 or y.shape[1] != model.d:
            raise ValueError(f"y must be [N, {model.d}] for this model, got {tuple(y.shape)}")
    else:
        ok = theta.dim() == 2 and theta.shape[0] == model.K
        want = f"[{model.K}, M]"
        if y.dim() != 1:
            raise ValueError(f"y must be one-dimensional for this model, got {tuple(y.shape)}")
    if not ok:
        raise ValueError(f"{name} must be {want} for this model, got {tuple(theta.shape)}")


def loglik_batch(ctx: Context, model: GMM, y, theta, out=None, grad=None, stream=None):
    """Per-particle mixture log-likelihood (and optional gradient)."""
    _match_model(model, y, theta)
    if isinstance(model, DiagGMM):
        N = y.shape[0]
        M = theta.shape[0]
    else:
        N = y.numel()
        M = theta.shape[1]
    out = torch.empty(M, dtype=torch.float64, device=theta.device) if out is None else out
    _need(y, torch.float32, "y")
    _need(theta, torch.float32, "theta")
    _need(out, torch.float64, "loglik_out", (M,))
    _need(grad, torch.float32, "grad_out", tuple(theta.shape))
    m = model.cstruct()
    _chk(L.load().smc_loglik_batch(ctx.handle, C.byref(m), _ptr(y), N, _ptr(theta), M,
                                   _ptr(out), _ptr(grad), _stream(stream)), "smc_loglik_batch")
    return out


def reweight(ctx: Context, loglik, dbeta: float, logw, W_out=None, scalars=None, flag=None,
             ess_frac: float = 0.5, stream=None):
    M = logw.numel()
    _need(loglik, torch.float64, "loglik", (M,))
    _need(logw, torch.float64, "logw", (M,))
    _need(W_out, torch.float64, "W_out", (M,))
    _need(scalars, torch.float64, "scalars", (4,))
    _need(flag, torch.int32, "flag", (1,))
    _chk(L.load().smc_reweight(ctx.handle, _ptr(loglik), float(dbeta), _ptr(logw), M, _ptr(W_out),
                               _ptr(scalars), _ptr(flag), float(ess_frac), _stream(stream)),
         "smc_reweight")


def reweight_resample(ctx: Context, loglik, dbeta: float, logw, W_out, seed: int, step: int,
                      scalars=None, flag=None, ess_frac: float = 0.5, anc=None, counts=None,
                      stream=None):
    """reweight followed by systematic resampling of its weights (logw reset
    where resampled), one pass fewer; flag None resamples unconditionally."""
    M = logw.numel()
    anc = torch.empty(M, dtype=torch.int32, device=logw.device) if anc is None else anc
    _need(loglik, torch.float64, "loglik", (M,))
    _need(logw, torch.float64, "logw", (M,))
    _need(W_out, torch.float64, "W_out", (M,))
    _need(scalars, torch.float64, "scalars", (4,))
    _need(flag, torch.int32, "flag", (1,))
    _need(anc, torch.int32, "ancestors", (M,))
    _need(counts, torch.int32, "counts", (M,))
    _chk(L.load().smc_reweight_resample(ctx.handle, _ptr(loglik), float(dbeta), _ptr(logw), M,
                                        _ptr(W_out), _ptr(scalars), _ptr(flag), float(ess_frac),
                                        int(seed), int(step), _ptr(anc), _ptr(counts),
                                        _stream(stream)), "smc_reweight_resample")
    return anc


def ess(ctx: Context, logw, out=None, stream=None):
    M = logw.numel()
    out = torch.empty(1, dtype=torch.float64, device=logw.device) if out is None else out
    _need(logw, torch.float64, "logw", (M,))
    _need(out, torch.float64, "ess_out", (1,))
    _chk(L.load().smc_ess(ctx.handle, _ptr(logw), M, _ptr(out), _stream(stream)), "smc_ess")
    return out


def resample_systematic(ctx: Context, W, seed: int, step: int, anc=None, counts=None,
                        do_flag=None, logw_reset=None, stream=None):
    M = W.numel()
    anc = torch.empty(M, dtype=torch.int32, device=W.device) if anc is None else anc
    _need(W, torch.float64, "W", (M,))
    _need(anc, torch.int32, "ancestors", (M,))
    _need(counts, torch.int32, "counts", (M,))
    _need(do_flag, torch.int32, "do_flag", (1,))
    _need(logw_reset, torch.float64, "logw_reset", (M,))
    _chk(L.load().smc_resample_systematic(ctx.handle, _ptr(W), M, int(seed), int(step), _ptr(anc),
                                          _ptr(counts), _ptr(do_flag), _ptr(logw_reset),
                                          _stream(stream)), "smc_resample_systematic")
    return anc


def _resample_var(fn, where, ctx, W, seed, step, anc, do_flag, logw_reset, stream):
    M = W.numel()
    anc = torch.empty(M, dtype=torch.int32, device=W.device) if anc is None else anc
    _need(W, torch.float64, "W", (M,))
    _need(anc, torch.int32, "ancestors", (M,))
    _need(do_flag, torch.int32, "do_flag", (1,))
    _need(logw_reset, torch.float64, "logw_reset", (M,))
    _chk(fn(ctx.handle, _ptr(W), M, int(seed), int(step), _ptr(anc), _ptr(do_flag),
            _ptr(logw_reset), _stream(stream)), where)
    return anc


def resample_multinomial(ctx: Context, W, seed: int, step: int, anc=None, do_flag=None,
                         logw_reset=None, stream=None):
    """Exact-integer multinomial resampling (ancestors in draw order)."""
    return _resample_var(L.load().smc_resample_multinomial, "smc_resample_multinomial", ctx, W,
                         seed, step, anc, do_flag, logw_reset, stream)


def resample_residual(ctx: Context, W, seed: int, step: int, anc=None, do_flag=None,
                      logw_reset=None, stream=None):
    """Exact-integer residual resampling (deterministic copies, then residual draws)."""
    return _resample_var(L.load().smc_resample_residual, "smc_resample_residual", ctx, W, seed,
                         step, anc, do_flag, logw_reset, stream)


RESAMPLERS = ("systematic", "multinomial", "residual")


def resample(ctx: Context, kind: str, W, seed: int, step: int, anc=None, do_flag=None,
             logw_reset=None, stream=None):
    """Dispatch on the scheme name (one of RESAMPLERS)."""
    if kind == "systematic":
        return resample_systematic(ctx, W, seed, step, anc=anc, do_flag=do_flag,
                                   logw_reset=logw_reset, stream=stream)
    if kind == "multinomial":
        return resample_multinomial(ctx, W, seed, step, anc, do_flag, logw_reset, stream)
    if kind == "residual":
        return resample_residual(ctx, W, seed, step, anc, do_flag, logw_reset, stream)
    raise ValueError(f"unknown resampling scheme {kind!r}")


def gather(ctx: Context, anc, src32=None, dst32=None, src64=None, dst64=None, stream=None):
    """dst[..., i] = src[..., anc[i]]: float32 rows [rows][M] (or [M]) and a
    float64 vector [M]; sources and destinations come in pairs of one shape."""
    if (src32 is None) != (dst32 is None) or (src64 is None) != (dst64 is None):
        raise ValueError("each source needs its destination and vice versa")
    if dst32 is None and dst64 is None:
        raise ValueError("nothing to gather")
    M = (dst64 if dst64 is not None else dst32).shape[-1]
    if dst32 is not None and (dst32.dim() not in (1, 2) or dst32.shape[-1] != M):
        raise ValueError(f"dst_f32 must be [rows, {M}] or [{M}], got {tuple(dst32.shape)}")
    rows = 0 if src32 is None else (dst32.shape[0] if dst32.dim() == 2 else 1)
    _need(anc, torch.int32, "anc", (M,))
    _need(src32, torch.float32, "src_f32", None if dst32 is None else dst32.shape)
    _need(dst32, torch.float32, "dst_f32")
    _need(src64, torch.float64, "src_f64", (M,))
    _need(dst64, torch.float64, "dst_f64", (M,))
    _chk(L.load().smc_gather(ctx.handle, _ptr(anc), M, rows, _ptr(src32), _ptr(dst32), _ptr(src64),
                             _ptr(dst64), _stream(stream)), "smc_gather")


def mh_move(ctx: Context, model: GMM, y, theta_in, ll_in, theta_out, ll_out, beta, scale: float,
            seed: int, step: int, kind: int = L.MOVE_RW, grad_in=None, grad_out=None, anc=None,
            do_flag=None, accept_count=None, stream=None):
    _match_model(model, y, theta_in, "theta_in")
    K, M = theta_in.shape
    _need(y, torch.float32, "y")
    for t, n in ((theta_in, "theta_in"), (theta_out, "theta_out")):
        _need(t, torch.float32, n, (K, M))
    for t, n in ((grad_in, "grad_in"), (grad_out, "grad_out")):
        _need(t, torch.float32, n, (K, M))
    _need(ll_in, torch.float64, "loglik_in", (M,))
    _need(ll_out, torch.float64, "loglik_out", (M,))
    _need(beta, torch.float32, "beta")
    _need(anc, torch.int32, "anc", (M,))
    _need(do_flag, torch.int32, "do_flag", (1,))
    _need(accept_count, torch.int32, "accept_count", (1,))
    bstride = 0 if beta.numel() == 1 else 1
    if bstride and beta.numel() != M:
        raise ValueError("beta must have 1 or M entries")
    m = model.cstruct()
    _chk(L.load().smc_mh_move(ctx.handle, C.byref(m), _ptr(y), y.numel(), _ptr(theta_in),
                              _ptr(ll_in), _ptr(grad_in), _ptr(anc), _ptr(do_flag),
                              _ptr(theta_out), _ptr(ll_out), _ptr(grad_out), M, _ptr(beta),
                              bstride, float(scale), int(kind), int(seed), int(step),
                              _ptr(accept_count), _stream(stream)), "smc_mh_move")


def popmcmc_sweep(ctx: Context, model: GMM, y, theta, loglik, beta, offsets, scale: float,
                  seed: int, sweep: int, stats=None, stream=None):
    """One population-MCMC sweep in place.  `offsets` (int32, device) must
    run non-decreasing from 0 to M: its values live on the device and are
    not checked here (PopulationMCMC checks them once, on the host)."""
    _match_model(model, y, theta)
    K, M = theta.shape
    n_pops = offsets.numel() - 1
    _need(y, torch.float32, "y")
    _need(theta, torch.float32, "theta", (K, M))
    _need(loglik, torch.float64, "loglik", (M,))
    _need(beta, torch.float32, "beta", (M,))
    _need(offsets, torch.int32, "pop_offsets", (n_pops + 1,))
    _need(stats, torch.int64, "stats", (3,))
    m = model.cstruct()
    _chk(L.load().smc_popmcmc_sweep(ctx.handle, C.byref(m), _ptr(y), y.numel(), _ptr(theta),
                                    _ptr(loglik), M, _ptr(beta), _ptr(offsets), n_pops,
                                    float(scale), int(seed), int(sweep), _ptr(stats),
                                    _stream(stream)), "smc_popmcmc_sweep")


def pf_step(ctx: Context, model: PFModel, y_t, x_in, x_out, logg_out, seed: int, t: int,
            anc=None, stream=None):
    if x_in.dim() != 2 or x_in.shape[0] != model.state_dim:
        raise ValueError(f"x_in must be [{model.state_dim}, M] for this model, "
                         f"got {tuple(x_in.shape)}")
    d, M = x_in.shape
    _need(y_t, torch.float32, "y_t", (model.obs_dim,))
    _need(x_in, torch.float32, "x_in", (d, M))
    _need(x_out, torch.float32, "x_out", (d, M))
    _need(logg_out, torch.float64, "logg_out", (M,))
    _need(anc, torch.int32, "anc", (M,))
    m = model.cstruct_cached()
    _chk(L.load().pf_step(ctx.handle, C.byref(m), _ptr(y_t), _ptr(x_in), _ptr(anc), _ptr(x_out),
                          _ptr(logg_out), M, int(seed), int(t), _stream(stream)), "pf_step")


def pf_filter_step(ctx: Context, model: PFModel, y_t, x_in, x_out, anc, logw, W_out, logg_out,
                   seed: int, t: int, scalars=None, flag=None, ess_frac: float = 0.5,
                   counts=None, stream=None):
    """One whole bootstrap-filter step in one call: pf_step, reweight
    (dbeta = 1) and systematic resampling; anc is read as this step's
    ancestors and overwritten with the next step's (the identity when flag
    says no resampling)."""
    if x_in.dim() != 2 or x_in.shape[0] != model.state_dim:
        raise ValueError(f"x_in must be [{model.state_dim}, M] for this model, "
                         f"got {tuple(x_in.shape)}")
    d, M = x_in.shape
    _need(y_t, torch.float32, "y_t", (model.obs_dim,))
    _need(x_in, torch.float32, "x_in", (d, M))
    _need(x_out, torch.float32, "x_out", (d, M))
    _need(anc, torch.int32, "anc", (M,))
    _need(logw, torch.float64, "logw", (M,))
    _need(W_out, torch.float64, "W_out", (M,))
    if logg_out is None:
        raise TypeError("logg_out must be a CUDA tensor")
    _need(logg_out, torch.float64, "logg_out", (M,))
    _need(scalars, torch.float64, "scalars", (4,))
    _need(flag, torch.int32, "flag", (1,))
    _need(counts, torch.int32, "counts", (M,))
    m = model.cstruct_cached()
    _chk(L.load().smc_pf_filter_step(ctx.handle, C.byref(m), _ptr(y_t), _ptr(x_in), _ptr(anc),
                                     _ptr(x_out), _ptr(logg_out), _ptr(logw), M, _ptr(W_out),
                                     _ptr(scalars), _ptr(flag), float(ess_frac), int(seed), int(t),
                                     _ptr(counts), _stream(stream)), "smc_pf_filter_step")


@dataclass
class ISProblem:
    """Gaussian-mixture target sum_k a_k N(mu_k, var), Gaussian proposal, test
    function x^power (Section 2.1's example by default)."""
    mu: tuple = (-1.0, 1.5)
    a: tuple = (0.5, 0.5)
    var: float = 0.25
    prop_mean: float = 0.0
    prop_sd: float = 1.0
    power: int = 2

    def cstruct(self) -> L.SmcIsProblem:
        c = L.SmcIsProblem()
        c.K = len(self.mu)
        if c.K < 1 or c.K > 8 or len(self.a) != c.K:
            raise ValueError("1..8 components, one weight each")
        for k in range(c.K):
            c.mu[k] = float(self.mu[k])
            c.a[k] = float(self.a[k])
        c.var, c.prop_mean, c.prop_sd = float(self.var), float(self.prop_mean), float(self.prop_sd)
        c.power = int(self.power)
        return c


def is_moments(ctx: Context, prob: ISProblem, x=None, N: int | None = None, seed: int = 0,
               step: int = 0, out=None, stream=None):
    """{sum w, sum w phi, sum w^2} over N proposal draws (x, or drawn on the device)."""
    if x is not None:
        _need(x, torch.float32, "x")
        N = x.numel()
    elif N is None:
        raise ValueError("give the draws x or their number N")
    out = torch.empty(3, dtype=torch.float64, device="cuda") if out is None else out
    _need(out, torch.float64, "out", (3,))
    c = prob.cstruct()
    _chk(L.load().smc_is_moments(ctx.handle, C.byref(c), _ptr(x), int(N), int(seed), int(step),
                                 _ptr(out), _stream(stream)), "smc_is_moments")
    return out


def rng_mrg32k3a(ctx: Context, seed=(12345,) * 6, offset: int = 0, n_threads: int = 1,
                 per_thread: int = 1, out=None, dtype=torch.float32, stream=None):
    """MRG32k3a uniforms: thread t's contiguous block of per_thread numbers
    starting at stream position offset + t * per_thread; returns a
    [per_thread, n_threads] tensor (float32: 24-bit uniforms; float64: the
    generator's z / (m1 + 1))."""
    out = (torch.empty(per_thread * n_threads, dtype=dtype, device="cuda")
           if out is None else out)
    if out.dtype not in (torch.float32, torch.float64):
        raise TypeError("out must be float32 or float64")
    _need(out, out.dtype, "out")
    if out.numel() != per_thread * n_threads:
        raise ValueError("out must hold per_thread * n_threads numbers")
    sd = (C.c_uint32 * 6)(*[int(v) for v in seed])
    f32 = out if out.dtype == torch.float32 else None
    f64 = out if out.dtype == torch.float64 else None
    _chk(L.load().smc_rng_mrg32k3a(ctx.handle, C.byref(sd), int(offset) & (2**64 - 1),
                                   int(n_threads), int(per_thread), _ptr(f32), _ptr(f64),
                                   _stream(stream)), "smc_rng_mrg32k3a")
    return out.view(per_thread, n_threads)


def rng_words(ctx: Context, seed: int, purpose: int, step: int, n_index: int, n_block: int = 1,
              stream=None):
    out = torch.empty(n_index * n_block * 4, dtype=torch.int32, device="cuda")
    _chk(L.load().smc_rng_words(ctx.handle, int(seed), purpose, int(step), n_index, n_block,
                                _ptr(out), _stream(stream)), "smc_rng_words")
    return out.view(n_index, n_block, 4)


def rng_normals(ctx: Context, seed: int, purpose: int, step: int, n_index: int, n: int,
                stream=None):
    out = torch.empty(n_index * n, dtype=torch.float32, device="cuda")
    _chk(L.load().smc_rng_normals(ctx.handle, int(seed), purpose, int(step), n_index, n,
                                  _ptr(out), _stream(stream)), "smc_rng_normals")
    return out.view(n_index, n)


# NVTX ranges (environment SMC_NVTX=1 at import): every call of the functions
# below runs inside a range named after it (torch.cuda.nvtx), so that a
# profiler can attribute the kernels a call launches (ncu --nvtx
# --nvtx-include "smc.reweight/").  Off by default: no wrapper, no cost.
RANGED = ("loglik_batch", "reweight", "reweight_resample", "ess", "resample_systematic",
          "resample_multinomial", "resample_residual", "resample", "gather", "mh_move",
          "popmcmc_sweep", "pf_step", "pf_filter_step", "is_moments", "rng_mrg32k3a", "rng_words",
          "rng_normals")


def _ranged(fn):
    name = "smc." + fn.__name__

    @functools.wraps(fn)
    def call(*args, **kwargs):
        torch.cuda.nvtx.range_push(name)
        try:
            return fn(*args, **kwargs)
        finally:
            torch.cuda.nvtx.range_pop()
    return call


if os.environ.get("SMC_NVTX") == "1":
    for _name in RANGED:
        globals()[_name] = _ranged(globals()[_name])
