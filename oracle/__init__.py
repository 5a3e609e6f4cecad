"""FP64 CPU oracle for the SMC / population-MCMC hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C, double
precision, one particle at a time) through ctypes and shares nothing with the
CUDA library: no code, header, table or helper.

Every function states the passage of Lee, Yau, Giles, Doucet & Holmes (2009)
it follows; the C source carries the full definitions.  Parity status: every
function here is pinned by a CPU test (brute-force enumeration, closed-form
evidence, Kalman filter, an independent Philox implementation, exact
invariants); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

P_MOVE, P_ACCEPT, P_RESAMPLE, P_EXCHANGE, P_PFNOISE, P_MULTINOMIAL, P_PROPOSAL = 1, 2, 3, 4, 5, 6, 7


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, IEEE semantics, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-std=gnu11",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_vp = C.c_void_p
_i64 = C.c_int64
_u64 = C.c_uint64


def _declare(L):
    L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.orc_draw_words.argtypes = [_u64, C.c_uint32, _u64, C.c_uint32, C.c_uint32, _u32p]
    L.orc_u01.argtypes = [C.c_uint32]
    L.orc_u01.restype = C.c_double
    L.orc_normals.argtypes = [_u64, C.c_uint32, _u64, C.c_uint32, C.c_int, _f64p]
    L.orc_gmm1d_loglik.argtypes = [_f32p, _i64, C.c_int, _f64p, C.c_double, _f32p, _i64, _f64p]
    L.orc_gmm1d_loglik_at.argtypes = [_f32p, _i64, C.c_int, _f64p, C.c_double, _f64p]
    L.orc_gmm1d_loglik_at.restype = C.c_double
    L.orc_gmm1d_grad.argtypes = [_f32p, _i64, C.c_int, _f64p, C.c_double, _f32p, _i64, _f64p]
    L.orc_gmm1d_grad_at.argtypes = [_f32p, _i64, C.c_int, _f64p, C.c_double, _f64p, _f64p]
    L.orc_gmmdiag_loglik.argtypes = [_f32p, _i64, C.c_int, C.c_int, _f64p, C.c_double, _f32p,
                                     _i64, _f64p]
    L.orc_reweight.argtypes = [_vp, C.c_double, _f64p, _i64, _f64p, _f64p]
    L.orc_reweight.restype = C.c_int
    L.orc_ess.argtypes = [_f64p, _i64]
    L.orc_ess.restype = C.c_double
    L.orc_resample_systematic.argtypes = [_f64p, _i64, C.c_uint32, _i32p, _vp]
    L.orc_resample_systematic.restype = C.c_int
    L.orc_word_array.argtypes = [_u64, C.c_uint32, _u64, _i64, _u32p]
    L.orc_mrg32k3a.argtypes = [_u32p, _u64, _i64, _vp, _vp]
    L.orc_is_moments.argtypes = [C.c_int, _f64p, _f64p, C.c_double, C.c_double, C.c_double, C.c_int,
                                 _vp, _i64, _u64, _u64, _f64p]
    L.orc_resample_multinomial.argtypes = [_f64p, _i64, _u32p, _i32p]
    L.orc_resample_multinomial.restype = C.c_int
    L.orc_resample_residual.argtypes = [_f64p, _i64, _u32p, _i32p, C.POINTER(C.c_int64)]
    L.orc_resample_residual.restype = C.c_int
    L.orc_rwmh_move.argtypes = [_f32p, _i64, C.c_int, _f64p, C.c_double, C.c_double, C.c_double,
                                _f32p, _f64p, _vp, _f32p, _f64p, _i64, _f32p, _i64, C.c_float,
                                _u64, _u64, _i32p]
    L.orc_rwmh_move_slots.argtypes = L.orc_rwmh_move.argtypes + [_vp, _i64, _vp]
    L.orc_mala_move.argtypes = [_f32p, _i64, C.c_int, _f64p, C.c_double, C.c_double, C.c_double,
                                _f32p, _f64p, _f32p, _vp, _f32p, _f64p, _f32p, _i64, _f32p, _i64,
                                C.c_float, _u64, _u64, _i32p]
    L.orc_mala_move_slots.argtypes = L.orc_mala_move.argtypes + [_vp, _i64, _vp]
    L.orc_popmcmc_sweep.argtypes = [_f32p, _i64, C.c_int, _f64p, C.c_double, C.c_double,
                                    C.c_double, _f32p, _f64p, _i64, _f32p, _i32p, C.c_int32,
                                    C.c_float, _u64, _u64, _i64p]
    L.orc_popmcmc_exchange.argtypes = [C.c_int, _f32p, _f64p, _i64, _f32p, _i32p, C.c_int32,
                                       C.c_int32, _u64, _u64, _i64p, _vp, _vp]
    L.orc_pf_step.argtypes = [C.c_int, C.c_int, _f64p, _f64p, C.c_double, _f32p, _f32p, _vp,
                              _f32p, _f64p, _i64, _u64, _u64]
    L.orc_pf_run.argtypes = [C.c_int, C.c_int, _f64p, _f64p, C.c_double, _f32p, _i64, _i64, _u64,
                             C.POINTER(C.c_double), _vp]
    L.orc_pf_run.restype = C.c_int
    L.orc_fsv_step.argtypes = [C.c_int, C.c_int, _f64p, _f64p, _f64p, _f64p, _f32p, _f32p, _vp,
                               _f32p, _f64p, _i64, _u64, _u64]
    L.orc_fsv_run.argtypes = [C.c_int, C.c_int, _f64p, _f64p, _f64p, _f64p, _f32p, _i64, _i64,
                              _u64, C.POINTER(C.c_double), _vp]
    L.orc_fsv_run.restype = C.c_int
    L.orc_kalman_lg.argtypes = [C.c_int, _f64p, _f64p, C.c_double, _f32p, _i64, _vp]
    L.orc_kalman_lg.restype = C.c_double
    L.orc_smc_run.argtypes = [_f32p, _i64, C.c_int, _f64p, C.c_double, C.c_double, C.c_double,
                              _f32p, _i64, _f64p, _i64, C.c_int, C.c_float, C.c_int, C.c_double,
                              _u64, C.POINTER(C.c_double), _vp, _vp]
    L.orc_smc_run.restype = C.c_int


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    pass


# --------------------------------------------------------------------------- RNG
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al. 2011); replaces the Section 2.5 streams."""
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def draw_words(seed, purpose, step, index, block) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().orc_draw_words(seed, purpose, step, index, block, out)
    return out


def u01(x: int) -> float:
    return lib().orc_u01(int(x))


def normals(seed, purpose, step, index, n) -> np.ndarray:
    z = np.zeros(max(n, 1), np.float64)
    lib().orc_normals(seed, purpose, step, index, n, z)
    return z[:n]


def resample_u32(seed: int, step: int) -> int:
    """The resampling uniform word: purpose RESAMPLE, index 0, block 0, word 0."""
    return int(draw_words(seed, P_RESAMPLE, step, 0, 0)[0])


# ---------------------------------------------------------------------- loglik
def gmm1d_loglik(y, logw, sigma, theta) -> np.ndarray:
    """Section 4.1 mixture log-likelihood per particle; theta is [K][M] float32."""
    y, theta, logw = _f32(y), _f32(theta), _f64(logw)
    K, M = theta.shape
    out = np.zeros(M, np.float64)
    lib().orc_gmm1d_loglik(y, y.size, K, logw, float(sigma), theta, M, out)
    return out


def gmm1d_loglik_at(y, logw, sigma, mu) -> float:
    """Section 4.1 log-likelihood at FP64 means mu [K]."""
    y, logw, mu = _f32(y), _f64(logw), _f64(mu)
    return lib().orc_gmm1d_loglik_at(y, y.size, mu.size, logw, float(sigma), mu)


def gmm1d_grad(y, logw, sigma, theta) -> np.ndarray:
    """d loglik / d mu, [K][M] float64 (derivative of the Section 4.1 density)."""
    y, theta, logw = _f32(y), _f32(theta), _f64(logw)
    K, M = theta.shape
    out = np.zeros((K, M), np.float64)
    lib().orc_gmm1d_grad(y, y.size, K, logw, float(sigma), theta, M, out)
    return out


def gmm1d_grad_at(y, logw, sigma, mu) -> np.ndarray:
    y, logw, mu = _f32(y), _f64(logw), _f64(mu)
    g = np.zeros(mu.size, np.float64)
    lib().orc_gmm1d_grad_at(y, y.size, mu.size, logw, float(sigma), mu, g)
    return g


def gmmdiag_loglik(Y, logw, sigma, theta) -> np.ndarray:
    """Diagonal d-dimensional mixture; Y [N][d], theta [M][K][d] float32."""
    Y, theta, logw = _f32(Y), _f32(theta), _f64(logw)
    N, d = Y.shape
    M, K, d2 = theta.shape
    assert d == d2
    out = np.zeros(M, np.float64)
    lib().orc_gmmdiag_loglik(Y, N, d, K, logw, float(sigma), theta, M, out)
    return out


# --------------------------------------------------------------------- weights
def reweight(loglik, dbeta, lw):
    """Section 3 weights + Section 4.1.2 incremental weight + ESS.

    Returns (lw_new, W, scalars) with scalars = (logZ_inc, ess, max, lse)."""
    lw = _f64(lw).copy()
    M = lw.size
    W = np.zeros(M, np.float64)
    sc = np.zeros(4, np.float64)
    ll = None if loglik is None else _f64(loglik)
    rc = lib().orc_reweight(_ptr(ll), float(dbeta), lw, M, W, sc)
    if rc:
        raise OracleError(f"reweight status {rc}")
    return lw, W, sc


def ess(lw) -> float:
    lw = _f64(lw)
    return lib().orc_ess(lw, lw.size)


def resample_systematic(W, u32):
    """Exact-integer systematic resampling; returns (ancestors, counts)."""
    W = _f64(W)
    M = W.size
    anc = np.zeros(M, np.int32)
    counts = np.zeros(M, np.int32)
    rc = lib().orc_resample_systematic(W, M, int(u32) & 0xFFFFFFFF, anc, _ptr(counts))
    if rc:
        raise OracleError(f"resample status {rc}")
    return anc, counts


def is_moments(mu, a, var, prop_mean, prop_sd, power, x=None, N=None, seed=0, step=0):
    """Importance-sampling sums {sum w, sum w phi, sum w^2} (Section 2.1);
    x None draws N proposal samples from (seed, PROPOSAL, step)."""
    mu, a = _f64(mu), _f64(a)
    xa = None if x is None else _f32(x)
    n = xa.size if xa is not None else int(N)
    out = np.zeros(3, np.float64)
    lib().orc_is_moments(mu.size, mu, a, float(var), float(prop_mean), float(prop_sd), int(power),
                         _ptr(xa), n, seed, step, out)
    return out


def mrg32k3a(seed, start, n, dtype=np.float32) -> np.ndarray:
    """n MRG32k3a uniforms from stream position `start`: float32 (24-bit
    uniforms) or float64 (z / (m1 + 1))."""
    out = np.zeros(max(int(n), 1), dtype)
    f32 = out if out.dtype == np.float32 else None
    f64 = out if out.dtype == np.float64 else None
    lib().orc_mrg32k3a(np.ascontiguousarray(seed, np.uint32), int(start) & (2**64 - 1), int(n),
                       _ptr(f32), _ptr(f64))
    return out[:n]


def slot_uniforms(seed, step, n) -> np.ndarray:
    """Word 0 of (seed, MULTINOMIAL, step, index i) for i < n."""
    out = np.zeros(max(int(n), 1), np.uint32)
    lib().orc_word_array(seed, P_MULTINOMIAL, step, int(n), out)
    return out[:n]


def resample_multinomial(W, u):
    """Exact-integer multinomial resampling with slot uniforms u (uint32[M])."""
    W = _f64(W)
    M = W.size
    u = np.ascontiguousarray(u, np.uint32)
    if u.size < M:
        raise ValueError("need one uniform per slot")
    anc = np.zeros(M, np.int32)
    rc = lib().orc_resample_multinomial(W, M, u, anc)
    if rc:
        raise OracleError(f"resample status {rc}")
    return anc


def resample_residual(W, v):
    """Exact-integer residual resampling; v (uint32, at least M entries) are
    the residual draws' uniforms.  Returns (ancestors, R)."""
    W = _f64(W)
    M = W.size
    v = np.ascontiguousarray(v, np.uint32)
    if v.size < M:
        raise ValueError("need M uniforms")
    anc = np.zeros(M, np.int32)
    R = C.c_int64(0)
    rc = lib().orc_resample_residual(W, M, v, anc, C.byref(R))
    if rc:
        raise OracleError(f"resample status {rc}")
    return anc, R.value


# ----------------------------------------------------------------------- moves
def _beta_arr(beta, M):
    b = np.atleast_1d(np.asarray(beta, np.float32))
    return _f32(b), (0 if b.size == 1 else 1)


def rwmh_move(y, logw, sigma, box, theta, loglik, beta, scale, seed, step, anc=None,
              slots=None, want_log_alpha=False):
    """Random-walk MH on prior * L^beta (Sections 4.1.1-4.1.2).

    slots (optional): compute only these output slots; outputs are compact.
    want_log_alpha: also return the log acceptance ratios (-inf outside the box)."""
    y, theta, loglik, logw = _f32(y), _f32(theta), _f64(loglik), _f64(logw)
    K, M = theta.shape
    b, bs = _beta_arr(beta, M)
    sl = None if slots is None else np.ascontiguousarray(slots, np.int32)
    n = M if sl is None else sl.size
    th_out = np.zeros((K, n), np.float32)
    l_out = np.zeros(n, np.float64)
    acc = np.zeros(n, np.int32)
    a = None if anc is None else np.ascontiguousarray(anc, np.int32)
    la = np.zeros(n, np.float64)
    lib().orc_rwmh_move_slots(y, y.size, K, logw, float(sigma), float(box[0]), float(box[1]),
                              theta, loglik, _ptr(a), th_out, l_out, M, b, bs, float(scale), seed,
                              step, acc, _ptr(sl), n, _ptr(la))
    return (th_out, l_out, acc, la) if want_log_alpha else (th_out, l_out, acc)


def mala_move(y, logw, sigma, box, theta, loglik, grad, beta, h, seed, step, anc=None,
              slots=None, want_log_alpha=False):
    """MALA move on prior * L^beta with the adjoint gradient (slots as rwmh_move)."""
    y, theta, loglik, logw, grad = _f32(y), _f32(theta), _f64(loglik), _f64(logw), _f32(grad)
    K, M = theta.shape
    b, bs = _beta_arr(beta, M)
    sl = None if slots is None else np.ascontiguousarray(slots, np.int32)
    n = M if sl is None else sl.size
    th_out = np.zeros((K, n), np.float32)
    g_out = np.zeros((K, n), np.float32)
    l_out = np.zeros(n, np.float64)
    acc = np.zeros(n, np.int32)
    a = None if anc is None else np.ascontiguousarray(anc, np.int32)
    la = np.zeros(n, np.float64)
    lib().orc_mala_move_slots(y, y.size, K, logw, float(sigma), float(box[0]), float(box[1]),
                              theta, loglik, grad, _ptr(a), th_out, l_out, g_out, M, b, bs,
                              float(h), seed, step, acc, _ptr(sl), n, _ptr(la))
    return (th_out, l_out, g_out, acc, la) if want_log_alpha else (th_out, l_out, g_out, acc)


def popmcmc_sweep(y, logw, sigma, box, theta, loglik, beta, offsets, scale, seed, sweep):
    """One population-MCMC sweep (Sections 3.1, 4.1.1); returns new state + stats."""
    y, logw = _f32(y), _f64(logw)
    theta = _f32(theta).copy()
    loglik = _f64(loglik).copy()
    K, M = theta.shape
    offsets = np.ascontiguousarray(offsets, np.int32)
    stats = np.zeros(3, np.int64)
    lib().orc_popmcmc_sweep(y, y.size, K, logw, float(sigma), float(box[0]), float(box[1]),
                            theta, loglik, M, _f32(beta), offsets, offsets.size - 1, float(scale),
                            seed, sweep, stats)
    return theta, loglik, stats


def popmcmc_exchange(theta, loglik, beta, offsets, seed, sweep, q0=0, q1=None, want_la=False,
                     flip=None):
    """Stage 2 of a population-MCMC sweep (the exchange moves of Section
    4.1.1) on populations q0 .. q1-1; returns the new state and stats.
    want_la: also the log alpha - log u of every pair attempted (populations
    in order, then pairs); flip: int8 per pair, nonzero takes the opposite
    decision (test hooks for replaying the stage with chosen decisions)."""
    theta = _f32(theta).copy()
    loglik = _f64(loglik).copy()
    K, M = theta.shape
    offsets = np.ascontiguousarray(offsets, np.int32)
    q1 = offsets.size - 1 if q1 is None else int(q1)
    stats = np.zeros(3, np.int64)
    npairs = int(sum(int(offsets[q + 1] - offsets[q]) // 2 + 1 for q in range(q0, q1)))
    la = np.zeros(max(npairs, 1), np.float64) if want_la else None
    fl = None if flip is None else np.ascontiguousarray(flip, np.int8)
    lib().orc_popmcmc_exchange(K, theta, loglik, M, _f32(beta), offsets, int(q0), q1, seed, sweep,
                               stats, _ptr(la), _ptr(fl))
    if want_la:
        return theta, loglik, stats, la[: int(stats[2])]
    return theta, loglik, stats


# -------------------------------------------------------------- particle filter
PF_MSV, PF_LG = 0, 1


def pf_step(kind, phi, chol, bscale, yt, x_in, anc, seed, t):
    """Bootstrap propagate + weight (Sections 3.2, 4.2); x is [d][M]."""
    x_in = _f32(x_in)
    d, M = x_in.shape
    x_out = np.zeros_like(x_in)
    lg = np.zeros(M, np.float64)
    a = None if anc is None else np.ascontiguousarray(anc, np.int32)
    lib().orc_pf_step(kind, d, _f64(phi), _f64(chol), float(bscale), _f32(yt), x_in, _ptr(a),
                      x_out, lg, M, seed, t)
    return x_out, lg


def pf_run(kind, phi, chol, bscale, y, M, seed, want_means=False):
    y = _f32(y)
    T, d = y.shape
    z = C.c_double(0.0)
    means = np.zeros((T, d), np.float64) if want_means else None
    rc = lib().orc_pf_run(kind, d, _f64(phi), _f64(chol), float(bscale), y, T, M, seed,
                          C.byref(z), _ptr(means))
    if rc:
        raise OracleError(f"pf_run status {rc}")
    return (z.value, means) if want_means else z.value


def fsv_step(phi, cholU, B, psi, yt, x_in, anc, seed, t):
    """Factor stochastic volatility (Section 4.2): propagate x ([K][M]) and
    weight by log N(y_t; 0, B diag(exp x) B^T + diag(psi)) (plain m x m
    Cholesky, FP64)."""
    x_in = _f32(x_in)
    K, M = x_in.shape
    B = _f64(B)
    m = B.shape[0]
    x_out = np.zeros_like(x_in)
    lg = np.zeros(M, np.float64)
    a = None if anc is None else np.ascontiguousarray(anc, np.int32)
    lib().orc_fsv_step(K, m, _f64(phi), _f64(cholU), B, _f64(psi), _f32(yt), x_in, _ptr(a),
                       x_out, lg, M, seed, t)
    return x_out, lg


def fsv_run(phi, cholU, B, psi, y, M, seed, want_means=False):
    """Bootstrap filter on the factor SV model (resampling every step)."""
    y = _f32(y)
    T, m = y.shape
    K = len(phi)
    z = C.c_double(0.0)
    means = np.zeros((T, K), np.float64) if want_means else None
    rc = lib().orc_fsv_run(K, m, _f64(phi), _f64(cholU), _f64(B), _f64(psi), y, T, M, seed,
                           C.byref(z), _ptr(means))
    if rc:
        raise OracleError(f"fsv_run status {rc}")
    return (z.value, means) if want_means else z.value


def kalman_lg(phi, Sigma, bscale, y, want_means=False):
    y = _f32(y)
    T, d = y.shape
    means = np.zeros((T, d), np.float64) if want_means else None
    ll = lib().orc_kalman_lg(d, _f64(phi), _f64(Sigma), float(bscale), y, T, _ptr(means))
    return (ll, means) if want_means else ll


def smc_run(y, logw, sigma, box, theta0, betas, kind, scale, ess_frac, seed, n_moves=1):
    """Tempered SMC sampler (Sections 3.3, 4.1.2) with n_moves MH / MALA moves per
    temperature; returns (logZ, theta, ess, resampled)."""
    y, logw = _f32(y), _f64(logw)
    theta = _f32(theta0).copy()
    K, M = theta.shape
    betas = _f64(betas)
    T = betas.size - 1
    z = C.c_double(0.0)
    ess_out = np.zeros(T, np.float64)
    rs = np.zeros(T, np.int32)
    rc = lib().orc_smc_run(y, y.size, K, logw, float(sigma), float(box[0]), float(box[1]), theta,
                           M, betas, T, int(kind), float(scale), int(n_moves), float(ess_frac),
                           seed,
                           C.byref(z), _ptr(ess_out), _ptr(rs))
    if rc:
        raise OracleError(f"smc_run status {rc}")
    return z.value, theta, ess_out, rs
