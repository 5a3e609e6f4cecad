"""Sampler drivers over the C ABI: the tempered SMC sampler (Sections 3.3,
4.1.2), population MCMC over many populations (Sections 3.1, 4.1.1) and the
bootstrap particle filter (Sections 3.2, 4.2).

Each driver owns its device buffers (torch tensors), issues the C-ABI calls
of one step on the current stream, and can capture a whole run into one CUDA
graph: every per-step decision (resample or not) is taken on the device
(the ESS flag), so nothing syncs with the host until the run ends.  The
plain and captured forms issue identical kernels with identical Philox
counters, so their outputs are bitwise equal.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib as L
from . import api


def _p(t):
    return None if t is None else t.data_ptr()


def step_records(hist, betas, M, flags=None, accepts=None, n_moves=1):
    """Per-step metrics of a tempered SMC run as plain dicts (one per step
    t = 1..len(hist)-1): temperature, log-evidence increment, ESS (before
    resampling), whether it resampled, the acceptance rate of the moves,
    and the running log Z.  `hist` rows are the reweight scalars
    {log Z increment, ESS, max log-weight, log-sum-exp} (host arrays)."""
    hist = np.asarray(hist, np.float64)
    out, logz = [], 0.0
    for t in range(1, hist.shape[0]):
        logz += float(hist[t, 0])
        r = {"t": t, "beta": float(betas[t]), "log_z_inc": float(hist[t, 0]),
             "log_z": logz, "ess": float(hist[t, 1]), "ess_frac": float(hist[t, 1]) / M}
        if flags is not None:
            r["resampled"] = bool(flags[t])
        if accepts is not None:
            r["accept_rate"] = float(accepts[t]) / (M * n_moves)
        out.append(r)
    return out


def write_jsonl(records, path):
    """One JSON object per line."""
    import json
    with open(path, "w") as f:
        for r in records:
            f.write(json.dumps(r) + "\n")


def _dev(a, dtype):
    if isinstance(a, torch.Tensor):
        return a.to(device="cuda", dtype=dtype).contiguous()
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _check_replacement(name, old, new):
    """A sampler's steps pass its buffers' pointers and sizes to the C ABI
    without re-checking them, so a device tensor (or a tuple of them) may
    only be replaced by one of the same dtype, shape and device, contiguous."""
    if isinstance(old, tuple):
        if not isinstance(new, tuple) or len(new) != len(old):
            raise ValueError(f"{name} must stay a tuple of {len(old)} buffers")
        for i, (o, n) in enumerate(zip(old, new)):
            _check_replacement(f"{name}[{i}]", o, n)
        return
    if isinstance(old, torch.Tensor):
        ok = (isinstance(new, torch.Tensor) and new.dtype == old.dtype and
              new.shape == old.shape and new.device == old.device and new.is_contiguous())
        if not ok:
            raise ValueError(f"{name} may only be replaced by a contiguous tensor of dtype "
                             f"{old.dtype}, shape {tuple(old.shape)} on {old.device}")
    elif old is None and isinstance(new, torch.Tensor):
        raise ValueError(f"{name} is not used by this sampler")



def _sum_increments(hist, t_done: int) -> float:
    """log Z = the sum of the per-step increments the reweighting kernels
    wrote to hist[t, 0]: at most T numbers, read once and added exactly
    rounded on the host (no device arithmetic outside the library)."""
    return math.fsum(hist[1:t_done + 1, 0].cpu().tolist())

class _Graphable:
    """run(graph=True) captures `_body(...)` once and replays it.  Device
    buffers set at construction may later be replaced only by tensors of the
    same dtype, shape and device (`_check_replacement`)."""

    _FIXED = ("M", "K", "T", "d", "n_pops")  # sizes the C calls take with the buffers

    def __setattr__(self, name, value):
        if name in self.__dict__:
            old = self.__dict__[name]
            if name in self._FIXED and value != old:
                raise ValueError(f"{name} is fixed when the sampler is built")
            _check_replacement(name, old, value)
        object.__setattr__(self, name, value)

    def _capture(self, fn):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                fn()
        torch.cuda.current_stream().wait_stream(s)
        return g


class SMCSampler(_Graphable):
    """Tempered SMC sampler: particles from the uniform prior, beta_0 = 0; per
    step t: reweight by (beta_t - beta_{t-1}) l, resample (systematic) iff
    ESS < ess_frac * M, then n_moves RW-MH or MALA moves targeting
    prior * L^beta_t (Section 4.1.2 uses 10).  Move r of step t draws with the
    step counter t + r 2^32; only the first move gathers the ancestors."""

    def __init__(self, ctx: api.Context, model: api.GMM, y, theta0, betas, kind=L.MOVE_RW,
                 scale=0.1, seed=1234, ess_frac=0.5, n_moves=1, resampler="systematic"):
        self.ctx, self.model, self.kind = ctx, model, kind
        self.scale, self.seed, self.ess_frac = float(scale), int(seed), float(ess_frac)
        self.n_moves = int(n_moves)
        if self.n_moves < 1:
            raise ValueError("n_moves must be at least 1")
        if resampler not in api.RESAMPLERS:
            raise ValueError(f"resampler must be one of {api.RESAMPLERS}")
        self.resampler = resampler
        self.y = _dev(y, torch.float32)
        th = _dev(theta0, torch.float32)
        if th.dim() != 2 or self.y.dim() != 1:
            raise ValueError("theta0 must be [K, M] and y one-dimensional")
        self.K, self.M = th.shape
        self.betas_host = np.asarray(betas, np.float64)
        self.T = self.betas_host.size - 1
        self.betas = _dev(self.betas_host.astype(np.float32), torch.float32)
        self.theta = (th.clone(), torch.empty_like(th))
        self.ll = tuple(torch.empty(self.M, dtype=torch.float64, device="cuda") for _ in range(2))
        mala = kind == L.MOVE_MALA
        self.grad = tuple(torch.empty_like(th) for _ in range(2)) if mala else (None, None)
        self.lw = torch.zeros(self.M, dtype=torch.float64, device="cuda")
        self.W = torch.empty(self.M, dtype=torch.float64, device="cuda")
        self.anc = torch.empty(self.M, dtype=torch.int32, device="cuda")
        self.flags = torch.zeros(self.T + 1, dtype=torch.int32, device="cuda")
        self.hist = torch.zeros(self.T + 1, 4, dtype=torch.float64, device="cuda")
        self.accepts = torch.zeros(self.T + 1, dtype=torch.int32, device="cuda")
        # per-step views, made once (a step issues its calls without building tensors)
        self._views = [(self.flags[t:t + 1], self.hist[t], self.betas[t:t + 1],
                        self.accepts[t:t + 1]) for t in range(self.T + 1)]
        ctx.reserve(self.M)
        self.reset(theta0)

    def reset(self, theta0=None):
        if theta0 is not None:
            self.theta[0].copy_(_dev(theta0, torch.float32))
        self.cur = 0
        self.t_done = 0  # steps completed
        self.lw.zero_()
        self.accepts.zero_()
        self.flags.zero_()
        self.hist.zero_()
        api.loglik_batch(self.ctx, self.model, self.y, self.theta[0], out=self.ll[0],
                         grad=self.grad[0])

    def step(self, t: int):
        c, n = self.cur, 1 - self.cur
        ctx = self.ctx
        db = float(self.betas_host[t] - self.betas_host[t - 1])
        flag, hist, beta, accepts = self._views[t]
        # the sampler's own buffers were checked when it was built: the calls
        # go to the C ABI directly (the api layer's per-call checks cost more
        # host time than a small step's kernels)
        lib, h, st = L.load(), ctx.handle, api._stream()
        fp = flag.data_ptr()
        if self.resampler == "systematic":  # one call, one pass fewer
            api._chk(lib.smc_reweight_resample(h, self.ll[c].data_ptr(), db, self.lw.data_ptr(),
                                               self.M, self.W.data_ptr(), hist.data_ptr(), fp,
                                               self.ess_frac, self.seed, t, self.anc.data_ptr(),
                                               None, st), "smc_reweight_resample")
        else:
            api.reweight(ctx, self.ll[c], db, self.lw, self.W, hist, flag, self.ess_frac)
            api.resample(ctx, self.resampler, self.W, self.seed, t, anc=self.anc, do_flag=flag,
                         logw_reset=self.lw)
        m = C.byref(self.model.cstruct())
        nd, bp, ap = self.y.numel(), beta.data_ptr(), accepts.data_ptr()
        for r in range(self.n_moves):
            first = r == 0
            api._chk(lib.smc_mh_move(h, m, self.y.data_ptr(), nd, self.theta[c].data_ptr(),
                                     self.ll[c].data_ptr(), _p(self.grad[c]),
                                     self.anc.data_ptr() if first else None,
                                     fp if first else None, self.theta[n].data_ptr(),
                                     self.ll[n].data_ptr(), _p(self.grad[n]), self.M, bp, 0,
                                     self.scale, self.kind, self.seed, t + (r << 32), ap, st),
                     "smc_mh_move")
            c, n = n, c
        self.cur = c

    def _body(self, t0: int = 1, t1: int | None = None):
        for t in range(t0, (self.T if t1 is None else t1) + 1):
            self.step(t)

    def run(self, graph: bool = False, stop: int | None = None):
        """Run the steps after the last completed one up to `stop` (default
        T); returns log Z so far (sum of the per-step increments).  Step t
        draws from counters fixed by (seed, t), so a run split anywhere, or
        resumed from a saved state, is bitwise the uninterrupted run."""
        t0, t1 = self.t_done + 1, (self.T if stop is None else int(stop))
        if t1 >= t0:
            if graph:
                start = self.cur
                g = self._capture(lambda: self._body(t0, t1))
                self.cur = start
                # the capture recorded the buffer swaps; replay from the same state
                self._graph = g
                g.replay()
                self.cur = (start + (t1 - t0 + 1) * self.n_moves) % 2
            else:
                self._body(t0, t1)
            self.t_done = t1
        return self.log_evidence()

    def log_evidence(self) -> float:
        return _sum_increments(self.hist, self.t_done)

    def history(self) -> list:
        """Per-step metrics of the completed steps (see step_records)."""
        n = self.t_done + 1
        return step_records(self.hist[:n].cpu().numpy(), self.betas_host[:n], self.M,
                            self.flags[:n].cpu().numpy(), self.accepts[:n].cpu().numpy(),
                            self.n_moves)

    def state_dict(self) -> dict:
        """Everything a resumed run needs (host copies): the particles, their
        log-likelihoods (and gradients), log-weights, per-step records and
        the number of completed steps."""
        c = self.cur
        return {"theta": self.theta[c].cpu(), "ll": self.ll[c].cpu(),
                "grad": None if self.grad[c] is None else self.grad[c].cpu(),
                "lw": self.lw.cpu(), "flags": self.flags.cpu(), "hist": self.hist.cpu(),
                "accepts": self.accepts.cpu(), "t_done": self.t_done}

    def load_state_dict(self, d: dict):
        self.cur = 0
        self.theta[0].copy_(d["theta"])
        self.ll[0].copy_(d["ll"])
        if self.grad[0] is not None:
            self.grad[0].copy_(d["grad"])
        for name in ("lw", "flags", "hist", "accepts"):
            getattr(self, name).copy_(d[name])
        self.t_done = int(d["t_done"])

    @property
    def state(self):
        return self.theta[self.cur], self.ll[self.cur]


class PopulationMCMC(_Graphable):
    """Many independent populations of tempered chains (ragged sizes), one
    persistent launch per sweep: RW-MH for every chain, then the exchange
    moves on the paper's alternating adjacent pairs."""

    def __init__(self, ctx: api.Context, model: api.GMM, y, offsets, betas, theta0, scale=0.1,
                 seed=1):
        self.ctx, self.model, self.scale, self.seed = ctx, model, float(scale), int(seed)
        self.y = _dev(y, torch.float32)
        off = np.asarray(offsets, np.int32)
        self.offsets = _dev(off, torch.int32)
        self.n_pops = off.size - 1
        self.beta = _dev(betas, torch.float32)
        self.theta = _dev(theta0, torch.float32).clone()
        if self.theta.dim() != 2 or self.y.dim() != 1:
            raise ValueError("theta0 must be [K, M] and y one-dimensional")
        self.K, self.M = self.theta.shape
        if self.beta.numel() != self.M or off[-1] != self.M:
            raise ValueError("betas and the population offsets must cover the M chains")
        self.ll = torch.empty(self.M, dtype=torch.float64, device="cuda")
        self.stats = torch.zeros(3, dtype=torch.int64, device="cuda")
        ctx.reserve(self.M, self.n_pops)
        api.loglik_batch(ctx, model, self.y, self.theta, out=self.ll)

    def sweep(self, s: int):
        # buffers checked at construction (shapes fixed): straight to the C ABI
        api._chk(L.load().smc_popmcmc_sweep(
            self.ctx.handle, C.byref(self.model.cstruct()), self.y.data_ptr(), self.y.numel(),
            self.theta.data_ptr(), self.ll.data_ptr(), self.M, self.beta.data_ptr(),
            self.offsets.data_ptr(), self.n_pops, self.scale, self.seed, s,
            self.stats.data_ptr(), api._stream()), "smc_popmcmc_sweep")

    def state_dict(self) -> dict:
        """The chains' states, log-likelihoods and the move statistics (host
        copies); sweep s draws from counters fixed by (seed, s)."""
        return {"theta": self.theta.cpu(), "ll": self.ll.cpu(), "stats": self.stats.cpu()}

    def load_state_dict(self, d: dict):
        self.theta.copy_(d["theta"])
        self.ll.copy_(d["ll"])
        self.stats.copy_(d["stats"])

    def run(self, n_sweeps: int, start: int = 0, graph: bool = False):
        if graph:
            g = self._capture(lambda: [self.sweep(start + i) for i in range(n_sweeps)])
            g.replay()
            self._graph = g
        else:
            for i in range(n_sweeps):
                self.sweep(start + i)


class ParticleFilter(_Graphable):
    """Bootstrap particle filter resampling after every step (systematic by
    default; multinomial or residual on request); log Z = sum_t [LSE(log g_t)
    - log M]."""

    def __init__(self, ctx: api.Context, model: api.PFModel, y, M: int, seed: int = 77,
                 resampler: str = "systematic"):
        self.ctx, self.model, self.M, self.seed = ctx, model, int(M), int(seed)
        if resampler not in api.RESAMPLERS:
            raise ValueError(f"resampler must be one of {api.RESAMPLERS}")
        self.resampler = resampler
        self.y = _dev(y, torch.float32)
        self.T = self.y.shape[0]
        self.d = int(np.asarray(model.phi).size)  # state dimension (FSV: factors)
        if self.y.shape[1] != model.obs_dim:
            raise ValueError("observations do not match the model's dimension")
        self.x = tuple(torch.zeros(self.d, self.M, device="cuda") for _ in range(2))
        self.logg = torch.empty(self.M, dtype=torch.float64, device="cuda")
        self.lw = torch.zeros(self.M, dtype=torch.float64, device="cuda")
        self.W = torch.empty(self.M, dtype=torch.float64, device="cuda")
        self.anc = torch.arange(self.M, dtype=torch.int32, device="cuda")
        self.hist = torch.zeros(self.T + 1, 4, dtype=torch.float64, device="cuda")
        self._views = [(self.y[max(t - 1, 0)], self.hist[t]) for t in range(self.T + 1)]
        ctx.reserve(self.M)
        self.cur = 0
        self.t_done = 0  # steps completed

    def reset(self):
        for x in self.x:
            x.zero_()
        self.lw.zero_()
        self.hist.zero_()
        self.anc.copy_(torch.arange(self.M, dtype=torch.int32, device="cuda"))
        self.cur = 0
        self.t_done = 0

    def step(self, t: int):
        c, n = self.cur, 1 - self.cur
        y_t, hist = self._views[t]
        lib, h, st = L.load(), self.ctx.handle, api._stream()
        # buffers checked at construction: straight to the C ABI
        if self.resampler == "systematic":
            # one call: step, reweighting, normalisation with the tile sums,
            # resampling into anc
            api._chk(lib.smc_pf_filter_step(h, C.byref(self.model.cstruct_cached()),
                                            y_t.data_ptr(), self.x[c].data_ptr(),
                                            self.anc.data_ptr(), self.x[n].data_ptr(),
                                            self.logg.data_ptr(),
                                            self.lw.data_ptr(), self.M, self.W.data_ptr(),
                                            hist.data_ptr(), None, 0.5, self.seed, t, None, st),
                     "smc_pf_filter_step")
        else:
            api._chk(lib.pf_step(h, C.byref(self.model.cstruct_cached()), y_t.data_ptr(),
                                 self.x[c].data_ptr(), self.anc.data_ptr(), self.x[n].data_ptr(),
                                 self.logg.data_ptr(), self.M, self.seed, t, st), "pf_step")
            api.reweight(self.ctx, self.logg, 1.0, self.lw, self.W, hist, None, 0.5)
            api.resample(self.ctx, self.resampler, self.W, self.seed, t, anc=self.anc,
                         logw_reset=self.lw)
        self.cur = n

    def run(self, graph: bool = False, steps: int | None = None):
        """Run the steps after the last completed one up to step `steps`
        (default T); returns log Z so far.  Split or resumed runs are bitwise
        the uninterrupted run (step t's draws are fixed by (seed, t))."""
        t0, t1 = self.t_done + 1, (self.T if steps is None else int(steps))
        if t1 >= t0:
            if graph:
                start = self.cur
                g = self._capture(lambda: [self.step(t) for t in range(t0, t1 + 1)])
                self.cur = start
                g.replay()
                self._graph = g
                self.cur = (start + (t1 - t0 + 1)) % 2
            else:
                for t in range(t0, t1 + 1):
                    self.step(t)
            self.t_done = t1
        return _sum_increments(self.hist, self.t_done)

    def state_dict(self) -> dict:
        """The particles, log-weights, ancestors of the last resampling (the
        next step gathers through them), per-step records and the number of
        completed steps (host copies)."""
        return {"x": self.x[self.cur].cpu(), "lw": self.lw.cpu(), "anc": self.anc.cpu(),
                "hist": self.hist.cpu(), "t_done": self.t_done}

    def load_state_dict(self, d: dict):
        self.cur = 0
        self.x[0].copy_(d["x"])
        for name in ("lw", "anc", "hist"):
            getattr(self, name).copy_(d[name])
        self.t_done = int(d["t_done"])
