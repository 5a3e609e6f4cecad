"""Autotuner for the launch shape of the likelihood-bearing kernels: lanes
per particle (Section 4.1.3 splits one likelihood over several threads) and
threads per block, chosen by timing every candidate with CUDA events on the
caller's own inputs, and cached per (op, K, N, M, device name) in a JSON file.
"""
from __future__ import annotations

import json
import os

import torch

from . import _lib as L
from . import api

CACHE = os.environ.get("SMC_AUTOTUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "smc_gb300_autotune.json"))
LANES = (1, 2, 4, 8, 16, 32)
THREADS = (128, 256)
# the population sweep: few lanes per chain win (its chains are many), and
# odd block sizes change how items fall on the SMs
POP_LANES = (1, 2, 4, 8, 16)
POP_THREADS = (128, 192, 256)


def _key(op, K, N, M):
    from . import build
    return f"{torch.cuda.get_device_name()}|{build.source_digest()}|op{op}|K{K}|N{N}|M{M}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass


def time_call(fn, reps=5, inner=1):
    """Median device time (ms) per call of fn(): CUDA events on the current
    stream around `inner` back-to-back calls, median over `reps`."""
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(inner):
            fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) / inner)
    ts.sort()
    return ts[len(ts) // 2]


def tune(ctx: api.Context, op: int, K: int, N: int, M: int, fn, use_cache=True, reps=5,
         inner=1, lanes_list=LANES, threads_list=THREADS):
    """Pick (lanes, threads) for `op` by timing `fn` (which issues the op with
    the context's current override) over all candidates; apply and cache."""
    key = _key(op, K, N, M)
    cache = _load() if use_cache else {}
    if key in cache:
        lanes, threads = cache[key]["lanes"], cache[key]["threads"]
        ctx.set_launch(op, lanes, threads)
        return lanes, threads, cache[key]
    results = []
    for lanes in lanes_list:
        if lanes > 1 and N // lanes < 2:
            continue
        for threads in threads_list:
            if threads % lanes:
                continue
            ctx.set_launch(op, lanes, threads)
            ms = time_call(fn, reps, inner)
            results.append((ms, lanes, threads))
    results.sort()
    ms, lanes, threads = results[0]
    ctx.set_launch(op, lanes, threads)
    entry = {"lanes": lanes, "threads": threads, "ms": ms,
             "all": [[l_, t_, round(m_, 5)] for m_, l_, t_ in results]}
    if use_cache:
        cache = _load()
        cache[key] = entry
        _save(cache)
    return lanes, threads, entry


def tune_loglik(ctx, model, y, theta, **kw):
    out = torch.empty(theta.shape[1], dtype=torch.float64, device="cuda")
    return tune(ctx, L.OP_LOGLIK, model.K, y.numel(), theta.shape[1],
                lambda: api.loglik_batch(ctx, model, y, theta, out=out), **kw)


# data counts and components for which smc_popmcmc_sweep takes the binned
# sweep (data sorted into bins in shared memory), whose launch shape is fixed
BINNED_MIN_N, BINNED_MAX_N, BINNED_MAX_K = 512, 4096, 16


def tune_popmcmc(ctx, sampler, **kw):
    """Chains-per-block / lanes for the persistent sweep of a PopulationMCMC.
    Candidate sweeps advance the chains; the caller re-initialises if needed.
    Where the library takes the binned sweep (one 512-thread block per SM,
    chain groups of 32: no launch parameter to choose) nothing is timed and
    (0, 512, entry) is returned."""
    n, k = sampler.y.numel(), sampler.model.K
    if BINNED_MIN_N <= n <= BINNED_MAX_N and k <= BINNED_MAX_K:
        return 0, 512, {"binned": "one 512-thread CTA per SM, chain groups of 32"}
    s = [10_000]

    def fn():
        sampler.sweep(s[0])
        s[0] += 1
    kw.setdefault("reps", 3)
    kw.setdefault("inner", 10)
    return tune(ctx, L.OP_POPMCMC, sampler.model.K, sampler.y.numel(), sampler.M, fn,
                lanes_list=POP_LANES, threads_list=POP_THREADS, **kw)
