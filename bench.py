#!/usr/bin/env python
"""Benchmark of the SMC / population-MCMC hot path on GB300.

Default workload (the batched population-MCMC configuration): 512
independent populations with 8..128 tempered chains each (34.8k chains),
univariate 8-component mixture, N = 1000 observations.  One step = one sweep
= one persistent launch (random-walk MH with the fused likelihood for every
chain, then the exchange moves).  Metric: particle-datum log-likelihood
evaluations per second (chains x N per sweep).

Other workloads (--workload): pf (d = 3 MSV particle filter, M = 2^20; step
= one filter step), resample (reweight + systematic resampling bandwidth at
M = 2^24), diag (diagonal mixture d = 32, K = 16, N = 65536, M = 4096 on the
tensor cores; step = one likelihood call), fsv (the paper's factor SV particle
filter, Table 3 sizes; step = one whole T = 200 run), tables (the paper's
Tables 1 and 2 configurations, every size; step = one whole run of each),
mala (the MALA tempered sampler; step = one whole 50-temperature run),
is (Section 2.1's importance-sampling example, N = 2^24 draws; step = one
call), mrg (MRG32k3a, 155,648 streams x 1024 numbers; step = one call),
peaks (the MUFU / FMA / FP64 /
conversion rates used as roofline denominators).  The default run also
reports, under "secondary", the paper's Tables 1 and 2 replicated, the
tempered SMC sampler (M = 8192), the MALA
sampler (M = 65536), the particle filter and the tensor-core likelihood,
each in its plain and CUDA-graph forms where both exist.

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs its own independent copy of the workload
(weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 2**20
FLUSH_BYTES = 256 * 2**20


def l2_note(what):
    return (f"256 MiB buffer (2x L2) written, then another read, before every timed {what}, "
            "outside its events")


class L2Flush:
    """Between timed iterations: write a 256 MiB buffer (twice L2), then read
    a second one, so that L2 holds none of the timed data and none of the
    flush's own dirty lines either (their write-back to HBM happens here,
    outside the events, instead of inside the next timed kernel)."""

    def __init__(self, torch):
        self.torch = torch
        self.w = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        self.r = torch.zeros(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        self.out = torch.empty((), dtype=torch.float32, device="cuda")

    def __call__(self, v=0.5):
        self.w.fill_(float(v))
        self.torch.sum(self.r, dim=0, out=self.out)


# ------------------------------------------------------------------ helpers
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms in the
    background.  Entering waits (up to 3 s) for the first reading, so that
    the sampler is running when the timed region starts; the summary keeps
    the readings taken after that point."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.start = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except OSError:
            self.proc = None
        self.start = len(self.lines)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[self.start:] or self.lines
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "_fallback": True}


def profile_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(kernel)
    if not e:
        return None
    from paper_0905_2441_gb300 import build as b
    try:
        now = b.source_digest(e.get("sources"))
    except FileNotFoundError:
        return None
    if e.get("source_digest") != now:
        return None  # the kernel changed since the counters were taken
    return e.get("bytes_per_launch")


class Dist:
    """One process per GPU (torchrun's RANK / WORLD_SIZE / LOCAL_RANK): a
    barrier and the max / sum of per-rank numbers, over NCCL on the GPUs (or
    gloo on the CPU, as the multi-process tests run it).  No data-path
    collective: every rank runs an independent replica of the workload."""

    def __init__(self, backend=None):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.backend = backend
        self.pg = False

    def init(self, torch):
        if self.world > 1:
            import torch.distributed as dist
            if self.backend is None:
                self.backend = "nccl" if torch.cuda.is_available() else "gloo"
            if self.backend == "nccl":
                dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
            else:
                dist.init_process_group(self.backend)
            self.pg = True

    def _dev(self):
        return "cuda" if self.backend == "nccl" else "cpu"

    def barrier(self, torch):
        if self.pg:
            import torch.distributed as dist
            dist.barrier()

    def max(self, torch, v: float) -> float:
        if not self.pg:
            return v
        import torch.distributed as dist
        t = torch.tensor([v], dtype=torch.float64, device=self._dev())
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, torch, v: float) -> float:
        if not self.pg:
            return v
        import torch.distributed as dist
        t = torch.tensor([v], dtype=torch.float64, device=self._dev())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    def throughput(self, torch, units: float, seconds: float):
        """Whole-job rate: the units every rank processed over the slowest
        rank's time (weak scaling: each rank keeps its own fixed work)."""
        t_max = self.max(torch, seconds)
        return self.sum(torch, units) / t_max, t_max

    def close(self):
        if self.pg:
            import torch.distributed as dist
            dist.destroy_process_group()


# ------------------------------------------------------------------ CPU baseline (oracle)
def popmcmc_config(w, M):
    """The population-MCMC workload's description, shared by both arms."""
    return {"workload": w.name, "n_pops": w.n_pops, "chains": M, "K": w.K, "N": w.N,
            "pop_sizes": "uniform 8..128", "temperatures": "geometric 1e-3..1 per population",
            "rw_scale": w.scale}


class CpuPopSample:
    """The FP64 oracle on a bounded sample of the population-MCMC workload
    (its first `sample_pops` populations), set up once; `run` continues the
    chains for as many sweeps as fit in ~budget_s (at least one)."""

    def __init__(self, w, sample_pops):
        import oracle
        import synth
        self.w, self.pops = w, sample_pops
        off = synth.population_offsets(w.n_pops, seed=w.pop_seed)
        self.M_total = int(off[-1])
        self.y = w.data()
        th = synth.population_particles(w.K, off)
        beta = synth.population_betas(off)
        self.sub = off[: sample_pops + 1].copy()
        self.m = int(self.sub[-1])
        self.ths, self.bs = th[:, :self.m].copy(), beta[:self.m].copy()
        self.ll = oracle.gmm1d_loglik(self.y, w.logw(), w.sigma, self.ths)
        self.sweep = 0

    def run(self, budget_s, max_sweeps):
        import oracle
        w = self.w
        t0 = time.perf_counter()
        n = 0
        while n < max_sweeps and (time.perf_counter() - t0) < budget_s:
            self.ths, self.ll, _ = oracle.popmcmc_sweep(self.y, w.logw(), w.sigma, (-10, 10),
                                                        self.ths, self.ll, self.bs, self.sub,
                                                        w.scale, 3, self.sweep)
            self.sweep += 1
            n += 1
        dt = time.perf_counter() - t0
        return {"value": self.m * w.N * n / dt, "unit": "p*d/s", "cores": 1, "kind": "oracle",
                "seconds": dt,
                "sample": f"{self.pops} of {w.n_pops} populations ({self.m} chains), {n} sweeps, "
                          f"{dt:.2f} s single-threaded FP64"}


def cpu_popmcmc(w, budget_s=10.0, sample_pops=16, max_sweeps=200):
    """The FP64 oracle on a bounded sample: the first `sample_pops`
    populations of the same workload, as many sweeps as fit in ~budget_s."""
    return CpuPopSample(w, sample_pops).run(budget_s, max_sweeps)


def _cpu_worker(job):
    """One process of the all-cores oracle timing: a slice of populations."""
    first, count, budget_s = job
    import oracle
    import synth
    w = synth.GMM8_POP
    off = synth.population_offsets(w.n_pops, seed=w.pop_seed)
    y = w.data()
    th = synth.population_particles(w.K, off)
    beta = synth.population_betas(off)
    sub = (off[first: first + count + 1] - off[first]).astype(np.int32)
    a, b = int(off[first]), int(off[first + count])
    ths, bs = th[:, a:b].copy(), beta[a:b].copy()
    ll = oracle.gmm1d_loglik(y, w.logw(), w.sigma, ths)
    t0 = time.perf_counter()
    n = 0
    while n < 1000 and (time.perf_counter() - t0) < budget_s:
        ths, ll, _ = oracle.popmcmc_sweep(y, w.logw(), w.sigma, (-10, 10), ths, ll, bs, sub,
                                          w.scale, 3, n)
        n += 1
    return (b - a) * w.N * n, time.perf_counter() - t0


def cpu_popmcmc_all_cores(budget_s=8.0, per_worker=16):
    """The same oracle on every host core: independent slices of populations
    in a process pool (started with spawn), each for ~budget_s; the value is
    all particle-data evaluated over the longest worker's time."""
    import multiprocessing as mp
    import synth
    n = max(1, os.cpu_count() or 1)
    n = min(n, synth.GMM8_POP.n_pops // per_worker)
    jobs = [(i * per_worker, per_worker, budget_s) for i in range(n)]
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_cpu_worker, jobs)
    pd = sum(r[0] for r in res)
    t = max(r[1] for r in res)
    return {"value": pd / t, "unit": "p*d/s", "cores": n,
            "sample": f"{n} processes x {per_worker} populations, ~{budget_s:.0f} s each, FP64"}


# ------------------------------------------------------------------ GPU workloads
def bench_popmcmc(args, torch, dist):
    """The configured workload: 512 populations, 34,591 chains, K = 8,
    N = 1000, one persistent launch per sweep, 1000 sweeps captured in one
    CUDA graph.  One step = one replay of that graph (the sweep counters are
    fixed at capture), the L2 flushed before every step outside its events.
    The plain form (one launch per sweep, L2 flushed before each) is timed
    beside it, as is the end-to-end form through the public API with host
    buffers."""
    import paper_0905_2441_gb300 as P
    from paper_0905_2441_gb300 import autotune, samplers
    import synth
    w = synth.GMM8_POP
    off = synth.population_offsets(w.n_pops, seed=w.pop_seed)
    y = w.data()
    th0 = synth.population_particles(w.K, off, seed=4 + dist.rank)
    beta = synth.population_betas(off)
    ctx = P.Context()
    model = P.GMM(w.K, w.sigma)
    smp = samplers.PopulationMCMC(ctx, model, y, off, beta, th0, scale=w.scale, seed=3 + dist.rank)
    M, N = smp.M, w.N
    # launch shape: the binned sweep (data in shared memory) has one shape;
    # the lanes-per-chain sweep (longer data) is autotuned
    binned = (autotune.BINNED_MIN_N <= N <= autotune.BINNED_MAX_N and
              w.K <= autotune.BINNED_MAX_K)
    lanes, threads, tune = autotune.tune_popmcmc(ctx, smp, use_cache=not args.retune)
    smp.theta.copy_(torch.from_numpy(th0).cuda())
    P.loglik_batch(ctx, model, smp.y, smp.theta, out=smp.ll)
    ctx.check()
    flush = L2Flush(torch)
    stream = torch.cuda.current_stream()
    S = args.graph_sweeps
    # ---- the captured run of S sweeps
    capt = torch.cuda.Stream()
    capt.wait_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(capt):
        with torch.cuda.graph(g, stream=capt):
            for i in range(S):
                smp.sweep(100_000 + i)
    stream.wait_stream(capt)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    # ---- timed: K replays, L2 flushed before each, CUDA events per replay
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    dist.barrier(torch)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush(i)
            ev[i][0].record(stream)
            g.replay()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    dist.barrier(torch)
    ctx.check()
    per = [a.elapsed_time(b) for a, b in ev]
    t_dev = sum(per) / 1e3
    t_max = dist.max(torch, t_dev)
    pd_rank = float(M) * N * S * args.steps
    value = dist.sum(torch, pd_rank) / t_max
    t_sweep = t_dev / (args.steps * S)
    # the state after the timed run and one more plain sweep from it, kept
    # for the oracle's check (outside every timed region)
    snap = {"theta": smp.theta.cpu().numpy(), "ll": smp.ll.cpu().numpy(), "sweep": 7_000_000}
    smp.sweep(snap["sweep"])
    snap["theta1"], snap["ll1"] = smp.theta.cpu().numpy(), smp.ll.cpu().numpy()
    ctx.check()
    # ---- plain form: one launch per sweep, L2 flushed before each
    Kp = max(20, min(200, args.steps * 10))
    evp = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(Kp)]
    for i in range(Kp):
        flush(i)
        _hold(torch)
        evp[i][0].record(stream)
        smp.sweep(200_000 + i)
        evp[i][1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    t_plain = sum(a.elapsed_time(b) for a, b in evp) / 1e3 / Kp
    # ---- end to end through the public API with host buffers
    # two population groups on two streams (four measured slower: the host
    # then takes longer to issue a step's twelve calls than the GPU to run them)
    dist.barrier(torch)
    e2e = e2e_popmcmc_pipelined(args, torch, P, smp, lanes, threads, 2)
    dist.barrier(torch)
    single = e2e_popmcmc(args, torch, P, ctx, smp)
    for r in (e2e, single):  # whole job: all ranks' units over the slowest rank's time
        r["value"] = dist.sum(torch, r.pop("_units")) / dist.max(torch, r.pop("_seconds"))
    e2e["single_stream"] = single
    # ---- roofline: MUFU ops of the sweep kernel vs the measured ex2 rate
    ex2_rate, ex2_ms = measure_peak(P, 0)
    mufu_per_launch = float(M) * N * (w.K + 1)  # K ex2 + 1 lg2 per particle-datum
    kname = "k_popmcmc_binned<8>" if binned else "k_popmcmc_sweep<8,true>"
    sm_mhz = clk.summary()["sm_mhz"]

    def roofline(t_launch, what):
        return {"bound": "alu", "pipe": "MUFU (ex2)", "achieved": mufu_per_launch / t_launch / 1e9,
                "peak": ex2_rate / 1e9, "unit": "Gop/s",
                "frac": mufu_per_launch / t_launch / ex2_rate,
                "traffic": profile_traffic("k_popmcmc_binned" if binned else "k_popmcmc_sweep"),
                "kernel": kname, "ops_per_launch": mufu_per_launch, "launch_time": what,
                "peak_source": "measured in this run: ex2.approx issue rate, all SMs, "
                               f"{ex2_ms:.2f} ms microbenchmark",
                # per datum the kernel issues the K ex2 (the logarithm is taken
                # once per chain segment, not per datum)
                "issued_count": "K ex2 per particle-datum",
                "frac_issued_count": float(M) * N * w.K / t_launch / ex2_rate}
    roof = roofline(t_sweep, f"average sweep launch inside the captured {S}-sweep run")
    if sm_mhz:
        roof["sm_mhz_under_load"] = sm_mhz
    out = {
        "metric": "particle-datum loglik evals/s (population MCMC sweeps)",
        "value": value, "unit": "p*d/s", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded mixture data and chain states; no dataset)",
        "config": {**popmcmc_config(w, M), "sweeps_per_step": S,
                   "step": f"one replay of a CUDA graph of {S} sweeps (one launch per sweep, "
                           "sweep counters fixed at capture)",
                   "launch": tune.get("binned") if binned else
                   {"lanes_per_chain": lanes, "threads_per_block": threads},
                   "l2": l2_note("step"),
                   "parallelism": f"independent populations per rank x{dist.world}"},
        "forms": {"graph_captured": {"sweeps": S, "value": float(M) * N / t_sweep,
                                     "us_per_sweep": 1e6 * t_sweep},
                  "plain_per_step": {"value": float(M) * N / t_plain, "us_per_sweep": 1e6 * t_plain,
                                     "sweeps": Kp, "l2": "flushed before every sweep",
                                     "roofline_frac": roofline(t_plain, "plain")["frac"]}},
        # per replay: the S sweeps and the binned layout's build (captured at
        # the head of the graph when the binned sweep runs)
        "roofline": roof, "e2e": e2e, "gpu_launches": args.steps * (S + (1 if binned else 0)),
        "clocks": clk.summary(), "wall_s": wall, "autotune": tune,
        "_oracle_check": snap,
    }
    ctx.close()
    return out


def popmcmc_oracle_check(w, snap, n_chains=400, sample_pops=16):
    """Observed error against the FP64 oracle (part of the CPU leg, outside
    every timed region): (1) the relative error of the stored
    log-likelihoods of sampled chains after the timed run, (2) one plain
    sweep from that state replayed by the oracle on the first populations:
    chains that differ, and how many MH decisions lay inside the FP32 band
    |log alpha - log u| < 5e-3 where the two may legitimately part."""
    import oracle
    import synth
    off = synth.population_offsets(w.n_pops, seed=w.pop_seed)
    y, logw = w.data(), w.logw()
    th, ll = snap["theta"], snap["ll"]
    M = th.shape[1]
    idx = np.random.default_rng(11).choice(M, n_chains, replace=False)
    ref = oracle.gmm1d_loglik(y, logw, w.sigma, th[:, idx])
    rel = float(np.max(np.abs(ll[idx] - ref) / np.abs(ref)))
    sub = off[: sample_pops + 1].copy()
    m = int(sub[-1])
    beta = synth.population_betas(off)[:m]
    ths, lls = th[:, :m].copy(), ll[:m].copy()
    seed = 3
    rt, rl, _ = oracle.popmcmc_sweep(y, logw, w.sigma, (-10, 10), ths, lls, beta, sub, w.scale,
                                     seed, snap["sweep"])
    g_th, g_ll = snap["theta1"][:, :m], snap["ll1"][:m]
    same = np.all(np.isclose(g_th, rt, rtol=3e-7, atol=2e-6), axis=0) & \
        np.isclose(g_ll, rl, rtol=1e-5, atol=0)
    _, _, _, la = oracle.rwmh_move(y, logw, w.sigma, (-10, 10), ths, lls, beta, w.scale, seed,
                                   snap["sweep"], want_log_alpha=True)
    lu = np.log(np.array([oracle.u01(int(oracle.draw_words(seed, oracle.P_ACCEPT, snap["sweep"],
                                                               c, 0)[0])) for c in range(m)]))
    band = int(np.sum(np.isfinite(la) & (np.abs(la - lu) < 5e-3)))
    pops_diff = int(sum(1 for q in range(sample_pops) if not same[sub[q]:sub[q + 1]].all()))
    return {"max_rel_loglik_err": rel, "chains_checked": n_chains,
            "sweep_replayed": {"populations": sample_pops, "chains": m,
                               "chains_differing": int((~same).sum()),
                               "populations_differing": pops_diff,
                               "mh_decisions_in_fp32_band": band},
            "tolerance": "relative 1e-5 per log-likelihood"}


def e2e_popmcmc(args, torch, P, ctx, smp):
    """Per step, on one stream: pinned host -> device copy of the chain
    state, one sweep through the public API, device -> host copy of the new
    state.  The state
    (log-likelihoods, then the K x M means) sits in one device buffer with a
    pinned host mirror, so each direction is one copy."""
    M, K, N = smp.M, smp.K, smp.y.numel()
    nb = M * 8 + K * M * 4
    dev = torch.empty(nb, dtype=torch.uint8, device="cuda")
    host = torch.empty(nb, dtype=torch.uint8).pin_memory()
    ll_v = dev[: M * 8].view(torch.float64)
    th_v = dev[M * 8:].view(torch.float32).view(K, M)
    ll_v.copy_(smp.ll)
    th_v.copy_(smp.theta)
    host.copy_(dev)
    smp.theta, smp.ll = th_v, ll_v  # the sampler's state now lives in the one buffer
    stream = torch.cuda.current_stream()
    steps = max(3, min(args.steps, 200))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for i in range(steps):
        dev.copy_(host, non_blocking=True)
        smp.sweep(50_000 + i)
        host.copy_(dev, non_blocking=True)
    b.record(stream)
    b.synchronize()
    t = a.elapsed_time(b) / 1e3
    return {"value": float(M) * N * steps / t, "unit": "p*d/s", "h2d_bytes_per_step": nb,
            "d2h_bytes_per_step": nb, "steps": steps, "_units": float(M) * N * steps,
            "_seconds": t}


def e2e_popmcmc_pipelined(args, torch, P, smp, lanes, threads, parts=2):
    """The same step end to end with the populations in `parts` contiguous
    groups, each a sampler with its own context, device buffer, pinned host
    mirror and stream, so that one group's copies overlap another group's
    sweep.  Every population is swept once per step as before; a group keys
    its draws by its own chain and population indices."""
    from paper_0905_2441_gb300 import _lib, samplers
    off = smp.offsets.cpu().numpy().astype(np.int64)
    n_pops = off.size - 1
    cuts = [round(i * n_pops / parts) for i in range(parts + 1)]
    groups = []
    for i in range(parts):
        c0, c1 = int(off[cuts[i]]), int(off[cuts[i + 1]])
        gctx = P.Context()
        gctx.set_launch(_lib.OP_POPMCMC, lanes, threads)
        sub = samplers.PopulationMCMC(gctx, smp.model, smp.y, off[cuts[i]:cuts[i + 1] + 1] - c0,
                                      smp.beta[c0:c1], smp.theta[:, c0:c1], scale=smp.scale,
                                      seed=smp.seed)
        M, K = sub.M, sub.K
        nb = M * 8 + K * M * 4
        dev = torch.empty(nb, dtype=torch.uint8, device="cuda")
        host = torch.empty(nb, dtype=torch.uint8).pin_memory()
        ll_v = dev[: M * 8].view(torch.float64)
        th_v = dev[M * 8:].view(torch.float32).view(K, M)
        ll_v.copy_(sub.ll)
        th_v.copy_(sub.theta)
        host.copy_(dev)
        sub.theta, sub.ll = th_v, ll_v
        groups.append((gctx, sub, dev, host, torch.cuda.Stream(), nb))
    main = torch.cuda.current_stream()
    steps = max(3, min(args.steps, 200))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(2):  # warm: each group's first sweep on its stream
        for gctx, sub, dev, host, st, nb in groups:
            with torch.cuda.stream(st):
                dev.copy_(host, non_blocking=True)
                sub.sweep(40_000 + i)
                host.copy_(dev, non_blocking=True)
    torch.cuda.synchronize()
    a.record(main)
    for g in groups:
        g[4].wait_stream(main)
    for i in range(steps):
        for gctx, sub, dev, host, st, nb in groups:
            with torch.cuda.stream(st):
                dev.copy_(host, non_blocking=True)
                sub.sweep(50_000 + i)
                host.copy_(dev, non_blocking=True)
    for g in groups:
        main.wait_stream(g[4])
    b.record(main)
    b.synchronize()
    t = a.elapsed_time(b) / 1e3
    nbytes = sum(g[5] for g in groups)
    for g in groups:
        g[0].check()
        g[0].close()
    units = float(smp.M) * smp.y.numel() * steps
    return {"value": units / t, "unit": "p*d/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": steps,
            "pipeline": f"{parts} population groups on {parts} streams, one context each",
            "_units": units, "_seconds": t}


def measure_peak(P, kind):
    import ctypes as C
    from paper_0905_2441_gb300 import _lib
    ops, ms = C.c_double(), C.c_double()
    st = _lib.load().smc_measure_peak(kind, 8, 4096, C.byref(ops), C.byref(ms))
    if st != 0:
        raise RuntimeError(f"smc_measure_peak failed ({st})")
    return ops.value, ms.value


def bench_secondary(torch, P):
    """Plain per-step vs CUDA-graph forms of the SMC sampler (4-component
    mixture, M = 8192, 20 temperatures), the differentiable MALA sampler
    (M = 65536, K = 8, N = 1000, 50 temperatures) and the particle filter
    (d = 3 MSV, M = 2^20, T = 200): steps/s of each, same kernels and Philox
    counters in both forms (bitwise-equal outputs)."""
    from paper_0905_2441_gb300 import samplers
    import synth
    out, snaps = {}, {}
    ctx = P.Context()
    ex2_rate, ex2_ms = measure_peak(P, 0)
    stream = torch.cuda.current_stream()
    flush = L2Flush(torch)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / 1e3

    for name, w, kind in (("smc_sampler", synth.GMM4, P.MOVE_RW),
                          ("mala_sampler", synth.GMM8_MALA, P.MOVE_MALA)):
        y = w.data()
        th0 = synth.prior_particles(w.K, w.M, seed=w.particle_seed)
        betas = synth.geometric_betas(w.T, w.beta_min)
        smp = samplers.SMCSampler(ctx, P.GMM(w.K, w.sigma), y, th0, betas, kind=kind,
                                  scale=w.scale, seed=w.method_seed)
        smp.run()  # warm
        smp.reset(th0)
        t_plain = timed(lambda: smp.run())
        z_plain = smp.log_evidence()
        th_plain = smp.state[0].clone()
        smp.reset(th0)
        g = smp._capture(smp._body)
        smp.reset(th0)
        t_graph = timed(lambda: g.replay())
        z_graph = smp.log_evidence()
        th_graph = smp.theta[(smp.T) % 2]
        th_f, ll_f = smp.state
        snaps[name] = {"w": w, "theta": th_f.cpu().numpy(), "ll": ll_f.cpu().numpy()}
        out[name] = {"workload": w.name, "steps": w.T, "M": w.M, "K": w.K, "N": w.N,
                     "plain_steps_per_s": w.T / t_plain, "graph_steps_per_s": w.T / t_graph,
                     "plain_pd_per_s": w.M * w.N * w.T / t_plain,
                     "graph_pd_per_s": w.M * w.N * w.T / t_graph,
                     "logZ_plain": z_plain, "logZ_graph": z_graph,
                     "graph_equals_plain": bool(torch.equal(th_plain, th_graph)) and z_plain == z_graph,
                     "resampled_steps": int(smp.flags[1:].sum().item())}
        ctx.check()
        if kind == P.MOVE_MALA:  # the fused likelihood + gradient move kernel, timed alone
            th, ll = smp.state
            gsrc = smp.grad[smp.cur]
            tho, llo, go = torch.empty_like(th), torch.empty_like(ll), torch.empty_like(gsrc)
            bl = smp.betas[-1:]
            mv = (lambda: P.mh_move(ctx, smp.model, smp.y, th, ll, tho, llo, bl, w.scale, 99, 1,
                                    kind=P.MOVE_MALA, grad_in=gsrc, grad_out=go))
            for _ in range(3):
                mv()
            tm = statistics.median([_whole_run(torch, flush, stream, mv) for _ in range(10)])
            ops = float(w.M) * w.N * (w.K + 1)
            out[name]["move_ms"] = 1e3 * tm
            out[name]["roofline"] = {
                "bound": "alu", "pipe": "MUFU", "achieved": ops / tm / 1e9, "peak": ex2_rate / 1e9,
                "unit": "Gop/s", "frac": ops / tm / ex2_rate,
                "traffic": profile_traffic("k_mh_move_mala"), "kernel": "k_mh_move<8,MALA,EQW>",
                "ops_per_launch": ops, "count": "K ex2 + 1 reciprocal per particle-datum",
                "launch_time": "one launch after an L2 flush (median of 10)",
                "peak_source": f"measured in this run: ex2.approx issue rate ({ex2_ms:.2f} ms)"}
            snaps["mala_move"] = {"w": w, "theta": th.cpu().numpy(), "ll": ll.cpu().numpy(),
                                  "grad": gsrc.cpu().numpy(), "theta1": tho.cpu().numpy(),
                                  "ll1": llo.cpu().numpy(), "grad1": go.cpu().numpy(),
                                  "beta": float(bl.item())}
    w = synth.MSV3
    phi, Sigma, beta = synth.msv_params(w.d, w.phi, w.rho, w.beta)
    _, yobs = synth.simulate_ssm("msv", w.T, phi, Sigma, beta, seed=w.data_seed)
    pf = samplers.ParticleFilter(ctx, P.PFModel(P.PF_MSV, phi, synth.chol(Sigma), beta), yobs, w.M,
                                 seed=w.method_seed)
    pf.run()
    pf.reset()
    t_plain = timed(lambda: pf.run())
    z_plain = float(pf.hist[1:, 0].sum().item())
    pf.reset()
    g = pf._capture(lambda: [pf.step(t) for t in range(1, w.T + 1)])
    pf.reset()
    t_graph = timed(lambda: g.replay())
    z_graph = float(pf.hist[1:, 0].sum().item())
    # one more filter step from the final state, kept for the oracle's check
    c, n = pf.cur, 1 - pf.cur
    xin = pf.x[c].cpu().numpy()
    ancs = pf.anc.cpu().numpy()
    P.pf_step(ctx, pf.model, pf.y[w.T - 1], pf.x[c], pf.x[n], pf.logg, pf.seed, w.T + 1,
              anc=pf.anc)
    snaps["particle_filter"] = {"phi": phi, "chol": synth.chol(Sigma), "beta": beta,
                                "yt": pf.y[w.T - 1].cpu().numpy(), "x_in": xin, "anc": ancs,
                                "seed": pf.seed, "t": w.T + 1, "logg": pf.logg.cpu().numpy(),
                                "x_out": pf.x[n].cpu().numpy()}
    out["particle_filter"] = {"workload": w.name, "steps": w.T, "M": w.M,
                              "plain_particle_steps_per_s": w.M * w.T / t_plain,
                              "graph_particle_steps_per_s": w.M * w.T / t_graph,
                              "ms_per_step_graph": 1e3 * t_graph / w.T,
                              "logZ_plain": z_plain, "logZ_graph": z_graph}
    ctx.check()
    # the diagonal mixture on the tensor cores (d=32, K=16, N=65536, M=4096),
    # and the widest shape the path takes (d=64, K=32)
    w = synth.DIAG32
    out["diag_tensor_core"], snaps["diag_tensor_core"] = diag_tc_entry(
        torch, P, ctx, flush, stream, ex2_rate, w.name, w.N, w.M, w.d, w.K, w.sigma, w.logw(),
        w.truth_seed, w.data_seed, w.particle_seed)
    out["is_example"] = is_example(torch, P, ctx)
    out["mrg32k3a"] = mrg_blocks(torch, P, ctx)
    K64 = 32
    out["diag_tensor_core_d64"], snaps["diag_tensor_core_d64"] = diag_tc_entry(
        torch, P, ctx, flush, stream, ex2_rate, "diag-d64-K32-N65536-M2048", 65536, 2048, 64,
        K64, 1.3, np.full(K64, -np.log(K64)), 64, 65, 66)
    try:
        out["reweight_resample"], snaps["reweight_resample"] = reweight_resample_roofline(
            torch, P, ctx, 1 << 24, 20)
    except Exception as e:  # noqa: BLE001
        out["reweight_resample"] = {"error": repr(e)}
    ctx.close()
    out["_snaps"] = snaps
    return out


def diag_tc_entry(torch, P, ctx, flush, stream, ex2_rate, name, N, M, d, K, sigma, logw,
                  truth_seed, data_seed, particle_seed):
    """The tensor-core diagonal-mixture likelihood on one synthetic shape:
    time per call (warm and after an L2 flush) and its two rooflines, issued
    bf16 MMA flops (three split products) and MUFU ops (K ex2 + 1 lg2 per
    particle-datum, K padded to 4, 8, 16 or 32).  Returns the entry and the
    snapshot for the oracle's check."""
    import synth
    truth = synth.diag_truth(K, d, seed=truth_seed)
    Y = torch.from_numpy(synth.diag_data(N, truth, seed=data_seed)).cuda()
    th = torch.from_numpy(synth.diag_particles(M, truth, seed=particle_seed)).cuda()
    tc = P.DiagGMM(K, sigma, d=d, log_w=np.asarray(logw), precision=P.PREC_BF16SPLIT)
    ll = torch.empty(M, dtype=torch.float64, device="cuda")
    P.loglik_batch(ctx, tc, Y, th, out=ll)
    reps = 10
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        P.loglik_batch(ctx, tc, Y, th, out=ll)
    b.record()
    b.synchronize()
    t_tc = a.elapsed_time(b) / 1e3 / reps
    ctx.check()
    kp = max(4, 1 << (K - 1).bit_length())
    flops = 3 * 2.0 * (-(-N // 128) * 128) * (M * kp) * d
    mufu = float(N) * M * (kp + 1)
    pk = measured_peaks()
    t_tcf = statistics.median([_whole_run(torch, flush, stream,
                                          lambda: P.loglik_batch(ctx, tc, Y, th, out=ll))
                               for _ in range(5)])
    snap = {"N": N, "d": d, "K": K, "sigma": sigma, "logw": np.asarray(logw),
            "seeds": (truth_seed, data_seed), "theta": th.cpu().numpy(), "ll": ll.cpu().numpy()}
    mu = {"bound": "alu", "pipe": "MUFU (ex2)", "achieved": mufu / t_tcf / 1e9,
          "peak": ex2_rate / 1e9, "unit": "Gop/s", "frac": mufu / t_tcf / ex2_rate,
          "ops_per_launch": mufu, "peak_source": "measured in this run: ex2.approx issue rate"}
    tens = {"bound": "tensor", "achieved": flops / t_tcf / 1e12, "peak": pk["bf16_tflops"],
            "unit": "TFLOP/s", "frac": flops / t_tcf / 1e12 / pk["bf16_tflops"],
            "flops_per_call": flops, "peak_source": "MEASURED_PEAKS.json bf16_tflops, burst"}
    # the primary bound is the unit nearer its peak; the other is kept beside it
    main, other, oname = (tens, mu, "mufu") if tens["frac"] > mu["frac"] else (mu, tens, "tensor")
    roof = dict(main)
    roof.update({"traffic": profile_traffic("k_dtc_main") if d == 32 else None,
                 "kernel": "k_dtc_main (+ prep, combine)",
                 "launch_time": "one call after an L2 flush (median of 5)", oname: other})
    entry = {
        "workload": name, "d": d, "K": K, "N": N, "M": M,
        "ms_per_call": 1e3 * t_tc, "ms_per_call_l2_flushed": 1e3 * t_tcf,
        "pd_per_s": M * N / t_tc,
        "form": "tcgen05 bf16 hi/lo split, FP32 accumulation in tensor memory",
        "roofline": roof}
    return entry, snap


def reweight_resample_roofline(torch, P, ctx, M, reps, seed=5):
    """smc_reweight (lw += l, W, log Z increment, ESS) and
    smc_resample_systematic (with the log-weight reset) at M particles,
    each timed alone after an L2 flush; algorithmic bytes per particle:
    reweight 32 (l read, lw read + write, W write), resampling 20 (W read,
    ancestor write, lw reset write).  Returns the entry and the inputs and
    outputs of one call for the oracle's check."""
    ctx.reserve(M)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    ll = torch.randn(M, dtype=torch.float64, device="cuda", generator=g)
    lw0 = torch.randn(M, dtype=torch.float64, device="cuda", generator=g) * 0.5
    lw = lw0.clone()
    W = torch.empty(M, dtype=torch.float64, device="cuda")
    anc = torch.empty(M, dtype=torch.int32, device="cuda")
    sc = torch.empty(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = L2Flush(torch)
    rw = lambda: P.reweight(ctx, ll, 1.0, lw, W, sc, None, 0.5)
    rs = lambda: P.resample_systematic(ctx, W, 9, 1, anc=anc, logw_reset=lw)
    for _ in range(3):
        lw.copy_(lw0)
        rw()
        rs()
    t_rw, t_rs = [], []
    for _ in range(reps):
        lw.copy_(lw0)
        e = _flush_timed(torch, flush, stream, [rw, rs])
        torch.cuda.synchronize()
        t_rw.append(e[0].elapsed_time(e[1]) / 1e3)
        t_rs.append(e[1].elapsed_time(e[2]) / 1e3)
    ctx.check()
    hbm = measured_peaks()["hbm_gbs"]
    trw, trs = statistics.median(t_rw), statistics.median(t_rs)
    lw.copy_(lw0)
    rw()
    snap = {"ll": ll.cpu().numpy(), "lw0": lw0.cpu().numpy(), "W": W.cpu().numpy(),
            "scalars": sc.cpu().numpy()}
    rs()
    snap["anc"] = anc.cpu().numpy()
    entry = {"M": M, "ms_reweight": 1e3 * trw, "ms_resample": 1e3 * trs,
             "roofline": {
                 "reweight": {"bound": "hbm", "achieved": 32 * M / trw / 1e9, "peak": hbm,
                              "unit": "GB/s", "frac": 32 * M / trw / 1e9 / hbm,
                              "traffic": profile_traffic("reweight"), "bytes_per_particle": 32,
                              "kernel": "k_reweight_reduce + k_reweight_normalize"},
                 "resample": {"bound": "hbm", "achieved": 20 * M / trs / 1e9, "peak": hbm,
                              "unit": "GB/s", "frac": 20 * M / trs / 1e9 / hbm,
                              "traffic": profile_traffic("resample_systematic"),
                              "bytes_per_particle": 20,
                              "kernel": "systematic resampling (total, finalize, scan)"}},
             "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
             "launch_time": f"each call alone after an L2 flush, median of {reps}"}
    return entry, snap


def secondary_oracle_checks(snaps):
    """Observed error of each secondary result against the FP64 oracle (part
    of the CPU leg, outside every timed region)."""
    import oracle
    res = {}
    rng = np.random.default_rng(12)
    for name in ("smc_sampler", "mala_sampler"):
        if name in snaps:
            d = snaps[name]
            w = d["w"]
            idx = rng.choice(d["theta"].shape[1], 200, replace=False)
            ref = oracle.gmm1d_loglik(w.data(), w.logw(), w.sigma, d["theta"][:, idx])
            res[name] = {"max_rel_loglik_err": float(np.max(np.abs(d["ll"][idx] - ref) /
                                                           np.abs(ref))),
                         "particles_checked": 200, "tolerance": "relative 1e-5"}
    if "mala_move" in snaps:
        d = snaps["mala_move"]
        w = d["w"]
        slots = np.sort(rng.choice(d["theta"].shape[1], 100, replace=False)).astype(np.int32)
        rt, rl, rg, racc, la = oracle.mala_move(w.data(), w.logw(), w.sigma, (-10, 10), d["theta"],
                                                d["ll"], d["grad"], d["beta"], w.scale, 99, 1,
                                                slots=slots, want_log_alpha=True)
        same = np.all(np.isclose(d["theta1"][:, slots], rt, rtol=3e-7, atol=2e-6), axis=0)
        ok = same & np.isclose(d["ll1"][slots], rl, rtol=1e-5)
        res["mala_move"] = {"slots_checked": int(slots.size), "slots_differing": int((~ok).sum()),
                            "max_rel_loglik_err_agreeing": float(np.max(
                                np.abs(d["ll1"][slots][ok] - rl[ok]) / np.abs(rl[ok])))
                            if ok.any() else None}
    for name in ("diag_tensor_core", "diag_tensor_core_d64"):
        if name not in snaps:
            continue
        d = snaps[name]
        import synth
        truth = synth.diag_truth(d["K"], d["d"], seed=d["seeds"][0])
        Yh = synth.diag_data(d["N"], truth, seed=d["seeds"][1])
        M = d["theta"].shape[0]
        idx = np.array([0, 1, M // 2 - 1, M // 2, M - 1])
        ref = oracle.gmmdiag_loglik(Yh, d["logw"], d["sigma"], d["theta"][idx])
        res[name] = {"max_rel_loglik_err": float(np.max(np.abs(d["ll"][idx] - ref) /
                                                       np.abs(ref))),
                     "particles_checked": int(idx.size), "tolerance": "relative 1e-3 (BF16 split)"}
    if "particle_filter" in snaps:
        d = snaps["particle_filter"]
        sl = rng.choice(d["x_in"].shape[1], 20000, replace=False)
        rx, rlg = oracle.pf_step(0, d["phi"], d["chol"], d["beta"], d["yt"], d["x_in"], d["anc"],
                                 d["seed"], d["t"])
        res["particle_filter"] = {"max_abs_logg_err": float(np.max(np.abs(d["logg"][sl] - rlg[sl]))),
                                  "max_rel_logg_err": float(np.max(np.abs(d["logg"][sl] - rlg[sl]) /
                                                                   np.maximum(np.abs(rlg[sl]), 1))),
                                  "state_max_abs_err": float(np.max(np.abs(d["x_out"] - rx))),
                                  "particles_checked": 20000}
    if "reweight_resample" in snaps:
        d = snaps["reweight_resample"]
        nlw, rW, rsc = oracle.reweight(d["ll"], 1.0, d["lw0"])
        ranc, _ = oracle.resample_systematic(d["W"], oracle.resample_u32(9, 1))
        res["reweight_resample"] = {
            "W_max_rel_err": float(np.max(np.abs(d["W"] - rW) / np.maximum(rW, 1e-300))),
            "ess_rel_err": float(abs(d["scalars"][1] - rsc[1]) / rsc[1]),
            "logz_inc_abs_err": float(abs(d["scalars"][0] - rsc[0])),
            "ancestors_differing": int(np.sum(d["anc"] != ranc)),
            "note": "ancestors from the GPU's own W (bit-exact given the same W)"}
    return res


def is_example(torch, P, ctx, reps=10):
    """Section 2.1's importance-sampling example at its size (N = 2^24
    draws): draws in device memory (HBM-bound, 4 bytes a draw), drawn on the
    device, and end to end from pinned host memory as in the example; L2
    flushed before each timed call, medians over `reps`."""
    prob = P.ISProblem()
    n_is = 1 << 24
    x_d = torch.randn(n_is, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    x_h = x_d.cpu().pin_memory()
    res = torch.empty(3, dtype=torch.float64, device="cuda")
    res_h = torch.empty(3, dtype=torch.float64).pin_memory()
    flush = L2Flush(torch)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        P.is_moments(ctx, prob, x_d, out=res)
    t_mem, t_dev, t_e2e = [], [], []
    for _ in range(reps):
        e = _flush_timed(torch, flush, stream, [lambda: P.is_moments(ctx, prob, x_d, out=res)])
        torch.cuda.synchronize()
        t_mem.append(e[0].elapsed_time(e[1]) / 1e3)
        e = _flush_timed(torch, flush, stream,
                         [lambda: P.is_moments(ctx, prob, N=n_is, seed=1, step=1, out=res)])
        torch.cuda.synchronize()
        t_dev.append(e[0].elapsed_time(e[1]) / 1e3)

        def e2e():
            x_d.copy_(x_h, non_blocking=True)
            P.is_moments(ctx, prob, x_d, out=res)
            res_h.copy_(res, non_blocking=True)
        e = _flush_timed(torch, flush, stream, [e2e], hold=False)
        torch.cuda.synchronize()
        t_e2e.append(e[0].elapsed_time(e[1]) / 1e3)
    ctx.check()
    est = res_h.numpy()
    tm = statistics.median(t_mem)
    return {"workload": "is-section2.1-N16777216", "N": n_is,
            "ms_draws_in_hbm": 1e3 * tm, "gbs_draws_in_hbm": 4 * n_is / tm / 1e9,
            "hbm_frac": 4 * n_is / tm / 1e9 / measured_peaks()["hbm_gbs"],
            "ms_draws_on_device": 1e3 * statistics.median(t_dev),
            "ms_end_to_end_from_host": 1e3 * statistics.median(t_e2e),
            "estimate_plain": float(est[1] / n_is),
            "estimate_self_normalised": float(est[1] / est[0]), "exact": 1.875}


def mrg_blocks(torch, P, ctx, reps=10):
    """MRG32k3a as Section 2.5 runs it: per thread a skip-ahead to its block,
    then the block (float32 out, slot-major); L2 flushed before each timed
    call, medians over `reps`."""
    nt, per = 152 * 256 * 4, 1024
    mrg = torch.empty(nt * per, dtype=torch.float32, device="cuda")
    flush = L2Flush(torch)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        P.rng_mrg32k3a(ctx, (12345,) * 6, 0, nt, per, out=mrg)
    t_blk, t_jump = [], []
    for _ in range(reps):
        e = _flush_timed(torch, flush, stream,
                         [lambda: P.rng_mrg32k3a(ctx, (12345,) * 6, 2**40, nt, per, out=mrg),
                          lambda: P.rng_mrg32k3a(ctx, (12345,) * 6, 2**40, nt, 1,
                                                 out=mrg[:nt])])
        torch.cuda.synchronize()
        t_blk.append(e[0].elapsed_time(e[1]) / 1e3)
        t_jump.append(e[1].elapsed_time(e[2]) / 1e3)
    ctx.check()
    tb = statistics.median(t_blk)
    return {"threads": nt, "per_thread": per, "ms": 1e3 * tb,
            "numbers_per_s": nt * per / tb, "gbs_written": 4 * nt * per / tb / 1e9,
            "ms_skip_ahead_only": 1e3 * statistics.median(t_jump)}


def bench_is(args, torch, dist):
    """One step = one importance-sampling call over N = 2^24 draws held in
    HBM (Section 2.1's example); also its on-device-draw and host forms."""
    import paper_0905_2441_gb300 as P
    ctx = P.Context()
    reps = max(3, min(args.steps, 50))
    with ClockSampler(torch.cuda.current_device()) as clk:
        r = is_example(torch, P, ctx, reps)
    ctx.close()
    t = dist.max(torch, r["ms_draws_in_hbm"] / 1e3)
    hbm = measured_peaks()["hbm_gbs"]
    ach = 4 * r["N"] / t / 1e9
    return {"metric": "importance-sampling draws/s (Section 2.1 example, draws in HBM)",
            "value": dist.sum(torch, float(r["N"])) / t, "unit": "draws/s", "n_gpus": dist.world,
            "steps": reps, "warmup": 3, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 per draw, f64 sums",
            "data": "synthetic (N(0,1) draws, seed 3)",
            "config": {"workload": r["workload"], "N": r["N"],
                       "l2": l2_note("call")},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "traffic": profile_traffic("k_is_moments"),
                         "bytes_per_draw": 4},
            "is_example": r, "gpu_launches": reps, "clocks": clk.summary()}


def bench_mrg(args, torch, dist):
    """One step = 155,648 MRG32k3a streams, each skipping ahead to its block
    and writing 1024 uniforms (Section 2.5's generator, float32 out)."""
    import paper_0905_2441_gb300 as P
    ctx = P.Context()
    reps = max(3, min(args.steps, 50))
    with ClockSampler(torch.cuda.current_device()) as clk:
        r = mrg_blocks(torch, P, ctx, reps)
    ctx.close()
    t = dist.max(torch, r["ms"] / 1e3)
    n = r["threads"] * r["per_thread"]
    hbm = measured_peaks()["hbm_gbs"]
    ach = 4 * n / t / 1e9
    return {"metric": "MRG32k3a uniforms/s (per-thread skip-ahead, then a block each)",
            "value": dist.sum(torch, float(n)) / t, "unit": "numbers/s", "n_gpus": dist.world,
            "steps": reps, "warmup": 3, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32 state, f32 out",
            "data": "synthetic (seed 12345 x 6)",
            "config": {"workload": "mrg32k3a-155648x1024", "threads": r["threads"],
                       "per_thread": r["per_thread"],
                       "l2": l2_note("call")},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "traffic": profile_traffic("k_mrg32k3a"),
                         "bytes_per_number": 4},
            "mrg32k3a": r, "gpu_launches": 2 * reps, "clocks": clk.summary()}


# A spin of about 0.13 ms on the device, queued after the L2 flush and
# before the first event: the host issues the timed calls meanwhile, so the
# events time the device work rather than the host's launch overhead (short
# calls after a flush would otherwise start when their launch arrives).
HOLD_CYCLES = 1 << 18


def _hold(torch):
    spin = getattr(torch.cuda, "_sleep", None)  # torch's device spin kernel
    if spin is not None:
        spin(HOLD_CYCLES)


def _flush_timed(torch, flush, stream, fns, hold=True):
    """Flush L2, then time each callable of one step with CUDA events on the
    launching stream; returns per-callable elapsed seconds.  hold=False for
    an end-to-end measurement, whose host side belongs to what it times."""
    flush()
    if hold:
        _hold(torch)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(fns) + 1)]
    evs[0].record(stream)
    for i, f in enumerate(fns):
        f()
        evs[i + 1].record(stream)
    return evs


def bench_pf(args, torch, dist):
    """One step = pf_step (gather + propagate + weight) -> reweight (log Z
    increment, W) -> systematic resampling, M = 2^20 particles (d = 3 MSV)."""
    import paper_0905_2441_gb300 as P
    from paper_0905_2441_gb300 import samplers
    import synth
    w = synth.MSV3
    phi, Sigma, beta = synth.msv_params(w.d, w.phi, w.rho, w.beta)
    _, yobs = synth.simulate_ssm("msv", w.T, phi, Sigma, beta, seed=w.data_seed)
    ctx = P.Context()
    pf = samplers.ParticleFilter(ctx, P.PFModel(P.PF_MSV, phi, synth.chol(Sigma), beta), yobs,
                                 w.M, seed=w.method_seed + dist.rank)
    flush = L2Flush(torch)
    stream = torch.cuda.current_stream()
    for t in range(1, args.warmup + 1):
        pf.step(t)
    torch.cuda.synchronize()
    K = min(args.steps, w.T - args.warmup)
    names = ["pf_step", "reweight", "resample"]
    rec = []
    dist.barrier(torch)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for t in range(args.warmup + 1, args.warmup + 1 + K):
            c, n = pf.cur, 1 - pf.cur
            fns = [lambda c=c, n=n, t=t: P.pf_step(ctx, pf.model, pf.y[t - 1], pf.x[c], pf.x[n],
                                                  pf.logg, pf.seed, t, anc=pf.anc),
                   lambda t=t: P.reweight(ctx, pf.logg, 1.0, pf.lw, pf.W, pf.hist[t], None, 0.5),
                   lambda t=t: P.resample_systematic(ctx, pf.W, pf.seed, t, anc=pf.anc,
                                                     logw_reset=pf.lw)]
            rec.append(_flush_timed(torch, flush, stream, fns))
            pf.cur = n
        torch.cuda.synchronize()
    ctx.check()
    per = np.array([[e[i].elapsed_time(e[i + 1]) / 1e3 for i in range(3)] for e in rec])
    t_dev = float(per.sum())
    t_max = dist.max(torch, t_dev)
    units = float(w.M) * K
    value = dist.sum(torch, units) / t_max
    share = per.sum(0) / per.sum()
    # algorithmic bytes per particle of each call
    bytes_pp = {"pf_step": 4 + 12 + 12 + 8,          # anc, x gather, x write, log g
                "reweight": 8 + 8 + 8 + 8,            # log g r, lw r/w, W w
                "resample": 8 + 4 + 8}                # W r, anc w, lw reset w
    i_dom = int(np.argmax(share))
    dom = names[i_dom]
    hbm = measured_peaks()["hbm_gbs"]
    ach = bytes_pp[dom] * w.M / (per[:, i_dom].mean()) / 1e9
    out = {"metric": "particle-steps/s (bootstrap particle filter, d=3 MSV)", "value": value,
           "unit": "particle-steps/s", "n_gpus": dist.world, "steps": K, "warmup": args.warmup,
           "ms_per_step": 1e3 * t_max / K, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded MSV observations)",
           "config": {"workload": w.name, "M": w.M, "d": w.d,
                      "l2": l2_note("step"),
                      "parallelism": f"independent filters per rank x{dist.world}"},
           "per_call_ms": {n: 1e3 * float(per[:, i].mean()) for i, n in enumerate(names)},
           "per_call_share": {n: float(share[i]) for i, n in enumerate(names)},
           "per_call_gbs": {n: bytes_pp[n] * w.M / float(per[:, i].mean()) / 1e9
                            for i, n in enumerate(names)},
           "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                        "frac": ach / hbm, "traffic": None, "kernel": dom,
                        "bytes_per_particle": bytes_pp[dom],
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
           "gpu_launches": 7 * K, "clocks": clk.summary()}  # 1 + 2 + 4 kernels a step
    ctx.close()
    return out


def bench_resample(args, torch, dist):
    """One step = smc_reweight (lw += l, W, scalars) + smc_resample_systematic
    (exact-integer systematic resampling) at M = 2^24: HBM-bound kernels.
    The multinomial and residual schemes are timed per call beside it."""
    import paper_0905_2441_gb300 as P
    M = 1 << 24
    ctx = P.Context()
    ctx.reserve(M)
    g = torch.Generator(device="cuda")
    g.manual_seed(5 + dist.rank)
    ll = torch.randn(M, dtype=torch.float64, device="cuda", generator=g)
    lw = torch.zeros(M, dtype=torch.float64, device="cuda")
    W = torch.empty(M, dtype=torch.float64, device="cuda")
    anc = torch.empty(M, dtype=torch.int32, device="cuda")
    sc = torch.empty(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = L2Flush(torch)
    fns = [lambda: P.reweight(ctx, ll, 1.0, lw, W, sc, None, 0.5),
           lambda: P.resample_systematic(ctx, W, 9, 1, anc=anc, logw_reset=lw)]
    for _ in range(args.warmup):
        for f in fns:
            f()
    torch.cuda.synchronize()
    K = min(args.steps, 200)
    rec = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for i in range(K):
            rec.append(_flush_timed(torch, flush, stream, fns))
        torch.cuda.synchronize()
    ctx.check()
    per = np.array([[e[i].elapsed_time(e[i + 1]) / 1e3 for i in range(2)] for e in rec])
    t_max = dist.max(torch, float(per.sum()))
    # the other two schemes on the same weights (4 and 6 kernels per call)
    variants = {}
    for name, fn in (("multinomial", P.resample_multinomial), ("residual", P.resample_residual)):
        call = (lambda fn=fn: fn(ctx, W, 9, 1, anc=anc))
        for _ in range(3):
            call()
        ts = []
        for _ in range(20):
            e = _flush_timed(torch, flush, stream, [call])
            torch.cuda.synchronize()
            ts.append(e[0].elapsed_time(e[1]) / 1e3)
        ctx.check()
        t = statistics.median(ts)
        variants[name] = {"ms_per_call": 1e3 * t, "particles_per_s": M / t}
    hbm = measured_peaks()["hbm_gbs"]
    b_rw, b_rs = 32, 20
    ach_rs = b_rs * M / per[:, 1].mean() / 1e9
    out = {"metric": "particles/s (reweight + systematic resampling)",
           "value": dist.sum(torch, float(M) * K) / t_max, "unit": "particles/s",
           "n_gpus": dist.world, "steps": K, "warmup": args.warmup,
           "ms_per_step": 1e3 * t_max / K, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (log-likelihoods ~ N(0,1))",
           "config": {"workload": "reweight+resample-M16777216", "M": M,
                      "l2": l2_note("step")},
           "per_call_gbs": {"reweight": b_rw * M / per[:, 0].mean() / 1e9,
                            "resample": ach_rs},
           "per_call_ms": {"reweight": 1e3 * per[:, 0].mean(), "resample": 1e3 * per[:, 1].mean()},
           "other_schemes": variants,
           "roofline": {"bound": "hbm", "achieved": ach_rs, "peak": hbm, "unit": "GB/s",
                        "frac": ach_rs / hbm, "traffic": profile_traffic("resample_systematic"),
                        "kernel": "resample (2 kernels)",
                        "bytes_per_particle": b_rs,
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
           "gpu_launches": 6 * K, "clocks": clk.summary()}
    ctx.close()
    return out


def bench_diag(args, torch, dist):
    """One step = smc_loglik_batch of the diagonal mixture (d=32, K=16,
    N=65536, M=4096) on the tensor cores (bf16 hi/lo split); the FP32
    CUDA-core path on the same inputs is timed beside it."""
    import paper_0905_2441_gb300 as P
    import synth
    import oracle
    w = synth.DIAG32
    if args.diag_shape == "d64k32":  # the widest shape the tensor-core path takes
        w = synth.DiagWorkload(name="diag-d64-K32-N65536-M2048", d=64, K=32, N=65536, M=2048,
                               sigma=1.3, truth_seed=64, data_seed=65, particle_seed=66)
    truth = synth.diag_truth(w.K, w.d, seed=w.truth_seed)
    Yh = synth.diag_data(w.N, truth, seed=w.data_seed)
    thh = synth.diag_particles(w.M, truth, seed=w.particle_seed + dist.rank)
    Y = torch.from_numpy(Yh).cuda()
    th = torch.from_numpy(thh).cuda()
    ctx = P.Context()
    tc = P.DiagGMM(w.K, w.sigma, d=w.d, precision=P.PREC_BF16SPLIT)
    fp = P.DiagGMM(w.K, w.sigma, d=w.d)
    out = torch.empty(w.M, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = L2Flush(torch)
    call = lambda: P.loglik_batch(ctx, tc, Y, th, out=out)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    K = min(args.steps, 200)
    rec = []
    dist.barrier(torch)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(K):
            rec.append(_flush_timed(torch, flush, stream, [call]))
        torch.cuda.synchronize()
    ctx.check()
    per = np.array([e[0].elapsed_time(e[1]) / 1e3 for e in rec])
    t_dev = float(per.sum())
    t_max = dist.max(torch, t_dev)
    pd = float(w.M) * w.N
    value = dist.sum(torch, pd * K) / t_max
    got = out.cpu().numpy()
    # error against the oracle on sampled particles
    idx = np.array([0, w.M // 2 - 1, w.M // 2, w.M - 1])
    ref = oracle.gmmdiag_loglik(Yh, w.logw(), w.sigma, thh[idx])
    err = float(np.max(np.abs(got[idx] - ref) / np.abs(ref)))
    # the FP32 CUDA-core path on the same inputs
    outf = torch.empty_like(out)
    P.loglik_batch(ctx, fp, Y, th, out=outf)
    torch.cuda.synchronize()
    recf = [_flush_timed(torch, flush, stream, [lambda: P.loglik_batch(ctx, fp, Y, th, out=outf)])
            for _ in range(3)]
    torch.cuda.synchronize()
    t_fp = float(np.mean([e[0].elapsed_time(e[1]) / 1e3 for e in recf]))
    # rooflines: issued bf16 MMA flops (3 split products) and MUFU ops
    t_call = float(per.mean())
    kp = max(4, 1 << (w.K - 1).bit_length())
    flops = 3 * 2.0 * (-(-w.N // 128) * 128) * (w.M * kp) * w.d
    mufu = float(w.N) * w.M * (kp + 1)
    pk = measured_peaks()
    ex2_rate, _ = measure_peak(P, 0)
    tens = {"bound": "tensor", "achieved": flops / t_call / 1e12, "peak": pk["bf16_tflops"],
            "unit": "TFLOP/s", "frac": flops / t_call / 1e12 / pk["bf16_tflops"],
            "traffic": profile_traffic("k_dtc_main") if w.d == 32 else None,
            "kernel": f"k_dtc_main<{kp}> (+ prep, combine)",
            "flops_per_call": flops,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops, burst (of measured)"}
    mu = {"achieved": mufu / t_call / 1e9, "peak": ex2_rate / 1e9, "unit": "Gop/s",
          "frac": mufu / t_call / ex2_rate, "ops_per_call": mufu,
          "count": "K ex2 + 1 lg2 per particle-datum"}
    roof = dict(tens)
    if mu["frac"] > tens["frac"]:
        roof = {"bound": "alu", "pipe": "MUFU (ex2)", "achieved": mu["achieved"],
                "peak": mu["peak"], "unit": "Gop/s", "frac": mu["frac"],
                "traffic": tens["traffic"], "kernel": tens["kernel"], "ops_per_call": mufu}
    roof["tensor"] = {k: tens[k] for k in ("achieved", "peak", "unit", "frac")}
    roof["mufu"] = {k: mu[k] for k in ("achieved", "peak", "unit", "frac")}
    res = {"metric": "particle-datum loglik evals/s (diagonal mixture, tensor cores)",
           "value": value, "unit": "p*d/s", "n_gpus": dist.world, "steps": K,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_max / K, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3->f32",
           "data": "synthetic (seeded mixture data and particles; no dataset)",
           "config": {"workload": w.name, "d": w.d, "K": w.K, "N": w.N, "M": w.M,
                      "l2": l2_note("call"),
                      "parallelism": f"independent particle sets per rank x{dist.world}"},
           "forms": {"tensor_bf16_split": {"ms_per_call": 1e3 * t_call, "max_rel_err": err},
                     "cuda_core_fp32": {"ms_per_call": 1e3 * t_fp, "value": pd / t_fp}},
           "roofline": roof, "gpu_launches": 4 * K, "clocks": clk.summary()}
    ctx.close()
    return res


# Table 3 of the paper: GTX 280 seconds for the whole T = 200 factor-SV filter
PAPER_FSV_GTX280_S = {8192: 0.082, 16384: 0.144, 32768: 0.249, 65536: 0.465, 131072: 0.929}


def bench_fsv(args, torch, dist):
    """The paper's particle-filter workload (Section 4.2, Table 3): the
    bootstrap filter on the factor SV model (m = 5 series, K = 3 factors,
    T = 200, resampling every step) for each N of the table; one step = one
    whole filter run (pf_step + reweight + resampling, T times), timed with
    CUDA events after an L2 flush, in its plain and CUDA-graph forms."""
    import paper_0905_2441_gb300 as P
    from paper_0905_2441_gb300 import samplers
    import synth
    w = synth.FSV
    phi, U, B, psi = synth.fsv_params()
    _, y = synth.simulate_fsv(w.T, phi, U, B, psi, seed=w.data_seed)
    ctx = P.Context()
    mod = P.PFModel(P.PF_FSV, phi, synth.chol(U), B=B, psi=psi)
    stream = torch.cuda.current_stream()
    flush = L2Flush(torch)
    reps = max(1, min(args.steps, 10))
    rows = {}
    with ClockSampler(torch.cuda.current_device()) as clk:
        for N in w.Ns:
            pf = samplers.ParticleFilter(ctx, mod, y, N, seed=w.method_seed + dist.rank)
            for _ in range(max(1, args.warmup // 3)):
                pf.reset()
                pf.run()
            t_plain, t_graph = [], []
            for r in range(reps):
                pf.reset()
                ev = _flush_timed(torch, flush, stream, [pf.run])
                torch.cuda.synchronize()
                t_plain.append(ev[0].elapsed_time(ev[1]) / 1e3)
            pf.reset()
            g = pf._capture(lambda: [pf.step(t) for t in range(1, w.T + 1)])
            for r in range(reps):
                pf.reset()
                ev = _flush_timed(torch, flush, stream, [g.replay])
                torch.cuda.synchronize()
                t_graph.append(ev[0].elapsed_time(ev[1]) / 1e3)
            logz = float(pf.hist[1:, 0].sum().item())
            tp, tg = statistics.median(t_plain), statistics.median(t_graph)
            rows[N] = {"plain_s": tp, "graph_s": tg, "paper_gtx280_s": PAPER_FSV_GTX280_S[N],
                       "speedup_plain_vs_paper_gpu": PAPER_FSV_GTX280_S[N] / tp,
                       "particle_steps_per_s_plain": N * w.T / tp,
                       "particle_steps_per_s_graph": N * w.T / tg, "logZ": logz}
    ctx.check()
    N = w.Ns[-1]
    t_max = dist.max(torch, rows[N]["plain_s"])
    value = dist.sum(torch, float(N) * w.T) / t_max
    paper_rate = N * w.T / PAPER_FSV_GTX280_S[N]
    out = {"metric": "particle-steps/s (factor SV particle filter, T=200, plain per-step launches)",
           "value": value, "unit": "particle-steps/s", "n_gpus": dist.world, "steps": reps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_max, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": value / dist.world / paper_rate,
           "vs_baseline_note": "against Table 3's GTX 280 time for the same N (another machine: context)",
           "dtype": "f32", "data": "synthetic (observations simulated from the model, seed 7)",
           "config": {"workload": w.name, "N": N, "T": w.T, "m": 5, "K": 3,
                      "l2": l2_note("filter run"),
                      "parallelism": f"independent filters per rank x{dist.world}"},
           "table3": rows, "gpu_launches": 7 * w.T * reps, "clocks": clk.summary()}
    ctx.close()
    return out


def bench_mala(args, torch, dist):
    """The differentiable sampler: tempered SMC with MALA moves (M = 65536,
    K = 8, N = 1000, 50 temperatures).  value = whole-run SMC steps/s in the
    plain per-call form; the roofline is the fused likelihood + gradient
    move kernel, timed alone per launch after an L2 flush (MUFU ops: K ex2
    and one reciprocal per particle-datum)."""
    import paper_0905_2441_gb300 as P
    from paper_0905_2441_gb300 import samplers
    import synth
    w = synth.GMM8_MALA
    y = w.data()
    th0 = synth.prior_particles(w.K, w.M, seed=w.particle_seed + dist.rank)
    betas = synth.geometric_betas(w.T, w.beta_min)
    ctx = P.Context()
    model = P.GMM(w.K, w.sigma)
    smp = samplers.SMCSampler(ctx, model, y, th0, betas, kind=P.MOVE_MALA, scale=w.scale,
                              seed=w.method_seed + dist.rank)
    stream = torch.cuda.current_stream()
    flush = L2Flush(torch)
    for _ in range(max(1, args.warmup // 3)):
        smp.reset(th0)
        smp.run()
    reps = max(1, min(args.steps, 5))
    with ClockSampler(torch.cuda.current_device()) as clk:
        t_run = []
        for _ in range(reps):
            smp.reset(th0)
            e = _flush_timed(torch, flush, stream, [smp.run])
            torch.cuda.synchronize()
            t_run.append(e[0].elapsed_time(e[1]) / 1e3)
        # the move kernel alone, from the sampler's final state
        th, ll = smp.state
        g = smp.grad[smp.cur]
        tho, llo, go = torch.empty_like(th), torch.empty_like(ll), torch.empty_like(g)
        beta = smp.betas[-1:]
        mv = (lambda: P.mh_move(ctx, model, smp.y, th, ll, tho, llo, beta, w.scale, 99, 1,
                                kind=P.MOVE_MALA, grad_in=g, grad_out=go))
        for _ in range(3):
            mv()
        t_mv = []
        for _ in range(20):
            e = _flush_timed(torch, flush, stream, [mv])
            torch.cuda.synchronize()
            t_mv.append(e[0].elapsed_time(e[1]) / 1e3)
    ctx.check()
    tr = statistics.median(t_run)
    t_max = dist.max(torch, tr)
    value = dist.sum(torch, float(w.T)) / t_max
    tm = statistics.median(t_mv)
    ex2_rate, ex2_ms = measure_peak(P, 0)
    ops = float(w.M) * w.N * (w.K + 1)
    ctx.close()
    return {"metric": "SMC steps/s (MALA tempered sampler, plain per-call launches)",
            "value": value, "unit": "steps/s", "n_gpus": dist.world, "steps": reps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / w.T, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 terms, f64 totals",
            "data": "synthetic (8-component mixture, 1000 simulated data, seed 1)",
            "config": {"workload": w.name, "M": w.M, "K": w.K, "N": w.N, "T": w.T, "h": w.scale,
                       "l2": l2_note("run / move"),
                       "parallelism": f"independent samplers per rank x{dist.world}"},
            "move_ms": 1e3 * tm,
            "roofline": {"bound": "alu", "pipe": "MUFU", "achieved": ops / tm / 1e9,
                         "peak": ex2_rate / 1e9, "unit": "Gop/s", "frac": ops / tm / ex2_rate,
                         "traffic": profile_traffic("k_mh_move_mala"),
                         "kernel": "k_mh_move<8,true,true> (MALA)",
                         "ops_per_launch": ops,
                         "issued_count": "K ex2 + 1 reciprocal per particle-datum",
                         "peak_source": "measured in this run: ex2.approx issue rate, all SMs, "
                                        f"{ex2_ms:.2f} ms microbenchmark"},
            "gpu_launches": (w.T * 7) * reps + 20, "clocks": clk.summary()}


# Tables 1 and 2 (Section 4.1): GTX 280 seconds and single-core CPU minutes
PAPER_T1_GTX280_S = {8: 1.083, 32: 1.098, 128: 1.100, 512: 1.235, 2048: 1.427, 8192: 2.323,
                     32768: 7.729, 131072: 28.349}
PAPER_T1_CPU_MIN = {8: 0.0166, 32: 0.0656, 128: 0.262, 512: 1.04, 2048: 4.16, 8192: 16.64,
                    32768: 66.7, 131072: 270.3}
PAPER_T2_GTX280_S = {8192: 0.597, 16384: 1.114, 32768: 2.114, 65536: 4.270, 131072: 8.075,
                     262144: 16.219}
PAPER_T2_CPU_MIN = {8192: 4.44, 16384: 8.82, 32768: 17.7, 65536: 35.3, 131072: 70.6,
                    262144: 141.0}


def _whole_run(torch, flush, stream, fn):
    """CUDA-event seconds of one whole run, L2 flushed just before it."""
    ev = _flush_timed(torch, flush, stream, [fn])
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / 1e3


def paper_tables(torch, P, ctx, flush, reps=1, rank=0):
    """Table 1 (population MCMC: one population of M chains, beta_i = (i/M)^2,
    N(0, I_4) random walk, 8192 sweeps) and Table 2 (SMC sampler: N
    particles, 200 temperatures beta_t = (t/200)^2, 10 N(0, I_4) moves per
    temperature, resampling when ESS < N/2), each whole run timed in its
    plain (one C-ABI call per kernel step) and CUDA-graph forms."""
    from paper_0905_2441_gb300 import samplers
    import synth
    w = synth.PAPER_TABLES
    y = w.data()
    model = P.GMM(w.K, w.sigma)
    stream = torch.cuda.current_stream()
    t1 = {}
    for M in w.table1_M:
        off = np.array([0, M], np.int32)
        beta = synth.power_betas(M).astype(np.float32)
        th0 = synth.prior_particles(w.K, M, seed=w.particle_seed + rank)
        smp = samplers.PopulationMCMC(ctx, model, y, off, beta, th0, scale=w.scale,
                                      seed=w.method_seed + rank)
        smp.run(3)  # warm
        n = w.table1_sweeps
        tp = min(_whole_run(torch, flush, stream, lambda: smp.run(n, start=3)) for _ in range(reps))
        g = smp._capture(lambda: [smp.sweep(3 + n + i) for i in range(n)])
        tg = min(_whole_run(torch, flush, stream, g.replay) for _ in range(reps))
        del g
        st = smp.stats.cpu().numpy()
        split = M > 2 * 256
        t1[M] = {"plain_s": tp, "graph_s": tg, "paper_gtx280_s": PAPER_T1_GTX280_S[M],
                 "paper_cpu_min": PAPER_T1_CPU_MIN[M],
                 "speedup_plain_vs_paper_gpu": PAPER_T1_GTX280_S[M] / tp,
                 "speedup_graph_vs_paper_gpu": PAPER_T1_GTX280_S[M] / tg,
                 "pd_per_s_graph": M * w.N * n / tg,
                 "launches_per_sweep": 2 if split else 1,
                 "swap_rate": float(st[1]) / max(1.0, float(st[2])),
                 "mh_accept_rate": float(st[0]) / float(M * (3 + 2 * n * reps))}
        ctx.check()
    t2 = {}
    betas = synth.power_betas(w.table2_T, start=0)
    for N in w.table2_N:
        th0 = synth.prior_particles(w.K, N, seed=w.particle_seed + rank)
        smp = samplers.SMCSampler(ctx, model, y, th0, betas, scale=w.scale,
                                  seed=w.method_seed + rank, n_moves=w.table2_moves)
        smp.run()  # warm
        tps = []
        for _ in range(reps):
            smp.reset(th0)
            tps.append(_whole_run(torch, flush, stream, smp.run))
        z_plain = smp.log_evidence()
        smp.reset(th0)
        g = smp._capture(smp._body)
        tgs = []
        for _ in range(reps):
            smp.reset(th0)
            tgs.append(_whole_run(torch, flush, stream, g.replay))
        del g
        tp, tg = min(tps), min(tgs)
        t2[N] = {"plain_s": tp, "graph_s": tg, "paper_gtx280_s": PAPER_T2_GTX280_S[N],
                 "paper_cpu_min": PAPER_T2_CPU_MIN[N],
                 "speedup_plain_vs_paper_gpu": PAPER_T2_GTX280_S[N] / tp,
                 "speedup_graph_vs_paper_gpu": PAPER_T2_GTX280_S[N] / tg,
                 "pd_per_s_plain": N * w.N * w.table2_T * w.table2_moves / tp,
                 "logZ": z_plain, "resampled_steps": int(smp.flags[1:].sum().item())}
        ctx.check()
    # annealed importance sampling: the same sampler with no resampling
    # (Section 4.1.2 reports its running time as practically identical)
    N = w.table2_N[-1]
    th0 = synth.prior_particles(w.K, N, seed=w.particle_seed + rank)
    smp = samplers.SMCSampler(ctx, model, y, th0, betas, scale=w.scale, seed=w.method_seed + rank,
                              n_moves=w.table2_moves, ess_frac=0.0)
    smp.run()
    smp.reset(th0)
    t_ais = _whole_run(torch, flush, stream, smp.run)
    ais = {"N": N, "plain_s": t_ais, "logZ": smp.log_evidence(),
           "resampled_steps": int(smp.flags[1:].sum().item()),
           "vs_smc_plain": t_ais / t2[N]["plain_s"]}
    ctx.check()
    return {"workload": w.name, "table1": t1, "table2": t2, "table2_ais": ais,
            "launches_per_table2_step": 6 + w.table2_moves}


def bench_tables(args, torch, dist):
    """The paper's Tables 1 and 2 replicated on this GPU; the JSON line's
    value is Table 2's largest run (N = 262144) in its plain form."""
    import paper_0905_2441_gb300 as P
    import synth
    w = synth.PAPER_TABLES
    ctx = P.Context()
    flush = L2Flush(torch)
    reps = max(1, min(args.steps, 5))
    with ClockSampler(torch.cuda.current_device()) as clk:
        tab = paper_tables(torch, P, ctx, flush, reps=reps, rank=dist.rank)
    ctx.close()
    N = w.table2_N[-1]
    work = float(N) * w.N * w.table2_T * w.table2_moves
    t_max = dist.max(torch, tab["table2"][N]["plain_s"])
    value = dist.sum(torch, work) / t_max
    paper_rate = work / PAPER_T2_GTX280_S[N]
    launches = (w.table2_T * tab["launches_per_table2_step"]) * reps * 2
    return {"metric": "particle-datum loglik evals/s (Table 2 SMC sampler, 200 temperatures x 10 "
                      "RW moves, plain per-call launches)",
            "value": value, "unit": "p*d/s", "n_gpus": dist.world, "steps": reps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": value / dist.world / paper_rate,
            "vs_baseline_note": "against Table 2's GTX 280 time for N = 262144 (another machine: "
                                "context)",
            "dtype": "f32 likelihood terms, f64 totals and weights",
            "data": "synthetic (Section 4.1 model, 100 simulated observations, seed 1)",
            "config": {"workload": w.name, "N": N, "T": w.table2_T, "moves": w.table2_moves,
                       "m": w.N, "k": w.K,
                       "l2": l2_note("run"),
                       "parallelism": f"independent samplers per rank x{dist.world}"},
            "table1": tab["table1"], "table2": tab["table2"], "table2_ais": tab["table2_ais"],
            "gpu_launches": launches,
            "clocks": clk.summary()}


def all_peaks(torch):
    import paper_0905_2441_gb300 as P
    out = {}
    for k, n in enumerate(["ex2", "lg2", "ffma", "dfma", "i2f", "frnd"]):
        ops, ms = measure_peak(P, k)
        out[n] = ops
    return out


# ------------------------------------------------------------------ reference arm
def reference_arm(args):
    """The oracle timed on the host cores on bounded samples of the same
    workload: each step continues four populations' chains for a share of
    ~ref_total seconds (at least one sweep), so any --steps ends in minutes."""
    import synth
    w = synth.GMM8_POP
    smp = CpuPopSample(w, sample_pops=4)
    budget = min(args.ref_budget, args.ref_total / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        smp.run(budget, 1)
    vals, samples, secs = [], [], []
    for i in range(args.steps):
        r = smp.run(budget, 1000)
        vals.append(r["value"])
        samples.append(r["sample"])
        secs.append(r["seconds"])
    v = statistics.median(vals)
    return {"impl": "reference", "metric": "particle-datum loglik evals/s (population MCMC sweeps)",
            "value": v, "unit": "p*d/s", "n_gpus": args.gpus, "devices": "host cores (rank 0)",
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded mixture data and chain states; no dataset)",
            "config": popmcmc_config(w, smp.M_total),
            "cpu_baseline": {"value": v, "unit": "p*d/s", "cores": 1, "kind": "oracle",
                             "sample": samples[0] + f"; median of {args.steps} samples"},
            "e2e": {"value": v, "unit": "p*d/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="popmcmc", choices=["popmcmc", "pf", "resample",
                                                              "diag", "fsv", "tables", "mala",
                                                              "is", "mrg", "peaks"])
    ap.add_argument("--graph-sweeps", type=int, default=1000)
    ap.add_argument("--diag-shape", default="d32k16", choices=["d32k16", "d64k32"],
                    help="--workload diag: d = 32 / K = 16 (default) or d = 64 / K = 32")
    ap.add_argument("--retune", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-secondary", action="store_true", help="skip the sampler / filter lines")
    ap.add_argument("--ref-budget", type=float, default=3.0,
                    help="reference arm: at most this many seconds of oracle work per step")
    ap.add_argument("--ref-total", type=float, default=120.0,
                    help="reference arm: about this many seconds over all steps")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    dist = Dist()
    if args.impl == "reference":
        if dist.rank == 0:
            print(json.dumps(reference_arm(args)), flush=True)
        return 0
    import torch
    torch.cuda.set_device(dist.local)
    dist.init(torch)
    from paper_0905_2441_gb300 import build as b
    if dist.rank == 0 and not os.path.exists(b.LIB):
        b.build()
    dist.barrier(torch)
    if args.workload == "pf":
        out = bench_pf(args, torch, dist)
    elif args.workload == "resample":
        out = bench_resample(args, torch, dist)
    elif args.workload == "diag":
        out = bench_diag(args, torch, dist)
    elif args.workload == "fsv":
        out = bench_fsv(args, torch, dist)
    elif args.workload == "tables":
        out = bench_tables(args, torch, dist)
    elif args.workload == "mala":
        out = bench_mala(args, torch, dist)
    elif args.workload == "is":
        out = bench_is(args, torch, dist)
    elif args.workload == "mrg":
        out = bench_mrg(args, torch, dist)
    elif args.workload == "peaks":
        out = {"peaks_ops_per_s": all_peaks(torch)}
    else:
        out = bench_popmcmc(args, torch, dist)
    if dist.rank == 0 and not args.no_secondary and args.workload == "popmcmc":
        # context lines; a failure here is reported in the line, it does not
        # take the headline measurement down with it
        import paper_0905_2441_gb300 as P
        try:
            out["secondary"] = bench_secondary(torch, P)
        except Exception as e:  # noqa: BLE001
            out["secondary"] = {"error": repr(e)}
        try:
            ctx = P.Context()
            flush = L2Flush(torch)
            out["secondary"]["paper_tables"] = paper_tables(torch, P, ctx, flush, reps=1)
            ctx.close()
        except Exception as e:  # noqa: BLE001
            out["secondary"]["paper_tables"] = {"error": repr(e)}
    if dist.rank == 0:
        snap = out.pop("_oracle_check", None)
        if args.no_cpu or dist.world != 1:
            out.get("secondary", {}).pop("_snaps", None)
        if not args.no_cpu and dist.world == 1 and args.workload == "popmcmc":
            import synth
            if snap is not None:
                out["error_vs_oracle"] = popmcmc_oracle_check(synth.GMM8_POP, snap)
            snaps = out.get("secondary", {}).pop("_snaps", None)
            if snaps:
                try:
                    for k, v in secondary_oracle_checks(snaps).items():
                        tgt = "mala_sampler" if k == "mala_move" else k
                        out["secondary"].setdefault(tgt, {})["error_vs_oracle" if k != "mala_move"
                                                             else "move_error_vs_oracle"] = v
                except Exception as e:  # noqa: BLE001
                    out["secondary"]["oracle_check_error"] = repr(e)
            out["cpu_baseline"] = cpu_popmcmc(synth.GMM8_POP)
            try:  # the same oracle on every host core (context beside the 1-core figure)
                out["cpu_baseline"]["all_cores"] = cpu_popmcmc_all_cores()
            except Exception as e:  # noqa: BLE001
                out["cpu_baseline"]["all_cores"] = {"error": repr(e)}
        print(json.dumps(out), flush=True)
    dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
