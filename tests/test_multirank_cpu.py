"""The multi-process path of bench.py on the CPU: two ranks over gloo (the
GPUs use NCCL the same way).  Each rank runs its own replica of the work and
only the timings are combined: the whole-job rate is the units of all ranks
over the slowest rank's time (weak scaling), with no data-path collective.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch
import bench
d = bench.Dist(backend="gloo")
d.init(torch)
d.barrier(torch)
r = d.rank
units = 1000.0 * (r + 1)          # rank r did (r + 1) thousand units
secs = 0.5 + r                    # in 0.5 + r seconds
value, tmax = d.throughput(torch, units, secs)
out = {"rank": r, "world": d.world, "max": d.max(torch, float(r)), "sum": d.sum(torch, 1.0 + r),
       "value": value, "tmax": tmax}
d.barrier(torch)
d.close()
print(json.dumps(out))
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run_ranks(world, script, timeout=120):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", script, ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, e[-2000:]
        outs.append(o)
    return outs


def test_two_ranks_gloo_aggregates():
    outs = _run_ranks(2, RANK_SCRIPT)
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o in outs), key=lambda d: d["rank"])
    for d in res:
        assert d["world"] == 2
        assert d["max"] == 1.0            # max over ranks of the rank number
        assert d["sum"] == 3.0            # 1 + 2
        assert d["tmax"] == 1.5           # the slowest rank's time
        assert d["value"] == pytest.approx(3000.0 / 1.5)  # all units over the slowest time


def test_reference_arm_non_zero_rank_does_no_work():
    # under torchrun only rank 0 runs and prints the reference arm
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_reference_arm_line_matches_the_gpu_arm_contract():
    # rank 0 prints one JSON line: the oracle's rate on the same workload
    # config as the GPU arm, within a bounded time for any --steps
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    env["CUDA_VISIBLE_DEVICES"] = ""
    steps = 400
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", str(steps), "--warmup", "3", "--ref-total", "4"], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    sys.path.insert(0, ROOT)
    import bench
    import synth
    w = synth.GMM8_POP
    off = synth.population_offsets(w.n_pops, seed=w.pop_seed)
    assert d["impl"] == "reference" and d["config"] == bench.popmcmc_config(w, int(off[-1]))
    assert d["metric"] == "particle-datum loglik evals/s (population MCMC sweeps)"
    assert d["unit"] == "p*d/s" and d["higher_is_better"] is True and d["steps"] == steps
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["ms_per_step"] > 0


def test_single_process_dist_is_identity():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    env_keep = {k: os.environ.pop(k) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK") if k in os.environ}
    try:
        d = bench.Dist()
        d.init(torch)
        assert not d.pg and d.world == 1 and d.rank == 0
        assert d.max(torch, 2.5) == 2.5 and d.sum(torch, 2.5) == 2.5
        v, t = d.throughput(torch, 10.0, 2.0)
        assert (v, t) == (5.0, 2.0)
    finally:
        os.environ.update(env_keep)
