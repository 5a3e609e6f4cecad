"""The bounds-checked build (build(debug=True): -DSMC_DEBUG_BOUNDS,
libsmc_debug.so), in a child process: the entry points whose kernels check
their indices, on tiny and ragged shapes against the oracle, none reporting
SMC_ERR_BOUNDS; an ancestor one past the end reported as SMC_ERR_BOUNDS with
the access redirected.  This is the bounds evidence the pool allows (no
sanitizer)."""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_bounds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0905_2441_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, SMC_LIB_VARIANT="debug")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_debug_bounds_run.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-4000:], r.stderr[-4000:])
    assert "all ok" in r.stdout


def test_nvtx_ranged_calls_run():
    """With SMC_NVTX=1 the calls run inside NVTX ranges and give the same
    result as without (a reweighting and a resampling, child process)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    code = (
        "import numpy as np, torch, paper_0905_2441_gb300 as P\n"
        "ctx = P.Context()\n"
        "lw = torch.from_numpy(np.random.default_rng(1).normal(0, 2, 4099)).cuda()\n"
        "W = torch.empty_like(lw)\n"
        "P.reweight(ctx, None, 0.0, lw, W)\n"
        "a = P.resample_systematic(ctx, W, 3, 4)\n"
        "ctx.check()\n"
        "print(hasattr(P.reweight, '__wrapped__'), float(W.sum()), int(a.sum()))\n")
    root = os.path.dirname(HERE)
    outs = []
    for flag in ("1", "0"):
        r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                           env=dict(os.environ, SMC_NVTX=flag), timeout=600)
        assert r.returncode == 0, r.stderr[-3000:]
        outs.append(r.stdout.split())
    assert outs[0][0] == "True" and outs[1][0] == "False"
    assert outs[0][1:] == outs[1][1:]
