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
