"""Host-side checks of the Python binding (no GPU): a tensor whose layout
does not match the model is refused before any call reaches the C ABI (the
ABI takes bare pointers and sizes, so the kernel would read past the end of
a smaller tensor), and a sampler's device buffers can only be replaced by
tensors of the same dtype, shape and device."""
import numpy as np
import pytest
import torch

import paper_0905_2441_gb300 as P
from paper_0905_2441_gb300 import samplers as S


def test_one_dimensional_model_shapes():
    m = P.GMM(8, 0.5)
    y = torch.zeros(10)
    with pytest.raises(ValueError, match=r"\[8, M\]"):
        P.loglik_batch(None, m, y, torch.zeros(4, 100))
    with pytest.raises(ValueError, match="one-dimensional"):
        P.loglik_batch(None, m, torch.zeros(10, 2), torch.zeros(8, 100))
    with pytest.raises(ValueError, match=r"\[8, M\]"):
        P.mh_move(None, m, y, torch.zeros(4, 50), None, None, None, None, 0.1, 1, 1)
    with pytest.raises(ValueError, match=r"\[8, M\]"):
        P.popmcmc_sweep(None, m, y, torch.zeros(8), None, None, None, 0.1, 1, 0)


def test_diagonal_model_shapes():
    m = P.DiagGMM(4, 1.0, d=16)
    with pytest.raises(ValueError, match=r"\[M, 4, 16\]"):
        P.loglik_batch(None, m, torch.zeros(5, 16), torch.zeros(10, 4, 8))
    with pytest.raises(ValueError, match=r"\[M, 4, 16\]"):
        P.loglik_batch(None, m, torch.zeros(5, 16), torch.zeros(10, 64))
    with pytest.raises(ValueError, match=r"\[N, 16\]"):
        P.loglik_batch(None, m, torch.zeros(5, 8), torch.zeros(10, 4, 16))


def test_filter_state_dimension():
    pf = P.PFModel(P.PF_MSV, np.full(3, 0.9), np.eye(3), 0.5)
    assert pf.state_dim == 3 and pf.obs_dim == 3
    with pytest.raises(ValueError, match=r"\[3, M\]"):
        P.pf_step(None, pf, torch.zeros(3), torch.zeros(2, 10), torch.zeros(2, 10),
                  torch.zeros(10, dtype=torch.float64), 1, 1)
    B = np.ones((5, 3))
    fsv = P.PFModel(P.PF_FSV, np.full(3, 0.9), np.eye(3), 1.0, B=B, psi=np.full(5, 0.5))
    assert fsv.state_dim == 3 and fsv.obs_dim == 5


def test_buffer_replacement_rules():
    t = torch.zeros(4, 10)
    S._check_replacement("theta", t, torch.ones(4, 10))  # same layout: accepted
    for bad in (torch.zeros(4, 11), torch.zeros(4, 10, dtype=torch.float64),
                torch.zeros(10, 4).t(), np.zeros((4, 10)), None):
        with pytest.raises(ValueError):
            S._check_replacement("theta", t, bad)
    pair = (torch.zeros(3), torch.zeros(3))
    S._check_replacement("ll", pair, (torch.ones(3), torch.ones(3)))
    with pytest.raises(ValueError):
        S._check_replacement("ll", pair, (torch.ones(3), torch.ones(4)))
    with pytest.raises(ValueError):
        S._check_replacement("ll", pair, [torch.ones(3), torch.ones(3)])
    with pytest.raises(ValueError):  # a buffer the sampler does not use stays unset
        S._check_replacement("grad[0]", None, torch.zeros(3))
    S._check_replacement("cur", 0, 1)  # plain attributes are free


def test_sizes_are_fixed_after_construction():
    class Fake(S._Graphable):
        pass
    f = Fake()
    f.M, f.K = 100, 4
    f.M = 100  # unchanged: fine
    with pytest.raises(ValueError, match="fixed"):
        f.M = 200
    with pytest.raises(ValueError, match="fixed"):
        f.K = 8
    f.buf = torch.zeros(5)
    with pytest.raises(ValueError):
        f.buf = torch.zeros(6)


def test_gather_pairs_and_shapes():
    with pytest.raises(ValueError, match="destination"):
        P.gather(None, None, src32=torch.zeros(3, 5))
    with pytest.raises(ValueError, match="destination"):
        P.gather(None, None, src64=torch.zeros(5, dtype=torch.float64))
    with pytest.raises(ValueError, match="nothing"):
        P.gather(None, None)
    with pytest.raises(ValueError, match=r"dst_f32 must be"):
        P.gather(None, None, torch.zeros(3, 5), torch.zeros(3, 4),
                 torch.zeros(5, dtype=torch.float64), torch.zeros(5, dtype=torch.float64))


def test_nvtx_ranges_wrap_the_calls_when_asked():
    """SMC_NVTX=1 at import wraps every ranged call (checked without a GPU, in
    a child interpreter); without it the functions are the plain ones."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import paper_0905_2441_gb300.api as a; "
            "print(all(hasattr(getattr(a, n), '__wrapped__') for n in a.RANGED))")
    for flag, want in (("1", "True"), ("0", "False")):
        r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                           env=dict(os.environ, SMC_NVTX=flag), timeout=300)
        assert r.returncode == 0, r.stderr
        assert r.stdout.strip() == want
