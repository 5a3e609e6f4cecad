"""Child process of tests/test_gpu_debug_bounds.py: loads the bounds-checked
library (SMC_LIB_VARIANT=debug) and runs the entry points whose kernels carry
index checks on tiny shapes against the oracle; then an ancestor outside
[0, M) must come back as SMC_ERR_BOUNDS with the access redirected (no
fault).  Prints "all ok" at the end."""
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import synth  # noqa: E402
from _popcheck import explain_sweep  # noqa: E402

import paper_0905_2441_gb300 as P  # noqa: E402
from paper_0905_2441_gb300 import _lib  # noqa: E402

assert os.path.basename(_lib.LIB_PATH) == "libsmc_debug.so", _lib.LIB_PATH
SIG, BOX = 0.55, (-10.0, 10.0)


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def np_(t):
    return t.detach().cpu().numpy()


ctx = P.Context()
n_cases = 0

# pf_step with ancestors (MSV and LG), d = 1..3
for kind in (0, 1):
    for d in (1, 2, 3):
        for M in (1, 7, 33):
            phi, Sigma, beta = synth.msv_params(d)
            L = synth.chol(Sigma)
            g = np.random.default_rng(100 * d + M)
            x_in = g.normal(0, 1, (d, M)).astype(np.float32)
            anc = g.integers(0, M, M).astype(np.int32)
            yt = g.normal(0, 1, d).astype(np.float32)
            xo = torch.empty(d, M, device="cuda")
            lg = torch.empty(M, dtype=torch.float64, device="cuda")
            P.pf_step(ctx, P.PFModel(kind, phi, L, beta), cu(yt), cu(x_in), xo, lg, 3, 2,
                      anc=cu(anc))
            ctx.check()
            rx, rlg = oracle.pf_step(kind, phi, L, beta, yt, x_in, anc, 3, 2)
            np.testing.assert_allclose(np_(xo), rx, rtol=2e-6, atol=2e-6)
            np.testing.assert_allclose(np_(lg), rlg, rtol=1e-5, atol=2e-5)
            n_cases += 1

# gather
for M in (1, 5, 33):
    g = np.random.default_rng(M)
    anc = g.integers(0, M, M).astype(np.int32)
    src = g.normal(0, 1, (2, M)).astype(np.float32)
    src64 = g.normal(0, 1, M)
    dst = torch.empty(2, M, device="cuda")
    dst64 = torch.empty(M, dtype=torch.float64, device="cuda")
    P.gather(ctx, cu(anc), cu(src), dst, cu(src64), dst64)
    ctx.check()
    assert np.array_equal(np_(dst), src[:, anc]) and np.array_equal(np_(dst64), src64[anc])
    n_cases += 1

# reweight + the three resamplers on tiny and ragged sizes, several weight shapes
for M in (1, 2, 3, 17, 33, 2049):
    for shape in ("gauss", "peaked", "onehot"):
        g = np.random.default_rng(M + len(shape))
        lw0 = g.normal(0, 2 if shape == "gauss" else 30, M)
        if shape == "onehot":
            lw0 = np.full(M, -np.inf)
            lw0[g.integers(0, M)] = 0.0
        lw = cu(lw0)
        W = torch.empty(M, dtype=torch.float64, device="cuda")
        P.reweight(ctx, None, 0.0, lw, W)
        ctx.check()
        Wn = np_(W)
        counts = torch.empty(M, dtype=torch.int32, device="cuda")
        anc = P.resample_systematic(ctx, W, 11, 4, counts=counts)
        ctx.check()
        ranc, rcounts = oracle.resample_systematic(Wn, oracle.resample_u32(11, 4))
        assert np.array_equal(np_(anc), ranc) and np.array_equal(np_(counts), rcounts)
        u = oracle.slot_uniforms(12, 5, M)
        a_mn = P.resample_multinomial(ctx, W, 12, 5)
        ctx.check()
        assert np.array_equal(np_(a_mn), oracle.resample_multinomial(Wn, u))
        a_rs = P.resample_residual(ctx, W, 12, 5)
        ctx.check()
        assert np.array_equal(np_(a_rs), oracle.resample_residual(Wn, u)[0])
        n_cases += 1

# population sweeps: the lanes-per-chain sweep (N < 512, N = 1..65) and the
# binned one (N = 600), small ragged populations
for K, N in ((1, 1), (2, 17), (3, 65), (4, 600)):
    y = synth.gmm1d_data(N, [-3, 0, 3, 6][:max(K, 1)], SIG, seed=N)
    logw = np.full(K, -np.log(K))
    off = np.array([0, 1, 3, 8, 16, 17, 40], np.int32)
    beta = synth.population_betas(off)
    th = synth.population_particles(K, off, seed=K)
    ll = oracle.gmm1d_loglik(y, logw, SIG, th)
    tt, lt = cu(th), cu(ll)
    P.popmcmc_sweep(ctx, P.GMM(K, SIG), cu(y), tt, lt, cu(beta), cu(off), 0.3, 5, 1)
    ctx.check()
    rep = explain_sweep(y, logw, SIG, BOX, th, ll, beta, off, 0.3, 5, 1, np_(tt), np_(lt))
    assert rep.unexplained == [], rep
    n_cases += 1

# an ancestor one past the end: reported, the access redirected
M = 33
phi, Sigma, beta = synth.msv_params(2)
x_in = np.zeros((2, M), np.float32)
anc = np.arange(M, dtype=np.int32)
anc[5] = M
xo = torch.empty(2, M, device="cuda")
lg = torch.empty(M, dtype=torch.float64, device="cuda")
P.pf_step(ctx, P.PFModel(0, phi, synth.chol(Sigma), beta), cu(np.zeros(2, np.float32)),
          cu(x_in), xo, lg, 3, 2, anc=cu(anc))
try:
    ctx.check()
    raise AssertionError("an out-of-range ancestor was not reported")
except P.SmcError as e:
    assert e.status == _lib.SMC_ERR_BOUNDS, e.status
dst = torch.empty(1, M, device="cuda")
P.gather(ctx, cu(anc), cu(np.zeros((1, M), np.float32)), dst)
try:
    ctx.check()
    raise AssertionError("an out-of-range ancestor was not reported")
except P.SmcError as e:
    assert e.status == _lib.SMC_ERR_BOUNDS, e.status
ctx.check()  # the status word was cleared
ctx.close()
print(f"all ok ({n_cases} cases)")
