"""GPU parity of the factor stochastic volatility particle filter (Section
4.2): pf_step with kind FSV against the FP64 oracle (plain m x m
covariance), and the whole filter against the oracle filter.

Tolerances: states within 2e-6 (FP32 Box-Muller normals against the FP64
ones of the oracle, one rounding of the stored state); log g within 1e-4
absolute + 1e-5 relative: the GPU forms it in FP32 through the Woodbury
identity, where q - |w|^2 (terms of size 10..100) cancels to the quadratic
form and carries ~1e-5 absolute error.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0905_2441_gb300 as P
    from paper_0905_2441_gb300 import build, samplers
    build.build()
    ctx = P.Context()
    yield P, samplers, ctx
    ctx.close()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def model(P):
    phi, U, B, psi = synth.fsv_params()
    return P.PFModel(P.PF_FSV, phi, synth.chol(U), B=B, psi=psi), (phi, U, B, psi)


@pytest.mark.parametrize("M", [1, 257, 5000, 1 << 20])
def test_fsv_step_parity(env, M):
    P, S, ctx = env
    mod, (phi, U, B, psi) = model(P)
    g = np.random.default_rng(M)
    x_in = g.normal(0, 1.6, (3, M)).astype(np.float32)
    anc = np.sort(g.integers(0, M, M)).astype(np.int32)
    yt = g.normal(0, 2.0, 5).astype(np.float32)
    xo = torch.empty(3, M, device="cuda")
    lg = torch.empty(M, dtype=torch.float64, device="cuda")
    P.pf_step(ctx, mod, cu(yt), cu(x_in), xo, lg, 31, 4, anc=cu(anc))
    ctx.check()
    if M > 100_000:  # the oracle on a sample of particles
        idx = np.sort(g.choice(M, 4000, replace=False))
        rx, rlg = oracle.fsv_step(phi, synth.chol(U), B, psi, yt, x_in, anc, 31, 4)
        got_x, got_l = xo.cpu().numpy()[:, idx], lg.cpu().numpy()[idx]
        rx, rlg = rx[:, idx], rlg[idx]
    else:
        rx, rlg = oracle.fsv_step(phi, synth.chol(U), B, psi, yt, x_in, anc, 31, 4)
        got_x, got_l = xo.cpu().numpy(), lg.cpu().numpy()
    np.testing.assert_allclose(got_x, rx, rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(got_l, rlg, rtol=1e-5, atol=1e-4)


def test_fsv_rejects_bad_models(env):
    P, S, ctx = env
    phi, U, B, psi = synth.fsv_params()
    x = torch.zeros(3, 8, device="cuda")
    lg = torch.empty(8, dtype=torch.float64, device="cuda")
    y = torch.zeros(5, device="cuda")
    bad = P.PFModel(P.PF_FSV, phi, synth.chol(U), B=B, psi=np.array([0.5, 0.5, 0.0, 0.5, 0.5]))
    with pytest.raises(P.SmcError):
        P.pf_step(ctx, bad, y, x, torch.empty_like(x), lg, 1, 1)
    big = P.PFModel(P.PF_FSV, np.full(5, 0.9), np.eye(5), B=np.ones((5, 5)), psi=psi)
    x5 = torch.zeros(5, 8, device="cuda")
    with pytest.raises(P.SmcError):
        P.pf_step(ctx, big, y, x5, torch.empty_like(x5), lg, 1, 1)


def test_fsv_filter_matches_oracle_filter(env):
    P, S, ctx = env
    mod, (phi, U, B, psi) = model(P)
    _, y = synth.simulate_fsv(60, phi, U, B, psi, seed=7)
    gz = []
    for s in range(6):
        pf = S.ParticleFilter(ctx, mod, y, 65536, seed=500 + s)
        gz.append(pf.run(graph=(s % 2 == 0)))
    ctx.check()
    oz = [oracle.fsv_run(phi, synth.chol(U), B, psi, y, 8000, 600 + s) for s in range(3)]
    gz, oz = np.array(gz), np.array(oz)
    spread = max(np.std(gz, ddof=1), np.std(oz, ddof=1), 0.05)
    assert abs(gz.mean() - oz.mean()) < 4 * spread + 0.1, (gz, oz)


def test_fsv_graph_equals_plain(env):
    P, S, ctx = env
    mod, (phi, U, B, psi) = model(P)
    _, y = synth.simulate_fsv(40, phi, U, B, psi, seed=9)
    pf = S.ParticleFilter(ctx, mod, y, 131072, seed=5)
    z1 = pf.run()
    x1 = pf.x[pf.cur].clone()
    pf.reset()
    z2 = pf.run(graph=True)
    ctx.check()
    assert z1 == z2 and torch.equal(x1, pf.x[pf.cur]) and np.isfinite(z1)
