"""GPU parity of the multinomial and residual resampling schemes (exact
integers on the systematic scheme's quantised CDF): ancestors bit-exact
against the oracle for every size and weight shape, the identity flag, the
log-weight reset and the error path."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0905_2441_gb300 as P
    from paper_0905_2441_gb300 import build
    build.build()
    ctx = P.Context()
    yield P, ctx
    ctx.close()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def np_(t):
    return t.detach().cpu().numpy()


def _weights(M, kind, seed):
    g = np.random.default_rng(seed)
    if kind == "gauss":
        lw = g.normal(0, 2, M)
    elif kind == "peaked":
        lw = g.normal(0, 30, M)
    elif kind == "uniform":
        lw = np.zeros(M)
    elif kind == "onehot":
        lw = np.full(M, -np.inf)
        lw[g.integers(0, M)] = 0.0
    else:  # sparse: most weights exactly zero
        lw = np.where(g.random(M) < 0.01, g.normal(0, 1, M), -np.inf)
        lw[0] = 0.0
    return oracle.reweight(None, 0.0, lw)[1]


def _oracle(scheme, W, seed, step):
    u = oracle.slot_uniforms(seed, step, W.size)
    if scheme == "multinomial":
        return oracle.resample_multinomial(W, u)
    return oracle.resample_residual(W, u)[0]


def _gpu(P, ctx, scheme, Wd, seed, step, **kw):
    fn = P.resample_multinomial if scheme == "multinomial" else P.resample_residual
    return fn(ctx, Wd, seed, step, **kw)


@pytest.mark.parametrize("scheme", ["multinomial", "residual"])
@pytest.mark.parametrize("M", [1, 2, 3, 100, 2047, 2048, 2049, 65537, 1 << 20, 3 << 20])
@pytest.mark.parametrize("kind", ["gauss", "peaked", "uniform", "onehot", "sparse"])
def test_bit_exact(smc, scheme, M, kind):
    P, ctx = smc
    if M > 70000 and kind in ("uniform", "sparse"):
        pytest.skip("covered at smaller sizes")
    W = _weights(M, kind, M + 7 * len(kind))
    seed, step = 777 + M, 23
    lwr = torch.full((M,), 5.0, dtype=torch.float64, device="cuda")
    anc = _gpu(P, ctx, scheme, cu(W), seed, step, logw_reset=lwr)
    ctx.check()
    ref = _oracle(scheme, W, seed, step)
    got = np_(anc)
    assert np.array_equal(got, ref), (np.flatnonzero(got != ref)[:10], got[:10], ref[:10])
    assert np.all(np_(lwr) == 0.0)


@pytest.mark.parametrize("scheme", ["multinomial", "residual"])
def test_identity_flag_and_repeated_calls(smc, scheme):
    P, ctx = smc
    M = 50000
    W = _weights(M, "gauss", 1)
    Wd = cu(W)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    lwr = torch.full((M,), 3.0, dtype=torch.float64, device="cuda")
    for step in range(4):
        flag.fill_(step % 2)
        anc = _gpu(P, ctx, scheme, Wd, 9, step, do_flag=flag, logw_reset=lwr)
        ctx.check()
        if step % 2:
            assert np.array_equal(np_(anc), _oracle(scheme, W, 9, step))
            assert np.all(np_(lwr) == 0.0)
        else:
            assert np.array_equal(np_(anc), np.arange(M))
            if step == 0:
                assert np.all(np_(lwr) == 3.0)  # untouched without resampling


@pytest.mark.parametrize("scheme", ["multinomial", "residual"])
def test_bad_weights(smc, scheme):
    P, ctx = smc
    _gpu(P, ctx, scheme, cu(np.array([0.5, np.nan, 0.5])), 1, 1)
    with pytest.raises(P.SmcError):
        ctx.check()
    _gpu(P, ctx, scheme, cu(np.zeros(100)), 1, 1)
    with pytest.raises(P.SmcError) as e:
        ctx.check()
    assert e.value.status == -4
    W = _weights(3000, "gauss", 3)
    anc = _gpu(P, ctx, scheme, cu(W), 2, 2)
    ctx.check()
    assert np.array_equal(np_(anc), _oracle(scheme, W, 2, 2))


def test_residual_keeps_integer_shares(smc):
    """Each particle keeps at least floor(M W_j) copies, in particle order at
    the front; the offspring counts add up to M."""
    P, ctx = smc
    M = 1 << 16
    W = _weights(M, "gauss", 5)
    anc = np_(P.resample_residual(ctx, cu(W), 3, 4))
    ctx.check()
    cnt = np.bincount(anc, minlength=M)
    share = np.floor(M * W - 1e-9).astype(np.int64)
    assert cnt.sum() == M and np.all(cnt >= share)
    nd = int(share.sum())
    assert np.all(np.diff(anc[:nd]) >= 0)


@pytest.mark.parametrize("scheme", ["multinomial", "residual"])
def test_samplers_with_other_schemes(smc, scheme):
    """The SMC sampler and the particle filter with the other schemes: graph
    form equals the plain form bit for bit, and the filter's evidence agrees
    with the Kalman filter (linear-Gaussian model) within Monte Carlo error."""
    import synth
    from paper_0905_2441_gb300 import samplers as S
    P, ctx = smc
    y = synth.gmm1d_data(100, [-3, 0, 3, 6], 0.55, seed=1)
    th0 = synth.prior_particles(4, 4096, seed=3)
    smp = S.SMCSampler(ctx, P.GMM(4, 0.55), y, th0, synth.power_betas(12, start=0), scale=1.0,
                       seed=5, n_moves=2, resampler=scheme)
    z1 = smp.run()
    th1 = smp.state[0].clone()
    smp.reset(th0)
    z2 = smp.run(graph=True)
    ctx.check()
    assert z1 == z2 and torch.equal(th1, smp.state[0]) and int(smp.flags.sum()) >= 1
    phi, Sigma, beta = synth.msv_params()
    _, yo = synth.simulate_ssm("lg", 40, phi, Sigma, beta, seed=4)
    exact = oracle.kalman_lg(phi, Sigma, beta, yo)
    zs = []
    for s in range(8):
        pf = S.ParticleFilter(ctx, P.PFModel(P.PF_LG, phi, synth.chol(Sigma), beta), yo, 1 << 14,
                              seed=100 + s, resampler=scheme)
        zs.append(pf.run())
    ctx.check()
    zs = np.array(zs)
    se = max(zs.std(ddof=1) / np.sqrt(zs.size), 0.01)
    assert abs(zs.mean() - exact) < 5 * se + 0.05, (zs.mean(), exact, se)


@pytest.mark.parametrize("frac", [0.0, 0.1, 0.5, 0.9, 1.0, 1.5])
def test_ess_threshold_decision(smc, frac):
    """The resampling decision is ESS < frac * M, taken on the device for any
    threshold (0: never, as in annealed importance sampling; >= 1: at every
    step unless all weights are equal), matching the oracle's ESS."""
    P, ctx = smc
    M = 20000
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    sc = torch.empty(4, dtype=torch.float64, device="cuda")
    W = torch.empty(M, dtype=torch.float64, device="cuda")
    for spread in (0.01, 0.5, 2.0, 8.0):
        g = np.random.default_rng(int(spread * 100))
        lw0 = g.normal(0, spread, M)
        P.reweight(ctx, None, 0.0, cu(lw0), W, sc, flag, frac)
        ctx.check()
        ess = oracle.ess(lw0)
        if abs(ess - frac * M) > 1e-6 * M:  # away from the threshold itself
            assert int(np_(flag)[0]) == int(ess < frac * M), (spread, ess)
