"""GPU parity: every C-ABI call against the FP64 oracle on identical seeded
inputs and identical Philox draws.

Tolerances, derived from the arithmetic of each kernel:
  * 1-D / diagonal FP32 log-likelihoods: relative 1e-5 per particle.
  * gradient: |g - g_oracle| <= 1e-4 * sum_n |r_nk (y_n - mu_k)| / sigma^2
    (the scale of the summed terms; cancellation makes plain relative error
    meaningless for components near a stationary point).
  * weights W: relative 1e-6 + 1e-7 |ln(W / W_max)| (FP32 exponential of the
    hi/lo float difference lw - max); ESS and log-evidence increment:
    relative 1e-6 / absolute 1e-6.
  * ancestors and offspring counts: bit-exact given the oracle's W.
  * moves: identical accept decisions except where |log alpha - log u| is
    inside the FP32 band 1e-3 (counted, must be rare); states within 2 ulp.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from _popcheck import explain_sweep

pytestmark = pytest.mark.gpu

SIG = 0.55
BOX = (-10.0, 10.0)


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


def cu(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def np_(t):
    return t.detach().cpu().numpy()


# ------------------------------------------------------------------ RNG
def test_philox_words_bit_exact(smc):
    P, ctx = smc
    for seed, purpose, step in [(0, 1, 0), (1234, 2, 7), (2**64 - 1, 3, (5 << 32) + 3),
                                (0x243F6A8885A308D3, 5, 2**32 - 1)]:
        w = np_(P.rng_words(ctx, seed, purpose, step, 300, 3)).view(np.uint32)
        for i in [0, 1, 77, 299]:
            for b in range(3):
                assert w[i, b].tolist() == oracle.draw_words(seed, purpose, step, i, b).tolist()


def test_normals_match_oracle(smc):
    P, ctx = smc
    z = np_(P.rng_normals(ctx, 99, 1, 4, 2000, 7)).astype(np.float64)
    ref = np.array([oracle.normals(99, 1, 4, i, 7) for i in range(2000)])
    np.testing.assert_allclose(z, ref, rtol=2e-6, atol=2e-6)


# ------------------------------------------------------------------ log-likelihood
def _ll_case(P, ctx, K, N, M, unequal=False, seed=0, lanes=None, offset=0):
    g = np.random.default_rng(seed)
    means = np.linspace(-6, 6, K)
    y_full = synth.gmm1d_data(N + offset, means, SIG, seed=seed + 1)
    logw = np.log(g.dirichlet(np.ones(K))) if unequal else np.full(K, -np.log(K))
    theta = g.uniform(-10, 10, (K, M)).astype(np.float32)
    theta[:, : M // 2] = (means[:, None] + 0.3 * g.standard_normal((K, M // 2))).astype(np.float32)
    model = P.GMM(K, SIG, logw)
    yt = cu(y_full)[offset:]
    if lanes:
        ctx.set_launch(P.OP_LOGLIK, lanes, 256)
    try:
        out = P.loglik_batch(ctx, model, yt, cu(theta))
        ctx.check()
    finally:
        ctx.set_launch(P.OP_LOGLIK, 0, 0)
    ref = oracle.gmm1d_loglik(y_full[offset:], logw, SIG, theta)
    return np_(out), ref


@pytest.mark.parametrize("K,N,M", [(1, 50, 33), (2, 1, 7), (3, 100, 257), (4, 100, 8192),
                                   (5, 333, 100), (8, 1000, 2048), (16, 257, 64), (32, 64, 40),
                                   (4, 8193, 70), (8, 20000, 50)])
def test_loglik_1d_parity(smc, K, N, M):
    P, ctx = smc
    got, ref = _ll_case(P, ctx, K, N, M)
    np.testing.assert_allclose(got, ref, rtol=1e-5)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_loglik_every_lane_count(smc, lanes):
    P, ctx = smc
    got, ref = _ll_case(P, ctx, 4, 1000, 999, lanes=lanes)
    np.testing.assert_allclose(got, ref, rtol=1e-5)


def test_loglik_unequal_weights_and_unaligned_data(smc):
    P, ctx = smc
    for off in (1, 2, 3):
        got, ref = _ll_case(P, ctx, 6, 9001, 300, unequal=True, offset=off)
        np.testing.assert_allclose(got, ref, rtol=1e-5)


def test_loglik_empty_inputs(smc):
    P, ctx = smc
    model = P.GMM(4, SIG)
    out = P.loglik_batch(ctx, model, torch.zeros(0, device="cuda"),
                         torch.zeros(4, 5, device="cuda"))
    ctx.check()
    assert np.all(np_(out) == 0.0)
    out = P.loglik_batch(ctx, model, torch.zeros(10, device="cuda"),
                         torch.zeros(4, 0, device="cuda"))
    assert out.numel() == 0


def test_loglik_full_size_sampled(smc):
    """Population-MCMC size (34.8k chains, K=8, N=1000): every particle on the
    GPU, a sample of 400 on the oracle."""
    P, ctx = smc
    w = synth.GMM8_POP
    off = synth.population_offsets(w.n_pops, seed=w.pop_seed)
    y = w.data()
    th = synth.population_particles(w.K, off)
    out = np_(P.loglik_batch(ctx, P.GMM(w.K, w.sigma), cu(y), cu(th)))
    ctx.check()
    idx = np.random.default_rng(0).choice(th.shape[1], 400, replace=False)
    ref = oracle.gmm1d_loglik(y, w.logw(), w.sigma, th[:, idx])
    np.testing.assert_allclose(out[idx], ref, rtol=1e-5)


def _grad_scale(y, logw, theta):
    """sum_n |r_nk (y_n - mu_k)| / sigma^2 per component and particle (FP64)."""
    y = y.astype(np.float64)[:, None, None]
    mu = theta.astype(np.float64)[None]
    a = logw[None, :, None] - (y - mu) ** 2 / (2 * SIG**2)
    r = np.exp(a - a.max(1, keepdims=True))
    r /= r.sum(1, keepdims=True)
    return np.abs(r * (y - mu)).sum(0) / SIG**2


@pytest.mark.parametrize("K,N,M", [(1, 100, 10), (4, 100, 512), (8, 1000, 300), (3, 77, 65),
                                   (4, 9001, 70)])  # data streamed through shared memory
def test_gradient_parity(smc, K, N, M):
    P, ctx = smc
    g = np.random.default_rng(K)
    y = synth.gmm1d_data(N, np.linspace(-5, 5, K), SIG, seed=3)
    logw = np.full(K, -np.log(K))
    theta = g.uniform(-6, 6, (K, M)).astype(np.float32)
    grad = torch.empty(K, M, device="cuda")
    out = P.loglik_batch(ctx, P.GMM(K, SIG), cu(y), cu(theta), grad=grad)
    ctx.check()
    ref = oracle.gmm1d_grad(y, logw, SIG, theta)
    scale = _grad_scale(y, logw, theta)
    assert np.all(np.abs(np_(grad) - ref) <= 1e-4 * scale + 1e-6)
    np.testing.assert_allclose(np_(out), oracle.gmm1d_loglik(y, logw, SIG, theta), rtol=1e-5)


@pytest.mark.parametrize("d,K,N,M", [(32, 16, 700, 10), (1, 1, 5, 3), (3, 2, 100, 17),
                                     (7, 5, 1000, 33), (64, 64, 50, 5), (16, 3, 1, 7),
                                     (5, 4, 0, 3)])
def test_diag_fp32_parity(smc, d, K, N, M):
    """FP32 CUDA-core path of the diagonal mixture over the accepted shapes
    (d, K in 1..64), a single datum and no data (the empty sum)."""
    P, ctx = smc
    truth = synth.diag_truth(K, d, seed=d + K)
    Y = synth.diag_data(max(N, 1), truth, seed=N + 1)[:N]
    th = synth.diag_particles(M, truth, seed=M)
    logw = np.log(np.random.default_rng(K).dirichlet(np.ones(K)))
    model = P.DiagGMM(K, 0.8, d=d, log_w=logw)
    out = np_(P.loglik_batch(ctx, model, cu(Y), cu(th)))
    ctx.check()
    if N == 0:
        assert np.all(out == 0.0)
    else:
        np.testing.assert_allclose(out, oracle.gmmdiag_loglik(Y, logw, 0.8, th), rtol=1e-5)


# ------------------------------------------------------------------ weights
@pytest.mark.parametrize("M", [1, 5, 1000, 100003, 1 << 20])
def test_reweight_parity(smc, M):
    P, ctx = smc
    g = np.random.default_rng(M)
    lw0 = g.normal(0, 2, M)
    ll = g.normal(-300, 20, M)
    lw = cu(lw0)
    W = torch.empty(M, dtype=torch.float64, device="cuda")
    sc = torch.empty(4, dtype=torch.float64, device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.reweight(ctx, cu(ll), 0.05, lw, W, sc, flag, 0.5)
    ctx.check()
    rlw, rW, rsc = oracle.reweight(ll, 0.05, lw0)
    np.testing.assert_allclose(np_(lw), rlw, rtol=0, atol=1e-12 * np.abs(rlw).max())
    big = rW > 1e-30
    # FP32 exponential of the hi/lo difference d = lw - max: relative error
    # <= 2^-21 (ex2, products) + 2^-24 |d| (one rounding of the difference)
    d = np.abs(np.log(rW[big] / rW.max()))
    assert np.all(np.abs(np_(W)[big] - rW[big]) <= (1e-6 + 1e-7 * d) * rW[big])
    assert np.all(np_(W)[~big] < 1e-29)
    s = np_(sc)
    assert abs(s[0] - rsc[0]) <= 1e-6 * max(1, abs(rsc[0]))
    assert abs(s[1] - rsc[1]) <= 1e-6 * rsc[1]
    # the GPU forms lw + dbeta * l with one fused multiply-add, the oracle with
    # two roundings: the max may differ in the last bit
    assert abs(s[2] - rsc[2]) <= 4e-16 * abs(rsc[2])
    assert abs(s[3] - rsc[3]) <= 1e-6 * max(1, abs(rsc[3]))
    assert int(np_(flag)[0]) == int(rsc[1] < 0.5 * M)


def test_reweight_no_increment_and_equal_weights(smc):
    P, ctx = smc
    M = 4096
    lw = cu(np.full(M, -7.0))
    W = torch.empty(M, dtype=torch.float64, device="cuda")
    sc = torch.empty(4, dtype=torch.float64, device="cuda")
    P.reweight(ctx, None, 0.0, lw, W, sc)
    ctx.check()
    s = np_(sc)
    assert s[0] == 0.0 and abs(s[1] - M) < 1e-9 * M
    np.testing.assert_allclose(np_(W), 1.0 / M, rtol=1e-6)


def test_reweight_error_statuses(smc):
    P, ctx = smc
    lw = cu(np.full(10, -np.inf))
    sc = torch.empty(4, dtype=torch.float64, device="cuda")
    P.reweight(ctx, None, 0.0, lw, None, sc)
    with pytest.raises(P.SmcError) as e:
        ctx.check()
    assert e.value.status == -4
    lw = cu(np.array([0.0, np.nan, 1.0]))
    P.reweight(ctx, None, 0.0, lw, None, sc)
    with pytest.raises(P.SmcError) as e:
        ctx.check()
    assert e.value.status == -3
    ctx.check()  # cleared


@pytest.mark.parametrize("M", [1, 3, 4097, 1 << 20])
def test_ess_parity(smc, M):
    P, ctx = smc
    lw0 = np.random.default_rng(M).normal(0, 3, M)
    out = np_(P.ess(ctx, cu(lw0)))
    ctx.check()
    assert abs(out[0] - oracle.ess(lw0)) <= 1e-6 * oracle.ess(lw0)


# ------------------------------------------------------------------ resampling
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


@pytest.mark.parametrize("M", [1, 2, 3, 100, 2047, 2048, 2049, 65537, 1 << 20, 3 << 20])
@pytest.mark.parametrize("kind", ["gauss", "peaked", "uniform", "onehot", "sparse"])
def test_resample_bit_exact(smc, M, kind):
    P, ctx = smc
    if M > 70000 and kind in ("uniform", "sparse"):
        pytest.skip("covered at smaller sizes")
    W = _weights(M, kind, M + len(kind))
    seed, step = 4242 + M, 17
    counts = torch.empty(M, dtype=torch.int32, device="cuda")
    lwr = torch.full((M,), 5.0, dtype=torch.float64, device="cuda")
    anc = P.resample_systematic(ctx, cu(W), seed, step, counts=counts, logw_reset=lwr)
    ctx.check()
    ranc, rcounts = oracle.resample_systematic(W, oracle.resample_u32(seed, step))
    assert np.array_equal(np_(anc), ranc)
    assert np.array_equal(np_(counts), rcounts)
    assert np.all(np_(lwr) == 0.0)


@pytest.mark.parametrize("M", [2049, 65537, 1 << 20])
@pytest.mark.parametrize("scale", [2.0 ** -25, 2.0 ** -34])
def test_resample_unnormalised_bit_exact(smc, M, scale):
    """Weights that do not sum to one: a total S below 2^32 (the wide-carry
    form) and, at the larger sizes, below M (the FP64 quotient estimates)."""
    P, ctx = smc
    W = _weights(M, "gauss", M + 7) * scale
    W[M // 3] = scale  # a heavy item (q = scale 2^52): S > 0, yet S < 2^32
    seed, step = 99 + M, 5
    counts = torch.empty(M, dtype=torch.int32, device="cuda")
    anc = P.resample_systematic(ctx, cu(W), seed, step, counts=counts)
    ctx.check()
    ranc, rcounts = oracle.resample_systematic(W, oracle.resample_u32(seed, step))
    assert np.array_equal(np_(anc), ranc)
    assert np.array_equal(np_(counts), rcounts)


def test_resample_repeated_calls_and_identity_flag(smc):
    P, ctx = smc
    M = 50000
    W = _weights(M, "gauss", 1)
    Wd = cu(W)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    for step in range(5):
        flag.fill_(step % 2)
        anc = P.resample_systematic(ctx, Wd, 9, step, do_flag=flag)
        ctx.check()
        if step % 2:
            assert np.array_equal(np_(anc), oracle.resample_systematic(W, oracle.resample_u32(9, step))[0])
        else:
            assert np.array_equal(np_(anc), np.arange(M))


def test_resample_bad_weights(smc):
    P, ctx = smc
    P.resample_systematic(ctx, cu(np.array([0.5, np.nan, 0.5])), 1, 1)
    with pytest.raises(P.SmcError):
        ctx.check()
    P.resample_systematic(ctx, cu(np.zeros(100)), 1, 1)
    with pytest.raises(P.SmcError) as e:
        ctx.check()
    assert e.value.status == -4
    # and the next good call still works (counters were reset)
    W = _weights(3000, "gauss", 3)
    anc = P.resample_systematic(ctx, cu(W), 2, 2)
    ctx.check()
    assert np.array_equal(np_(anc), oracle.resample_systematic(W, oracle.resample_u32(2, 2))[0])


def test_gather(smc):
    P, ctx = smc
    M = 10001
    g = np.random.default_rng(0)
    src = g.normal(size=(3, M)).astype(np.float32)
    s64 = g.normal(size=M)
    anc = np.sort(g.integers(0, M, M)).astype(np.int32)
    d32 = torch.empty(3, M, device="cuda")
    d64 = torch.empty(M, dtype=torch.float64, device="cuda")
    P.gather(ctx, cu(anc), cu(src), d32, cu(s64), d64)
    ctx.check()
    assert np.array_equal(np_(d32), src[:, anc]) and np.array_equal(np_(d64), s64[anc])


# ------------------------------------------------------------------ moves
def _band_check(got_acc, ref_acc, log_alpha, logu, band=1e-3):
    diff = got_acc != ref_acc
    near = np.abs(log_alpha - logu) < band
    assert np.all(near[diff]), np.flatnonzero(diff & ~near)[:10]
    return diff


def _move_case(P, ctx, K, N, M, kind, beta, scale, anc=False, seed=5, step=3, slots=None):
    g = np.random.default_rng(seed)
    means = np.linspace(-6, 6, K)
    y = synth.gmm1d_data(N, means, SIG, seed=seed)
    logw = np.full(K, -np.log(K))
    theta = (means[:, None] + 0.4 * g.standard_normal((K, M))).astype(np.float32)
    theta[:, ::7] = g.uniform(-10, 10, (K, theta[:, ::7].shape[1]))
    theta[:, 1::11] = 9.97  # near the box edge
    ll = oracle.gmm1d_loglik(y, logw, SIG, theta)
    grad = oracle.gmm1d_grad(y, logw, SIG, theta).astype(np.float32)
    a = np.sort(g.integers(0, M, M)).astype(np.int32) if anc else None
    b = np.float32(beta) if np.isscalar(beta) else beta
    model = P.GMM(K, SIG)
    to = torch.empty(K, M, device="cuda")
    lo = torch.empty(M, dtype=torch.float64, device="cuda")
    go = torch.empty(K, M, device="cuda") if kind == 1 else None
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.mh_move(ctx, model, cu(y), cu(theta), cu(ll), to, lo, cu(np.atleast_1d(b).astype(np.float32)),
              scale, 77, step, kind=kind, grad_in=cu(grad) if kind == 1 else None, grad_out=go,
              anc=cu(a) if anc else None, accept_count=cnt)
    ctx.check()
    if kind == 0:
        rt, rl, racc, la = oracle.rwmh_move(y, logw, SIG, BOX, theta, ll, b, scale, 77, step,
                                            anc=a, slots=slots, want_log_alpha=True)
        rg = None
    else:
        rt, rl, rg, racc, la = oracle.mala_move(y, logw, SIG, BOX, theta, ll, grad, b, scale, 77,
                                                step, anc=a, slots=slots, want_log_alpha=True)
    sl = np.arange(M) if slots is None else slots
    gt, gl = np_(to)[:, sl], np_(lo)[sl]
    src = a[sl] if anc else sl
    gacc = np.any(gt != theta[:, src], axis=0)   # the GPU moved the particle
    racc_b = racc.astype(bool)
    logu = np.log([oracle.u01(int(oracle.draw_words(77, oracle.P_ACCEPT, step, int(p), 0)[0]))
                   for p in sl])
    # the FP32 likelihood's absolute error grows with the number of data: the
    # band allowed to decide differently grows with it
    band = 5e-3 * max(1.0, N / 1000.0)
    diff = _band_check(gacc, racc_b, la, logu, band=band)
    ok = ~diff
    np.testing.assert_allclose(gt[:, ok], rt[:, ok], rtol=3e-7, atol=2e-6)
    np.testing.assert_allclose(gl[ok], rl[ok], rtol=1e-5)
    if kind == 1:
        gg = np_(go)[:, sl]
        sc = _grad_scale(y, logw, np.where(racc_b, rt, theta[:, src])[:, ok])
        assert np.all(np.abs(gg[:, ok] - rg[:, ok]) <= 1e-4 * sc + 1e-5)
    if slots is None:
        assert int(np_(cnt)[0]) == int(gacc.sum())
    return diff.sum(), racc.mean()


@pytest.mark.parametrize("K,N,M", [(1, 100, 500), (4, 100, 8192), (8, 1000, 2000), (5, 60, 333),
                                   (4, 9001, 300)])  # data streamed through shared memory
def test_rwmh_parity(smc, K, N, M):
    P, ctx = smc
    flips, rate = _move_case(P, ctx, K, N, M, 0, 0.7, 0.1)
    assert flips <= max(2, M // 500, int(M * 5e-3 * N / 1000)) and 0.01 < rate < 0.99


def test_rwmh_with_ancestors_and_per_particle_beta(smc):
    P, ctx = smc
    M = 3000
    beta = np.random.default_rng(1).uniform(0.01, 1, M).astype(np.float32)
    flips, _ = _move_case(P, ctx, 4, 100, M, 0, beta, 0.2, anc=True)
    assert flips <= 6


@pytest.mark.parametrize("K,N,M", [(1, 100, 400), (8, 1000, 1500), (4, 100, 4096),
                                   (4, 9001, 300)])  # data streamed through shared memory
def test_mala_parity(smc, K, N, M):
    P, ctx = smc
    flips, rate = _move_case(P, ctx, K, N, M, 1, 0.5, 0.05, anc=(K == 4))
    assert flips <= max(2, M // 500, int(M * 5e-3 * N / 1000))


def test_mala_full_size_sampled(smc):
    """Differentiable-sampler size (M=65536, K=8, N=1000): GPU for all, oracle on 300 slots."""
    P, ctx = smc
    slots = np.sort(np.random.default_rng(2).choice(65536, 300, replace=False)).astype(np.int32)
    flips, _ = _move_case(P, ctx, 8, 1000, 65536, 1, 1.0, 0.05, slots=slots)
    assert flips <= 3


@pytest.mark.parametrize("N", [100, 9001])  # resident data / streamed through shared memory
def test_popmcmc_sweep_parity(smc, N):
    P, ctx = smc
    K = 4
    y = synth.gmm1d_data(N, [-3, 0, 3, 6], SIG, seed=1)
    logw = np.full(K, -np.log(K))
    off = np.array([0, 1, 3, 8, 16, 17, 57, 185, 200, 264, 300], np.int32)
    Mt = int(off[-1])
    beta = synth.population_betas(off)
    th = synth.population_particles(K, off, seed=9)
    ll = oracle.gmm1d_loglik(y, logw, SIG, th)
    tt, lt = cu(th), cu(ll)
    stats = torch.zeros(3, dtype=torch.int64, device="cuda")
    P.popmcmc_sweep(ctx, P.GMM(K, SIG), cu(y), tt, lt, cu(beta), cu(off), 0.3, 55, 0,
                    stats=stats)
    ctx.check()
    rt, rl, rst = oracle.popmcmc_sweep(y, logw, SIG, BOX, th, ll, beta, off, 0.3, 55, 0)
    # a population may differ only through decisions inside the FP32 band
    rep = explain_sweep(y, logw, SIG, BOX, th, ll, beta, off, 0.3, 55, 0, np_(tt), np_(lt))
    assert rep.unexplained == [] and len(rep.differing) <= 1, rep
    s = np_(stats)
    assert s[2] == rst[2] and abs(int(s[0]) - int(rst[0])) <= 2 and abs(int(s[1]) - int(rst[1])) <= 2


@pytest.mark.parametrize("N", [600, 5000])  # binned sweep (shape fixed) / lanes-per-chain sweep
@pytest.mark.parametrize("lanes,threads", [(1, 256), (8, 128), (16, 128), (32, 256)])
def test_popmcmc_sweep_launch_shapes(smc, lanes, threads, N):
    """Every sweep shape the autotuner may choose gives the oracle's sweep."""
    P, ctx = smc
    K = 4
    y = synth.gmm1d_data(N, [-3, 0, 3, 6], SIG, seed=2)
    logw = np.full(K, -np.log(K))
    off = np.array([0, 2, 9, 40, 41, 130, 131, 300], np.int32)
    beta = synth.population_betas(off)
    th = synth.population_particles(K, off, seed=3)
    ll = oracle.gmm1d_loglik(y, logw, SIG, th)
    tt, lt = cu(th), cu(ll)
    ctx.set_launch(P.OP_POPMCMC, lanes, threads)
    try:
        P.popmcmc_sweep(ctx, P.GMM(K, SIG), cu(y), tt, lt, cu(beta), cu(off), 0.3, 66, 1)
        ctx.check()
    finally:
        ctx.set_launch(P.OP_POPMCMC, 0, 0)
    rep = explain_sweep(y, logw, SIG, BOX, th, ll, beta, off, 0.3, 66, 1, np_(tt), np_(lt))
    assert rep.unexplained == [] and len(rep.differing) <= 1, rep


def test_popmcmc_binned_layout_follows_the_data(smc):
    """The binned sweep keeps the data's binned layout between calls (keyed
    on the data pointer, N, the bin width and c) and checks the data against
    the layout's own copy: data overwritten in place under the same pointer,
    or another sigma on the same data, still give the oracle's sweep."""
    P, ctx = smc
    K, N = 4, 800
    off = np.array([0, 2, 9, 40, 41, 130, 131, 300], np.int32)
    beta = synth.population_betas(off)
    logw = np.full(K, -np.log(K))
    y_d = cu(synth.gmm1d_data(N, [-3, 0, 3, 6], SIG, seed=4))
    cases = [(synth.gmm1d_data(N, [-3, 0, 3, 6], SIG, seed=4), SIG),   # builds the layout
             (synth.gmm1d_data(N, [-3, 0, 3, 6], SIG, seed=4), SIG),   # uses it
             (synth.gmm1d_data(N, [-2, 1, 2, 7], SIG, seed=5), SIG),   # overwritten in place
             (synth.gmm1d_data(N, [-2, 1, 2, 7], SIG, seed=5), 1.5 * SIG)]  # another bin width
    for i, (y, sig) in enumerate(cases):
        y_d.copy_(cu(y))
        th = synth.population_particles(K, off, seed=10 + i)
        ll = oracle.gmm1d_loglik(y, logw, sig, th)
        tt, lt = cu(th), cu(ll)
        P.popmcmc_sweep(ctx, P.GMM(K, sig), y_d, tt, lt, cu(beta), cu(off), 0.3, 77, i)
        ctx.check()
        rep = explain_sweep(y, logw, sig, BOX, th, ll, beta, off, 0.3, 77, i, np_(tt), np_(lt))
        assert rep.unexplained == [] and len(rep.differing) <= 1, (i, rep)


def test_popmcmc_full_size_runs_and_reuses_queue(smc):
    P, ctx = smc
    w = synth.GMM8_POP
    off = synth.population_offsets(w.n_pops, seed=w.pop_seed)
    y = w.data()
    th = synth.population_particles(w.K, off)
    beta = synth.population_betas(off)
    tt = cu(th)
    lt = P.loglik_batch(ctx, P.GMM(w.K, w.sigma), cu(y), tt)
    stats = torch.zeros(3, dtype=torch.int64, device="cuda")
    for s in range(3):
        P.popmcmc_sweep(ctx, P.GMM(w.K, w.sigma), cu(y), tt, lt, cu(beta), cu(off), 0.1, 3, s,
                        stats=stats)
    ctx.check()
    st = np_(stats)
    npairs = 0
    for s in range(3):
        for q in range(w.n_pops):
            m = int(off[q + 1] - off[q])
            b = int(oracle.draw_words(3, oracle.P_EXCHANGE, s, q, 0)[0]) & 1
            npairs += m // 2 if b == 0 else (m - 1) // 2 + (1 if m % 2 == 0 else 0)
    assert st[2] == npairs and 0 < st[0] < 3 * off[-1]
    # the sweep keeps l consistent with theta
    sample = np.random.default_rng(0).choice(int(off[-1]), 200, replace=False)
    ref = oracle.gmm1d_loglik(y, w.logw(), w.sigma, np_(tt)[:, sample])
    np.testing.assert_allclose(np_(lt)[sample], ref, rtol=1e-5)


@pytest.mark.parametrize("shape", [(4, 256), (0, 0)])  # the benchmark's tuned shape; default
def test_popmcmc_full_size_parity(smc, shape):
    """One sweep of the full batched configuration (512 populations, 34,591
    chains, K = 8, N = 1000: the benchmarked workload and seeds) against the
    oracle's sweep, population by population, in the launch shape the
    benchmark times and in the default one.  A population may differ only
    through an accept decision taken inside the FP32 likelihood's error band."""
    P, ctx = smc
    w = synth.GMM8_POP
    off = synth.population_offsets(w.n_pops, seed=w.pop_seed)
    y = w.data()
    th = synth.population_particles(w.K, off, seed=4)
    beta = synth.population_betas(off)
    ll = oracle.gmm1d_loglik(y, w.logw(), w.sigma, th)
    tt, lt = cu(th), cu(ll)
    stats = torch.zeros(3, dtype=torch.int64, device="cuda")
    ctx.set_launch(P.OP_POPMCMC, *shape)
    try:
        P.popmcmc_sweep(ctx, P.GMM(w.K, w.sigma), cu(y), tt, lt, cu(beta), cu(off), w.scale, 3, 7,
                        stats=stats)
        ctx.check()
    finally:
        ctx.set_launch(P.OP_POPMCMC, 0, 0)
    rt, rl, rst = oracle.popmcmc_sweep(y, w.logw(), w.sigma, BOX, th, ll, beta, off, w.scale, 3,
                                       7)
    gt, gl = np_(tt), np_(lt)
    # every population that differs is reproduced by the oracle's sweep with
    # in-band decisions taken the other way; such populations stay rare
    rep = explain_sweep(y, w.logw(), w.sigma, BOX, th, ll, beta, off, w.scale, 3, 7, gt, gl)
    assert rep.unexplained == [], rep
    assert len(rep.differing) <= 3, rep
    s = np_(stats)
    assert s[2] == rst[2]
    assert abs(int(s[0]) - int(rst[0])) <= 4 and abs(int(s[1]) - int(rst[1])) <= 4
    assert rst[0] > 0 and rst[1] > 0  # moves and swaps both happened


# ------------------------------------------------------------------ particle filter
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("M", [1, 1000, 1 << 20])
def test_pf_step_parity(smc, kind, M):
    P, ctx = smc
    phi, Sigma, beta = synth.msv_params()
    L = synth.chol(Sigma)
    g = np.random.default_rng(M)
    x_in = g.normal(0, 1, (3, M)).astype(np.float32)
    anc = np.sort(g.integers(0, M, M)).astype(np.int32)
    yt = np.array([0.4, -1.1, 0.2], np.float32)
    model = P.PFModel(kind, phi, L, beta)
    xo = torch.empty(3, M, device="cuda")
    lg = torch.empty(M, dtype=torch.float64, device="cuda")
    P.pf_step(ctx, model, cu(yt), cu(x_in), xo, lg, 21, 8, anc=cu(anc))
    ctx.check()
    rx, rlg = oracle.pf_step(kind, phi, L, beta, yt, x_in, anc, 21, 8)
    np.testing.assert_allclose(np_(xo), rx, rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(np_(lg), rlg, rtol=1e-5, atol=2e-5)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("d", [1, 2, 5, 8])
def test_pf_step_state_dimensions(smc, kind, d):
    """pf_step over the accepted state dimensions (1..8), identity ancestors."""
    P, ctx = smc
    phi, Sigma, beta = synth.msv_params(d)
    L = synth.chol(Sigma)
    M = 3001
    g = np.random.default_rng(d)
    x_in = g.normal(0, 1, (d, M)).astype(np.float32)
    yt = g.normal(0, 1, d).astype(np.float32)
    xo = torch.empty(d, M, device="cuda")
    lg = torch.empty(M, dtype=torch.float64, device="cuda")
    P.pf_step(ctx, P.PFModel(kind, phi, L, beta), cu(yt), cu(x_in), xo, lg, 4, 2)
    ctx.check()
    rx, rlg = oracle.pf_step(kind, phi, L, beta, yt, x_in, None, 4, 2)
    np.testing.assert_allclose(np_(xo), rx, rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(np_(lg), rlg, rtol=1e-5, atol=2e-5)


def _fsv_or_msv(kind):
    if kind == 2:
        phi, Sigma, B, psi = synth.fsv_params()
        return dict(kind=kind, phi=phi, L=synth.chol(Sigma), B=B, psi=psi), B.shape[0]
    phi, Sigma, beta = synth.msv_params()
    return dict(kind=kind, phi=phi, L=synth.chol(Sigma), beta=beta), 3


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("M", [1, 2049, 100003, 1 << 20])
@pytest.mark.parametrize("with_flag", [False, True])
def test_pf_filter_step_equals_the_three_calls(smc, kind, M, with_flag):
    """smc_pf_filter_step against pf_step + smc_reweight (dbeta = 1) +
    smc_resample_systematic: the same states, log g, log-weights, W and
    scalars bit for bit; the ancestors exactly the oracle's systematic
    resampling of W (and the identity when the flag says no)."""
    P, ctx = smc
    spec, m = _fsv_or_msv(kind)
    if kind == 2:
        model = P.PFModel(P.PF_FSV, spec["phi"], spec["L"], B=spec["B"], psi=spec["psi"])
    else:
        model = P.PFModel(kind, spec["phi"], spec["L"], spec["beta"])
    d = len(spec["phi"])
    g = np.random.default_rng(M + kind)
    x_in = g.normal(0, 1, (d, M)).astype(np.float32)
    anc0 = np.sort(g.integers(0, M, M)).astype(np.int32)
    yt = g.normal(0, 1, m).astype(np.float32)
    lw0 = g.normal(0, 0.3, M)
    seed, t = 31, 5
    # the three calls
    xo_a = torch.empty(d, M, device="cuda")
    lg_a = torch.empty(M, dtype=torch.float64, device="cuda")
    P.pf_step(ctx, model, cu(yt), cu(x_in), xo_a, lg_a, seed, t, anc=cu(anc0))
    lw_a = cu(lw0)
    W_a = torch.empty(M, dtype=torch.float64, device="cuda")
    sc_a = torch.empty(4, dtype=torch.float64, device="cuda")
    fl_a = torch.zeros(1, dtype=torch.int32, device="cuda") if with_flag else None
    P.reweight(ctx, lg_a, 1.0, lw_a, W_a, sc_a, fl_a, 0.9)
    ctx.check()
    lw_new = np_(lw_a).copy()
    # the fused call
    xo_b = torch.empty(d, M, device="cuda")
    lg_b = torch.empty(M, dtype=torch.float64, device="cuda")
    anc_b = cu(anc0)
    lw_b = cu(lw0)
    W_b = torch.empty(M, dtype=torch.float64, device="cuda")
    sc_b = torch.empty(4, dtype=torch.float64, device="cuda")
    fl_b = torch.full((1,), 7, dtype=torch.int32, device="cuda") if with_flag else None
    counts = torch.empty(M, dtype=torch.int32, device="cuda")
    P.pf_filter_step(ctx, model, cu(yt), cu(x_in), xo_b, anc_b, lw_b, W_b, lg_b, seed, t,
                     scalars=sc_b, flag=fl_b, ess_frac=0.9, counts=counts)
    ctx.check()
    assert np.array_equal(np_(xo_a), np_(xo_b))
    assert np.array_equal(np_(lg_a), np_(lg_b))
    assert np.array_equal(np_(W_a), np_(W_b))
    assert np.array_equal(np_(sc_a), np_(sc_b))
    resampled = True
    if with_flag:
        assert int(np_(fl_b)[0]) == int(np_(fl_a)[0])
        resampled = bool(np_(fl_b)[0])
    if resampled:
        ranc, rcounts = oracle.resample_systematic(np_(W_b), oracle.resample_u32(seed, t))
        assert np.array_equal(np_(anc_b), ranc)
        assert np.array_equal(np_(counts), rcounts)
        assert np.all(np_(lw_b) == 0.0)
    else:
        assert np.array_equal(np_(anc_b), np.arange(M))
        assert np.array_equal(np_(lw_b), lw_new)


@pytest.mark.parametrize("M", [1, 3, 2047, 2049, 100003, 1 << 20])
@pytest.mark.parametrize("with_flag", [False, True])
def test_reweight_resample_equals_the_two_calls(smc, M, with_flag):
    """smc_reweight_resample gives, bit for bit, the log-weights, weights,
    scalars, flag, ancestors and counts of smc_reweight followed by
    smc_resample_systematic."""
    P, ctx = smc
    g = np.random.default_rng(M + with_flag)
    ll = cu(g.normal(-50, 3, M))
    lw0 = g.normal(0, 1.5, M)
    out = []
    for fused in (False, True):
        lw = cu(lw0)
        W = torch.empty(M, dtype=torch.float64, device="cuda")
        sc = torch.empty(4, dtype=torch.float64, device="cuda")
        flag = torch.zeros(1, dtype=torch.int32, device="cuda") if with_flag else None
        anc = torch.empty(M, dtype=torch.int32, device="cuda")
        cnt = torch.empty(M, dtype=torch.int32, device="cuda")
        if fused:
            P.reweight_resample(ctx, ll, 0.3, lw, W, 5, 9, scalars=sc, flag=flag, ess_frac=0.9,
                                anc=anc, counts=cnt)
        else:
            P.reweight(ctx, ll, 0.3, lw, W, sc, flag, 0.9)
            P.resample_systematic(ctx, W, 5, 9, anc=anc, counts=cnt, do_flag=flag, logw_reset=lw)
        ctx.check()
        out.append([np_(t) for t in (lw, W, sc, anc, cnt)] + ([np_(flag)] if with_flag else []))
    for a, b in zip(*out):
        assert np.array_equal(a, b)
