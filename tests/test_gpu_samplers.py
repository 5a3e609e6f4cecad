"""GPU sampler drivers: CUDA-graph form equals the plain form bit for bit,
whole-run estimates agree with closed forms / the Kalman filter / the oracle
sampler within Monte Carlo error, and the autograd wrapper returns the
adjoint gradient."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
SIG = 0.55


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


@pytest.mark.parametrize("kind", [0, 1])
def test_smc_graph_equals_plain(env, kind):
    P, S, ctx = env
    w = synth.GMM4
    y = w.data()
    th0 = synth.prior_particles(4, 4096, seed=3)
    betas = synth.geometric_betas(20)
    smp = S.SMCSampler(ctx, P.GMM(4, SIG), y, th0, betas, kind=kind,
                       scale=0.1 if kind == 0 else 0.05, seed=11)
    z1 = smp.run()
    th1, l1 = [t.clone() for t in smp.state]
    f1 = smp.flags.clone()
    smp.reset(th0)
    z2 = smp.run(graph=True)
    th2, l2 = smp.state
    ctx.check()
    assert z1 == z2 and torch.equal(th1, th2) and torch.equal(l1, l2)
    assert torch.equal(f1, smp.flags) and int(f1.sum()) >= 1


def _log_int_normal_product(ys, sigma, lo=-10.0, hi=10.0):
    from scipy import stats
    ys = np.asarray(ys, np.float64)
    n = ys.size
    yb = ys.mean()
    S = np.sum((ys - yb) ** 2)
    mass = stats.norm.cdf((hi - yb) * np.sqrt(n) / sigma) - stats.norm.cdf((lo - yb) * np.sqrt(n) / sigma)
    return (-np.log(hi - lo) - 0.5 * (n - 1) * np.log(2 * np.pi * sigma**2) - 0.5 * np.log(n)
            - S / (2 * sigma**2) + np.log(mass))


@pytest.mark.parametrize("kind,scale", [(0, 0.1), (1, 0.05)])
def test_smc_evidence_closed_form_on_gpu(env, kind, scale):
    P, S, ctx = env
    y = synth.gmm1d_data(30, [1.0], SIG, seed=31)
    exact = _log_int_normal_product(y, SIG)
    betas = synth.geometric_betas(20)
    zs = []
    for s in range(16):
        th0 = synth.prior_particles(1, 16384, seed=2000 + s)
        smp = S.SMCSampler(ctx, P.GMM(1, SIG), y, th0, betas, kind=kind, scale=scale, seed=700 + s)
        zs.append(smp.run(graph=True))
    ctx.check()
    zs = np.array(zs)
    se = zs.std(ddof=1) / np.sqrt(zs.size)
    assert abs(zs.mean() - exact) < 4 * se + 0.02, (zs.mean(), exact, se)


def test_smc_paper_model_matches_oracle_sampler_statistically(env):
    """Section 4.1.2 model (four components, 100 data, 8192 particles): the GPU
    and oracle samplers use the same Philox draws; their paths part once an
    accept decision falls inside the FP32 band, so compare log Z across seeds."""
    P, S, ctx = env
    w = synth.GMM4
    y = w.data()
    betas = synth.geometric_betas(w.T)
    g, o = [], []
    for s in range(4):
        th0 = synth.prior_particles(4, 2048, seed=50 + s)
        smp = S.SMCSampler(ctx, P.GMM(4, SIG), y, th0, betas, scale=w.scale, seed=90 + s)
        g.append(smp.run())
        o.append(oracle.smc_run(y, w.logw(), SIG, (-10, 10), th0, betas, 0, w.scale, 0.5, 90 + s)[0])
    ctx.check()
    g, o = np.array(g), np.array(o)
    spread = max(np.std(g, ddof=1), np.std(o, ddof=1), 0.05)
    assert abs(g.mean() - o.mean()) < 4 * spread, (g, o)


def test_pf_lg_matches_kalman(env):
    P, S, ctx = env
    phi, Sigma, beta = synth.msv_params()
    L = synth.chol(Sigma)
    _, y = synth.simulate_ssm("lg", 60, phi, Sigma, beta, seed=4)
    exact = oracle.kalman_lg(phi, Sigma, beta, y)
    zs = []
    for s in range(12):
        pf = S.ParticleFilter(ctx, P.PFModel(P.PF_LG, phi, L, beta), y, 65536, seed=300 + s)
        zs.append(pf.run(graph=(s % 2 == 0)))
    ctx.check()
    zs = np.array(zs)
    se = zs.std(ddof=1) / np.sqrt(zs.size)
    assert abs(zs.mean() - exact) < 4 * se + 0.05, (zs.mean(), exact, se)


def test_pf_graph_equals_plain_msv_full_size(env):
    P, S, ctx = env
    w = synth.MSV3
    phi, Sigma, beta = synth.msv_params()
    _, y = synth.simulate_ssm("msv", 50, phi, Sigma, beta, seed=w.data_seed)
    pf = S.ParticleFilter(ctx, P.PFModel(P.PF_MSV, phi, synth.chol(Sigma), beta), y, w.M, seed=5)
    z1 = pf.run()
    x1 = pf.x[pf.cur].clone()
    pf.reset()
    z2 = pf.run(graph=True)
    ctx.check()
    assert z1 == z2 and torch.equal(x1, pf.x[pf.cur]) and np.isfinite(z1)


def test_autograd_loglik(env):
    P, S, ctx = env
    from paper_0905_2441_gb300 import autograd
    y = synth.gmm1d_data(200, [-2, 0, 2], SIG, seed=8)
    th = torch.from_numpy(np.random.default_rng(0).uniform(-3, 3, (3, 50)).astype(np.float32)).cuda()
    th.requires_grad_(True)
    yd = torch.from_numpy(y).cuda()
    l = autograd.loglik(th, yd, P.GMM(3, SIG), ctx)
    w = torch.linspace(0.5, 1.5, 50, device="cuda", dtype=torch.float64)
    (l * w).sum().backward()
    ctx.check()
    ref = oracle.gmm1d_grad(y, np.full(3, -np.log(3)), SIG, th.detach().cpu().numpy())
    got = th.grad.cpu().numpy() / w.cpu().numpy()[None, :]
    np.testing.assert_allclose(got, ref, rtol=2e-4, atol=2e-3)
    np.testing.assert_allclose(l.detach().cpu().numpy(),
                               oracle.gmm1d_loglik(y, np.full(3, -np.log(3)), SIG,
                                                   th.detach().cpu().numpy()), rtol=1e-5)


def test_popmcmc_graph_equals_plain(env):
    P, S, ctx = env
    w = synth.GMM8_POP
    off = synth.population_offsets(64, seed=w.pop_seed)
    y = w.data()
    th0 = synth.population_particles(w.K, off)
    beta = synth.population_betas(off)
    a = S.PopulationMCMC(ctx, P.GMM(w.K, w.sigma), y, off, beta, th0, seed=9)
    a.run(20)
    b = S.PopulationMCMC(ctx, P.GMM(w.K, w.sigma), y, off, beta, th0, seed=9)
    b.run(20, graph=True)
    ctx.check()
    assert torch.equal(a.theta, b.theta) and torch.equal(a.ll, b.ll)
    assert torch.equal(a.stats, b.stats)


def test_autotuner_picks_a_valid_shape(env, tmp_path, monkeypatch):
    P, S, ctx = env
    from paper_0905_2441_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "cache.json"))
    y = torch.from_numpy(synth.gmm1d_data(1000, np.linspace(-7, 7, 8), SIG)).cuda()
    th = torch.from_numpy(synth.prior_particles(8, 20000)).cuda()
    lanes, threads, entry = autotune.tune_loglik(ctx, P.GMM(8, SIG), y, th, reps=2)
    assert lanes in autotune.LANES and threads in autotune.THREADS
    again = autotune.tune_loglik(ctx, P.GMM(8, SIG), y, th, reps=2)
    assert again[:2] == (lanes, threads)
    ctx.set_launch(P.OP_LOGLIK, 0, 0)


@pytest.mark.parametrize("graph", [False, True])
def test_resume_is_bitwise_the_uninterrupted_run(env, graph):
    """Checkpoint / resume: 6 steps, save, a fresh sampler loads the state and
    runs the rest -- the same particles, log-likelihoods, log-weights and
    log Z as one uninterrupted run (counter-based draws need no RNG state)."""
    P, S, ctx = env
    y = synth.gmm1d_data(100, [-3, 0, 3, 6], SIG, seed=1)
    th0 = synth.prior_particles(4, 4096, seed=3)
    betas = synth.power_betas(12, start=0)
    mk = lambda: S.SMCSampler(ctx, P.GMM(4, SIG), y, th0, betas, scale=1.0, seed=17, n_moves=2)
    a = mk()
    za = a.run(graph=graph)
    b = mk()
    b.run(graph=graph, stop=6)
    sd = b.state_dict()
    c = mk()
    c.load_state_dict(sd)
    zc = c.run(graph=graph)
    ctx.check()
    assert za == zc
    for u, v in zip(a.state, c.state):
        assert torch.equal(u, v)
    assert torch.equal(a.lw, c.lw) and torch.equal(a.flags, c.flags)
    hist = a.history()  # per-step metrics, identical for the resumed run
    assert hist == c.history() and len(hist) == 12 and abs(hist[-1]["log_z"] - za) < 1e-9
    # the particle filter and population MCMC resume the same way
    phi, Sigma, beta = synth.msv_params()
    _, yo = synth.simulate_ssm("msv", 30, phi, Sigma, beta, seed=4)
    mkf = lambda: S.ParticleFilter(ctx, P.PFModel(P.PF_MSV, phi, synth.chol(Sigma), beta), yo,
                                   20000, seed=8)
    fa = mkf()
    zfa = fa.run(graph=graph)
    fb = mkf()
    fb.run(graph=graph, steps=13)
    fc = mkf()
    fc.load_state_dict(fb.state_dict())
    zfc = fc.run(graph=graph)
    assert zfa == zfc and torch.equal(fa.x[fa.cur], fc.x[fc.cur])
    w = synth.GMM8_POP
    off = synth.population_offsets(64, seed=w.pop_seed)
    yp = w.data()
    beta_p = synth.population_betas(off)
    thp = synth.population_particles(w.K, off)
    mkp = lambda: S.PopulationMCMC(ctx, P.GMM(w.K, w.sigma), yp, off, beta_p, thp, scale=0.1,
                                   seed=3)
    pa = mkp()
    pa.run(10, graph=graph)
    pb = mkp()
    pb.run(4, graph=graph)
    pc = mkp()
    pc.load_state_dict(pb.state_dict())
    pc.run(6, start=4, graph=graph)
    ctx.check()
    assert torch.equal(pa.theta, pc.theta) and torch.equal(pa.ll, pc.ll)
    assert torch.equal(pa.stats, pc.stats)
