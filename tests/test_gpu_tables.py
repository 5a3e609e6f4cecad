"""GPU parity for the paper's Table 1 and Table 2 configurations (Section
4.1): one large population of tempered chains (the exchange stage then runs
as its own grid-wide launch) and the SMC sampler with several random-walk
moves per temperature, each against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from _popcheck import explain_sweep
import synth

pytestmark = pytest.mark.gpu
SIG = 0.55
BOX = (-10.0, 10.0)


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


def np_(t):
    return t.detach().cpu().numpy()


def _pop_betas(off):
    """beta_i = (i/M_q)^2 along each population (Section 4.1.1)."""
    b = np.zeros(int(off[-1]), np.float32)
    for q in range(off.size - 1):
        m = int(off[q + 1] - off[q])
        if m:
            b[off[q]:off[q + 1]] = synth.power_betas(m).astype(np.float32)
    return b


@pytest.mark.parametrize("off", [
    [0, 3000],                        # Table 1 shape: one population
    [0, 1, 1, 1000, 1003, 4000],      # large and tiny (even, odd, empty) populations
    [0, 4096],                        # even population: the wrap pair (M-1, 0)
])
def test_large_population_sweep_parity(env, off):
    P, S, ctx = env
    off = np.array(off, np.int32)
    Mt = int(off[-1])
    assert Mt > 2 * 256 * (off.size - 1)  # the grid-wide exchange launch is taken
    w = synth.PAPER_TABLES
    y = w.data()
    beta = _pop_betas(off)
    th = synth.population_particles(w.K, off, seed=21)
    ll = oracle.gmm1d_loglik(y, w.logw(), SIG, th)
    model = P.GMM(w.K, SIG)
    for sweep in range(3):
        tt, lt = cu(th), cu(ll)
        stats = torch.zeros(3, dtype=torch.int64, device="cuda")
        P.popmcmc_sweep(ctx, model, cu(y), tt, lt, cu(beta), cu(off), w.scale, 808, sweep,
                        stats=stats)
        ctx.check()
        rt, rl, rst = oracle.popmcmc_sweep(y, w.logw(), SIG, BOX, th, ll, beta, off, w.scale, 808,
                                           sweep)
        gt, gl = np_(tt), np_(lt)
        # a population may differ only through decisions inside the FP32 band
        rep = explain_sweep(y, w.logw(), SIG, BOX, th, ll, beta, off, w.scale, 808, sweep, gt, gl)
        assert rep.unexplained == [], (sweep, rep)
        s = np_(stats)
        assert s[2] == rst[2]
        assert abs(int(s[0]) - int(rst[0])) <= 2 and abs(int(s[1]) - int(rst[1])) <= 2
        th, ll = rt, rl  # next sweep from the oracle's state


def test_large_population_graph_equals_plain(env):
    P, S, ctx = env
    w = synth.PAPER_TABLES
    y = w.data()
    M = 8192
    off = np.array([0, M], np.int32)
    beta = synth.power_betas(M).astype(np.float32)
    th0 = synth.prior_particles(w.K, M, seed=5)
    a = S.PopulationMCMC(ctx, P.GMM(w.K, SIG), y, off, beta, th0, scale=w.scale, seed=9)
    a.run(6)
    b = S.PopulationMCMC(ctx, P.GMM(w.K, SIG), y, off, beta, th0, scale=w.scale, seed=9)
    b.run(6, graph=True)
    ctx.check()
    assert torch.equal(a.theta, b.theta) and torch.equal(a.ll, b.ll)
    assert torch.equal(a.stats, b.stats)
    st = np_(a.stats)
    assert st[2] > 0 and 0 < st[1] <= st[2] and st[0] > 0


def test_inline_and_split_exchange_agree(env):
    """The same populations swept with the in-sweep exchange (many small
    populations) and with the grid-wide exchange launch (the same chains
    regrouped so the average population is large): chains of populations
    common to both take the same moves and swaps.  Their log-likelihoods
    agree to the rounding of the FP32 partial sums, whose split over the
    data follows the launch geometry (here two different chain counts)."""
    P, S, ctx = env
    w = synth.PAPER_TABLES
    y = w.data()
    small = np.arange(0, 64 * 40 + 1, 64, dtype=np.int32)       # 40 populations of 64
    big = np.concatenate([small[:2], [small[-1] + 6000]]).astype(np.int32)  # 64, then 8496
    assert small[-1] <= 2 * 256 * (small.size - 1) and big[-1] > 2 * 256 * (big.size - 1)
    th_big = synth.population_particles(w.K, big, seed=31)
    res = {}
    for name, off in (("inline", small), ("split", big)):
        Mt = int(off[-1])
        th = th_big[:, :Mt].copy()
        beta = _pop_betas(off)
        tt = cu(th)
        lt = cu(oracle.gmm1d_loglik(y, w.logw(), SIG, th))
        for s in range(2):
            P.popmcmc_sweep(ctx, P.GMM(w.K, SIG), cu(y), tt, lt, cu(beta), cu(off), w.scale, 4, s)
        ctx.check()
        res[name] = (np_(tt), np_(lt))
    # population 0 (chains 0..63) is the same population in both layouts
    assert np.array_equal(res["inline"][0][:, :64], res["split"][0][:, :64])
    np.testing.assert_allclose(res["inline"][1][:64], res["split"][1][:64], rtol=1e-7, atol=0)


@pytest.mark.parametrize("kind", [0, 1])
def test_smc_several_moves_graph_equals_plain(env, kind):
    P, S, ctx = env
    w = synth.PAPER_TABLES
    y = w.data()
    th0 = synth.prior_particles(4, 4096, seed=3)
    betas = synth.power_betas(12, start=0)
    smp = S.SMCSampler(ctx, P.GMM(4, SIG), y, th0, betas, kind=kind,
                       scale=w.scale if kind == 0 else 0.05, seed=11, n_moves=3)
    z1 = smp.run()
    th1, l1 = [t.clone() for t in smp.state]
    f1 = smp.flags.clone()
    acc1 = smp.accepts.clone()
    smp.reset(th0)
    z2 = smp.run(graph=True)
    th2, l2 = smp.state
    ctx.check()
    assert z1 == z2 and torch.equal(th1, th2) and torch.equal(l1, l2)
    assert torch.equal(f1, smp.flags) and torch.equal(acc1, smp.accepts)


def test_smc_several_moves_trajectories_match_oracle(env):
    """Two small temperature steps (no resampling), three RW moves each:
    every particle follows the oracle's trajectory unless one of its six
    accept decisions falls inside the FP32 band."""
    P, S, ctx = env
    w = synth.PAPER_TABLES
    y = w.data()
    M = 4096
    th0 = synth.prior_particles(4, M, seed=8)
    betas = np.array([0.0, 1e-5, 2e-5])
    smp = S.SMCSampler(ctx, P.GMM(4, SIG), y, th0, betas, scale=w.scale, seed=23, n_moves=3)
    zg = smp.run()
    ctx.check()
    zo, tho, esso, rso = oracle.smc_run(y, w.logw(), SIG, BOX, th0, betas, 0, w.scale, 0.5, 23,
                                        n_moves=3)
    assert rso.sum() == 0 and int(smp.flags[1:].sum()) == 0
    thg = np_(smp.state[0])
    same = np.all(np.isclose(thg, tho, rtol=3e-7, atol=2e-6), axis=0)
    assert (~same).sum() <= max(2, M // 500), (~same).sum()
    assert abs(zg - zo) <= 1e-6 * abs(zo) + 1e-6


def test_smc_paper_table2_setting_matches_oracle_statistically(env):
    """Table 2's sampler (beta_t = (t/T)^2, ten N(0, I_4) moves per
    temperature) at reduced size: GPU and oracle log Z agree across seeds."""
    P, S, ctx = env
    w = synth.PAPER_TABLES
    y = w.data()
    betas = synth.power_betas(10, start=0)
    g, o = [], []
    for s in range(4):
        th0 = synth.prior_particles(4, 1024, seed=60 + s)
        smp = S.SMCSampler(ctx, P.GMM(4, SIG), y, th0, betas, scale=w.scale, seed=70 + s,
                           n_moves=10)
        g.append(smp.run())
        o.append(oracle.smc_run(y, w.logw(), SIG, BOX, th0, betas, 0, w.scale, 0.5, 70 + s,
                                n_moves=10)[0])
    ctx.check()
    g, o = np.array(g), np.array(o)
    spread = max(np.std(g, ddof=1), np.std(o, ddof=1), 0.05)
    assert abs(g.mean() - o.mean()) < 4 * spread, (g, o)


def test_ais_on_gpu_never_resamples_and_matches_oracle(env):
    """Annealed importance sampling (Section 4.1.2: the SMC sampler with no
    resampling): no step resamples, and the GPU and oracle evidence
    estimates agree across seeds."""
    P, S, ctx = env
    w = synth.PAPER_TABLES
    y = w.data()
    betas = synth.power_betas(10, start=0)
    g, o = [], []
    for s in range(4):
        th0 = synth.prior_particles(4, 1024, seed=80 + s)
        smp = S.SMCSampler(ctx, P.GMM(4, SIG), y, th0, betas, scale=w.scale, seed=90 + s,
                           n_moves=5, ess_frac=0.0)
        g.append(smp.run())
        assert int(smp.flags.sum()) == 0
        zo, _, _, rs = oracle.smc_run(y, w.logw(), SIG, BOX, th0, betas, 0, w.scale, 0.0, 90 + s,
                                      n_moves=5)
        assert rs.sum() == 0
        o.append(zo)
    ctx.check()
    g, o = np.array(g), np.array(o)
    spread = max(np.std(g, ddof=1), np.std(o, ddof=1), 0.1)
    assert abs(g.mean() - o.mean()) < 4 * spread, (g, o)
