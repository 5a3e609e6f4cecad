"""Pins for the oracle's particle filter (Sections 3.2, 4.2), its Kalman
filter, and the tempered SMC sampler's evidence (Sections 3.3, 4.1.2)."""
import itertools

import numpy as np
import pytest
from scipy import stats

import oracle
import synth

# ------------------------------------------------------------------ particle filter


def test_pf_weight_matches_library_densities():
    phi, Sigma, beta = synth.msv_params()
    L = synth.chol(Sigma)
    g = np.random.default_rng(0)
    M = 500
    x_in = g.normal(0, 1, (3, M)).astype(np.float32)
    yt = np.array([0.3, -1.2, 0.05], np.float32)
    for kind in (oracle.PF_MSV, oracle.PF_LG):
        x_out, lg = oracle.pf_step(kind, phi, L, beta, yt, x_in, None, 3, 5)
        x = x_out.astype(np.float64)
        if kind == oracle.PF_MSV:
            want = stats.norm.logpdf(yt[:, None].astype(np.float64), 0.0, beta * np.exp(0.5 * x)).sum(0)
        else:
            want = stats.norm.logpdf(yt[:, None].astype(np.float64), x, beta).sum(0)
        np.testing.assert_allclose(lg, want, rtol=1e-12, atol=1e-12)


def test_pf_propagation_distribution_and_gather():
    phi, Sigma, beta = synth.msv_params()
    L = synth.chol(Sigma)
    M = 100000
    x0 = np.tile(np.array([[1.0], [-2.0], [0.5]], np.float32), (1, M))
    x_out, _ = oracle.pf_step(oracle.PF_MSV, phi, L, beta, np.zeros(3, np.float32), x0, None, 9, 1)
    eta = x_out.astype(np.float64) - phi[:, None] * x0.astype(np.float64)
    assert np.all(np.abs(eta.mean(1)) < 4 * np.sqrt(np.diag(Sigma) / M))
    np.testing.assert_allclose(np.cov(eta), Sigma, atol=0.02)
    # zero noise: slot i holds phi * x_in[anc[i]] exactly
    xi = np.random.default_rng(1).normal(0, 1, (3, 50)).astype(np.float32)
    anc = np.random.default_rng(2).integers(0, 50, 50).astype(np.int32)
    xo, _ = oracle.pf_step(oracle.PF_LG, phi, np.zeros((3, 3)), beta, np.zeros(3, np.float32), xi,
                           anc, 9, 1)
    np.testing.assert_array_equal(xo, (phi[:, None] * xi[:, anc].astype(np.float64)).astype(np.float32))


def test_kalman_matches_dense_gaussian():
    """The linear-Gaussian y_{1:T} is jointly Gaussian; its exact log-density
    from the dense covariance pins the Kalman recursion."""
    phi, Sigma, beta = synth.msv_params()
    T, d = 8, 3
    _, y = synth.simulate_ssm("lg", T, phi, Sigma, beta, seed=3)
    A = np.diag(phi)
    cov_x = np.zeros((T * d, T * d))
    P = [None] * T
    Pt = np.zeros((d, d))
    for t in range(T):
        Pt = A @ Pt @ A.T + Sigma
        P[t] = Pt
    for s in range(T):
        for t in range(s, T):
            c = np.linalg.matrix_power(A, t - s) @ P[s]
            cov_x[t * d:(t + 1) * d, s * d:(s + 1) * d] = c
            cov_x[s * d:(s + 1) * d, t * d:(t + 1) * d] = c.T
    cov_y = cov_x + beta**2 * np.eye(T * d)
    want = stats.multivariate_normal.logpdf(y.astype(np.float64).ravel(), np.zeros(T * d), cov_y)
    got = oracle.kalman_lg(phi, Sigma, beta, y)
    assert abs(got - want) < 1e-9 * abs(want)


def test_pf_evidence_matches_kalman():
    phi, Sigma, beta = synth.msv_params()
    L = synth.chol(Sigma)
    _, y = synth.simulate_ssm("lg", 40, phi, Sigma, beta, seed=4)
    exact, kmeans = oracle.kalman_lg(phi, Sigma, beta, y, want_means=True)
    zs, mse = [], []
    for s in range(12):
        z, means = oracle.pf_run(oracle.PF_LG, phi, L, beta, y, 4096, 100 + s, want_means=True)
        zs.append(z)
        mse.append(np.abs(means - kmeans).mean())
    zs = np.array(zs)
    se = zs.std(ddof=1) / np.sqrt(zs.size)
    assert abs(zs.mean() - exact) < 4 * se + 0.05, (zs.mean(), exact, se)
    # filter means: Monte Carlo error ~ 0.02 per entry at this particle count
    assert np.mean(mse) < 0.05


def test_pf_msv_runs_and_tracks_volatility():
    phi, Sigma, beta = synth.msv_params()
    L = synth.chol(Sigma)
    x, y = synth.simulate_ssm("msv", 60, phi, Sigma, beta, seed=7)
    z, means = oracle.pf_run(oracle.PF_MSV, phi, L, beta, y, 4096, 5, want_means=True)
    assert np.isfinite(z)
    # the filter means correlate with the true log-volatilities
    assert np.corrcoef(means.ravel(), x.ravel())[0, 1] > 0.5


# ------------------------------------------------------------------ SMC sampler evidence
SIG = 0.55


def _log_int_normal_product(ys, sigma, lo=-10.0, hi=10.0):
    """log of (1/(hi-lo)) * int_lo^hi prod_n N(y_n | mu, sigma^2) dmu."""
    n = len(ys)
    if n == 0:
        return 0.0
    ys = np.asarray(ys, np.float64)
    yb = ys.mean()
    S = np.sum((ys - yb) ** 2)
    mass = stats.norm.cdf((hi - yb) * np.sqrt(n) / sigma) - stats.norm.cdf((lo - yb) * np.sqrt(n) / sigma)
    return (-np.log(hi - lo) - 0.5 * (n - 1) * np.log(2 * np.pi * sigma**2) - 0.5 * np.log(n)
            - S / (2 * sigma**2) + np.log(mass))


def _smc_logZ(y, K, M, T, kind, scale, seeds, n_moves=1):
    betas = synth.geometric_betas(T, 1e-3)
    out = []
    for s in seeds:
        th0 = synth.prior_particles(K, M, seed=1000 + s)
        z, _, ess, rs = oracle.smc_run(y, np.full(K, -np.log(K)), SIG, (-10, 10), th0, betas, kind,
                                       scale, 0.5, 500 + s, n_moves=n_moves)
        out.append(z)
    return np.array(out)


@pytest.mark.parametrize("kind,scale,n_moves", [(0, 0.1, 1), (1, 0.05, 1), (0, 0.3, 3)])
def test_smc_evidence_one_component_closed_form(kind, scale, n_moves):
    y = synth.gmm1d_data(30, [1.0], SIG, seed=31)
    exact = _log_int_normal_product(y, SIG)
    zs = _smc_logZ(y, 1, 2048, 20, kind, scale, range(12), n_moves=n_moves)
    se = zs.std(ddof=1) / np.sqrt(zs.size)
    assert abs(zs.mean() - exact) < 4 * se + 0.02, (zs.mean(), exact, se)


def test_smc_evidence_two_components_brute_force():
    """Z = sum over assignments z of prod_n w_{z_n} prod_k (1/20) int prod_{n: z_n=k} N(y_n|mu)."""
    y = synth.gmm1d_data(6, [-2.0, 2.0], SIG, seed=32)
    K = 2
    terms = []
    for z in itertools.product(range(K), repeat=y.size):
        t = y.size * np.log(1.0 / K)
        for k in range(K):
            t += _log_int_normal_product([y[n] for n in range(y.size) if z[n] == k], SIG)
        terms.append(t)
    exact = np.logaddexp.reduce(terms)
    zs = _smc_logZ(y, K, 4096, 20, 0, 0.3, range(12))
    se = zs.std(ddof=1) / np.sqrt(zs.size)
    assert abs(zs.mean() - exact) < 4 * se + 0.02, (zs.mean(), exact, se)


def test_smc_paper_model_covers_symmetric_modes():
    """Section 4.1.2: the tempered SMC sampler represents all 24 relabelled
    modes; each ordering of the four means carries about 1/24 of the mass."""
    y = synth.gmm1d_data(100, [-3, 0, 3, 6], SIG, seed=1)
    betas = synth.geometric_betas(20, 1e-3)
    th0 = synth.prior_particles(4, 8192, seed=2)
    z, th, ess, rs = oracle.smc_run(y, np.full(4, -np.log(4)), SIG, (-10, 10), th0, betas, 0, 0.1,
                                    0.5, 1234)
    order = np.argsort(th, axis=0)
    perms = {tuple(o) for o in order.T}
    # 20 temperatures and one random-walk move per step (far fewer than the
    # paper's 200 x 10) still leave many relabelled modes populated
    assert len(perms) >= 12
    assert rs.sum() >= 1


def test_smc_several_moves_per_temperature():
    """Section 4.1.2 runs 10 random-walk moves per temperature.  Move r of
    step t draws from step counter t + r 2^32 and starts from move r-1's
    output (identity ancestors): one move reproduces the single-move run,
    and the second move's proposals are fresh draws."""
    y = synth.gmm1d_data(20, [-3, 3], SIG, seed=5)
    logw = np.full(2, -np.log(2))
    th0 = synth.prior_particles(2, 256, seed=6)
    betas = synth.power_betas(3, start=0)
    a = oracle.smc_run(y, logw, SIG, (-10, 10), th0, betas, 0, 1.0, 0.5, 17)
    b = oracle.smc_run(y, logw, SIG, (-10, 10), th0, betas, 0, 1.0, 0.5, 17, n_moves=1)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    # two moves at one (small) temperature, written out from the single-move primitive
    b2 = np.array([0.0, 1e-5])
    bt = np.float32(b2[1])
    l0 = oracle.gmm1d_loglik(y, logw, SIG, th0)
    z, th, ess, rs = oracle.smc_run(y, logw, SIG, (-10, 10), th0, b2, 0, 1.0, 0.5, 17,
                                    n_moves=2)
    assert rs[0] == 0  # one small temperature step: no resampling
    t1, l1, _ = oracle.rwmh_move(y, logw, SIG, (-10, 10), th0, l0, bt, 1.0, 17, 1)
    t2, l2, _ = oracle.rwmh_move(y, logw, SIG, (-10, 10), t1, l1, bt, 1.0, 17, 1 + (1 << 32))
    np.testing.assert_array_equal(th, t2)
    assert not np.array_equal(t1, t2)


def test_smc_paper_table2_schedule_covers_all_modes():
    """Section 4.1.2 / Table 2 setting at reduced size: beta_t = (t/T)^2,
    ten N(0, I_4) random-walk moves per temperature.  The sampler then
    represents all 24 relabelled modes of the four-component posterior."""
    y = synth.gmm1d_data(100, [-3, 0, 3, 6], SIG, seed=1)
    betas = synth.power_betas(30, start=0)
    th0 = synth.prior_particles(4, 1024, seed=2)
    z, th, ess, rs = oracle.smc_run(y, np.full(4, -np.log(4)), SIG, (-10, 10), th0, betas, 0, 1.0,
                                    0.5, 4321, n_moves=10)
    order = np.argsort(th, axis=0)
    perms = {tuple(o) for o in order.T}
    assert len(perms) == 24
    assert 1 <= rs.sum() < 30


def test_ais_no_resampling_closed_form():
    """Section 4.1.2: the sampler with no resampling at all is annealed
    importance sampling; its evidence estimate still targets the closed-form
    marginal likelihood (one component), and it never resamples."""
    y = synth.gmm1d_data(30, [1.0], SIG, seed=31)
    exact = _log_int_normal_product(y, SIG)
    betas = synth.geometric_betas(20, 1e-3)
    zs = []
    for s in range(12):
        th0 = synth.prior_particles(1, 2048, seed=1000 + s)
        z, _, ess, rs = oracle.smc_run(y, np.zeros(1), SIG, (-10, 10), th0, betas, 0, 0.3, 0.0,
                                       500 + s, n_moves=2)
        assert rs.sum() == 0
        zs.append(z)
    zs = np.array(zs)
    se = zs.std(ddof=1) / np.sqrt(zs.size)
    assert abs(zs.mean() - exact) < 4 * se + 0.05, (zs.mean(), exact, se)
