"""Pins for the oracle's random-walk MH, MALA and population-MCMC sweep
(Sections 3.1, 4.1.1, 4.1.2).

A pi-invariant kernel started from exact draws of pi must leave them
distributed as pi: with one component the tempered posterior
prior * L^beta is (up to negligible truncation) N(ybar, sigma^2/(beta N)),
so each kernel is checked against that closed form.  The exchange pairing is
checked deterministically against the paper's two pair sets."""
import numpy as np
import pytest
from scipy import stats

import oracle
import synth

SIG = 0.55
BOX = (-10.0, 10.0)


def _posterior(y, beta):
    return float(np.mean(y.astype(np.float64))), SIG / np.sqrt(beta * y.size)


def _exact_draws(y, beta, M, seed):
    m, s = _posterior(y, beta)
    return (m + s * np.random.default_rng(seed).standard_normal((1, M))).astype(np.float32)


@pytest.mark.parametrize("beta", [1.0, 0.2])
def test_rwmh_leaves_tempered_posterior_invariant(beta):
    y = synth.gmm1d_data(100, [1.0], SIG, seed=21)
    m, s = _posterior(y, beta)
    M = 40000
    th = _exact_draws(y, beta, M, 1)
    ll = oracle.gmm1d_loglik(y, np.zeros(1), SIG, th)
    acc_tot = 0
    for step in range(6):
        th, ll, acc = oracle.rwmh_move(y, np.zeros(1), SIG, BOX, th, ll, beta, 1.5 * s, 99, step)
        acc_tot += acc.sum()
    assert 0.2 < acc_tot / (6 * M) < 0.9
    assert stats.kstest((th[0].astype(np.float64) - m) / s, "norm").pvalue > 1e-4
    np.testing.assert_allclose(ll, oracle.gmm1d_loglik(y, np.zeros(1), SIG, th), rtol=1e-14)


def test_rwmh_wrong_temperature_is_detected():
    """The invariance check has power: a kernel targeting beta=1 does not
    preserve draws from beta=0.2."""
    y = synth.gmm1d_data(100, [1.0], SIG, seed=21)
    m, s = _posterior(y, 0.2)
    th = _exact_draws(y, 0.2, 40000, 2)
    ll = oracle.gmm1d_loglik(y, np.zeros(1), SIG, th)
    for step in range(6):
        th, ll, _ = oracle.rwmh_move(y, np.zeros(1), SIG, BOX, th, ll, 1.0, 1.5 * s, 99, step)
    assert stats.kstest((th[0].astype(np.float64) - m) / s, "norm").pvalue < 1e-6


def test_rwmh_proposal_and_box():
    y = synth.gmm1d_data(20, [0.0, 1.0], SIG, seed=22)
    K, M = 2, 2000
    th = np.full((K, M), 9.9, np.float32)
    ll = oracle.gmm1d_loglik(y, np.log([0.5, 0.5]), SIG, th)
    out, lo, acc = oracle.rwmh_move(y, np.log([0.5, 0.5]), SIG, BOX, th, ll, 1.0, 0.5, 5, 3)
    assert np.all(out <= 10.0) and np.all(out >= -10.0)
    assert np.all(out[:, acc == 0] == 9.9)
    # accepted moves equal theta + s z with the documented normals
    for p in np.flatnonzero(acc)[:20]:
        z = oracle.normals(5, oracle.P_MOVE, 3, int(p), K)
        np.testing.assert_array_equal(out[:, p], np.float32(float(np.float32(9.9)) + 0.5 * z))
    # a proposal leaving the box is always rejected
    z_all = np.array([oracle.normals(5, oracle.P_MOVE, 3, p, K) for p in range(M)]).T
    outside = np.any(th.astype(np.float64) + 0.5 * z_all > 10.0, axis=0)
    assert np.all(acc[outside] == 0)


def test_rwmh_gathers_ancestors():
    y = synth.gmm1d_data(20, [0.0], SIG, seed=23)
    th = np.arange(10, dtype=np.float32)[None] * 0.5
    ll = oracle.gmm1d_loglik(y, np.zeros(1), SIG, th)
    anc = np.array([3, 3, 3, 0, 9, 9, 1, 2, 2, 2], np.int32)
    out, lo, acc = oracle.rwmh_move(y, np.zeros(1), SIG, BOX, th, ll, 1.0, 0.0, 1, 1, anc=anc)
    # zero scale: the proposal equals the gathered state and is accepted
    np.testing.assert_array_equal(out[0], th[0, anc])
    np.testing.assert_array_equal(lo, ll[anc])


@pytest.mark.parametrize("beta", [1.0, 0.3])
def test_mala_leaves_tempered_posterior_invariant(beta):
    y = synth.gmm1d_data(100, [-2.0], SIG, seed=24)
    m, s = _posterior(y, beta)
    M = 40000
    th = _exact_draws(y, beta, M, 3)
    ll = oracle.gmm1d_loglik(y, np.zeros(1), SIG, th)
    g = oracle.gmm1d_grad(y, np.zeros(1), SIG, th).astype(np.float32)
    h = 1.6 * s  # large step: an uncorrected Langevin step would inflate the variance 2.8x
    for step in range(6):
        th, ll, g, acc = oracle.mala_move(y, np.zeros(1), SIG, BOX, th, ll, g, beta, h, 7, step)
    z = (th[0].astype(np.float64) - m) / s
    assert stats.kstest(z, "norm").pvalue > 1e-4
    np.testing.assert_allclose(g, oracle.gmm1d_grad(y, np.zeros(1), SIG, th), rtol=1e-6, atol=1e-6)


def _paper_pairs(m, b):
    """Section 4.1.1 (0-based): {0,1},{2,3},... or {1,2},{3,4},...,{m-1,0};
    with an odd chain count the chain left without a partner sits out."""
    if b == 0:
        return [(2 * j, 2 * j + 1) for j in range(m // 2)]
    pairs = [(2 * j + 1, 2 * j + 2) for j in range((m - 1) // 2)]
    if m % 2 == 0:
        pairs.append((m - 1, 0))
    return pairs


def test_exchange_pairing_is_the_papers():
    y = synth.gmm1d_data(30, [0.0, 2.0], SIG, seed=25)
    logw = np.log([0.5, 0.5])
    offsets = np.array([0, 2, 5, 9, 16, 17, 25], np.int32)
    Mt = int(offsets[-1])
    th = np.stack([np.arange(Mt, dtype=np.float32) * 0.1, -np.arange(Mt, dtype=np.float32) * 0.1])
    ll = oracle.gmm1d_loglik(y, logw, SIG, th)
    beta = np.full(Mt, 0.7, np.float32)  # equal temperatures: every swap is accepted
    for sweep in range(4):
        new_th, new_ll, stats_ = oracle.popmcmc_sweep(y, logw, SIG, BOX, th, ll, beta, offsets,
                                                      0.0, 31, sweep)
        want = np.arange(Mt)
        npairs = 0
        for q in range(offsets.size - 1):
            b = int(oracle.draw_words(31, oracle.P_EXCHANGE, sweep, q, 0)[0]) & 1
            m = int(offsets[q + 1] - offsets[q])
            if m < 2:
                continue
            for a, c in _paper_pairs(m, b):
                want[offsets[q] + a], want[offsets[q] + c] = offsets[q] + c, offsets[q] + a
                npairs += 1
        np.testing.assert_array_equal(new_th, th[:, want])
        np.testing.assert_array_equal(new_ll, ll[want])
        assert stats_[0] == Mt and stats_[1] == npairs and stats_[2] == npairs


def test_popmcmc_leaves_product_of_tempered_posteriors_invariant():
    y = synth.gmm1d_data(60, [0.5], SIG, seed=26)
    n_pops = 15000
    offsets = (np.arange(n_pops + 1) * 2).astype(np.int32)
    betas = np.tile(np.array([0.15, 1.0], np.float32), n_pops)
    Mt = 2 * n_pops
    m0, s0 = _posterior(y, 0.15)
    m1, s1 = _posterior(y, 1.0)
    g = np.random.default_rng(4)
    th = np.where(np.arange(Mt) % 2 == 0, m0 + s0 * g.standard_normal(Mt),
                  m1 + s1 * g.standard_normal(Mt)).astype(np.float32)[None]
    ll = oracle.gmm1d_loglik(y, np.zeros(1), SIG, th)
    swaps = 0
    for sweep in range(5):
        th, ll, st = oracle.popmcmc_sweep(y, np.zeros(1), SIG, BOX, th, ll, betas, offsets,
                                          float(1.2 * s1), 41, sweep)
        swaps += st[1]
    assert swaps > 0.05 * 5 * n_pops  # exchanges do happen
    cold = (th[0, 1::2].astype(np.float64) - m1) / s1
    hot = (th[0, 0::2].astype(np.float64) - m0) / s0
    assert stats.kstest(cold, "norm").pvalue > 1e-4
    assert stats.kstest(hot, "norm").pvalue > 1e-4
