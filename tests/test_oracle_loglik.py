"""Pins for the oracle's mixture log-likelihoods and gradient (Section 4.1).

Brute-force enumeration of the product-sum over all K^N component
assignments, closed forms for one component, the permutation symmetry the
paper states (24 symmetric modes), and finite differences for the gradient."""
import itertools
import json
import os

import numpy as np
from scipy import stats

import oracle
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _brute_force_loglik(y, mu, w, sigma):
    """log prod_n sum_k w_k N(y_n|mu_k, sigma^2) expanded as a sum over all
    assignments z in {0..K-1}^N of prod_n w_{z_n} N(y_n | mu_{z_n})."""
    K = len(mu)
    dens = np.array([[w[k] * stats.norm.pdf(yn, mu[k], sigma) for k in range(K)] for yn in y])
    total = 0.0
    for z in itertools.product(range(K), repeat=len(y)):
        total += np.prod(dens[np.arange(len(y)), list(z)])
    return np.log(total)


def test_loglik_brute_force_k2_n8_and_k3_n6():
    g = np.random.default_rng(1)
    for K, N in [(2, 8), (3, 6)]:
        y = g.normal(0, 2, N).astype(np.float32)
        w = g.dirichlet(np.ones(K))
        for _ in range(3):
            mu = g.uniform(-3, 3, K).astype(np.float32)
            got = oracle.gmm1d_loglik(y, np.log(w), 0.7, mu[:, None])[0]
            want = _brute_force_loglik(y.astype(np.float64), mu.astype(np.float64), w, 0.7)
            assert abs(got - want) <= 1e-12 * abs(want)


def test_loglik_one_component_closed_form():
    y = synth.gmm1d_data(200, [1.5], 0.55, seed=3)
    mu = np.array([[0.3], [1.4], [-9.0]], np.float32).T  # K=1, M=3
    got = oracle.gmm1d_loglik(y, np.zeros(1), 0.55, mu)
    want = [stats.norm.logpdf(y.astype(np.float64), float(m), 0.55).sum() for m in mu[0]]
    np.testing.assert_allclose(got, want, rtol=1e-13)


def test_loglik_far_tail_no_underflow():
    """Every component far from the data: the max shift keeps the result finite."""
    y = np.array([8.0, 9.5], np.float32)
    mu = np.full((4, 1), -10.0, np.float32)
    got = oracle.gmm1d_loglik(y, np.full(4, -np.log(4)), 0.55, mu)[0]
    want = stats.norm.logpdf(y.astype(np.float64), -10.0, 0.55).sum()
    assert np.isfinite(got) and abs(got - want) < 1e-9 * abs(want)


def test_paper_mixture_has_24_symmetric_modes():
    """Section 4.1: with exchangeable priors the posterior is invariant to
    relabelling, so all k! = 24 permutations of mu give the same likelihood."""
    c = GOLD["gmm_section_4_1"]
    y = synth.gmm1d_data(c["m"], c["mu"], c["sigma"], seed=1)
    perms = np.array(list(itertools.permutations(c["mu"])), np.float32)
    assert len(perms) == c["n_symmetric_modes"]
    ll = oracle.gmm1d_loglik(y, np.full(4, -np.log(4)), c["sigma"], perms.T.copy())
    assert np.ptp(ll) <= 1e-12 * abs(ll[0])
    # and the true means are (near) a mode: a shifted mu is less likely
    shifted = oracle.gmm1d_loglik(y, np.full(4, -np.log(4)), c["sigma"],
                                  (perms[:1] + 0.5).T.copy())
    assert shifted[0] < ll[0] - 10
    # unit count: k*m Gaussian evaluations per likelihood (Section 5)
    assert c["k"] * c["m"] == GOLD["likelihood_size_section_5"]["gaussian_evals_per_likelihood"]
    assert c["k"] + c["m"] == GOLD["likelihood_size_section_5"]["values_involved"]


def test_gradient_central_differences():
    g = np.random.default_rng(2)
    y = synth.gmm1d_data(300, [-3, 0, 3, 6], 0.55, seed=5)
    logw = np.log(np.array([0.1, 0.2, 0.3, 0.4]))
    theta = g.uniform(-5, 7, (4, 5)).astype(np.float32)
    G = oracle.gmm1d_grad(y, logw, 0.55, theta)
    h = 1e-4
    for p in range(theta.shape[1]):
        mu = theta[:, p].astype(np.float64)
        for k in range(4):
            e = np.zeros(4)
            e[k] = h
            fd = (oracle.gmm1d_loglik_at(y, logw, 0.55, mu + e) -
                  oracle.gmm1d_loglik_at(y, logw, 0.55, mu - e)) / (2 * h)
            assert abs(fd - G[k, p]) <= 1e-5 * max(1.0, abs(G[k, p]))


def test_gradient_one_component_closed_form():
    y = synth.gmm1d_data(50, [2.0], 0.8, seed=6)
    mu = np.array([[0.5, 2.0, 3.1]], np.float32)
    G = oracle.gmm1d_grad(y, np.zeros(1), 0.8, mu)
    want = [(y.astype(np.float64) - m).sum() / 0.64 for m in mu[0].astype(np.float64)]
    np.testing.assert_allclose(G[0], want, rtol=1e-12, atol=1e-10)


def test_diag_loglik_closed_form_and_brute_force():
    g = np.random.default_rng(3)
    d = 5
    Y = g.normal(0, 2, (7, d)).astype(np.float32)
    # K=1: sum of isotropic Gaussian log-densities
    th = g.normal(0, 1, (3, 1, d)).astype(np.float32)
    got = oracle.gmmdiag_loglik(Y, np.zeros(1), 1.3, th)
    for p in range(3):
        want = stats.multivariate_normal.logpdf(Y.astype(np.float64), th[p, 0].astype(np.float64),
                                                1.69 * np.eye(d)).sum()
        assert abs(got[p] - want) <= 1e-12 * abs(want)
    # K=2, N=4: enumerate assignments
    w = np.array([0.3, 0.7])
    th2 = g.normal(0, 1, (2, 2, d)).astype(np.float32)
    got2 = oracle.gmmdiag_loglik(Y[:4], np.log(w), 0.9, th2)
    for p in range(2):
        dens = np.array([[w[k] * stats.multivariate_normal.pdf(Y[n].astype(np.float64),
                                                              th2[p, k].astype(np.float64),
                                                              0.81 * np.eye(d))
                          for k in range(2)] for n in range(4)])
        tot = sum(np.prod(dens[np.arange(4), list(z)]) for z in itertools.product(range(2), repeat=4))
        assert abs(got2[p] - np.log(tot)) <= 1e-11 * abs(np.log(tot))


def test_diag_reduces_to_1d_when_d_is_1():
    y = synth.gmm1d_data(40, [-1, 2], 0.6, seed=8)
    th = np.array([[-1.1, 2.2], [0.0, 1.0]], np.float32)  # [M][K]
    a = oracle.gmmdiag_loglik(y[:, None], np.log([0.4, 0.6]), 0.6, th[:, :, None])
    b = oracle.gmm1d_loglik(y, np.log([0.4, 0.6]), 0.6, th.T.copy())
    np.testing.assert_allclose(a, b, rtol=1e-14)
