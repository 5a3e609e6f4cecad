"""Pins for the oracle's weights, ESS and exact-integer systematic resampling
(Section 3 normalised weights; Section 3.2 ESS and resampling; Section 4.1.2
incremental weight; Section 2.1 importance-sampling example)."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import special, stats

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_reweight_against_library_softmax_and_logsumexp():
    g = np.random.default_rng(0)
    for M in [1, 7, 1000]:
        lw0 = g.normal(0, 3, M)
        ll = g.normal(-200, 30, M)
        lw, W, sc = oracle.reweight(ll, 0.37, lw0)
        np.testing.assert_allclose(lw, lw0 + 0.37 * ll, rtol=0, atol=1e-12)
        np.testing.assert_allclose(W, special.softmax(lw0 + 0.37 * ll), rtol=1e-12, atol=1e-300)
        assert abs(W.sum() - 1) < 1e-14
        assert abs(sc[0] - (special.logsumexp(lw) - special.logsumexp(lw0))) < 1e-10
        assert abs(sc[1] - 1.0 / np.sum(W**2)) <= 1e-11 * sc[1]
        assert 1 - 1e-12 <= sc[1] <= M * (1 + 1e-12)
        assert sc[2] == lw.max()
        assert abs(sc[3] - special.logsumexp(lw)) < 1e-10


def test_reweight_special_cases():
    M = 64
    lw, W, sc = oracle.reweight(np.full(M, -5.0), 0.5, np.zeros(M))
    assert sc[1] == M and np.all(W == 1.0 / M)
    assert abs(sc[0] - (0.5 * -5.0)) < 1e-14  # equal likelihoods: log Z inc = dbeta * l
    one_hot = np.full(M, -np.inf)
    one_hot[5] = 0.0
    lw, W, sc = oracle.reweight(None, 0.0, one_hot)
    assert sc[1] == 1.0 and W[5] == 1.0 and W.sum() == 1.0
    with pytest.raises(oracle.OracleError):
        oracle.reweight(None, 0.0, np.full(4, -np.inf))
    with pytest.raises(oracle.OracleError):
        oracle.reweight(np.array([0.0, np.nan]), 1.0, np.zeros(2))


def test_reweight_shift_invariance():
    g = np.random.default_rng(1)
    lw0, ll = g.normal(0, 1, 100), g.normal(0, 1, 100)
    _, W1, s1 = oracle.reweight(ll, 1.0, lw0)
    _, W2, s2 = oracle.reweight(ll, 1.0, lw0 + 1234.5)
    np.testing.assert_allclose(W1, W2, rtol=1e-9)
    assert abs(s1[0] - s2[0]) < 1e-9 and abs(s1[1] - s2[1]) < 1e-9 * s1[1]


def test_ess_matches_reweight():
    lw = np.random.default_rng(2).normal(0, 2, 500)
    _, _, sc = oracle.reweight(None, 0.0, lw)
    assert abs(oracle.ess(lw) - sc[1]) <= 1e-12 * sc[1]


def test_importance_sampling_example_section_2_1():
    """Self-normalised IS estimate of E[x^2] under the paper's two-component
    target with an N(0,1) proposal; the exact value is
    sum_i w_i (var + mean_i^2)."""
    c = GOLD["importance_sampling_example_section_2_1"]
    exact = sum(w * (c["target_var"] + m**2) for w, m in zip(c["target_weights"], c["target_means"]))
    x = np.random.default_rng(3).standard_normal(400000)
    tgt = sum(w * stats.norm.pdf(x, m, np.sqrt(c["target_var"]))
              for w, m in zip(c["target_weights"], c["target_means"]))
    lw = np.log(tgt) - stats.norm.logpdf(x)
    _, W, _ = oracle.reweight(None, 0.0, lw)
    est = np.sum(W * x**2)
    assert abs(est - exact) < 0.02, (est, exact)


# ------------------------------------------------------------------ resampling
def _resample_fraction(W, u32):
    """Brute force in exact rationals: slot i gets the first j whose CDF
    C_j / S exceeds (i + u) / M, u = u32 / 2^32, q_j = floor(W_j 2^52)."""
    q = [int(Fraction(w) * 2**52) for w in W]  # floor of an exact non-negative rational
    S = sum(q)
    C = np.cumsum(q).tolist()
    M = len(W)
    u = Fraction(u32, 2**32)
    out = []
    for i in range(M):
        t = (i + u) / M
        out.append(next(j for j in range(M) if Fraction(C[j], S) > t))
    return np.array(out, np.int32)


def test_resample_brute_force_small():
    g = np.random.default_rng(4)
    for M in [1, 2, 3, 4, 6]:
        for _ in range(20):
            W = g.dirichlet(np.ones(M) * 0.5)
            for u32 in [0, 1, 2**31, 2**32 - 1, int(g.integers(0, 2**32))]:
                anc, counts = oracle.resample_systematic(W, u32)
                assert np.array_equal(anc, _resample_fraction(W, u32))
                assert np.array_equal(counts, np.bincount(anc, minlength=M))


def test_resample_step_function_of_u():
    """For small M each offspring count is a step function of u that takes
    only the values floor(M q/S) and ceil(M q/S)."""
    W = np.array([0.1, 0.45, 0.05, 0.4])
    grid = np.linspace(0, 2**32 - 1, 257).astype(np.int64)
    seen = []
    for u32 in grid:
        _, c = oracle.resample_systematic(W, int(u32))
        seen.append(c)
    seen = np.array(seen)
    q = np.floor(W * 2**52)
    S = q.sum()
    for j in range(4):
        lo, hi = np.floor(4 * q[j] / S), np.ceil(4 * q[j] / S)
        assert set(seen[:, j]).issubset({lo, hi})
        # monotone steps: counts change at most twice across u for this size
        assert np.count_nonzero(np.diff(seen[:, j])) <= 2


def test_resample_invariants_large():
    g = np.random.default_rng(5)
    M = 100000
    _, W, _ = oracle.reweight(None, 0.0, g.normal(0, 2, M))
    anc, counts = oracle.resample_systematic(W, 0x9E3779B9)
    assert counts.sum() == M
    assert np.all(np.diff(anc) >= 0)
    q = np.floor(W * 2**52)
    S = q.sum()
    assert np.all(counts >= np.floor(M * q / S)) and np.all(counts <= np.ceil(M * q / S))
    # agreement with a textbook float systematic resampler away from ties
    u = 0x9E3779B9 / 2**32
    cdf = np.cumsum(W)
    t = (np.arange(M) + u) / M
    ref = np.searchsorted(cdf, t, side="right")
    near = np.abs(cdf[np.minimum(ref, M - 1)] - t) < 1e-9
    assert np.array_equal(anc[~near], ref[~near])


def test_resample_degenerate_and_uniform():
    M = 1000
    W = np.zeros(M)
    W[123] = 1.0
    anc, counts = oracle.resample_systematic(W, 777)
    assert np.all(anc == 123) and counts[123] == M
    anc, counts = oracle.resample_systematic(np.full(M, 1.0 / M), 2**32 - 1)
    assert np.array_equal(anc, np.arange(M))
    with pytest.raises(oracle.OracleError):
        oracle.resample_systematic(np.zeros(5), 0)
    with pytest.raises(oracle.OracleError):
        oracle.resample_systematic(np.array([0.5, np.nan]), 0)
    with pytest.raises(oracle.OracleError):
        oracle.resample_systematic(np.array([0.5, 1.5]), 0)


# ------------------------------------------------------------------ multinomial / residual
def _q_cdf(W):
    q = [int(Fraction(w) * 2**52) for w in W]
    return q, np.cumsum(q).tolist(), sum(q)


def test_multinomial_brute_force_rationals():
    """Slot i takes the particle whose CDF interval (C_{j-1}/S, C_j/S]
    contains (u_i + 1/2) / 2^32, evaluated in exact rationals."""
    g = np.random.default_rng(11)
    for M in [1, 2, 3, 5, 9, 40]:
        for _ in range(10):
            W = g.dirichlet(np.ones(M) * 0.4)
            u = g.integers(0, 2**32, M, dtype=np.uint64).astype(np.uint32)
            u[0] = 0
            u[-1] = 2**32 - 1
            q, C, S = _q_cdf(W)
            want = [next(j for j in range(M) if Fraction(C[j], S) > Fraction(2 * int(ui) + 1, 2**33))
                    for ui in u]
            assert np.array_equal(oracle.resample_multinomial(W, u), want)


def test_multinomial_frequencies_match_weights():
    """Counts over many independent calls follow Multinomial(M, W)."""
    W = np.array([0.05, 0.3, 0.0, 0.15, 0.5])
    M = W.size
    counts = np.zeros(M)
    for step in range(4000):
        a = oracle.resample_multinomial(W, oracle.slot_uniforms(3, step, M))
        counts += np.bincount(a, minlength=M)
    assert counts[2] == 0  # zero weight is never drawn
    keep = W > 0
    chi2 = np.sum((counts[keep] - counts.sum() * W[keep]) ** 2 / (counts.sum() * W[keep]))
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4, (counts, chi2)


def test_residual_brute_force_rationals():
    """Deterministic shares floor(M q_j / S), then the R remaining slots drawn
    on the remainders shifted to 32 bits, all in exact rationals."""
    g = np.random.default_rng(12)
    for M in [1, 2, 3, 7, 16, 50]:
        for _ in range(8):
            W = g.dirichlet(np.ones(M) * 0.5)
            v = g.integers(0, 2**32, M, dtype=np.uint64).astype(np.uint32)
            q, C, S = _q_cdf(W)
            n = [(M * qj) // S for qj in q]
            r = [M * qj - nj * S for qj, nj in zip(q, n)]
            sh = max(0, S.bit_length() - 32)
            E = np.cumsum([rj >> sh for rj in r]).tolist()
            P = E[-1]
            det = [j for j in range(M) for _ in range(n[j])]
            R = M - len(det)
            res = [next(j for j in range(M) if Fraction(E[j], P) > Fraction(2 * int(v[k]) + 1, 2**33))
                   for k in range(R)]
            anc, Rg = oracle.resample_residual(W, v)
            assert Rg == R and np.array_equal(anc, det + res)
            # every particle keeps at least its integer share floor(M W_j) up to the 2^-52 grid
            cnt = np.bincount(anc, minlength=M)
            assert np.all(cnt >= np.floor(M * W - 1e-9)) and cnt.sum() == M


def test_residual_special_cases():
    M = 64
    # equal weights: every particle keeps exactly one copy, no residual draw
    anc, R = oracle.resample_residual(np.full(M, 1.0 / M), oracle.slot_uniforms(1, 1, M))
    assert R == 0 and np.array_equal(anc, np.arange(M))
    # one-hot: all M slots deterministic
    W = np.zeros(M)
    W[17] = 1.0
    anc, R = oracle.resample_residual(W, oracle.slot_uniforms(1, 2, M))
    assert R == 0 and np.all(anc == 17)
    # expected counts over calls: E[count_j] = M W_j
    W = np.random.default_rng(3).dirichlet(np.ones(M))
    tot = np.zeros(M)
    reps = 3000
    for step in range(reps):
        anc, R = oracle.resample_residual(W, oracle.slot_uniforms(4, step, M))
        tot += np.bincount(anc, minlength=M)
    assert np.max(np.abs(tot / reps - M * W)) < 0.1


def test_multinomial_residual_errors():
    for f in (oracle.resample_multinomial, oracle.resample_residual):
        with pytest.raises(oracle.OracleError):
            f(np.array([0.5, np.nan]), np.zeros(2, np.uint32))
        with pytest.raises(oracle.OracleError):
            f(np.zeros(3), np.zeros(3, np.uint32))
        with pytest.raises(oracle.OracleError):
            f(np.array([0.5, 1.5]), np.zeros(2, np.uint32))


def test_is_moments_section_2_1_example():
    """The worked example of Section 2.1: E[x^2] under the two-component
    target is 1.875 (closed form); both the plain estimate sum w phi / N and
    the self-normalised one converge to it, and sum w / N to 1 (the target is
    normalised).  Given draws and device-style draws give the same sums."""
    c = GOLD["importance_sampling_example_section_2_1"]
    exact = sum(w * (c["target_var"] + m**2) for w, m in zip(c["target_weights"], c["target_means"]))
    assert abs(exact - 1.875) < 1e-15
    N = 400000
    out = oracle.is_moments(c["target_means"], c["target_weights"], c["target_var"], 0.0, 1.0, 2,
                            N=N, seed=5, step=1)
    ess = out[0] ** 2 / out[2]
    se = 4.0 / np.sqrt(ess)
    assert abs(out[1] / N - exact) < se and abs(out[1] / out[0] - exact) < se
    assert abs(out[0] / N - 1.0) < 4.0 / np.sqrt(ess)
    # the same draws passed in explicitly
    z = np.array([oracle.normals(5, oracle.P_PROPOSAL, 1, i, 1)[0] for i in range(1000)])
    x = (0.0 + 1.0 * z).astype(np.float32)
    a = oracle.is_moments(c["target_means"], c["target_weights"], c["target_var"], 0.0, 1.0, 2, x=x)
    b = oracle.is_moments(c["target_means"], c["target_weights"], c["target_var"], 0.0, 1.0, 2,
                          N=1000, seed=5, step=1)
    np.testing.assert_allclose(a, b, rtol=1e-12)
    # weights against independent densities: w = p / q with scipy's normal pdf
    wr = (0.5 * stats.norm.pdf(x, -1.0, 0.5) + 0.5 * stats.norm.pdf(x, 1.5, 0.5)) / stats.norm.pdf(x)
    np.testing.assert_allclose(a, [wr.sum(), (wr * x.astype(np.float64) ** 2).sum(), (wr ** 2).sum()],
                               rtol=1e-10)
