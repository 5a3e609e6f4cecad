"""Pins of the factor stochastic volatility oracle (Section 4.2): the
observation density against SciPy's multivariate normal and two closed
forms, the state transition by its moments, the paper's constants, and the
whole filter by its agreement across seeds and with the simulated truth."""
import json
import os

import numpy as np
import pytest
from scipy import stats

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def test_constants_are_the_papers():
    g = json.load(open(GOLD))["fsv_section_4_2"]
    phi, U, B, psi = synth.fsv_params()
    assert np.array_equal(B, np.array(g["B"])) and np.array_equal(U, np.array(g["U"]))
    assert np.all(phi == g["phi"]) and np.all(psi == g["psi"])
    assert B.shape == (g["M"], g["K"]) and np.all(np.triu(B, 1) == 0.0)


def test_logg_matches_scipy_multivariate_normal():
    phi, U, B, psi = synth.fsv_params()
    g = np.random.default_rng(3)
    M = 50
    x_in = g.normal(0, 1.5, (3, M)).astype(np.float32)
    yt = g.normal(0, 2.0, 5).astype(np.float32)
    x_out, lg = oracle.fsv_step(phi, synth.chol(U), B, psi, yt, x_in, None, 11, 3)
    for i in range(M):
        S = B @ np.diag(np.exp(x_out[:, i].astype(np.float64))) @ B.T + np.diag(psi)
        ref = stats.multivariate_normal(np.zeros(5), S).logpdf(yt.astype(np.float64))
        assert lg[i] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_zero_loadings_give_independent_noise():
    phi, U, _, psi = synth.fsv_params()
    B = np.zeros((5, 3))
    yt = np.array([0.3, -1.2, 2.0, 0.0, 0.7], np.float32)
    x_in = np.random.default_rng(1).normal(0, 1, (3, 7)).astype(np.float32)
    _, lg = oracle.fsv_step(phi, synth.chol(U), B, psi, yt, x_in, None, 2, 1)
    y = yt.astype(np.float64)
    ref = np.sum(-0.5 * np.log(2 * np.pi * psi) - y * y / (2 * psi))
    assert np.allclose(lg, ref, rtol=1e-13, atol=0)


def test_one_factor_one_series_closed_form():
    b, psi = 0.8, 0.3
    x_in = np.random.default_rng(2).normal(0, 1, (1, 9)).astype(np.float32)
    yt = np.array([1.1], np.float32)
    x_out, lg = oracle.fsv_step([0.9], [[0.7]], [[b]], [psi], yt, x_in, None, 4, 2)
    var = b * b * np.exp(x_out[0].astype(np.float64)) + psi
    yv = float(yt[0])  # the stored (FP32) observation
    ref = -0.5 * np.log(2 * np.pi * var) - yv ** 2 / (2 * var)
    assert np.allclose(lg, ref, rtol=1e-12)


def test_transition_moments():
    phi, U, B, psi = synth.fsv_params()
    M = 200_000
    c = np.array([1.0, -2.0, 0.5])
    x_in = np.repeat(c[:, None], M, 1).astype(np.float32)
    x_out, _ = oracle.fsv_step(phi, synth.chol(U), B, psi, np.zeros(5, np.float32), x_in, None,
                               5, 1)
    d = x_out.astype(np.float64) - (phi * c)[:, None]
    se = np.sqrt(np.diag(U) / M)
    assert np.all(np.abs(d.mean(1)) < 5 * se)
    assert np.allclose(np.cov(d), U, atol=0.01)


def test_ancestors_select_the_parents():
    phi, U, B, psi = synth.fsv_params()
    x_in = np.arange(12, dtype=np.float32).reshape(3, 4)
    anc = np.array([3, 3, 0, 2], np.int32)
    xa, la = oracle.fsv_step(phi, np.zeros((3, 3)), B, psi, np.ones(5, np.float32), x_in, anc,
                             1, 1)
    assert np.allclose(xa, (phi[:, None] * x_in[:, anc]).astype(np.float32))


def test_filter_tracks_the_truth_and_seeds_agree():
    phi, U, B, psi = synth.fsv_params()
    x, y = synth.simulate_fsv(60, phi, U, B, psi, seed=7)
    L = synth.chol(U)
    z1, m1 = oracle.fsv_run(phi, L, B, psi, y, 4000, 1, want_means=True)
    z2 = oracle.fsv_run(phi, L, B, psi, y, 4000, 2)
    assert np.isfinite(z1) and abs(z1 - z2) < 1.0   # Monte Carlo error of log Z at M = 4000
    # the filtered means follow the simulated states (the factor volatilities
    # are weakly identified from 5 series: correlations near 0.4-0.5 here)
    r = [np.corrcoef(m1[:, k], x[:, k])[0, 1] for k in range(3)]
    assert min(r) > 0.25 and np.mean(r) > 0.35
