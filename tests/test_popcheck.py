"""CPU tests of the population-sweep validity check (tests/_popcheck.py):
it must accept the oracle's own sweep, accept a sweep that differs from it
only by an in-band decision taken the other way, and reject a sweep made by
a copy of the oracle with a planted mistake (a wrong exchange pair index)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth
from _popcheck import explain_sweep

SIG = 0.55
BOX = (-10.0, 10.0)
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def case():
    K, N = 4, 100
    y = synth.gmm1d_data(N, [-3, 0, 3, 6], SIG, seed=1)
    logw = np.full(K, -np.log(K))
    off = synth.population_offsets(40, lo=8, hi=40, seed=5)
    beta = synth.population_betas(off)
    th = synth.population_particles(K, off, seed=6)
    ll = oracle.gmm1d_loglik(y, logw, SIG, th)
    return dict(y=y, logw=logw, off=off, beta=beta, th=th, ll=ll, scale=0.3, seed=17, sweep=3)


def _check(c, th_g, ll_g, band=5e-3):
    return explain_sweep(c["y"], c["logw"], SIG, BOX, c["th"], c["ll"], c["beta"], c["off"],
                         c["scale"], c["seed"], c["sweep"], th_g, ll_g, band=band)


def test_the_oracle_s_own_sweep_passes(case):
    c = case
    rt, rl, _ = oracle.popmcmc_sweep(c["y"], c["logw"], SIG, BOX, c["th"], c["ll"], c["beta"],
                                     c["off"], c["scale"], c["seed"], c["sweep"])
    r = _check(c, rt, rl)
    assert r.differing == [] and r.unexplained == []


def test_an_in_band_decision_taken_the_other_way_is_explained(case):
    c = case
    M = c["th"].shape[1]
    _, _, acc, la = oracle.rwmh_move(c["y"], c["logw"], SIG, BOX, c["th"], c["ll"], c["beta"],
                                     c["scale"], c["seed"], c["sweep"], want_log_alpha=True)
    lu = np.log([oracle.u01(int(oracle.draw_words(c["seed"], oracle.P_ACCEPT, c["sweep"], i, 0)[0]))
                 for i in range(M)])
    d = np.where(np.isfinite(la), np.abs(la - lu), np.inf)
    k = int(np.argmin(d))  # the decision nearest its threshold
    # the sweep with that one decision flipped: force it through the start
    # log-likelihood (-inf accepts; +inf rejects), then the exchange stage
    ll_f = c["ll"].copy()
    ll_f[k] = np.inf if acc[k] else -np.inf
    t1, l1, _ = oracle.rwmh_move(c["y"], c["logw"], SIG, BOX, c["th"], ll_f, c["beta"], c["scale"],
                                 c["seed"], c["sweep"])
    if acc[k]:
        l1[k] = c["ll"][k]  # rejected: the chain keeps its true log-likelihood
    tg, lg, _ = oracle.popmcmc_exchange(t1, l1, c["beta"], c["off"], c["seed"], c["sweep"])
    r = _check(c, tg, lg, band=1.01 * d[k] + 1e-12)
    assert len(r.differing) == 1 and r.unexplained == []
    assert list(r.explained.values())[0]["mh"] == [k]


def test_a_planted_wrong_exchange_pair_is_rejected(case, tmp_path):
    """A copy of oracle.c whose wrap-around exchange pair is (M_q - 1, 1)
    instead of (M_q - 1, 0), compiled on its own: its sweep must leave
    populations the check cannot explain."""
    src = open(os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")).read()
    good = "else { ia = Mq - 1; ib = 0; }"
    assert src.count(good) == 1
    planted = tmp_path / "oracle_planted.c"
    planted.write_text(src.replace(good, "else { ia = Mq - 1; ib = 1; }"))
    so = str(tmp_path / "liboracle_planted.so")
    subprocess.check_call([shutil.which("gcc") or "gcc", "-O2", "-fno-fast-math",
                           "-ffp-contract=off", "-std=gnu11", "-fPIC", "-shared", str(planted),
                           "-o", so, "-lm"])
    L = C.CDLL(so)
    oracle._declare(L)
    c = case
    th = np.ascontiguousarray(c["th"], np.float32).copy()
    ll = np.ascontiguousarray(c["ll"], np.float64).copy()
    off = np.ascontiguousarray(c["off"], np.int32)
    K, M = th.shape
    stats = np.zeros(3, np.int64)
    L.orc_popmcmc_sweep(np.ascontiguousarray(c["y"], np.float32), c["y"].size, K,
                        np.ascontiguousarray(c["logw"], np.float64), SIG, BOX[0], BOX[1], th, ll, M,
                        np.ascontiguousarray(c["beta"], np.float32), off, off.size - 1,
                        c["scale"], c["seed"], c["sweep"], stats)
    r = _check(c, th, ll)
    assert r.unexplained, "the planted pair index went unnoticed"
