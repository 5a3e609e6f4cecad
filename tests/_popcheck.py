"""Test helper: is a population-MCMC sweep that differs from the oracle's
sweep explained by FP32 rounding alone?

A GPU sweep and the oracle's sweep from the same state with the same Philox
draws take the same decisions, except where the FP32 likelihood's rounding
can turn one (Section 4.3 notes the same for the paper's own CPU / GPU
comparison): an MH decision whose log alpha - log u lies inside the FP32
band, or an exchange decision whose log alpha - log u does (it is formed from
log-likelihoods that carry the FP32 error).  `explain_sweep` compares the
two sweeps population by population and, for every population that
differs, searches the sets of in-band decisions of that population taken
the other way: the population is explained only if the oracle's sweep with
one such set of decisions reproduces the GPU's chains exactly (states
within 2 ulp, log-likelihoods within the FP32 tolerance).  Anything else
(a wrong pair, a wrong temperature, a lost move) stays unexplained.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

import oracle


@dataclass
class SweepReport:
    differing: list = field(default_factory=list)     # populations that differ
    explained: dict = field(default_factory=dict)     # population -> decisions flipped
    unexplained: list = field(default_factory=list)
    mh_in_band: int = 0                               # MH decisions inside the band (all chains)


def _same(th_a, l_a, th_b, l_b):
    return (np.allclose(th_a, th_b, rtol=3e-7, atol=2e-6) and
            np.allclose(l_a, l_b, rtol=1e-5, atol=0))


def explain_sweep(y, logw, sigma, box, theta0, ll0, beta, offsets, scale, seed, sweep,
                  theta_g, ll_g, band=5e-3, max_combos=4096, pops=None):
    """Compare a sweep's result (theta_g, ll_g) with the oracle's sweep from
    (theta0, ll0); return a SweepReport.  `pops` restricts the comparison to
    those populations (all by default)."""
    offsets = np.asarray(offsets, np.int64)
    K, M = theta0.shape
    beta = np.asarray(beta, np.float32)
    # stage 1: the oracle's MH move, its log alpha, and each chain's other outcome
    th1, l1, acc, la = oracle.rwmh_move(y, logw, sigma, box, theta0, ll0, beta, scale, seed, sweep,
                                        want_log_alpha=True)
    lu = np.log([oracle.u01(int(oracle.draw_words(seed, oracle.P_ACCEPT, sweep, c, 0)[0]))
                 for c in range(M)])
    d1 = la - lu
    # a start log-likelihood of -inf makes every in-box proposal accepted
    thp, lp, accp = oracle.rwmh_move(y, logw, sigma, box, theta0, np.full(M, -np.inf), beta,
                                     scale, seed, sweep)
    rep = SweepReport(mh_in_band=int(np.sum(np.isfinite(d1) & (np.abs(d1) < band))))
    th2, l2, _ = oracle.popmcmc_exchange(th1, l1, beta, offsets, seed, sweep)
    qs = range(offsets.size - 1) if pops is None else pops
    for q in qs:
        a, b = int(offsets[q]), int(offsets[q + 1])
        if _same(theta_g[:, a:b], ll_g[a:b], th2[:, a:b], l2[a:b]):
            continue
        rep.differing.append(q)
        mh = [c for c in range(a, b) if np.isfinite(d1[c]) and abs(d1[c]) < band]
        found = None
        tried = 0
        for r in range(len(mh) + 1):
            for sub in itertools.combinations(mh, r):
                t1, ll1 = th1.copy(), l1.copy()
                for c in sub:  # the other outcome of chain c's MH decision
                    if acc[c]:
                        t1[:, c], ll1[c] = theta0[:, c], ll0[c]
                    else:
                        t1[:, c], ll1[c] = thp[:, c], lp[c]
                t2, ll2, _, lax = oracle.popmcmc_exchange(t1, ll1, beta, offsets, seed, sweep,
                                                          q0=q, q1=q + 1, want_la=True)
                ex = [p for p in range(lax.size) if abs(lax[p]) < band]
                for r2 in range(len(ex) + 1):
                    for sub2 in itertools.combinations(ex, r2):
                        tried += 1
                        if tried > max_combos:
                            break
                        if sub2:
                            flip = np.zeros(lax.size, np.int8)
                            flip[list(sub2)] = 1
                            t2, ll2, _ = oracle.popmcmc_exchange(t1, ll1, beta, offsets, seed,
                                                                 sweep, q0=q, q1=q + 1, flip=flip)
                        if _same(theta_g[:, a:b], ll_g[a:b], t2[:, a:b], ll2[a:b]):
                            found = {"mh": list(sub), "exchange_pairs": list(sub2)}
                            break
                    if found:
                        break
                if found:
                    break
            if found:
                break
        if found is None:
            rep.unexplained.append(q)
        else:
            rep.explained[q] = found
    return rep
