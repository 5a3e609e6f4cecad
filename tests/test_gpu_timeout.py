"""The bounded device waits give up and report, without a GPU fault.

Every kernel that stages the data into shared memory by a bulk copy waits
on the copy's mbarrier with a bounded number of polls; when the bound runs
out the kernel latches SMC_ERR_TIMEOUT in the context, then waits again with
the full bound so that no copy is left in flight.  The context's test hook
sets the first bound to zero: every such wait gives up at once.  The calls
must report SMC_ERR_TIMEOUT through smc_ctx_check, their results must still
be correct (the second wait completed the copy), and the next calls with the
normal bound must report nothing.  No wait is made to hang and no fault is
raised: the data copies complete normally.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

SIG = 0.55


@pytest.fixture(scope="module")
def smc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0905_2441_gb300 as P
    from paper_0905_2441_gb300 import build
    build.build()
    ctx = P.Context()
    yield P, ctx
    ctx.set_wait_limit(4 << 20)
    ctx.close()


def _timeout_then_normal(P, ctx, call):
    """call() under a zero first-wait bound, then under the normal one;
    returns the two results."""
    ctx.check()
    ctx.set_wait_limit(0)
    try:
        r0 = call()
        with pytest.raises(P.SmcError) as ei:
            ctx.check()
        assert ei.value.status == -5  # SMC_ERR_TIMEOUT
    finally:
        ctx.set_wait_limit(4 << 20)
    r1 = call()
    ctx.check()  # nothing latched any more
    return r0, r1


@pytest.mark.parametrize("N", [1000, 20000])  # resident data / streamed in chunks
def test_loglik_wait_gives_up_and_reports_timeout(smc, N):
    P, ctx = smc
    K, M = 8, 4096
    y = synth.gmm1d_data(N, np.arange(-7, 8, 2), SIG, seed=1)
    th = synth.prior_particles(K, M, seed=2)
    yd, thd = torch.from_numpy(y).cuda(), torch.from_numpy(th).cuda()
    model = P.GMM(K, SIG)
    r0, r1 = _timeout_then_normal(P, ctx, lambda: P.loglik_batch(ctx, model, yd, thd).cpu().numpy())
    ref = oracle.gmm1d_loglik(y, np.full(K, -np.log(K)), SIG, th)
    np.testing.assert_allclose(r0, ref, rtol=1e-5)
    np.testing.assert_allclose(r1, ref, rtol=1e-5)


def test_population_sweep_wait_gives_up_and_reports_timeout(smc):
    P, ctx = smc
    w = synth.GMM8_POP
    off = synth.population_offsets(24, seed=w.pop_seed)
    y = w.data()
    th = synth.population_particles(w.K, off, seed=4)
    beta = synth.population_betas(off)
    ll = oracle.gmm1d_loglik(y, w.logw(), w.sigma, th)
    model = P.GMM(w.K, w.sigma)
    outs = []

    def call():
        tt, lt = torch.from_numpy(th).cuda(), torch.from_numpy(ll).cuda()
        P.popmcmc_sweep(ctx, model, torch.from_numpy(y).cuda(), tt, lt,
                        torch.from_numpy(beta).cuda(), torch.from_numpy(off).cuda(), w.scale, 3, 1)
        outs.append((tt.cpu().numpy(), lt.cpu().numpy()))
        return outs[-1]

    (t0, l0), (t1, l1) = _timeout_then_normal(P, ctx, call)
    # the same sweep from the same state: the timed-out call's result is the
    # normal one
    assert np.array_equal(t0, t1) and np.array_equal(l0, l1)
