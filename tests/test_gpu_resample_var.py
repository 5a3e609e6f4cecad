"""GPU parity of the multinomial and residual resampling schemes (exact
integers on the systematic scheme's quantised CDF): ancestors bit-exact
against the oracle for every size and weight shape, the identity flag, the
log-weight reset and the error path."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0905_2441_gb300 as P
    from paper_0905_2441_gb300 import build
    build.build()
    ctx = P.Context()
    yield P, ctx
    ctx.close()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def np_(t):
    return t.detach().cpu().numpy()


def _weights(M, kind, seed):
    g = np.random.default_rng(seed)
    if kind == "gauss":
        lw = g.normal(0, 2, M)
    elif kind == "peaked":
        lw = g.normal(0, 30, M)
    elif kind == "uniform":
        lw = np.zeros(M)
    elif kind == "onehot":
        lw = np.full(M, -np.inf)
        lw[g.integers(0, M)] = 0.0
    else:  # sparse: most weights exactly zero
        lw = np.where(g.random(M) < 0.01, g.normal(0, 1, M), -np.inf)
        lw[0] = 0.0
    return oracle.reweight(None, 0.0, lw)[1]


def _oracle(scheme, W, seed, step):
    u = oracle.slot_uniforms(seed, step, W.size)
    if scheme == "multinomial":
        return oracle.resample_multinomial(W, u)
    return oracle.resample_residual(W, u)[0]


def _gpu(P, ctx, scheme, Wd, seed, step, **kw):
    fn = P.resample_multinomial if scheme == "multinomial" else P.resample_residual
    return fn(ctx, Wd, seed, step, **kw)


@pytest.mark.parametrize("scheme", ["multinomial", "residual"])
@pytest.mark.parametrize("M", [1, 2, 3, 100, 2047, 2048, 2049, 65537, 1 << 20, 3 << 20])
@pytest.mark.parametrize("kind", ["gauss", "peaked", "uniform", "onehot", "sparse"])
def test_bit_exact(smc, scheme, M, kind):
    P, ctx = smc
    if M > 70000 and kind in ("uniform", "sparse"):
        pytest.skip("covered at smaller sizes")
    W = _weights(M, kind, M + 7 * len(kind))
    seed, step = 777 + M, 23
    lwr = torch.full((M,), 5.0, dtype=torch.float64, device="cuda")
    anc = _gpu(P, ctx, scheme, cu(W), seed, step, logw_reset=lwr)
    ctx.check()
    ref = _oracle(scheme, W, seed, step)
    got = np_(anc)
    assert np.array_equal(got, ref), (np.flatnonzero(got != ref)[:10], got[:10], ref[:10])
    assert np.all(np_(lwr) == 0.0)


@pytest.mark.parametrize("scheme", ["multinomial", "residual"])
def test_identity_flag_and_repeated_calls(smc, scheme):
    P, ctx = smc
    M = 50000
    W = _weights(M, "gauss", 1)
    Wd = cu(W)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    lwr = torch.full((M,), 3.0, dtype=torch.float64, device="cuda")
    for step in range(4):
        flag.fill_(step % 2)
        anc = _gpu(P, ctx, scheme, Wd, 9, step, do_flag=flag, logw_reset=lwr)
        ctx.check()
        if step % 2:
            assert np.array_equal(np_(anc), _oracle(scheme, W, 9, step))
            assert np.all(np_(lwr) == 0.0)
        else:
            assert np.array_equal(np_(anc), np.arange(M))
            if step == 0:
                assert np.all(np_(lwr) == 3.0)  # untouched without resampling


@pytest.mark.parametrize("scheme", ["multinomial", "residual"])
def test_bad_weights(smc, scheme):
    P, ctx = smc
    _gpu(P, ctx, scheme, cu(np.array([0.5, np.nan, 0.5])), 1, 1)
    with pytest.raises(P.SmcError):
        ctx.check()
    _gpu(P, ctx, scheme, cu(np.zeros(100)), 1, 1)
    with pytest.raises(P.SmcError) as e:
        ctx.check()
    assert e.value.status == -4
    W = _weights(3000, "gauss", 3)
    anc = _gpu(P, ctx, scheme, cu(W), 2, 2)
    ctx.check()
    assert np.array_equal(np_(anc), _oracle(scheme, W, 2, 2))


def test_residual_keeps_integer_shares(smc):
    """Each particle keeps at least floor(M W_j) copies, in particle order at
    the front; the offspring counts add up to M."""
    P, ctx = smc
    M = 1 << 16
    W = _weights(M, "gauss", 5)
    anc = np_(P.resample_residual(ctx, cu(W), 3, 4))
    ctx.check()
    cnt = np.bincount(anc, minlength=M)
    share = np.floor(M * W - 1e-9).astype(np.int64)
    assert cnt.sum() == M and np.all(cnt >= share)
    nd = int(share.sum())
    assert np.all(np.diff(anc[:nd]) >= 0)
