"""The allocation-free resampling entry point against the regular one.

smc_resample_systematic_noalloc serves callers that may not allocate device
memory (a pool or budget they must not bypass, or loops that cannot pay the
synchronisation of cudaMalloc/cudaFree); it keeps its scan scratch in a
static device array instead of a context.  Both entry points are called
through the C ABI on the same inputs, twice in a row, and must agree bit for
bit (ancestors and offspring counts are integers).  This file is collected
last on purpose and builds / loads everything it needs itself.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0905_2441_gb300 import _lib, build
    build.build()
    L = _lib.load()
    ctx = C.c_void_p()
    assert L.smc_create(C.byref(ctx), torch.cuda.current_device()) == 0
    yield L, ctx
    L.smc_destroy(ctx)


def _weights(M, seed, spread):
    lw = np.random.default_rng(seed).normal(0.0, spread, M)
    w = np.exp(lw - lw.max())
    return w / w.sum()


def _p(t):
    return C.c_void_p(t.data_ptr())


def _both(L, ctx, W, seed, step, flag=None):
    M = W.numel()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = {}
    for name in ("ctx", "noalloc"):
        anc = torch.full((M,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.full((M,), -1, dtype=torch.int32, device="cuda")
        lwr = torch.full((M,), 7.0, dtype=torch.float64, device="cuda")
        fl = None if flag is None else _p(flag)
        if name == "ctx":
            st = L.smc_resample_systematic(ctx, _p(W), M, seed, step, _p(anc), _p(cnt), fl, _p(lwr),
                                           stream)
            assert st == 0
            assert L.smc_ctx_check(ctx, stream) == 0
            status = 0
        else:
            sw = torch.zeros(1, dtype=torch.int32, device="cuda")
            st = L.smc_resample_systematic_noalloc(_p(W), M, seed, step, _p(anc), _p(cnt), fl,
                                                   _p(lwr), _p(sw), stream)
            assert st == 0
            torch.cuda.synchronize()
            status = int(sw.item())
        out[name] = (anc.cpu().numpy(), cnt.cpu().numpy(), lwr.cpu().numpy(), status)
    return out


def test_noalloc_matches_context_entry_point_twice(lib):
    L, ctx = lib
    # two calls in a row on different inputs (the second reuses the scratch)
    for M, seed, step, spread in [(1_000_003, 11, 1, 2.0), (70_001, 12, 2, 25.0)]:
        W = torch.from_numpy(_weights(M, seed, spread)).cuda()
        r = _both(L, ctx, W, seed, step)
        a0, c0, l0, _ = r["ctx"]
        a1, c1, l1, s1 = r["noalloc"]
        assert s1 == 0
        assert np.array_equal(a0, a1)
        assert np.array_equal(c0, c1)
        assert np.array_equal(l0, l1) and np.all(l1 == 0.0)
        assert c1.sum() == M and np.all(np.diff(a1) >= 0)


def test_noalloc_identity_flag_and_limits(lib):
    L, ctx = lib
    M = 5000
    W = torch.from_numpy(_weights(M, 3, 1.0)).cuda()
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    r = _both(L, ctx, W, 5, 9, flag=flag)
    assert np.array_equal(r["noalloc"][0], np.arange(M)) and np.array_equal(r["ctx"][0], r["noalloc"][0])
    # sizes beyond the static scratch are refused on the host, before any launch
    big = (1 << 24) + 1
    st = L.smc_resample_systematic_noalloc(_p(W), big, 1, 1, _p(W), None, None, None, None, None)
    assert st == -1
    # an all-zero weight vector is reported through the caller's status word
    Z = torch.zeros(M, dtype=torch.float64, device="cuda")
    anc = torch.empty(M, dtype=torch.int32, device="cuda")
    sw = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert L.smc_resample_systematic_noalloc(_p(Z), M, 1, 1, _p(anc), None, None, None, _p(sw),
                                             None) == 0
    torch.cuda.synchronize()
    assert int(sw.item()) & 2
    # and the next call is correct again
    r = _both(L, ctx, W, 6, 10)
    assert np.array_equal(r["ctx"][0], r["noalloc"][0]) and r["noalloc"][3] == 0


def test_noalloc_at_the_size_limit_matches_the_context_entry_point(lib):
    """The largest sizes the static array serves (2^24 weights: every tile
    sum of the array in use, the constants right after them) and one below."""
    L, ctx = lib
    for M, seed in [(1 << 24, 21), ((1 << 24) - 1, 22)]:
        W = torch.from_numpy(_weights(M, seed, 1.0)).cuda()
        r = _both(L, ctx, W, seed, 3)
        assert r["noalloc"][3] == 0
        assert np.array_equal(r["ctx"][0], r["noalloc"][0])
        assert np.array_equal(r["ctx"][1], r["noalloc"][1])


def test_noalloc_one_hot_and_peaked_weights_near_the_limit_match_the_oracle(lib):
    """Without heavy-chunk scratch a tile whose output range is long is
    expanded by its own CTA: one-hot weights (one particle takes every slot)
    and a few heavy particles among light ones, at M = 2^24 - 3, against
    the oracle's exact-integer resampling (ancestors bit-exact)."""
    import oracle
    L, _ = lib
    M = (1 << 24) - 3
    onehot = np.zeros(M)
    onehot[M // 3] = 1.0
    peaked = np.full(M, 1e-12)
    peaked[[7, M // 2, M - 2]] = [0.5, 0.3, 0.2]
    peaked /= peaked.sum()
    for name, Wh in (("one-hot", onehot), ("peaked", peaked)):
        W = torch.from_numpy(Wh).cuda()
        anc = torch.full((M,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.full((M,), -1, dtype=torch.int32, device="cuda")
        sw = torch.zeros(1, dtype=torch.int32, device="cuda")
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        assert L.smc_resample_systematic_noalloc(_p(W), M, 31, 4, _p(anc), _p(cnt), None, None,
                                                 _p(sw), None) == 0
        t1.record()
        torch.cuda.synchronize()
        assert int(sw.item()) == 0, name
        ranc, rcnt = oracle.resample_systematic(Wh, oracle.resample_u32(31, 4))
        assert np.array_equal(anc.cpu().numpy(), ranc), name
        assert np.array_equal(cnt.cpu().numpy(), rcnt), name
        print(f"{name}: {t0.elapsed_time(t1):.3f} ms per call (first call of this input)")
