"""GPU parity of the MRG32k3a stream (Section 2.5: every thread computes a
contiguous block of one stream, reached by skip-ahead): bit-exact against
the oracle for small and far offsets, ragged thread counts and blocks, and
the position arithmetic wrapping at 2^64."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
SEED6 = [12345] * 6


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


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("offset,n_threads,per_thread", [
    (0, 1, 1000), (0, 1000, 7), (3, 257, 33), (2**40 + 3, 333, 17), (2**63 + 11, 64, 5),
    (2**64 - 40, 9, 8),     # positions wrap past 2^64
])
def test_blocks_bit_exact(smc, offset, n_threads, per_thread, dtype):
    P, ctx = smc
    out = P.rng_mrg32k3a(ctx, SEED6, offset, n_threads, per_thread, dtype=dtype).cpu().numpy()
    ctx.check()
    npd = np.float32 if dtype == torch.float32 else np.float64
    for t in sorted({0, min(1, n_threads - 1), n_threads // 2, n_threads - 1}):
        start = (offset + t * per_thread) % 2**64
        assert np.array_equal(out[:, t], oracle.mrg32k3a(SEED6, start, per_thread, npd)), t


def test_blocks_tile_one_stream(smc):
    """Consecutive threads' blocks laid end to end are the stream itself."""
    P, ctx = smc
    out = P.rng_mrg32k3a(ctx, [1, 2, 3, 4, 5, 6], 100, 50, 40).cpu().numpy()
    ctx.check()
    assert np.array_equal(out.T.reshape(-1), oracle.mrg32k3a([1, 2, 3, 4, 5, 6], 100, 2000))


def test_bad_seeds(smc):
    P, ctx = smc
    for bad in ([0, 0, 0, 1, 1, 1], [1, 1, 1, 0, 0, 0], [4294967087, 1, 1, 1, 1, 1]):
        with pytest.raises(P.SmcError):
            P.rng_mrg32k3a(ctx, bad, 0, 4, 4)
