"""Pins for the oracle's Philox4x32-10 and its uniform / normal transforms.

The oracle's Philox is checked bit for bit against an independent
implementation (Triton's, executed by its CPU interpreter); the transforms
against their distributions.  Section 2.5 of the paper (parallel streams with
skip-ahead) is realised here by a counter-based generator."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _triton_philox(seeds, ctrs):
    pytest.importorskip("triton")
    req = json.dumps({"seeds": [int(s) for s in seeds], "ctr": [[int(v) for v in c] for c in ctrs]})
    out = subprocess.run([sys.executable, os.path.join(HERE, "_triton_philox.py")], input=req,
                         capture_output=True, text=True, timeout=600)
    if out.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + out.stderr[-300:])
    return json.loads(out.stdout)


def test_philox_matches_independent_implementation():
    g = np.random.default_rng(0)
    ctrs = g.integers(0, 2**32, size=(64, 4), dtype=np.uint64)
    ctrs[0] = 0
    ctrs[1] = 0xFFFFFFFF
    seeds = [0, 1, 0xFFFFFFFFFFFFFFFF, 0x243F6A8885A308D3, 1234]
    ref = _triton_philox(seeds, ctrs)
    for s in seeds:
        key = np.array([s & 0xFFFFFFFF, (s >> 32) & 0xFFFFFFFF], np.uint32)
        for c, want in zip(ctrs, ref[str(s)]):
            got = oracle.philox4x32_10(c.astype(np.uint32), key)
            assert got.tolist() == want, (s, c)


def test_counter_layout():
    """draw_words puts (index, block, step lo, purpose | step hi << 8) in the counter."""
    seed, purpose, step, index, block = 0x1122334455667788, 3, (5 << 32) | 77, 9, 2
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    ctr = np.array([index, block, 77, purpose | (5 << 8)], np.uint32)
    assert oracle.draw_words(seed, purpose, step, index, block).tolist() == \
        oracle.philox4x32_10(ctr, key).tolist()


def test_u01_endpoints_and_exactness():
    assert oracle.u01(0) == 2.0**-24
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0**-24
    # every value is an odd multiple of 2^-24, representable in float32
    for x in [1, 511, 512, 12345678, 0x80000000, 0xDEADBEEF]:
        u = oracle.u01(x)
        assert float(np.float32(u)) == u
        assert (u * 2**24) % 2 == 1


def test_uniform_and_normal_distributions():
    w = np.concatenate([oracle.draw_words(7, 1, 0, i, 0) for i in range(5000)])
    u = np.array([oracle.u01(int(x)) for x in w])
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    z = np.concatenate([oracle.normals(7, 1, 3, i, 5) for i in range(4000)])
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 4 * np.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # odd n: the last pair contributes only its cosine normal
    z5 = oracle.normals(7, 1, 3, 11, 5)
    z6 = oracle.normals(7, 1, 3, 11, 6)
    assert np.array_equal(z5, z6[:5])
    # pairs are uncorrelated
    zz = np.array([oracle.normals(9, 1, 0, i, 2) for i in range(20000)])
    assert abs(np.corrcoef(zz.T)[0, 1]) < 4 / np.sqrt(20000)


# ------------------------------------------------------------------ MRG32k3a (Section 2.5)
SEED6 = [12345] * 6


def test_mrg32k3a_skip_ahead_equals_stepping():
    """Section 2.5: a thread jumps to its block by skip-ahead in O(log n)
    products; the numbers it then draws are those sequential stepping
    reaches (repeated squaring against one-step iteration)."""
    seq = oracle.mrg32k3a(SEED6, 0, 20000)
    for start in [1, 2, 3, 7, 64, 1000, 12345, 19990]:
        n = min(10, 20000 - start)
        assert np.array_equal(oracle.mrg32k3a(SEED6, start, n), seq[start:start + n]), start
    other = [1, 2, 3, 4, 5, 6]
    seq2 = oracle.mrg32k3a(other, 0, 3000)
    assert np.array_equal(oracle.mrg32k3a(other, 2500, 500), seq2[2500:])


def test_mrg32k3a_far_jumps_are_consistent():
    """Jumps far beyond anything steppable: the block at 2^70 + 5 is the block
    at 2^70 moved by five places, and substreams 2^76 apart differ."""
    a = oracle.mrg32k3a(SEED6, 2**70, 20)
    b = oracle.mrg32k3a(SEED6, 2**70 + 5, 15)
    assert np.array_equal(a[5:], b)
    s76 = oracle.mrg32k3a(SEED6, 2**63, 8)
    assert not np.array_equal(s76, oracle.mrg32k3a(SEED6, 0, 8))


def test_mrg32k3a_float_output_is_the_double_cut_to_24_bits():
    u64 = oracle.mrg32k3a(SEED6, 0, 50000, np.float64)
    u32 = oracle.mrg32k3a(SEED6, 0, 50000).astype(np.float64)
    assert np.all((u32 > 0) & (u32 < 1)) and np.all((u64 > 0) & (u64 < 1))
    # the FP32 form is the centre of z's 2^-23 bin read as a fraction of 2^32
    # (within 2^-24 of z / 2^32); the FP64 form divides by m1 + 1 = 2^32 - 208
    # (within 209 * 2^-32 of z / 2^32)
    assert np.max(np.abs(u32 - u64)) <= 2.0**-24 + 209 * 2.0**-32
    assert np.array_equal(oracle.mrg32k3a(SEED6, 9000, 100, np.float64), u64[9000:9100])


def test_mrg32k3a_uniform_and_uncorrelated():
    u = oracle.mrg32k3a(SEED6, 777, 200000).astype(np.float64)
    assert np.all((u > 0) & (u < 1))
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 0.01
    # pairs fall evenly into a 16 x 16 grid
    h, _, _ = np.histogram2d(u[:-1:2], u[1::2], bins=16, range=[[0, 1], [0, 1]])
    chi2 = np.sum((h - h.mean()) ** 2 / h.mean())
    assert stats.chi2.sf(chi2, 255) > 1e-4
