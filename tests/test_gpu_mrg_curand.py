"""An independent pin of the oracle's MRG32k3a (Section 2.5's generator):
NVIDIA cuRAND's device generator, run from the same six-word state, must
produce the same stream.  cuRAND is a separate implementation of
L'Ecuyer's recurrence, so a wrong multiplier, modulus or lag in the
oracle's recurrence (which the skip-ahead and statistical pins cannot see,
since both sides of those share the oracle's constants) breaks the match.

The comparison is on the integer z in [1, m1] behind each uniform: the
oracle's double is z / (m1 + 1); cuRAND's is scaled back by m1 + 1 and by
m1 (the two normalisations in use) and one of the two must give the
oracle's z exactly for every output.  The state-word order of cuRAND's
struct is not documented, so both orders are tried for a state with
distinct words; the all-12345 state needs none."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
M1 = 4294967087


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("curand") / "libcurandmrg.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                    "-Xcompiler", "-fPIC", os.path.join(HERE, "_curand_mrg.cu"), "-o", out],
                   check=True, capture_output=True)
    L = C.CDLL(out)
    L.curand_mrg_run.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    return L


def _curand_u(L, seed6, rev, n):
    s = np.ascontiguousarray(seed6, np.uint32)
    u = np.zeros(n, np.float64)
    assert L.curand_mrg_run(s.ctypes.data, rev, n, u.ctypes.data) == 0
    return u


def _oracle_z(seed6, n):
    u = oracle.mrg32k3a(seed6, 0, n, np.float64)
    return np.rint(u * (M1 + 1.0)).astype(np.int64), u


def _same_stream(uc, zo):
    """cuRAND's uniforms carry the integers zo under one of the two
    normalisations, for every output."""
    return any(np.array_equal(np.rint(uc * scale).astype(np.int64), zo)
               for scale in (M1 + 1.0, float(M1)))


def test_oracle_mrg32k3a_equals_curand_from_the_all_12345_state(curand_lib):
    n = 100_000
    uc = _curand_u(curand_lib, [12345] * 6, 0, n)
    zo, uo = _oracle_z([12345] * 6, n)
    assert np.all((zo >= 1) & (zo <= M1))
    assert _same_stream(uc, zo)
    np.testing.assert_allclose(uc, uo, rtol=3e-10, atol=0)  # the same uniforms, to normalisation


def test_oracle_mrg32k3a_equals_curand_from_a_state_with_distinct_words(curand_lib):
    seed = [123456789, 2345678901, 345678901, 3456789012, 45678901, 567890123]
    n = 50_000
    zo, _ = _oracle_z(seed, n)
    matches = [rev for rev in (0, 1) if _same_stream(_curand_u(curand_lib, seed, rev, n), zo)]
    assert len(matches) == 1, matches


def test_a_planted_multiplier_error_is_caught(curand_lib):
    """The pin's power: the recurrence with one multiplier off by one
    (a copy of the oracle's recurrence in Python, on the same state) no
    longer matches cuRAND, while the oracle itself does."""
    n = 8
    uc = _curand_u(curand_lib, [12345] * 6, 0, n)
    zo, _ = _oracle_z([12345] * 6, n)
    assert _same_stream(uc, zo)
    x, yv, bad = [12345] * 3, [12345] * 3, []
    for _ in range(n):
        p1 = (1403580 * x[1] - 810728 * x[0]) % M1
        x = [x[1], x[2], p1]
        p2 = (527613 * yv[2] - 1370589 * yv[0]) % 4294944443  # 527612 planted as 527613
        yv = [yv[1], yv[2], p2]
        z = (p1 - p2) % M1
        bad.append(z if z > 0 else M1)
    assert not _same_stream(uc, np.array(bad, np.int64))
