"""The seeded synthetic inputs (no GPU): the workload recipes the benchmark
and the parity tests quote (sizes, schedules, seeds) and their determinism.
The generators draw numbers only; none of the method's arithmetic is here."""
import numpy as np

import synth


def test_population_workload_recipe():
    w = synth.GMM8_POP
    off = synth.population_offsets(w.n_pops, seed=w.pop_seed)
    sizes = np.diff(off)
    assert off[0] == 0 and off.size == 513 and off[-1] == 34591
    assert sizes.min() >= 8 and sizes.max() <= 128
    assert np.array_equal(off, synth.population_offsets(w.n_pops, seed=w.pop_seed))
    beta = synth.population_betas(off)
    for q in (0, 100, 511):  # per population: geometric from 1e-3 up to 1
        b = beta[off[q]:off[q + 1]].astype(np.float64)
        assert np.all(np.diff(b) > 0) and b[-1] == 1.0 and abs(b[0] - 1e-3) < 1e-9
        np.testing.assert_allclose(b[1:] / b[:-1], b[1] / b[0], rtol=1e-5)
    y = w.data()
    assert y.shape == (1000,) and y.dtype == np.float32
    th = synth.population_particles(w.K, off)
    assert th.shape == (8, 34591) and th.min() >= -10 and th.max() <= 10


def test_schedules():
    b = synth.geometric_betas(20, 1e-3)
    assert b.size == 21 and b[0] == 0.0 and b[-1] == 1.0 and abs(b[1] - 1e-3) < 1e-15
    p = synth.power_betas(200, start=0)  # Table 2: beta_t = (t / 200)^2, t = 0..200
    assert p.size == 201 and p[0] == 0.0 and p[-1] == 1.0 and p[100] == 0.25
    q = synth.power_betas(8)  # Table 1: chain i = 1..M gets (i / M)^2
    np.testing.assert_array_equal(q, (np.arange(1, 9) / 8.0) ** 2)


def test_paper_tables_recipe():
    w = synth.PAPER_TABLES
    assert (w.K, w.N, w.sigma, w.means) == (4, 100, 0.55, (-3.0, 0.0, 3.0, 6.0))
    assert w.table1_M == tuple(8 * 4 ** i for i in range(8)) and w.table1_sweeps == 8192
    assert w.table2_N == tuple(8192 * 2 ** i for i in range(6))
    assert (w.table2_T, w.table2_moves, w.scale) == (200, 10, 1.0)


def test_generators_are_deterministic_and_shaped():
    a = synth.gmm1d_data(100, [-3, 0, 3, 6], 0.55, seed=1)
    assert np.array_equal(a, synth.gmm1d_data(100, [-3, 0, 3, 6], 0.55, seed=1))
    assert not np.array_equal(a, synth.gmm1d_data(100, [-3, 0, 3, 6], 0.55, seed=2))
    truth = synth.diag_truth(16, 32)
    assert synth.diag_particles(4096, truth).shape == (4096, 16, 32)
    assert synth.diag_data(100, truth).shape == (100, 32)
    phi, Sigma, beta = synth.msv_params()
    L = synth.chol(Sigma)
    np.testing.assert_allclose(L @ L.T, Sigma, atol=1e-12)
    x, y = synth.simulate_ssm("msv", 50, phi, Sigma, beta, seed=7)
    assert y.shape == (50, 3)
