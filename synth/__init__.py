"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module simulates data from the paper's models and draws starting states;
it holds none of the samplers' arithmetic (no likelihood, weight, resampling
or move code).  Every generator is a numpy ``Generator(Philox(seed))`` stream,
so inputs are reproducible on any host.  The method's own random draws
(proposals, accept uniforms, resampling and exchange uniforms, filter noise)
are NOT made here: both implementations generate them from the same Philox
counters inside the method.

Workloads (Lee, Yau, Giles, Doucet & Holmes 2009):
  * gmm4   -- Section 4.1 mixture: k=4, sigma=0.55, w=1/4, mu=(-3,0,3,6),
              m=100 observations, prior U[-10,10]^4, 8192 particles,
              20 geometric temperatures 1e-3 -> 1.
  * gmm8   -- the same model with 8 components at (-7,-5,...,7) and 1000
              observations (population MCMC: 512 populations with 8..128
              chains each; differentiable sampler: 65536 particles, 50
              temperatures).
  * diag32 -- d=32 diagonal mixture, 16 components with means ~ N(0, 4 I),
              sigma=1, 65536 observations, 4096 particles.
  * msv3   -- d=3 multivariate stochastic volatility (the multivariate SV
              model of Section 4.2): phi=0.9, Sigma with unit diagonal and
              0.5 off-diagonal, beta=0.5, T=200, 2^20 particles; plus the
              linear-Gaussian variant y_t = x_t + eps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


# ----------------------------------------------------------------- mixtures
def gmm1d_data(N: int, means, sigma: float, weights=None, seed: int = 1) -> np.ndarray:
    """N observations from the univariate mixture (Section 4.1), float32."""
    means = np.asarray(means, np.float64)
    K = means.size
    w = np.full(K, 1.0 / K) if weights is None else np.asarray(weights, np.float64)
    g = rng(seed)
    comp = g.choice(K, size=N, p=w)
    y = means[comp] + sigma * g.standard_normal(N)
    return y.astype(np.float32)


def prior_particles(K: int, M: int, lo: float = -10.0, hi: float = 10.0,
                    seed: int = 2) -> np.ndarray:
    """Particles from the uniform prior on [lo, hi]^K, SoA layout [K][M]."""
    g = rng(seed)
    return g.uniform(lo, hi, size=(K, M)).astype(np.float32)


def geometric_betas(T: int, beta_min: float = 1e-3) -> np.ndarray:
    """Temperature schedule beta_0 = 0, beta_t = beta_min^((T-t)/(T-1)), t=1..T."""
    t = np.arange(1, T + 1, dtype=np.float64)
    b = beta_min ** ((T - t) / max(T - 1, 1))
    return np.concatenate([[0.0], b])


def power_betas(n: int, start: int = 1) -> np.ndarray:
    """(i/n)^2 for i = start..n: the cooling schedule of Section 4.1.1
    (chains i = 1..M, start=1) and Section 4.1.2 (beta_0..beta_T, start=0)."""
    return (np.arange(start, n + 1, dtype=np.float64) / n) ** 2


def population_offsets(n_pops: int, lo: int = 8, hi: int = 128, seed: int = 3) -> np.ndarray:
    """CSR offsets [n_pops+1] of populations with chain counts uniform in [lo, hi]."""
    g = rng(seed)
    sizes = g.integers(lo, hi + 1, size=n_pops)
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)


def population_betas(offsets, beta_min: float = 1e-3) -> np.ndarray:
    """Per-chain temperatures: chain c of a population of size m gets
    beta_min^((m-1-c)/(m-1)), so the last chain targets the posterior."""
    offsets = np.asarray(offsets, np.int64)
    out = np.empty(int(offsets[-1]), np.float64)
    for q in range(offsets.size - 1):
        m = int(offsets[q + 1] - offsets[q])
        c = np.arange(m, dtype=np.float64)
        out[offsets[q]:offsets[q + 1]] = beta_min ** ((m - 1 - c) / max(m - 1, 1))
    return out.astype(np.float32)


def population_particles(K: int, offsets, lo=-10.0, hi=10.0, seed: int = 4) -> np.ndarray:
    return prior_particles(K, int(np.asarray(offsets)[-1]), lo, hi, seed)


def diag_truth(K: int, d: int, seed: int = 1) -> np.ndarray:
    """True component means ~ N(0, 4 I_d), [K][d] float64."""
    return 2.0 * rng(seed).standard_normal((K, d))


def diag_data(N: int, truth: np.ndarray, sigma: float = 1.0, seed: int = 11) -> np.ndarray:
    """N observations [N][d] float32 from the equal-weight diagonal mixture."""
    K, d = truth.shape
    g = rng(seed)
    comp = g.integers(0, K, size=N)
    return (truth[comp] + sigma * g.standard_normal((N, d))).astype(np.float32)


def diag_particles(M: int, truth: np.ndarray, seed: int = 12) -> np.ndarray:
    """Particles [M][K][d] float32: the first half near the truth
    (truth + 0.1 N(0, I)), the second half prior-like draws N(0, 4 I)."""
    K, d = truth.shape
    g = rng(seed)
    h = M // 2
    near = truth[None] + 0.1 * g.standard_normal((h, K, d))
    far = 2.0 * g.standard_normal((M - h, K, d))
    return np.concatenate([near, far]).astype(np.float32)


# ----------------------------------------------------- state-space models
def msv_params(d: int = 3, phi: float = 0.9, rho: float = 0.5, beta: float = 0.5):
    Sigma = np.full((d, d), rho) + (1.0 - rho) * np.eye(d)
    return np.full(d, phi), Sigma, beta


def chol(Sigma) -> np.ndarray:
    return np.linalg.cholesky(np.asarray(Sigma, np.float64))


def simulate_ssm(kind: str, T: int, phi, Sigma, beta: float, seed: int = 7):
    """Simulate x_{1:T} (x_0 = 0) and y_{1:T} from the MSV model
    (y_t ~ N(0, beta^2 diag(exp(x_t)))) or the linear-Gaussian variant
    (y_t = x_t + N(0, beta^2 I)).  Returns (x [T][d] f64, y [T][d] f32)."""
    phi = np.asarray(phi, np.float64)
    L = chol(Sigma)
    d = phi.size
    g = rng(seed)
    x = np.zeros(d)
    xs = np.zeros((T, d))
    ys = np.zeros((T, d))
    for t in range(T):
        x = phi * x + L @ g.standard_normal(d)
        e = g.standard_normal(d)
        if kind == "msv":
            ys[t] = beta * np.exp(0.5 * x) * e
        else:
            ys[t] = x + beta * e
        xs[t] = x
    return xs, ys.astype(np.float32)


def fsv_params():
    """The factor stochastic volatility model of Section 4.2: K = 3 factors,
    m = 5 series, phi_i = 0.9, psi_i = 0.5, loading matrix B (m x K, zero
    above the diagonal) and state covariance U as printed there.  Returns
    (phi [K], U [K][K], B [m][K], psi [m])."""
    B = np.array([[1.0, 0.0, 0.0],
                  [0.5, 1.0, 0.0],
                  [0.5, 0.5, 1.0],
                  [0.2, 0.6, 0.3],
                  [0.8, 0.7, 0.5]])
    U = np.array([[0.5, 0.2, 0.1],
                  [0.2, 0.5, 0.2],
                  [0.1, 0.2, 0.5]])
    return np.full(3, 0.9), U, B, np.full(5, 0.5)


def simulate_fsv(T: int, phi, U, B, psi, seed: int = 7):
    """Simulate x_{1:T} (x_0 = 0) and y_{1:T} of the factor SV model:
    x_t = phi x_{t-1} + N(0, U), f_t ~ N(0, diag(exp x_t)), y_t = B f_t +
    N(0, diag(psi)).  Returns (x [T][K] f64, y [T][m] f32)."""
    phi = np.asarray(phi, np.float64)
    B = np.asarray(B, np.float64)
    L = chol(U)
    K, m = phi.size, B.shape[0]
    g = rng(seed)
    x = np.zeros(K)
    xs = np.zeros((T, K))
    ys = np.zeros((T, m))
    for t in range(T):
        x = phi * x + L @ g.standard_normal(K)
        f = np.exp(0.5 * x) * g.standard_normal(K)
        ys[t] = B @ f + np.sqrt(np.asarray(psi, np.float64)) * g.standard_normal(m)
        xs[t] = x
    return xs, ys.astype(np.float32)


def gaussian_logweights(M: int, scale: float = 1.0, seed: int = 5) -> np.ndarray:
    return scale * rng(seed).standard_normal(M)


# ------------------------------------------------------------- workloads
@dataclass
class GMMWorkload:
    name: str
    K: int
    N: int
    M: int
    means: tuple
    sigma: float = 0.55
    box: tuple = (-10.0, 10.0)
    T: int = 20
    beta_min: float = 1e-3
    scale: float = 0.1
    ess_frac: float = 0.5
    data_seed: int = 1
    particle_seed: int = 2
    method_seed: int = 1234
    n_pops: int = 0
    pop_lo: int = 8
    pop_hi: int = 128
    pop_seed: int = 3
    sweeps: int = 0
    extra: dict = field(default_factory=dict)

    def logw(self) -> np.ndarray:
        return np.full(self.K, -np.log(self.K))

    def data(self) -> np.ndarray:
        return gmm1d_data(self.N, self.means, self.sigma, seed=self.data_seed)


GMM4 = GMMWorkload("gmm4-smc-M8192-K4-N100", K=4, N=100, M=8192, means=(-3.0, 0.0, 3.0, 6.0), T=20)
GMM8_POP = GMMWorkload("gmm8-popmcmc-512pops-K8-N1000", K=8, N=1000, M=0,
                       means=tuple(float(v) for v in range(-7, 8, 2)), n_pops=512, sweeps=1000)
GMM8_MALA = GMMWorkload("gmm8-mala-smc-M65536-K8-N1000", K=8, N=1000, M=65536,
                        means=tuple(float(v) for v in range(-7, 8, 2)), T=50, scale=0.05)


@dataclass
class PaperTablesWorkload:
    """Section 4.1 model (m = 100 data, k = 4, sigma = 0.55, means
    (-3, 0, 3, 6), uniform prior on [-10, 10]^4), run as in Table 1
    (one population of M chains with beta_i = (i/M)^2, N(0, I_4) random
    walk, 8192 sweeps) and Table 2 (N particles, 200 temperatures with
    beta_t = (t/200)^2, 10 N(0, I_4) random-walk moves per temperature,
    resampling when ESS < N/2)."""
    name: str = "gmm4-paper-tables-1-2"
    K: int = 4
    N: int = 100
    means: tuple = (-3.0, 0.0, 3.0, 6.0)
    sigma: float = 0.55
    scale: float = 1.0
    table1_M: tuple = (8, 32, 128, 512, 2048, 8192, 32768, 131072)
    table1_sweeps: int = 8192
    table2_N: tuple = (8192, 16384, 32768, 65536, 131072, 262144)
    table2_T: int = 200
    table2_moves: int = 10
    data_seed: int = 1
    particle_seed: int = 2
    method_seed: int = 1234

    def logw(self) -> np.ndarray:
        return np.full(self.K, -np.log(self.K))

    def data(self) -> np.ndarray:
        return gmm1d_data(self.N, self.means, self.sigma, seed=self.data_seed)


PAPER_TABLES = PaperTablesWorkload()


@dataclass
class DiagWorkload:
    name: str = "diag-d32-K16-N65536-M4096"
    d: int = 32
    K: int = 16
    N: int = 65536
    M: int = 4096
    sigma: float = 1.0
    truth_seed: int = 1
    data_seed: int = 11
    particle_seed: int = 12

    def logw(self) -> np.ndarray:
        return np.full(self.K, -np.log(self.K))


DIAG32 = DiagWorkload()


@dataclass
class FSVWorkload:
    """Section 4.2 / Table 3: the bootstrap filter on the factor SV model,
    T = 200 steps, particle counts as in the table, resampling every step."""
    name: str = "fsv-m5-K3-T200"
    T: int = 200
    Ns: tuple = (8192, 16384, 32768, 65536, 131072)
    data_seed: int = 7
    method_seed: int = 77


FSV = FSVWorkload()


@dataclass
class PFWorkload:
    name: str = "msv3-pf-M1048576-T200"
    d: int = 3
    M: int = 1 << 20
    T: int = 200
    phi: float = 0.9
    rho: float = 0.5
    beta: float = 0.5
    data_seed: int = 7
    method_seed: int = 77


MSV3 = PFWorkload()
