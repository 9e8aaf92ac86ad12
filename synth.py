"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds workload shapes, parameter sets and arbitrary seeded states;
it contains none of the slip-spring method's arithmetic (no init sampling, no
step, no stress).  Both the CUDA library and the CPU oracle receive what it
produces.  The random numbers the method itself draws come from each side's own
Philox4x32-10, keyed by the seed given here.

Workloads (the paper's parameter ratios, Sec. 4.1: N0 = 4, Ns = 0.5,
zeta_s = 0.1, dt = 0.01, b = kT = zeta = 1):
  parity   256 chains, N = 16, FP64, 1e4 steps, seed 0       (<Z> = 4)
  lve      65536 chains, N = 32, FP32 beads / FP64 sums, 1e6 steps,
           multiple-tau 16 points x 24 levels, seed 1         (<Z> = 8)
  shear    N = 32, 16384 chains per rate, 8 rates 10^(-4 + 3k/7), 2e5 steps,
           logs every 100 steps, seeds 2 + k
  batched  4096 elements, M_e = round(exp(U[ln 64, ln 1024])), N_e uniform in
           {16, 24, 32, 48}, traceless kappa with N(0, 1e-2) entries redrawn
           every 1000 steps, 1e5 steps, seed 3
  adjoint  8192 chains, N = 24, 1e4-step windows, checkpoints every 256 steps
"""
import numpy as np

PAPER = dict(N0=4.0, Ns=0.5, zeta_s=0.1, dt=0.01, b=1.0, kT=1.0, zeta=1.0)

WORKLOADS = {
    "parity": dict(M=256, N=16, precision="fp64", steps=10_000, seed=0, levels=24),
    "lve": dict(M=65536, N=32, precision="fp32", steps=1_000_000, seed=1, levels=24),
    "shear": dict(M=16384, N=32, precision="fp32", steps=200_000, seed=2, levels=24,
                  log_every=100, rates=[10 ** (-4 + 3 * k / 7) for k in range(8)]),
    "batched": dict(n_elements=4096, lengths=(16, 24, 32, 48), m_lo=64, m_hi=1024,
                    precision="fp32", steps=100_000, seed=3, kappa_every=1000, kappa_std=1e-2),
    "adjoint": dict(M=8192, N=24, precision="fp32", steps=10_000, seed=4, checkpoint=256),
}


def shear_kappa(gdot: float) -> np.ndarray:
    """Velocity gradient of simple shear, kappa_xy = gdot (Sec. 4.1)."""
    k = np.zeros((3, 3))
    k[0, 1] = gdot
    return k


def element_table(n_elements: int, seed: int = 3, lengths=(16, 24, 32, 48), m_lo=64, m_hi=1024,
                  n_kappa: int = 100, kappa_std: float = 1e-2):
    """Batched multiscale workload: per element an ensemble size (log-uniform in
    [m_lo, m_hi], rounded), a chain length (uniform over `lengths`) and n_kappa
    traceless velocity gradients with Gaussian entries of std kappa_std."""
    rng = np.random.default_rng(seed)
    M = np.rint(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi), size=n_elements))).astype(np.int64)
    N = rng.choice(np.asarray(lengths, dtype=np.int64), size=n_elements)
    G = rng.normal(0.0, kappa_std, size=(n_elements, n_kappa, 3, 3))
    tr = np.trace(G, axis1=2, axis2=3)
    G -= (tr / 3.0)[:, :, None, None] * np.eye(3)[None, None]
    return M, N, G


def random_state(M: int, N: int, z_max: int, seed: int, z_mean: float = 4.0,
                 bond_std: float = 0.6, anchor_std: float = 0.4, offset: float = 0.0):
    """An arbitrary (not equilibrium-distributed) seeded chain state:
    R [M][N][3] random walks, Z [M] binomial-ish counts <= z_max, S [M][z_max]
    random bead indices (-1 beyond Z), A [M][z_max][3] near the chosen beads."""
    rng = np.random.default_rng(seed)
    R = np.cumsum(rng.normal(0.0, bond_std, size=(M, N, 3)), axis=1) + offset
    Z = np.minimum(rng.poisson(z_mean, size=M), z_max).astype(np.int32)
    S = -np.ones((M, z_max), dtype=np.int32)
    A = np.zeros((M, z_max, 3))
    for m in range(M):
        z = Z[m]
        S[m, :z] = rng.integers(0, N, size=z)
        A[m, :z] = R[m, S[m, :z]] + rng.normal(0.0, anchor_std, size=(z, 3))
    return {"R": R, "Z": Z, "S": S, "A": A}
