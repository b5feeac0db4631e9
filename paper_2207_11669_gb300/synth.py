"""Seeded synthetic RPCA instances (the problem generator of §4.1).

This module only builds inputs: it holds none of the DCF-PCA arithmetic and
is the one piece of code that both the CUDA path's tests/benchmarks and the
FP64 oracle's tests draw from.

Generator (§4.1 "Problem Generation"): a low-rank ground truth L* = A B^T
with Gaussian factors, plus a sparse corruption S* whose support is
Bernoulli(density).  The paper draws S* values from {-sqrt(mn), 0, sqrt(mn)};
the workloads used here draw them uniformly from [-a, a] (the magnitude
sqrt(mn) reads as a typo for a sign law), and ``values="paper"`` keeps the
printed law available.

Layout conventions shared by every consumer:
  * M is m x n, column-major (numpy ``order='F'``), float32; column block i
    is the contiguous slice of columns [c_i, c_i + n_i).
  * factors are row-major: U is m x r with row a at U[a, :], V is n x r.
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class Instance:
    M: np.ndarray          # (m, n) float32, Fortran order
    A: np.ndarray          # (m, k) float32 left truth factor
    B: np.ndarray          # (n, k) float32 right truth factor
    S_star: np.ndarray     # (m, n) float32, Fortran order (sparse part)
    n_i: np.ndarray        # (E,) int64 block widths, sum = n
    seed: int

    @property
    def m(self) -> int:
        return self.M.shape[0]

    @property
    def n(self) -> int:
        return self.M.shape[1]

    @property
    def E(self) -> int:
        return len(self.n_i)


def uneven_blocks(n: int, E: int, lo: int, hi: int, rng: np.random.Generator,
                  max_tries: int = 100000) -> np.ndarray:
    """E block widths drawn uniformly from [lo, hi] that sum to n.

    Seeded rejection sampling: draw E-1 widths, give the remainder to the
    last block, accept when the remainder is inside [lo, hi].
    """
    if E == 1:
        if not lo <= n <= hi:
            raise ValueError("single block outside [lo, hi]")
        return np.array([n], dtype=np.int64)
    for _ in range(max_tries):
        w = rng.integers(lo, hi + 1, size=E - 1)
        last = n - int(w.sum())
        if lo <= last <= hi:
            return np.concatenate([w, [last]]).astype(np.int64)
    raise ValueError(f"no split of n={n} into {E} blocks in [{lo},{hi}]")


def equal_blocks(n: int, E: int) -> np.ndarray:
    base = n // E
    w = np.full(E, base, dtype=np.int64)
    w[: n - base * E] += 1
    return w


def make_instance(m: int, n: int, k: int, *, seed: int, density: float,
                  amp: float, factor_std: float, n_i=None, E: int = 1,
                  values: str = "uniform") -> Instance:
    """M = A B^T + S*, all float32, with a fixed seed.

    ``factor_std`` is the standard deviation of the entries of A and B,
    ``density`` the Bernoulli rate of the support of S*, ``amp`` the bound
    of the uniform values of S* (``values="uniform"``) or ignored for the
    paper's {+-sqrt(mn)} law (``values="paper"``).
    """
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((m, k)) * factor_std).astype(np.float32)
    B = (rng.standard_normal((n, k)) * factor_std).astype(np.float32)
    if n_i is None:
        n_i = equal_blocks(n, E)
    n_i = np.asarray(n_i, dtype=np.int64)
    if int(n_i.sum()) != n:
        raise ValueError("block widths do not sum to n")
    # Build column-major M in column chunks to bound the temporaries.
    M = np.empty((m, n), dtype=np.float32, order="F")
    S = np.zeros((m, n), dtype=np.float32, order="F")
    chunk = max(1, (1 << 24) // max(m, 1))
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        w = c1 - c0
        support = rng.random((w, m)) < density          # column-major draw
        if values == "paper":
            sign = np.where(rng.random((w, m)) < 0.5, -1.0, 1.0)
            vals = (sign * np.sqrt(float(m) * float(n))).astype(np.float32)
        else:
            vals = rng.uniform(-amp, amp, size=(w, m)).astype(np.float32)
        Sc = np.where(support, vals, np.float32(0)).astype(np.float32)
        S[:, c0:c1] = Sc.T
        M[:, c0:c1] = (B[c0:c1] @ A.T).T + Sc.T
    return Instance(M=M, A=A, B=B, S_star=S, n_i=n_i, seed=seed)


def gaussian_u0(m: int, r: int, seed: int) -> np.ndarray:
    """Initial left factor U0 with i.i.d. N(0, 1/m) entries, float32, row-major."""
    rng = np.random.default_rng(seed ^ 0x5EED5EED)
    return (rng.standard_normal((m, r)) / np.sqrt(m)).astype(np.float32)


# ---------------------------------------------------------------------------
# The five workload families (sizes, value laws and seeds).
# ---------------------------------------------------------------------------
SEED_BASE = 20220723


@dataclasses.dataclass
class Workload:
    name: str
    m: int
    n: int
    k: int              # true rank of L*
    r: int              # factor rank used by the solver
    E: int
    density: float
    amp: float
    factor_std: float
    rho: float
    lam: float
    iters: int
    blocks: str         # "equal" or "uneven"
    block_lo: int = 0
    block_hi: int = 0
    seed: int = SEED_BASE

    def instance(self, seed=None, m=None, n=None) -> Instance:
        """Draw the instance; ``m``/``n`` shrink it while keeping the laws."""
        seed = self.seed if seed is None else seed
        m = self.m if m is None else m
        n = self.n if n is None else n
        rng = np.random.default_rng(seed + 7919)
        if self.blocks == "uneven" and n == self.n:
            n_i = uneven_blocks(n, self.E, self.block_lo, self.block_hi, rng)
        elif self.blocks == "uneven":
            scale = n / self.n
            lo = max(1, int(self.block_lo * scale))
            hi = max(lo, int(self.block_hi * scale))
            n_i = uneven_blocks(n, self.E, lo, hi, rng)
        else:
            n_i = equal_blocks(n, self.E)
        return make_instance(m, n, self.k, seed=seed, density=self.density,
                             amp=self.amp, factor_std=self.factor_std, n_i=n_i)


def workload_small() -> Workload:
    """m=n=200, E=4 equal blocks, L* rank 5 with N(0,1) factors, S* density
    0.05 with values U[-10,10]; r=5, rho=1e-2, lambda=1/sqrt(200), 200 iterations."""
    return Workload("dcf_m200_n200_r5_E4", 200, 200, 5, 5, 4, 0.05, 10.0, 1.0,
                    1e-2, 1.0 / np.sqrt(200.0), 200, "equal", seed=SEED_BASE + 0)


def workload_medium() -> Workload:
    """m=4096, n=65536 in E=16 uneven blocks of [2048, 6144] columns, L* rank
    32 with N(0,1/32) factors, S* density 0.05 with values U[-5,5]; r=32,
    rho=1e-2, lambda=1/sqrt(4096), 100 iterations."""
    return Workload("dcf_m4096_n65536_r32_E16", 4096, 65536, 32, 32, 16, 0.05, 5.0,
                    float(np.sqrt(1.0 / 32.0)), 1e-2, 1.0 / 64.0, 100, "uneven",
                    2048, 6144, seed=SEED_BASE + 1)


def workload_large() -> Workload:
    """m=16384, n=262144 in E=64 uneven blocks of [2048, 6144], L* rank 64 with
    N(0,1/64) factors, S* density 0.05 with values U[-5,5]; r=64,
    rho=1e-2, lambda=1/128."""
    return Workload("dcf_m16384_n262144_r64_E64", 16384, 262144, 64, 64, 64, 0.05, 5.0,
                    0.125, 1e-2, 1.0 / 128.0, 100, "uneven", 2048, 6144,
                    seed=SEED_BASE + 4)


def batched_instance_shapes(count: int, seed: int = SEED_BASE + 2):
    """Shapes of the batched workload: m ~ U[256,1024], n ~ U[512,8192],
    E ~ U{4..16} uneven blocks, rank ~ U{4..32} (r = true rank), density
    ~ U[0.01, 0.10], values U[-10,10], rho=1e-2, lambda=1/sqrt(m)."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        m = int(rng.integers(256, 1025))
        n = int(rng.integers(512, 8193))
        E = int(rng.integers(4, 17))
        k = int(rng.integers(4, 33))
        dens = float(rng.uniform(0.01, 0.10))
        lo = max(1, n // (2 * E))
        hi = max(lo, (3 * n) // (2 * E))
        n_i = uneven_blocks(n, E, lo, hi, rng)
        out.append(dict(m=m, n=n, E=E, k=k, r=k, density=dens, amp=10.0,
                        factor_std=1.0 / np.sqrt(k), rho=1e-2,
                        lam=1.0 / np.sqrt(m), n_i=n_i, seed=seed * 1000 + q))
    return out


def learned_instance(q: int, split: str = "train") -> Instance:
    """Problem q of the learned-network workload: m = 1024, n = 16384 in E = 8
    equal blocks, L* of rank 16 from N(0, 1/16) factors, S* density 0.10 with
    values U[-10, 10].  Training and held-out problems use disjoint seeds."""
    base = SEED_BASE + 3000 + (0 if split == "train" else 100000)
    return make_instance(1024, 16384, 16, seed=base + q, density=0.10, amp=10.0,
                         factor_std=0.25, E=8)


LEARNED_RHO = 1e-2
LEARNED_LAMBDA = 1.0 / 32.0     # 1 / sqrt(m)
LEARNED_K = 10


PHASE_N = 160
PHASE_RANKS = (0.05, 0.075, 0.1, 0.125, 0.15, 0.175, 0.2)
PHASE_DENSITIES = (0.05, 0.1, 0.15, 0.2, 0.25, 0.3)


def phase_grid(n: int = PHASE_N, ranks=PHASE_RANKS, densities=PHASE_DENSITIES,
               trials: int = 1, E: int = 4, seed: int = SEED_BASE + 5):
    """Cells of the sparsity x rank sweep of §4.2 (the phase-transition figure):
    m = n, truth rank r = ratio * n for each ratio in ``ranks`` (the solver runs
    with that rank), S* density s for each s in ``densities``, values U[-10, 10],
    N(0, 1/r) truth factors, E equal blocks, ``trials`` seeded instances per
    cell.  rho = 1e-2 and lambda = 1/sqrt(n).  Returns a list of dicts (shape,
    law and seed of every instance, cell coordinates under "cell")."""
    out = []
    for a, ratio in enumerate(ranks):
        k = max(1, int(round(ratio * n)))
        for b, dens in enumerate(densities):
            for t in range(trials):
                out.append(dict(m=n, n=n, k=k, r=k, density=float(dens), amp=10.0,
                                factor_std=1.0 / np.sqrt(k), rho=1e-2, lam=1.0 / np.sqrt(n),
                                n_i=equal_blocks(n, E), seed=seed * 1000 + 97 * a + 7 * b + t,
                                cell=(float(ratio), float(dens), t)))
    return out
