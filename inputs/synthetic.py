"""Synthetic stand-ins for the paper's data sets.

The paper's experiments (Sec. 2.1.2, Sec. 2.2.2, Sec. 5, Table 1) run on LIBSVM /
OpenML / UCI / QM9 / SUSY data, which are not available here.  These generators
produce seeded inputs with the shapes and structure of those workloads:
standardised-scale features, d between 4 and 32, N from thousands to millions,
clustered or ill-conditioned point sets.  Every array is float64, C-contiguous.

Layouts used throughout the library:
  X : (N, d) row-major, one point per row.
  Y : (m, N) row-major, i.e. the N x m right-hand-side block in column-major
      order (column r of the block is Y[r]).

Kernel codes: 0 = Gaussian (squared exponential), 1 = Laplace with the l1
distance, 2 = Matern-5/2.  ``mu`` is the regularisation per data point; the
shift applied to the kernel matrix is lambda = mu * N.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

GAUSSIAN = 0
LAPLACE_L1 = 1
MATERN52 = 2


@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray                 # (N, d) float64
    Y: np.ndarray                 # (m, N) float64
    kernel: int
    sigma: float
    mu: float                     # shift is lambda = mu * N
    k: int                        # RPCholesky rank or number of KRILL centers
    block: int                    # RPCholesky block size B
    tol: float
    seed: int
    precision: str = "fp64"       # "fp64" or "mixed"
    centers: Optional[np.ndarray] = None              # KRILL: int64[k], ascending
    settings: Optional[List[Tuple[int, float]]] = None  # batched: (kernel, sigma)
    mus: Optional[List[float]] = None                   # batched: mu values

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    @property
    def m(self) -> int:
        return int(self.Y.shape[0])

    @property
    def lam(self) -> float:
        return self.mu * self.N


def _sin_targets(rng: np.random.Generator, X: np.ndarray) -> np.ndarray:
    y = np.sin(X.sum(axis=1)) + 0.01 * rng.standard_normal(X.shape[0])
    return np.ascontiguousarray(y[None, :])


def make_c1_plain_fp64(n: int = 4096, seed: int = 0) -> Workload:
    """Plain full-data KRR: x ~ N(0, I_8), Gaussian sigma = 1.5, mu = 1e-5,
    y = sin(sum_j x_j) + N(0, 0.01^2); RPCholesky rank 200 with B = 20."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 8))
    Y = _sin_targets(rng, X)
    return Workload("c1_plain_fp64", np.ascontiguousarray(X), Y, GAUSSIAN, 1.5,
                    1e-5, k=min(200, n), block=20, tol=1e-10, seed=seed,
                    precision="fp64")


def make_c2_mixed(n: int = 100_000, seed: int = 1, m: int = 4,
                  k: int = 1000) -> Workload:
    """Ill-conditioned full-data KRR: x uniform on [0,1]^16, then 5% of the rows
    are overwritten by a copy of another (uniformly chosen) row plus 1e-6
    Gaussian jitter.  Gaussian sigma = 0.5, mu = 1e-7, m right-hand sides
    y_r = sum_j cos(2 pi r x_j) + N(0, 0.01^2), r = 1..m."""
    rng = np.random.default_rng(seed)
    d = 16
    X = rng.random((n, d))
    n_dup = n // 20
    dst = rng.choice(n, size=n_dup, replace=False)
    src = rng.integers(0, n, size=n_dup)
    # never copy a row onto itself
    src = np.where(src == dst, (src + 1) % n, src)
    X[dst] = X[src] + 1e-6 * rng.standard_normal((n_dup, d))
    Y = np.empty((m, n))
    for r in range(1, m + 1):
        Y[r - 1] = np.cos(2 * np.pi * r * X).sum(axis=1) + 0.01 * rng.standard_normal(n)
    return Workload("c2_mixed", np.ascontiguousarray(X), Y, GAUSSIAN, 0.5, 1e-7,
                    k=min(k, n), block=100, tol=1e-6, seed=seed, precision="mixed")


def make_c3_batched(n: int = 500_000, seed: int = 2, k: int = 2000) -> Workload:
    """Batched hyperparameters: x from an equal-weight 8-component Gaussian
    mixture in d = 8 (means ~ N(0, 9 I), component scales geomspace(0.1, 2, 8));
    Matern-5/2 and Laplace-l1 at sigma in {0.5, 1, 2, 4}, mu in {1e-6, 1e-8}."""
    rng = np.random.default_rng(seed)
    d, ncomp = 8, 8
    means = 3.0 * rng.standard_normal((ncomp, d))
    scales = np.geomspace(0.1, 2.0, ncomp)
    comp = rng.integers(0, ncomp, size=n)
    X = means[comp] + scales[comp, None] * rng.standard_normal((n, d))
    Y = _sin_targets(rng, X)
    settings = [(MATERN52, s) for s in (0.5, 1.0, 2.0, 4.0)] + \
               [(LAPLACE_L1, s) for s in (0.5, 1.0, 2.0, 4.0)]
    return Workload("c3_batched", np.ascontiguousarray(X), Y, MATERN52, 1.0, 1e-6,
                    k=min(k, n), block=100, tol=1e-6, seed=seed, precision="mixed",
                    settings=settings, mus=[1e-6, 1e-8])


def uniform_centers(rng: np.random.Generator, n: int, k: int) -> np.ndarray:
    """k distinct indices drawn uniformly from range(n), sorted ascending
    (Sec. 2.2: centers sampled uniformly at random)."""
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


def make_c4_krill(n: int = 2_000_000, seed: int = 3, k: int = 2000) -> Workload:
    """Restricted KRR: x ~ N(0, diag(j^-1)), d = 20, k uniform centers,
    Gaussian sigma = 2, mu = 1e-6, y = sin(sum_j x_j) + N(0, 0.01^2)."""
    rng = np.random.default_rng(seed)
    d = 20
    scale = 1.0 / np.sqrt(np.arange(1, d + 1, dtype=np.float64))
    X = rng.standard_normal((n, d)) * scale[None, :]
    Y = _sin_targets(rng, X)
    centers = uniform_centers(rng, n, min(k, n))
    return Workload("c4_krill", np.ascontiguousarray(X), Y, GAUSSIAN, 2.0, 1e-6,
                    k=min(k, n), block=0, tol=1e-6, seed=seed, precision="mixed",
                    centers=centers)


def make_serving_stream(n_requests: int = 512, seed: int = 4,
                        n_range=(2000, 200_000)) -> List[Dict]:
    """Request descriptors for the serving workload: N log-uniform, d in
    {4, 8, 16, 32}, kernel in {Gaussian, Laplace-l1, Matern-5/2}, sigma
    log-uniform in [0.3, 3], mu log-uniform in [1e-8, 1e-4], 1-16 RHS."""
    rng = np.random.default_rng(seed)
    reqs = []
    lo, hi = np.log(n_range[0]), np.log(n_range[1])
    for i in range(n_requests):
        n = int(np.exp(rng.uniform(lo, hi)))
        reqs.append(dict(
            id=i, N=n, d=int(rng.choice([4, 8, 16, 32])),
            kernel=int(rng.integers(0, 3)),
            sigma=float(np.exp(rng.uniform(np.log(0.3), np.log(3.0)))),
            mu=float(np.exp(rng.uniform(np.log(1e-8), np.log(1e-4)))),
            m=int(rng.integers(1, 17)), k=int(min(1000, n // 10)),
            seed=int(rng.integers(0, 2**31))))
    return reqs


def make_serving_request(desc: Dict) -> Tuple[np.ndarray, np.ndarray]:
    """Points and targets of one serving request: x ~ N(0, I_d) and m
    right-hand sides y_r = sin(r <w, x>) + N(0, 0.01^2), r = 1..m, for a
    random unit vector w (seeded by the request's seed)."""
    rng = np.random.default_rng(int(desc["seed"]) + 7919)
    n, d, m = int(desc["N"]), int(desc["d"]), int(desc["m"])
    X = rng.standard_normal((n, d))
    w = rng.standard_normal(d)
    w /= np.linalg.norm(w)
    proj = X @ w
    Y = np.empty((m, n))
    for r in range(1, m + 1):
        Y[r - 1] = np.sin(r * proj) + 0.01 * rng.standard_normal(n)
    return np.ascontiguousarray(X), Y


WORKLOADS: Dict[str, Callable[..., Workload]] = {
    "c1": make_c1_plain_fp64,
    "c2": make_c2_mixed,
    "c3": make_c3_batched,
    "c4": make_c4_krill,
}
