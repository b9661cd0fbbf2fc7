"""Seeded synthetic inputs shaped like the paper's regression workloads.

The paper's UCI datasets (Houseelectric n=2,049,280 d=11, Keggdirected d=20, Protein,
Elevators, Precipitation; Sec. 5, Table n_lattice) are not available, so these
generators stand in for them.  This module holds no arithmetic of the method: it only
draws inputs, and both the CUDA path and the oracle consume exactly the arrays it
returns (float32, C order).
"""

from __future__ import annotations

import numpy as np


def uniform_points(n: int, d: int, seed: int) -> np.ndarray:
    """X ~ Uniform[0, 1]^d (the small single-MVM workload: n=4096, d=3)."""
    rng = np.random.default_rng(seed)
    return rng.random((n, d)).astype(np.float32)


def gaussian_values(n: int, k: int, seed: int) -> np.ndarray:
    """Right-hand sides V ~ N(0, 1), shape [n][k]."""
    rng = np.random.default_rng(seed + 7919)
    return rng.standard_normal((n, k)).astype(np.float32)


def gmm_points(n: int, d: int, seed: int, components: int = 16) -> np.ndarray:
    """Standardised Gaussian mixture: means ~ N(0, I), diagonal scales ~ U[0.2, 1],
    equal weights, then each dimension shifted/scaled to zero mean and unit variance."""
    rng = np.random.default_rng(seed)
    means = rng.standard_normal((components, d))
    scales = rng.uniform(0.2, 1.0, (components, d))
    comp = rng.integers(0, components, n)
    X = means[comp] + scales[comp] * rng.standard_normal((n, d))
    X = (X - X.mean(0)) / X.std(0)
    return X.astype(np.float32)


def regression_targets(X: np.ndarray, seed: int, noise_std: float = 0.1) -> np.ndarray:
    """y = sum_j sin(2 x_j) + N(0, noise_std^2)."""
    rng = np.random.default_rng(seed + 104729)
    y = np.sin(2.0 * X.astype(np.float64)).sum(1) + noise_std * rng.standard_normal(X.shape[0])
    return y.astype(np.float32)


def rademacher(n: int, k: int, seed: int) -> np.ndarray:
    """Probe vectors with independent +-1 entries, shape [n][k]."""
    rng = np.random.default_rng(seed + 1299709)
    return (2.0 * rng.integers(0, 2, (n, k)) - 1.0).astype(np.float32)


def solve_rhs(X: np.ndarray, seed: int, probes: int = 8) -> np.ndarray:
    """B = [y, probes Rademacher columns] for a posterior-mean-and-variance solve."""
    y = regression_targets(X, seed)
    return np.ascontiguousarray(
        np.concatenate([y[:, None], rademacher(X.shape[0], probes, seed)], 1), np.float32)


def correlated_points(n: int, d: int, seed: int):
    """X ~ N(0, Q diag(lam) Q^T) with Q Haar-orthogonal and lam log-uniform[0.3, 3];
    ARD lengthscales log-uniform[0.5, 2].  Returns (X, lengthscales)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((d, d))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))[None, :]
    lam = np.exp(rng.uniform(np.log(0.3), np.log(3.0), d))
    X = (rng.standard_normal((n, d)) * np.sqrt(lam)[None, :]) @ Q.T
    ls = np.exp(rng.uniform(np.log(0.5), np.log(2.0), d))
    return X.astype(np.float32), ls.astype(np.float32)


def subsample(n: int, count: int, seed: int) -> np.ndarray:
    """Sorted, distinct row indices drawn by seed (for sampled parity checks)."""
    rng = np.random.default_rng(seed + 15485863)
    return np.sort(rng.choice(n, size=min(count, n), replace=False)).astype(np.int64)


def serving_stream(count: int, seed: int, rate_per_s: float = 50.0,
                   n_range=(5_000, 500_000), dims=(3, 8, 20, 50, 90), test_points: int = 256,
                   noise: float = 0.01):
    """GP posterior requests with Poisson arrivals (exponential gaps, mean 1 / rate).

    Each request: n log-uniform in n_range, d uniform over dims, n + test_points points
    from one standardised Gaussian mixture split into training and test inputs, targets
    as regression_targets, unit ARD lengthscales, outputscale 1, the given noise, and a
    probe seed.  Returns a list of dicts (arrival_s, X, y, Xs, lengthscales, outputscale,
    noise, seed) in arrival order.
    """
    rng = np.random.default_rng(seed + 32452843)
    gaps = rng.exponential(1.0 / rate_per_s, count)
    arrivals = np.cumsum(gaps) - gaps[0]
    lo, hi = np.log(n_range[0]), np.log(n_range[1])
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(lo, hi)))
        d = int(dims[rng.integers(0, len(dims))])
        rs = seed * 1000003 + i
        P = gmm_points(n + test_points, d, rs)
        X, Xs = P[:n], P[n:]
        out.append(dict(arrival_s=float(arrivals[i]), X=np.ascontiguousarray(X),
                        y=regression_targets(X, rs), Xs=np.ascontiguousarray(Xs),
                        lengthscales=np.ones(d, np.float32), outputscale=1.0, noise=noise,
                        seed=rs))
    return out


def repeated_stream(count: int, datasets: int, seed: int, rate_per_s: float = 50.0,
                    n_range=(5_000, 500_000), dims=(3, 8, 20, 50, 90),
                    test_points: int = 256, noise: float = 0.01):
    """Requests that reuse `datasets` point sets: each request takes one of them
    (round-robin over a seeded shuffle) with its own targets (regression_targets with the
    request's seed) and Poisson arrivals.  Each dict also carries "dataset" (0-based)."""
    base = serving_stream(datasets, seed, rate_per_s, n_range, dims, test_points, noise)
    rng = np.random.default_rng(seed + 49979687)
    gaps = rng.exponential(1.0 / rate_per_s, count)
    arrivals = np.cumsum(gaps) - gaps[0]
    order = rng.permutation(count) % datasets
    out = []
    for i in range(count):
        b = base[int(order[i])]
        rs = seed * 1000003 + 500009 + i
        out.append(dict(b, arrival_s=float(arrivals[i]), y=regression_targets(b["X"], rs),
                        seed=rs, dataset=int(order[i])))
    return out
