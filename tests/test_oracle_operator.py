"""Pins of the oracle's splat / blur / slice operator (Sec. 3.2, Eq. k_ski, Eq.
ski_to_bf) and of its stencils (Sec. 4.1, Eq. balance_coverage).

The blur is checked against matrices assembled here independently of the oracle's
own neighbour search (a Python dict over the exported keys), against the closed form
of a single point at the origin, and against the explicit d = 1 matrix built without
any hashing.
"""

import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy import integrate

import oracle
from oracle import MATERN32_COVERAGE, RBF_BINOMIAL, RBF_COVERAGE, OracleLattice
from paper_2106_06695_gb300 import synth


def test_binomial_stencil_golden(golden):
    taps = golden("binomial_stencil.txt")[0]
    s, c, g = oracle.stencil(RBF_BINOMIAL, 1)
    assert np.allclose([c[1], c[0], c[1]], taps, rtol=0, atol=1e-15)
    # the taps are kernel values at the lattice spacing (Sec. 4.1): k(s) = 1/2
    assert abs(math.exp(-0.5 * s * s) - 0.5) < 1e-15


@pytest.mark.parametrize("r", [1, 2, 3])
def test_rbf_coverage_closed_form(r):
    # Gaussian: both sides of Eq. balance_coverage are erf's, equal when s^2 = 2 pi / (2r+1)
    s, c, g = oracle.stencil(RBF_COVERAGE, r)
    assert abs(s - math.sqrt(2 * math.pi / (2 * r + 1))) < 1e-9


@pytest.mark.parametrize("kind", [RBF_COVERAGE, MATERN32_COVERAGE])
@pytest.mark.parametrize("r", [1, 2, 3])
def test_coverage_balance_by_quadrature(kind, r):
    """The spacing balances the two coverages of Eq. balance_coverage when both are
    integrated numerically (scipy quad) from the kernel and its spectral density."""
    s, c, g = oracle.stencil(kind, r)
    if kind == MATERN32_COVERAGE:
        b = math.sqrt(3.0)
        k = lambda t: (1 + b * abs(t)) * math.exp(-b * abs(t))  # noqa: E731
        S = lambda w: 1.0 / (b * b + w * w) ** 2  # noqa: E731
    else:
        k = lambda t: math.exp(-0.5 * t * t)  # noqa: E731
        S = lambda w: math.exp(-0.5 * w * w)  # noqa: E731
    m = 2 * r + 1
    lhs = integrate.quad(k, 0, s * m / 2)[0] / integrate.quad(k, 0, np.inf)[0]
    rhs = integrate.quad(S, 0, math.pi / s)[0] / integrate.quad(S, 0, np.inf)[0]
    assert abs(lhs - rhs) < 1e-8
    for t in range(r + 1):
        assert abs(c[t] - k(t * s)) < 1e-14


@pytest.mark.parametrize("kind", [RBF_BINOMIAL, MATERN32_COVERAGE])
def test_half_kernel_taps(kind):
    """g samples a kernel whose self-convolution is proportional to k, with
    sum_{t=-r..r} g_t^2 = 1."""
    r = 2
    s, c, g = oracle.stencil(kind, r)
    assert abs(g[0] ** 2 + 2 * (g[1:] ** 2).sum() - 1.0) < 1e-14
    if kind == MATERN32_COVERAGE:
        b = math.sqrt(3.0)
        kh = lambda t: math.exp(-b * abs(t))  # noqa: E731
        k = lambda t: (1 + b * abs(t)) * math.exp(-b * abs(t))  # noqa: E731
    else:
        kh = lambda t: math.exp(-t * t)  # noqa: E731
        k = lambda t: math.exp(-0.5 * t * t)  # noqa: E731
    conv = [integrate.quad(lambda x: kh(x) * kh(tau - x), -np.inf, np.inf)[0]
            for tau in (0.0, 0.7, 1.9)]
    assert np.allclose(np.array(conv) / conv[0], [k(0.0), k(0.7), k(1.9)], rtol=1e-7)
    for t in range(r + 1):
        assert abs(g[t] / g[0] - kh(t * s)) < 1e-14


@pytest.mark.parametrize("d", [1, 2, 3, 4, 8, 11])
def test_single_point_closed_form(golden, d):
    table = {int(row[0]): row[1] for row in golden("origin_self_covariance.txt")}
    expect = table.get(d, 1.0 + 2.0 ** -(d + 1))
    L = OracleLattice(np.zeros((1, d), np.float32), np.ones(d, np.float32))
    for mode in (0, 1):
        assert L.mvm(np.ones((1, 1)), mode=mode)[0, 0] == pytest.approx(expect, abs=1e-15)


def _d1_matrix(x, ls, coef, s):
    """Explicit d = 1 operator: hat-function interpolation on the grid s*Z, blur by the
    tridiagonal stencil restricted to occupied grid points, applied once per lattice
    direction (both directions lie on the same line)."""
    t = x.astype(np.float64)[:, 0] / float(np.float32(ls)) / s
    lo = np.floor(t).astype(int)
    frac = t - lo
    grid = np.unique(np.concatenate([lo, lo + 1]))
    pos = {g: i for i, g in enumerate(grid)}
    W = np.zeros((len(x), len(grid)))
    for i in range(len(x)):
        W[i, pos[lo[i]]] += 1.0 - frac[i]
        W[i, pos[lo[i] + 1]] += frac[i]
    S = np.eye(len(grid)) * coef[0]
    for a in range(len(grid)):
        for tt in range(1, len(coef)):
            for b in (grid[a] + tt, grid[a] - tt):
                if b in pos:
                    S[a, pos[b]] += coef[tt]
    return W, S


def test_d1_closed_form():
    rng = np.random.default_rng(7)
    x = (rng.standard_normal((60, 1)) * 3.0).astype(np.float32)
    for r in (1, 2):
        L = OracleLattice(x, np.array([0.8], np.float32), kind=RBF_COVERAGE, r=r)
        W, S = _d1_matrix(x, 0.8, L.coef, L.s)
        _, G = _d1_matrix(x, 0.8, L.half, L.s)
        V = rng.standard_normal((60, 3))
        assert np.allclose(L.mvm(V, mode=0), W @ S @ S @ W.T @ V, rtol=1e-12, atol=1e-12)
        assert np.allclose(L.mvm(V, mode=1), W @ S @ S @ W.T @ V, rtol=1e-12, atol=1e-12)
        G4 = np.linalg.matrix_power(G, 4)
        assert np.allclose(L.mvm(V, mode=2), W @ G4 @ W.T @ V, rtol=1e-12, atol=1e-12)
        U = rng.standard_normal((60, 3))
        assert abs((U * L.mvm(V)).sum() - (V * L.mvm(U)).sum()) < 1e-12 * np.abs(
            (U * L.mvm(V)).sum())


def _explicit_operator(L):
    """W and the per-direction shift matrices built from the exported keys with a
    Python dict (independent of the oracle's neighbour search)."""
    e = L.export()
    keys, D = e["keys"], L.D
    lut = {tuple(k): i for i, k in enumerate(keys)}
    W = sp.csr_matrix((e["w"].ravel(), (np.repeat(np.arange(L.n), D), e["idx"].ravel())),
                      shape=(L.n, L.m))
    shifts = []
    for j in range(D):
        u = -np.ones(D, int)
        u[j] += D
        rows, cols = [], []
        for v in range(L.m):
            t = lut.get(tuple(keys[v] + u))
            if t is not None:
                rows.append(v)
                cols.append(t)
        shifts.append(sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(L.m, L.m)))
    return W, shifts


@pytest.mark.parametrize("n,d,gen", [(300, 2, "u"), (400, 3, "g"), (300, 5, "g"),
                                     (250, 11, "g")])
def test_explicit_direction_products(n, d, gen):
    X = synth.uniform_points(n, d, 3) if gen == "u" else synth.gmm_points(n, d, 3)
    L = OracleLattice(X, np.full(d, 0.5, np.float32))
    W, S = _explicit_operator(L)
    V = synth.gaussian_values(n, 2, 4).astype(np.float64)

    def seq(taps, order, x):
        for j in order:
            x = taps[0] * x + taps[1] * (S[j] @ x + S[j].T @ x)
        return x

    c, g, D = L.coef, L.half, L.D
    fwd = W @ seq(c, range(D), W.T @ V)
    bwd = W @ seq(c, range(D - 1, -1, -1), W.T @ V)
    sym = W @ seq(g, range(D - 1, -1, -1), seq(g, range(D), W.T @ V))
    assert np.allclose(L.mvm(V, mode=0), fwd, rtol=1e-12, atol=1e-12)
    assert np.allclose(L.mvm(V, mode=1), bwd, rtol=1e-12, atol=1e-12)
    assert np.allclose(L.mvm(V, mode=2), sym, rtol=1e-12, atol=1e-12)
    # stages separately: splat is W^T, slice is W
    assert np.allclose(L.splat(V), W.T @ V, rtol=1e-13, atol=1e-13)
    lat = np.random.default_rng(1).standard_normal((L.m, 2))
    assert np.allclose(L.slice(lat), W @ lat, rtol=1e-13, atol=1e-13)
    assert np.allclose(L.blur(lat), seq(c, range(D), lat), rtol=1e-12, atol=1e-12)


def test_radius_two_blur_uses_two_step_neighbours():
    X = synth.gmm_points(300, 3, 11)
    L = OracleLattice(X, np.full(3, 0.4, np.float32), kind=RBF_COVERAGE, r=2)
    e = L.export()
    keys, D = e["keys"], L.D
    lut = {tuple(k): i for i, k in enumerate(keys)}
    lat = np.random.default_rng(2).standard_normal((L.m, 1))
    x = lat.copy()
    for j in range(D):
        u = -np.ones(D, int)
        u[j] += D
        y = L.coef[0] * x
        for v in range(L.m):
            for t in (1, 2):
                for sgn in (1, -1):
                    w = lut.get(tuple(keys[v] + sgn * t * u))
                    if w is not None:
                        y[v] += L.coef[t] * x[w]
        x = y
    assert np.allclose(L.blur(lat), x, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3, 8])
def test_adjoint_and_symmetry(d):
    X = synth.gmm_points(400, d, 5)
    L = OracleLattice(X, np.ones(d, np.float32))
    U = synth.gaussian_values(400, 3, 1).astype(np.float64)
    V = synth.gaussian_values(400, 3, 2).astype(np.float64)
    a = (U * L.mvm(V, 0)).sum()
    b = (V * L.mvm(U, 1)).sum()
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)
    a = (U * L.mvm(V, 2)).sum()
    b = (V * L.mvm(U, 2)).sum()
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)


def test_symmetric_operator_is_positive_semidefinite():
    X = synth.gmm_points(250, 4, 6)
    L = OracleLattice(X, np.ones(4, np.float32))
    K = L.mvm(np.eye(250), mode=2)
    assert np.abs(K - K.T).max() < 1e-13 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() > -1e-12 * np.abs(K).max()


def test_alpha_beta_epilogue():
    X = synth.gmm_points(200, 3, 8)
    L = OracleLattice(X, np.ones(3, np.float32))
    V = synth.gaussian_values(200, 2, 3).astype(np.float64)
    assert np.allclose(L.mvm(V, 0, alpha=2.5, beta=0.3), 2.5 * L.mvm(V, 0) + 0.3 * V,
                       rtol=1e-14, atol=1e-14)
