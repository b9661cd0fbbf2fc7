"""Pins of the oracle's stochastic Lanczos quadrature (the log-det term of Eq. gp_mll;
App. A: at most 100 Lanczos iterations) against dense linear algebra."""

import itertools

import numpy as np
import pytest

from oracle import OracleLattice, lanczos_quadrature, rademacher_sketch
from paper_2106_06695_gb300 import synth


def dense_operator(L, noise, outputscale):
    N = L.n
    return L.mvm(np.eye(N), mode=2, alpha=outputscale, beta=noise)


def logm_quadratic(A, z):
    lam, U = np.linalg.eigh(A)
    w = U.T @ z
    return float((w ** 2) @ np.log(lam))


def test_exhaustive_probes_give_the_exact_log_determinant():
    """n = 4 points, probes = all 16 sign patterns (their mean outer product is I): with
    CG run to its exact end the estimate equals log det A."""
    X = synth.gmm_points(4, 2, 5)
    L = OracleLattice(X, np.full(2, 0.7, np.float32))
    A = dense_operator(L, 0.05, 1.3)
    Z = np.array(list(itertools.product([-1.0, 1.0], repeat=4))).T
    est, quads = lanczos_quadrature(lambda P: L.mvm(P, mode=2, alpha=1.3, beta=0.05), Z,
                                    max_iter=4, tol=1e-14)
    sign, ld = np.linalg.slogdet(A)
    assert sign > 0
    assert est == pytest.approx(ld, rel=1e-10, abs=1e-10)


@pytest.mark.parametrize("d,noise", [(2, 0.01), (4, 0.1)])
def test_each_quadrature_converges_to_the_quadratic_form(d, noise):
    X = synth.gmm_points(60, d, 8)
    L = OracleLattice(X, np.ones(d, np.float32))
    A = dense_operator(L, noise, 1.0)
    Z = rademacher_sketch(60, 3, 4)
    _, quads = L.logdet(Z, noise, max_lanczos=60, tol=1e-13)
    for c in range(3):
        assert quads[c] == pytest.approx(logm_quadratic(A, Z[:, c]), rel=1e-8)


def test_cg_coefficients_give_the_lanczos_tridiagonal():
    """T from CG's alpha/beta equals the tridiagonal of textbook Lanczos (full
    reorthogonalisation) on (A, z / ||z||) for the first steps."""
    X = synth.gmm_points(80, 3, 2)
    L = OracleLattice(X, np.ones(3, np.float32))
    A = dense_operator(L, 0.02, 1.0)
    z = rademacher_sketch(80, 1, 9)[:, 0]
    m = 8
    Qs = [z / np.linalg.norm(z)]
    alphas, betas = [], []
    for j in range(m):
        w = A @ Qs[j]
        a = Qs[j] @ w
        w = w - a * Qs[j] - (betas[-1] * Qs[j - 1] if j > 0 else 0.0)
        for q in Qs:  # full reorthogonalisation
            w -= (q @ w) * q
        alphas.append(a)
        b = np.linalg.norm(w)
        betas.append(b)
        Qs.append(w / b)
    T_lanczos = np.diag(alphas) + np.diag(betas[:m - 1], 1) + np.diag(betas[:m - 1], -1)
    from oracle.oracle import _cg_columns

    hist = {}
    _cg_columns(lambda P: A @ P, z[:, None], 0.0, m, history=hist)
    a = np.asarray(hist["alpha"][0])
    b = np.asarray(hist["beta"][0][:m - 1])
    diag = 1.0 / a
    diag[1:] += b / a[:-1]
    off = np.sqrt(b) / a[:-1]
    T_cg = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    assert np.abs(T_cg - T_lanczos).max() <= 1e-10 * np.abs(T_lanczos).max()
