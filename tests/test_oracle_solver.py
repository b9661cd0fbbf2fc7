"""Pins of the oracle's CG solve (Sec. 2; App. A table: max 500 iterations) and of the
exact RBF MVM used for the approximation report (Sec. 3.1, Sec. 5.1 cosine error)."""

import numpy as np
import pytest
from scipy.spatial.distance import cdist

from oracle import OracleLattice, dense_rbf
from paper_2106_06695_gb300 import synth


@pytest.mark.parametrize("n,d,noise", [(300, 3, 0.05), (400, 6, 0.01)])
def test_cg_matches_dense_solve(n, d, noise):
    X = synth.gmm_points(n, d, 21)
    L = OracleLattice(X, np.ones(d, np.float32))
    B = synth.solve_rhs(X, 21, probes=3).astype(np.float64)
    A = L.mvm(np.eye(n), mode=2) + noise * np.eye(n)
    exact = np.linalg.solve(A, B)
    tol = 1e-6
    Xs, iters, rel = L.cg(B, noise, tol=tol, max_iter=2000, mode=2)
    assert (rel <= tol).all()
    assert (iters <= 2 * n).all()
    true_rel = np.linalg.norm(B - A @ Xs, axis=0) / np.linalg.norm(B, axis=0)
    assert (true_rel <= 10 * tol).all()
    cond = np.linalg.cond(A)
    err = np.linalg.norm(Xs - exact, axis=0) / np.linalg.norm(exact, axis=0)
    assert (err <= 10 * tol * cond).all()
    assert (err <= 1e-3).all()


def test_cg_stops_at_tolerance_and_caps_iterations():
    X = synth.gmm_points(500, 4, 22)
    L = OracleLattice(X, np.ones(4, np.float32))
    B = synth.solve_rhs(X, 22, probes=2).astype(np.float64)
    B[:, 2] = 0.0  # a zero right-hand side needs no iteration
    Xs, iters, rel = L.cg(B, 0.01, tol=1e-3, max_iter=500, mode=2)
    assert iters[2] == 0 and rel[2] == 0 and not Xs[:, 2].any()
    assert (rel[:2] <= 1e-3).all()
    A = lambda V: L.mvm(V, mode=2, beta=0.01)  # noqa: E731
    true_rel = np.linalg.norm(B[:, :2] - A(Xs[:, :2]), axis=0) / np.linalg.norm(B[:, :2], axis=0)
    assert np.allclose(true_rel, rel[:2], rtol=1e-6)
    Xc, it_c, rel_c = L.cg(B, 0.01, tol=1e-12, max_iter=7, mode=2)
    assert (it_c[:2] == 7).all() and (rel_c[:2] > 1e-12).all()
    # the first 7 iterations are the same iterations
    Xd, it_d, _ = L.cg(B, 0.01, tol=1e-12, max_iter=7, mode=2)
    assert np.array_equal(Xc, Xd)


def test_dense_rbf_matches_scipy_distances():
    X = synth.gmm_points(150, 5, 23)
    ls = np.array([0.5, 1.0, 2.0, 0.7, 1.3], np.float32)
    V = synth.gaussian_values(150, 2, 23).astype(np.float64)
    Z = X.astype(np.float64) / ls.astype(np.float64)
    K = np.exp(-0.5 * cdist(Z, Z, "sqeuclidean"))
    assert np.allclose(dense_rbf(X, ls, V), K @ V, rtol=1e-12, atol=1e-12)


def test_small_workload_approximation_report():
    """n=4096, d=3, X ~ U[0,1]^3, lengthscale 0.3, binomial stencil: the cosine error
    of Sec. 5.1 against the exact MVM.  The paper's figure values are lost, so this is
    a reported figure with a loose sanity bound, not a parity pin."""
    X = synth.uniform_points(4096, 3, 1)
    ls = np.full(3, 0.3, np.float32)
    V = synth.gaussian_values(4096, 1, 1).astype(np.float64)
    L = OracleLattice(X, ls)
    exact = dense_rbf(X, ls, V)
    for mode in (0, 2):
        z = L.mvm(V, mode=mode)
        cos_err = 1 - (z * exact).sum() / np.linalg.norm(z) / np.linalg.norm(exact)
        assert cos_err < 0.05
