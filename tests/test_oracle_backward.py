"""Pins of the oracle's MVM backward (Sec. 3.2) and of the Sec. 4.2 filter gradient.

The exact derivative is checked against central finite differences of the FP64 forward:
the product is linear in V (exact differences), and within one configuration of simplices
it is quadratic in the points (exact central differences); steps are powers of two so
that the perturbed fp32 inputs are exact, and a check counts only when the perturbation
left every point's vertex keys unchanged (across a simplex boundary the vertex set, and
with it the blurred values, jump).  The filter gradient's algebra is checked with the dense
kernel in place of the lattice, where it must equal the analytic dense gradient."""

import numpy as np
import pytest

from oracle import OracleLattice
from oracle.oracle import filter_gradient
from paper_2106_06695_gb300 import synth

H = 2.0 ** -14


def problem(n, d, k, seed):
    X, ls = synth.correlated_points(n, d, seed)
    X = X.astype(np.float64)
    ls = ls.astype(np.float64)
    V = synth.gaussian_values(n, k, seed + 1).astype(np.float64)
    G = synth.gaussian_values(n, k, seed + 2).astype(np.float64)
    return X, ls, V, G


def loss_and_ids(X, ls, V, G, mode, alpha):
    """Loss and the lattice structure (every point's vertex keys) it was computed on."""
    L = OracleLattice(X.astype(np.float32), ls.astype(np.float32))
    ex = L.export()
    return float((G * L.mvm(V, mode=mode, alpha=alpha)).sum()), ex["keys"][ex["idx"]]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_dV_is_the_transpose_product(mode):
    X, ls, V, G = problem(120, 3, 2, 1)
    L = OracleLattice(X.astype(np.float32), ls.astype(np.float32))
    dV, _, _ = L.mvm_backward(V, G, mode=mode, alpha=0.7)
    for i, c in [(3, 0), (50, 1), (119, 0)]:
        e = np.zeros_like(V)
        e[i, c] = 1.0
        fd = ((G * L.mvm(V + e, mode=mode, alpha=0.7)).sum()
              - (G * L.mvm(V - e, mode=mode, alpha=0.7)).sum()) / 2.0
        assert dV[i, c] == pytest.approx(fd, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("d,mode,alpha", [(2, 0, 1.0), (3, 2, 1.3), (5, 1, 0.8), (8, 2, 1.0)])
def test_dX_and_dls_match_central_differences(d, mode, alpha):
    X, ls, V, G = problem(150, d, 3, 2 + d)
    X = X.astype(np.float32).astype(np.float64)  # exact fp32 values, so X +- H is exact
    ls = ls.astype(np.float32).astype(np.float64)
    L = OracleLattice(X.astype(np.float32), ls.astype(np.float32))
    _, dX, dls = L.mvm_backward(V, G, mode=mode, alpha=alpha)
    ex = L.export()
    base = ex["keys"][ex["idx"]]
    checked = 0
    for i in (0, 37, 99, 149):
        for j in range(d):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, j] += H
            Xm[i, j] -= H
            (a, ia), (b, ib) = (loss_and_ids(Xp, ls, V, G, mode, alpha),
                                loss_and_ids(Xm, ls, V, G, mode, alpha))
            if not (ia.shape == base.shape and ib.shape == base.shape and (ia == base).all()
                    and (ib == base).all()):
                continue  # the step crossed a simplex boundary: not a smooth piece
            fd = (a - b) / (2 * H)
            assert abs(dX[i, j] - fd) <= 1e-6 * max(1.0, abs(fd))
            checked += 1
    assert checked >= 3 * d
    for j in range(d):
        lp, lm = ls.copy(), ls.copy()
        lp[j] += H
        lm[j] -= H
        (a, ia), (b, ib) = loss_and_ids(X, lp, V, G, mode, alpha), loss_and_ids(X, lm, V, G, mode, alpha)
        if ia.shape == base.shape and ib.shape == base.shape and (ia == base).all() and (
                ib == base).all():
            fd = (a - b) / (2 * H)
            assert abs(dls[j] - fd) <= 1e-5 * max(1.0, abs(fd))


def dense_rbf_grads(X, ls, V, G, alpha):
    """Analytic gradients of <G, alpha K V>, K_ij = exp(-|z_i - z_j|^2 / 2), z = x / l."""
    Z = X / ls
    diff = Z[:, None, :] - Z[None, :, :]
    D2 = diff ** 2
    K = np.exp(-0.5 * D2.sum(-1))
    W = alpha * (G @ V.T) * K
    dls = (W[:, :, None] * D2).sum((0, 1)) / ls
    dX = -((W + W.T)[:, :, None] * diff).sum(1) / ls
    return K, dX, dls


def test_filter_gradient_algebra_is_exact_with_the_dense_kernel():
    X, ls, V, G = problem(200, 4, 3, 9)
    K, dX0, dls0 = dense_rbf_grads(X, ls, V, G, 1.7)
    dX, dls = filter_gradient(lambda M: K @ M, X, ls, V, G, alpha=1.7)
    assert np.abs(dX - dX0).max() <= 1e-12 * np.abs(dX0).max()
    assert np.abs(dls - dls0).max() <= 1e-12 * np.abs(dls0).max()


def cos(a, b):
    a, b = a.ravel(), b.ravel()
    return float(a @ b / np.linalg.norm(a) / np.linalg.norm(b))


@pytest.mark.parametrize("mode", [0, 2])
def test_lattice_gradients_track_the_dense_kernel_gradient_at_low_d(mode):
    """Both lattice gradients against the exact RBF gradient on n = 2000, d = 3 (the
    lattice's own approximation error; measured cosines 0.83-0.99; dls has only d = 3
    entries, so its cosine is the noisier one)."""
    X, ls, V, G = problem(2000, 3, 8, 3)
    L = OracleLattice(X.astype(np.float32), ls.astype(np.float32))
    _, dX0, dls0 = dense_rbf_grads(X, ls, V, G, 1.0)
    _, dXl, dlsl = L.mvm_backward(V, G, mode=mode)
    dXf, dlsf = filter_gradient(lambda M: L.mvm(M, mode=mode), X, ls, V, G)
    print("mode %d: lattice derivative cos dX %.3f dls %.3f; Sec. 4.2 filter cos dX %.3f "
          "dls %.3f" % (mode, cos(dXl, dX0), cos(dlsl, dls0), cos(dXf, dX0), cos(dlsf, dls0)))
    assert cos(dXf, dX0) >= 0.95 and cos(dlsf, dls0) >= 0.8
    assert cos(dXl, dX0) >= 0.85 and cos(dlsl, dls0) >= 0.9


def test_dX_and_dls_match_central_differences_on_the_d20_workload_subsample():
    """The differentiation workload's own dimension: a seeded n = 2,000 subsample of the
    n = 500,000, d = 20 correlated-Gaussian points with their ARD lengthscales, symmetric
    blur, k = 2.  Central differences with steps that keep every vertex key (within one
    configuration of simplices the loss is quadratic in the points, so they are exact).
    A lengthscale step moves all 2,000 points and crosses some simplex boundary almost
    every time at d = 20, so dls counts only where it did not (its formula is pinned at
    d = 2..8 above)."""
    Xf, lsf = synth.correlated_points(500_000, 20, 3)
    rows = synth.subsample(500_000, 2000, 3)
    X = Xf[rows].astype(np.float64)
    ls = lsf.astype(np.float64)
    V = synth.gaussian_values(2000, 2, 4).astype(np.float64)
    G = synth.gaussian_values(2000, 2, 5).astype(np.float64)
    d, mode, alpha = 20, 2, 1.0
    L = OracleLattice(X.astype(np.float32), ls.astype(np.float32))
    _, dX, dls = L.mvm_backward(V, G, mode=mode, alpha=alpha)
    ex = L.export()
    base = ex["keys"][ex["idx"]]
    checked = 0
    for i in (0, 1999):
        for j in range(d):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, j] += H
            Xm[i, j] -= H
            (a, ia), (b, ib) = (loss_and_ids(Xp, ls, V, G, mode, alpha),
                                loss_and_ids(Xm, ls, V, G, mode, alpha))
            if not (ia.shape == base.shape and ib.shape == base.shape and (ia == base).all()
                    and (ib == base).all()):
                continue
            fd = (a - b) / (2 * H)
            assert abs(dX[i, j] - fd) <= 1e-6 * max(1.0, abs(fd))
            checked += 1
    assert checked >= d
    checked = 0
    for j in range(d):
        lp, lm = ls.copy(), ls.copy()
        lp[j] += H
        lm[j] -= H
        (a, ia), (b, ib) = loss_and_ids(X, lp, V, G, mode, alpha), loss_and_ids(X, lm, V, G, mode, alpha)
        if ia.shape == base.shape and ib.shape == base.shape and (ia == base).all() and (
                ib == base).all():
            fd = (a - b) / (2 * H)
            assert abs(dls[j] - fd) <= 1e-5 * max(1.0, abs(fd))
            checked += 1
    print("d = 20: %d of %d lengthscale steps kept every vertex key" % (checked, d))
