"""Pins of the oracle's rank-l Nystrom preconditioner and preconditioned CG (App. A: CG
pre-conditioner of rank 100)."""

import os

import numpy as np
import pytest

import oracle
from oracle import OracleLattice
from paper_2106_06695_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def test_splitmix64_reference_outputs():
    want = [int(l, 16) for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    got = oracle.splitmix64(np.array([1, 2, 3], np.uint64), seed=0)
    assert [int(v) for v in got] == want


def test_rademacher_sketch_is_balanced_and_reproducible():
    om = oracle.rademacher_sketch(4000, 50, seed=7)
    assert set(np.unique(om)) == {-1.0, 1.0}
    assert abs(om.mean()) < 0.01
    assert np.array_equal(om, oracle.rademacher_sketch(4000, 50, seed=7))
    assert not np.array_equal(om, oracle.rademacher_sketch(4000, 50, seed=8))
    # row i of a larger sketch with the same l is the same row
    assert np.array_equal(om[:100], oracle.rademacher_sketch(100, 50, seed=7))


@pytest.fixture(scope="module")
def small():
    X = synth.gmm_points(400, 4, 41)
    L = OracleLattice(X, np.ones(4, np.float32))
    A = L.mvm(np.eye(400), mode=2)
    return L, A


def test_nystrom_factor_matches_its_definition(small):
    L, A = small
    noise, rank = 0.05, 30
    Bm, Q = L.nystrom(rank, noise, seed=3)
    om = oracle.rademacher_sketch(400, rank, 3)
    Y = A @ om + 1e-3 * noise * om
    nys = Y @ np.linalg.solve(om.T @ Y, Y.T)  # Y C^-1 Y^T
    assert np.allclose(Bm @ Bm.T, 0.5 * (nys + nys.T), rtol=1e-8, atol=1e-8 * np.abs(nys).max())
    assert np.allclose(Q @ Q.T, noise * np.eye(rank) + Bm.T @ Bm, rtol=1e-12, atol=1e-10)


def test_woodbury_apply_is_the_inverse_of_p(small):
    L, A = small
    noise = 0.05
    Bm, Q = L.nystrom(30, noise, seed=3)
    P = Bm @ Bm.T + noise * np.eye(400)
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0
    R = np.random.default_rng(0).standard_normal((400, 3))
    assert np.allclose(OracleLattice.nystrom_apply(Bm, Q, noise, R), np.linalg.solve(P, R),
                       rtol=1e-8, atol=1e-8)


def test_nystrom_is_exact_for_low_rank_operators():
    # a lattice with fewer vertices than the sketch rank: A has rank <= m < l
    X = (np.random.default_rng(5).standard_normal((300, 2)) * 0.3).astype(np.float32)
    L = OracleLattice(X, np.ones(2, np.float32))
    assert L.m < 40
    A = L.mvm(np.eye(300), mode=2)
    Bm, _ = L.nystrom(40, 1.0, seed=1)
    # B B^T approximates A + nu I restricted to the sketch's range: exact on A's range
    err = np.linalg.norm(Bm @ Bm.T - A) / np.linalg.norm(A)
    assert err < 1e-2


def test_pcg_solves_the_same_system_in_fewer_iterations():
    X = synth.gmm_points(600, 5, 43)
    L = OracleLattice(X, np.ones(5, np.float32))
    B = synth.solve_rhs(X, 43, probes=2).astype(np.float64)
    noise = 0.01
    A = L.mvm(np.eye(600), mode=2) + noise * np.eye(600)
    exact = np.linalg.solve(A, B)
    xp, ip, rp = L.pcg(B, noise, rank=50, tol=1e-8, max_iter=2000)
    xc, ic, rc = L.cg(B, noise, tol=1e-8, max_iter=2000, mode=2)
    assert (rp <= 1e-8).all() and (rc <= 1e-8).all()
    assert (ip < ic).all()
    assert np.allclose(xp, exact, rtol=0, atol=1e-5 * np.abs(exact).max())
    true_rel = np.linalg.norm(B - A @ xp, axis=0) / np.linalg.norm(B, axis=0)
    assert np.allclose(true_rel, rp, rtol=1e-3, atol=1e-12)


def test_pcg_columns_edge_cases():
    """The preconditioned CG's start rule, as the device applies it: a zero right-hand
    side gives x = 0 with no iterations, tol >= 1 or max_iter = 0 run none, and an
    identity preconditioner reproduces plain CG's iterates and counts."""
    from oracle.oracle import _cg_columns, _pcg_columns

    rng = np.random.default_rng(4)
    M = rng.standard_normal((30, 30))
    A = M @ M.T + 30 * np.eye(30)
    B = rng.standard_normal((30, 3))
    B[:, 1] = 0.0
    apply_A = lambda V: A @ V  # noqa: E731
    X, it, rel = _pcg_columns(apply_A, B, lambda R: R.copy(), 1e-10, 200)
    assert it[1] == 0 and np.all(X[:, 1] == 0.0) and rel[1] == 0.0
    assert np.allclose(A @ X, B, atol=1e-8)
    Xc, itc, _ = _cg_columns(apply_A, B, 1e-10, 200)
    assert np.array_equal(it, itc) and np.allclose(X, Xc, atol=1e-12)
    for tol, mi in ((1.0, 200), (1e-10, 0)):
        X0, it0, rel0 = _pcg_columns(apply_A, B, lambda R: R.copy(), tol, mi)
        assert np.all(it0 == 0) and np.all(X0 == 0.0)
        assert np.array_equal(rel0, np.where(np.linalg.norm(B, axis=0) > 0, 1.0, 0.0))


# ---- the shifted large-rank preconditioner (library CG) --------------------------------
def test_nystrom_shifted_matches_its_definition(small):
    """B B^T = Y C^-1 Y^T with C = Q^T Y (+ the small diagonal shift), Q = Omega without
    power iteration and an orthonormal basis of A Omega with one; tau is the smallest
    eigenvalue of B^T B plus the noise; Minv = (tau I + B^T B)^-1."""
    L, A = small
    noise, rank = 0.05, 30
    for q in (0, 1):
        Bm, tau, Minv = oracle.nystrom_shifted(lambda V: A @ V, 400, rank, noise, seed=3,
                                               power_iters=q, rel_shift=0.0)
        om = oracle.rademacher_sketch(400, rank, 3)
        Q = om if q == 0 else np.linalg.qr(A @ om)[0]
        Y = A @ Q
        nys = Y @ np.linalg.solve(0.5 * (Q.T @ Y + Y.T @ Q), Y.T)
        assert np.allclose(Bm @ Bm.T, nys, rtol=1e-7, atol=1e-7 * np.abs(nys).max())
        G = Bm.T @ Bm
        assert abs(tau - noise - np.linalg.eigvalsh(G)[0]) <= 1e-10 * np.linalg.norm(G)
        assert np.allclose(Minv @ (tau * np.eye(rank) + G), np.eye(rank), atol=1e-8)


def test_nystrom_shifted_apply_is_the_inverse_of_p(small):
    L, A = small
    noise = 0.05
    Bm, tau, Minv = oracle.nystrom_shifted(lambda V: A @ V, 400, 30, noise, seed=3)
    P = Bm @ Bm.T + tau * np.eye(400)
    R = np.random.default_rng(0).standard_normal((400, 3))
    assert np.allclose(oracle.nystrom_shifted_apply(Bm, tau, Minv, R), np.linalg.solve(P, R),
                       rtol=1e-8, atol=1e-8)


def test_nystrom_shifted_on_a_low_rank_operator_converges_at_once():
    """When the operator's rank is below the sketch rank the approximation is exact on its
    range, tau = noise (B^T B has zero eigenvalues), P = A exactly up to the shift, and
    preconditioned CG stops after one or two iterations; a dropped term or a wrong sign
    in P^-1 would not."""
    X = (np.random.default_rng(5).standard_normal((300, 2)) * 0.3).astype(np.float32)
    L = OracleLattice(X, np.ones(2, np.float32))
    assert L.m < 40
    B = synth.solve_rhs(X, 5, probes=2).astype(np.float64)
    _, it, rel, tau = L.pcg_shifted(B, 0.01, rank=40, tol=1e-6, seed=1, power_iters=0)
    assert abs(tau - 0.01) < 1e-6
    assert (rel <= 1e-6).all() and (it <= 3).all()


def test_nystrom_shifted_pcg_beats_plain_cg_and_solves_the_system():
    X = synth.gmm_points(600, 5, 43)
    L = OracleLattice(X, np.ones(5, np.float32))
    B = synth.solve_rhs(X, 43, probes=2).astype(np.float64)
    noise = 0.01
    A = L.mvm(np.eye(600), mode=2) + noise * np.eye(600)
    exact = np.linalg.solve(A, B)
    _, ic, _ = L.cg(B, noise, tol=1e-8, max_iter=2000, mode=2)
    for q in (0, 1):
        xp, ip, rp, tau = L.pcg_shifted(B, noise, rank=50, tol=1e-8, max_iter=2000, power_iters=q)
        assert (rp <= 1e-8).all() and (ip < ic).all()
        assert np.allclose(xp, exact, rtol=0, atol=1e-5 * np.abs(exact).max())
    # one power iteration captures the top of the spectrum better: fewer iterations
    _, i0, _, _ = L.pcg_shifted(B, noise, rank=50, tol=1e-8, max_iter=2000, power_iters=0)
    _, i1, _, _ = L.pcg_shifted(B, noise, rank=50, tol=1e-8, max_iter=2000, power_iters=1)
    assert i1.sum() <= i0.sum()


def test_oracle_threads_are_bit_identical():
    """The multi-threaded oracle computes every output with the same operations in the same
    order as the single-threaded one: builds, products in all three blur modes and CG
    histories are bitwise equal."""
    X = synth.gmm_points(3000, 6, 47)
    B = synth.solve_rhs(X, 47, probes=3).astype(np.float64)
    out = {}
    try:
        for t in (1, 4):
            oracle.set_threads(t)
            L = OracleLattice(X, np.ones(6, np.float32))
            e = L.export()
            prods = [L.mvm(B, mode=m, beta=0.01) for m in (0, 1, 2)]
            _, it, rel, hist = L.cg(B, 0.01, tol=1e-4, max_iter=40, mode=2, history=True)
            out[t] = (e, prods, it, hist)
    finally:
        oracle.set_threads(1)
    a, b = out[1], out[4]
    assert all(np.array_equal(a[0][k], b[0][k]) for k in a[0])
    assert all(np.array_equal(p, q) for p, q in zip(a[1], b[1]))
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3], equal_nan=True)


def test_cg_history_matches_the_final_residual_and_stops_with_nan():
    X = synth.gmm_points(800, 4, 49)
    L = OracleLattice(X, np.ones(4, np.float32))
    B = synth.solve_rhs(X, 49, probes=2).astype(np.float64)
    _, it, rel, hist = L.cg(B, 0.05, tol=1e-3, max_iter=300, mode=2, history=True)
    for c in range(B.shape[1]):
        assert hist[it[c] - 1, c] == rel[c]
        assert np.isnan(hist[it[c]:, c]).all() and np.isfinite(hist[:it[c], c]).all()
