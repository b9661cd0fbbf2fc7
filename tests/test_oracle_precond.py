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
