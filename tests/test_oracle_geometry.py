"""Pins of the oracle's splat geometry (Sec. 3.2 "Splat", Eq. canon_simplex).

Everything here is checked against something other than the oracle itself: the
canonical simplex written out by hand, a brute-force search over all candidate
simplices around a point, the barycentric reconstruction of the point, and the
orthonormality of the elevation.
"""

import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import OracleLattice
from paper_2106_06695_gb300 import synth


def canonical(d):
    D = d + 1
    return np.array([[k] * (D - k) + [k - D] * k for k in range(D)], np.int64)


def test_canonical_simplex_golden(golden):
    rows = golden("canonical_simplex.txt")
    assert np.array_equal(canonical(2), np.array(rows[0:3], np.int64))
    assert np.array_equal(canonical(3), np.array(rows[3:7], np.int64))


@pytest.mark.parametrize("d", [1, 2, 3, 5, 11, 20])
def test_origin_has_canonical_vertices(d):
    L = OracleLattice(np.zeros((1, d), np.float32), np.ones(d, np.float32))
    e = L.export()
    assert L.m == d + 1
    assert np.array_equal(e["keys"], canonical(d))
    assert np.array_equal(e["idx"][0], np.arange(d + 1))
    assert np.array_equal(e["w"][0], np.eye(d + 1)[0])


@pytest.mark.parametrize("d", [1, 2, 3, 4, 7, 11, 20])
def test_elevation_is_scaled_isometry_into_hyperplane(d):
    rng = np.random.default_rng(d)
    s = 1.3
    scale = math.sqrt(d * (d + 1)) / s
    Z = rng.standard_normal((20, d))
    Y = np.stack([oracle.elevate(z, s) for z in Z])
    assert np.allclose(Y.sum(1), 0.0, atol=1e-12 * np.abs(Y).max())
    # Gram matrices agree: E has orthonormal columns and one lattice step is s units.
    assert np.allclose(Y @ Y.T, scale ** 2 * (Z @ Z.T), rtol=1e-12, atol=1e-10)
    # triangular basis: z = e_0 maps onto (1, -1, 0, ...) * scale / sqrt(2)
    y0 = oracle.elevate(np.eye(d)[0], s)
    expect = np.zeros(d + 1)
    expect[0], expect[1] = 1.0, -1.0
    assert np.allclose(y0, expect * scale / math.sqrt(2.0), rtol=1e-14)


def _brute_force_simplices(y, d):
    """All simplices rem0 + permuted canonical simplex around y with non-negative
    barycentric coordinates of y."""
    D = d + 1
    base = np.floor(y / D).astype(int)
    ranges = [range(b - 1, b + 3) for b in base]
    S = canonical(d)
    found = []
    for a in itertools.product(*ranges):
        if sum(a) != 0:
            continue
        rem0 = D * np.array(a)
        for perm in itertools.permutations(range(D)):
            verts = rem0[None, :] + S[:, perm]
            A = np.vstack([verts[:, :d].T.astype(float), np.ones(D)])
            rhs = np.concatenate([y[:d], [1.0]])
            w = np.linalg.solve(A, rhs)
            if w.min() >= -1e-12:
                found.append((verts, w))
    return found


@pytest.mark.parametrize("d", [1, 2, 3])
def test_enclosing_simplex_brute_force(d):
    rng = np.random.default_rng(100 + d)
    D = d + 1
    checked = 0
    for _ in range(40):
        y = 4.0 * D * rng.standard_normal(D)
        y -= y.mean()
        hits = _brute_force_simplices(y, d)
        if len(hits) != 1:  # on a shared face: more than one valid simplex
            continue
        verts, w = hits[0]
        got = oracle.simplex(y)
        # vertex k is the one whose coordinates are all k mod D
        order = [int(v[0] % D) for v in verts]
        want = np.zeros_like(verts)
        want_w = np.zeros(D)
        for row, k in enumerate(order):
            want[k] = verts[row]
            want_w[k] = w[row]
        assert np.array_equal(got["keys"], want)
        assert np.allclose(got["w"], want_w, atol=1e-12)
        checked += 1
    assert checked >= 30


@pytest.mark.parametrize("n,d,seed", [(500, 2, 1), (500, 3, 2), (400, 8, 3), (300, 11, 4),
                                      (200, 20, 5)])
def test_barycentric_reconstruction_and_key_invariants(n, d, seed):
    X = synth.gmm_points(n, d, seed)
    L = OracleLattice(X, np.full(d, 0.7, np.float32))
    e = L.export()
    D = d + 1
    w, idx, keys, y = e["w"], e["idx"], e["keys"], e["y"]
    assert L.m <= n * D
    assert np.allclose(w.sum(1), 1.0, atol=1e-12)
    assert w.min() >= -1e-12
    assert (keys.sum(1) == 0).all()
    assert ((keys % D) == (keys[:, :1] % D)).all()  # one remainder class per vertex
    vk = keys[idx]  # [n][D][D]: coordinates of vertex k of point i
    assert (vk[:, :, 0] % D == np.arange(D)[None, :]).all()
    recon = np.einsum("ik,ikc->ic", w, vk.astype(np.float64))
    assert np.allclose(recon, y, rtol=0, atol=1e-10 * max(1.0, np.abs(y).max()))
    # vertex k minus the remainder-0 vertex is s_k with permuted coordinates
    S = np.sort(canonical(d), axis=1)
    diff = np.sort(vk - vk[:, :1, :], axis=2)
    assert (diff == S[None]).all()
    assert len({tuple(r) for r in keys}) == L.m


def test_lattice_points_and_ties():
    d, D = 3, 4
    # a remainder-0 lattice point: rem0 is the point, ranks follow the coordinate index
    y = np.array([D, -D, 0, 0], np.float64)
    got = oracle.simplex(y)
    assert np.array_equal(got["rem0"], y.astype(int))
    assert np.array_equal(got["rank"], np.arange(D))
    assert np.array_equal(got["w"], np.eye(D)[0])
    # equal residuals: the lower index gets the smaller rank
    y = np.array([1.0, 1.0, -1.0, -1.0])
    got = oracle.simplex(y)
    assert np.array_equal(got["rank"], [0, 1, 2, 3])
    # a coordinate exactly half way between multiples of D rounds down
    y = np.array([2.0, -2.0, 0.5, -0.5])
    got = oracle.simplex(y)
    assert got["w"].min() >= 0 and abs(got["w"].sum() - 1) < 1e-15
    recon = got["w"] @ got["keys"]
    assert np.allclose(recon, y, atol=1e-14)


def test_first_occurrence_ids_and_permutation():
    X = synth.gmm_points(300, 5, 9)
    L = OracleLattice(X, np.ones(5, np.float32))
    e = L.export()
    first = e["idx"].ravel()
    # ids appear for the first time in increasing order
    seen = -1
    for v in first:
        if v > seen:
            assert v == seen + 1
            seen = v
    perm = np.random.default_rng(0).permutation(300)
    L2 = OracleLattice(X[perm], np.ones(5, np.float32))
    e2 = L2.export()
    assert {tuple(k) for k in e["keys"]} == {tuple(k) for k in e2["keys"]}
    assert np.array_equal(e["keys"][e["idx"][perm]], e2["keys"][e2["idx"]])
    V = synth.gaussian_values(300, 2, 1).astype(np.float64)
    assert np.allclose(L.mvm(V)[perm], L2.mvm(V[perm]), rtol=1e-12, atol=1e-12)
