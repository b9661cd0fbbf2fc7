"""Stochastic Lanczos quadrature of log det(outputscale K~ + noise I) on the GPU against
the oracle's (same probes, same iteration cap) and against a dense log-determinant."""

import numpy as np
import pytest
import torch

from oracle import OracleLattice, rademacher_sketch
from paper_2106_06695_gb300 import SGPError, synth
from paper_2106_06695_gb300.lattice import Lattice

pytestmark = pytest.mark.gpu


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("n,d,noise", [(3000, 3, 0.05), (4000, 8, 0.01), (2000, 20, 0.01)])
def test_quadratures_match_oracle(n, d, noise):
    X = synth.gmm_points(n, d, 6)
    Z = rademacher_sketch(n, 16, 3).astype(np.float32)
    lat = Lattice(gpu(X), 1.0)
    est, quads = lat.logdet(gpu(Z), noise=noise, max_lanczos=100, tol=1e-6)
    ref = OracleLattice(X, np.ones(d, np.float32))
    est_ref, q_ref = ref.logdet(Z.astype(np.float64), noise, max_lanczos=100, tol=1e-6)
    err = np.abs(quads - q_ref).max() / np.abs(q_ref).max()
    print("n=%d d=%d: logdet %.6e (oracle %.6e), worst probe rel %.1e"
          % (n, d, est, est_ref, err))
    assert err <= 1e-3
    assert est == pytest.approx(est_ref, rel=1e-4)


def test_estimate_against_dense_log_determinant():
    """n = 1200: the 64-probe estimate lies within 4 standard errors of slogdet."""
    n, d, noise = 1200, 3, 0.05
    X = synth.gmm_points(n, d, 2)
    ref = OracleLattice(X, np.ones(d, np.float32))
    A = ref.mvm(np.eye(n), mode=2, beta=noise)
    sign, exact = np.linalg.slogdet(A)
    assert sign > 0
    Z = rademacher_sketch(n, 64, 7).astype(np.float32)
    est, quads = Lattice(gpu(X), 1.0).logdet(gpu(Z), noise=noise, max_lanczos=100, tol=1e-7)
    se = quads.std(ddof=1) / np.sqrt(len(quads))
    print("logdet estimate %.4f, exact %.4f, standard error %.4f" % (est, exact, se))
    assert abs(est - exact) <= 4 * se + 1e-3 * abs(exact)


def test_argument_checks():
    X = synth.gmm_points(200, 3, 1)
    lat = Lattice(gpu(X), 1.0)
    with pytest.raises(SGPError):
        lat.logdet(gpu(np.ones((200, 2))), noise=0.1, max_lanczos=0)
