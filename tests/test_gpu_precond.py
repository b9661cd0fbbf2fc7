"""GPU preconditioned CG (shifted rank-l Nystrom preconditioner, App. A) against the oracle.

The sketch is the same counter-based Rademacher matrix on both sides and the subspace
iteration reaches the same subspace (the GPU takes its basis by Cholesky QR, the oracle
by Householder QR; the approximation depends only on the subspace).  The GPU forms the
factor from three-part bf16 panels with tensor-core (tcgen05) products, stores it rounded
to bf16, and estimates the smallest captured eigenvalue by inverse power iteration; the
oracle keeps it in fp64 and takes the eigenvalue from a dense eigensolver, so the two
preconditioners differ slightly and the iterates are compared through what does not
depend on that: each solve reaches its tolerance, the true residual of the GPU's answer
under the oracle's FP64 operator is within 1.5 x tol, and the iteration counts stay close
to the oracle's preconditioned count and below the unpreconditioned one.
"""

import numpy as np
import pytest
import torch

from oracle import OracleLattice
from paper_2106_06695_gb300 import synth

pytestmark = pytest.mark.gpu


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,d,k,rank,q", [(3000, 5, 4, 100, 1), (5000, 6, 9, 64, 0),
                                          (4000, 3, 16, 100, 1), (4000, 4, 20, 48, 1),
                                          (6000, 6, 5, 200, 1), (2500, 3, 17, 130, 0)])
def test_pcg_converges_like_the_oracle(n, d, k, rank, q):
    from paper_2106_06695_gb300.lattice import Lattice

    X = synth.gmm_points(n, d, 19)
    ls = np.ones(d, np.float32)
    ref = OracleLattice(X, ls)
    lat = Lattice(gpu(X), gpu(ls), precond_rank=rank, precond_seed=11, spacing=ref.s,
                  precond_power_iters=q)
    B = synth.solve_rhs(X, 19, probes=k - 1)
    tol, noise = 1e-3, 0.01
    xg, ig, rg = lat.cg(gpu(B), noise=noise, tol=tol, max_iter=500)
    Bd = B.astype(np.float64)
    _, io, ro, tau = ref.pcg_shifted(Bd, noise, rank=rank, tol=tol, max_iter=500, seed=11,
                                     power_iters=q)
    _, ic, rc = ref.cg(Bd, noise, tol=tol, max_iter=500, mode=2)
    R = Bd - ref.mvm(xg.cpu().numpy().astype(np.float64), mode=2, beta=noise)
    true_rel = np.linalg.norm(R, axis=0) / np.linalg.norm(Bd, axis=0)
    print("pcg iters gpu", ig, "oracle", io, "plain cg", ic, "tau", tau,
          "true rel", true_rel.max())
    assert (rg <= tol).all()
    assert (true_rel <= 1.5 * tol).all()
    assert (ig <= 1.3 * io + 3).all()
    assert (ig < ic).all()


@pytest.mark.parametrize("n,d,k,rank", [(40, 3, 4, 8), (300, 4, 3, 256), (129, 2, 16, 64),
                                       (70, 5, 5, 128)])
def test_pcg_on_tiny_and_ragged_systems(n, d, k, rank):
    """Fewer rows than one 128-row tile or one 64-row chunk, a rank close to n (C may be
    singular: the shifted Cholesky then either succeeds or the solve falls back to plain
    CG), and a rank equal to n's tile: every solve stops at its tolerance and its answer
    has the oracle's residual."""
    from paper_2106_06695_gb300.lattice import Lattice

    X = synth.gmm_points(n, d, 23)
    ls = np.ones(d, np.float32)
    ref = OracleLattice(X, ls)
    lat = Lattice(gpu(X), gpu(ls), precond_rank=rank, precond_seed=5, spacing=ref.s)
    B = synth.solve_rhs(X, 23, probes=k - 1)
    tol = 1e-4
    xg, ig, rg = lat.cg(gpu(B), noise=0.01, tol=tol, max_iter=500)
    Bd = B.astype(np.float64)
    R = Bd - ref.mvm(xg.cpu().numpy().astype(np.float64), mode=2, beta=0.01)
    true_rel = np.linalg.norm(R, axis=0) / np.linalg.norm(Bd, axis=0)
    assert (rg <= tol).all() and (true_rel <= 3 * tol).all(), (ig, rg, true_rel)


def test_pcg_rank_validation_and_noise_free_fallback():
    from paper_2106_06695_gb300 import SGPError
    from paper_2106_06695_gb300.lattice import Lattice

    X = synth.gmm_points(2000, 4, 3)
    with pytest.raises(SGPError, match="INVALID_ARG"):
        Lattice(gpu(X), 1.0, precond_rank=4097)
    with pytest.raises(SGPError, match="INVALID_ARG"):
        Lattice(gpu(X), 1.0, precond_rank=16, precond_power_iters=2)
    lat = Lattice(gpu(X), 1.0, precond_rank=32)
    B = gpu(synth.solve_rhs(X, 3, probes=1))
    # noise 0: the preconditioner needs noise > 0, the solve runs unpreconditioned
    _, it, rel = lat.cg(B, noise=0.0, tol=1e-2, max_iter=50)
    assert (it >= 1).all() and np.isfinite(rel).all()


def test_pooled_memory_is_reused_and_trimmed():
    """The library's pool keeps the blocks a solve frees; a second solve on the same handle
    gives bitwise the same answer, and so does one after the pool is trimmed."""
    from paper_2106_06695_gb300.lattice import Lattice, trim_memory

    n, d, k = 30000, 5, 8
    X = gpu(synth.gmm_points(n, d, 41))
    B = gpu(synth.gaussian_values(n, k, 41))
    lat = Lattice(X, gpu(np.ones(d, np.float32)), precond_rank=128, precond_seed=3)
    x1, it1, _ = lat.cg(B, noise=0.01, tol=1e-4, max_iter=300)
    x2, it2, _ = lat.cg(B, noise=0.01, tol=1e-4, max_iter=300)
    trim_memory()
    x3, it3, _ = lat.cg(B, noise=0.01, tol=1e-4, max_iter=300)
    assert torch.equal(x1, x2) and torch.equal(x1, x3)
    assert np.array_equal(it1, it2) and np.array_equal(it1, it3)
    lat.close()
    trim_memory()
