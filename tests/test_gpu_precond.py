"""GPU preconditioned CG (rank-l Nystrom preconditioner, App. A) against the FP64 oracle.

The sketch is the same counter-based Rademacher matrix on both sides; the GPU forms the
factor B in fp32 and the oracle in fp64, so the two preconditioners differ by rounding
and their iterates are compared through what does not depend on it: each solve reaches
its tolerance, the true residual of the GPU's answer under the oracle's FP64 operator is
within 1.5 x tol, and the iteration counts stay close to the oracle's preconditioned
count and below the unpreconditioned one.
"""

import numpy as np
import pytest
import torch

from oracle import OracleLattice
from paper_2106_06695_gb300 import synth

pytestmark = pytest.mark.gpu


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,d,k,rank", [(3000, 5, 4, 100), (5000, 6, 9, 64), (4000, 3, 16, 100), (4000, 4, 20, 48)])
def test_pcg_converges_like_the_oracle(n, d, k, rank):
    from paper_2106_06695_gb300.lattice import Lattice

    X = synth.gmm_points(n, d, 19)
    ls = np.ones(d, np.float32)
    lat = Lattice(gpu(X), gpu(ls), precond_rank=rank, precond_seed=11)
    s, _, _ = lat.stencil()
    ref = OracleLattice(X, ls, spacing=s)
    B = synth.solve_rhs(X, 19, probes=k - 1)
    tol, noise = 1e-3, 0.01
    xg, ig, rg = lat.cg(gpu(B), noise=noise, tol=tol, max_iter=500)
    Bd = B.astype(np.float64)
    _, io, ro = ref.pcg(Bd, noise, rank=rank, tol=tol, max_iter=500, seed=11)
    _, ic, rc = ref.cg(Bd, noise, tol=tol, max_iter=500, mode=2)
    R = Bd - ref.mvm(xg.cpu().numpy().astype(np.float64), mode=2, beta=noise)
    true_rel = np.linalg.norm(R, axis=0) / np.linalg.norm(Bd, axis=0)
    print("pcg iters gpu", ig, "oracle", io, "plain cg", ic, "true rel", true_rel.max())
    assert (rg <= tol).all()
    assert (true_rel <= 1.5 * tol).all()
    assert (ig <= 1.3 * io + 3).all()
    assert (ig < ic).all()


def test_pcg_rank_validation_and_noise_free_fallback():
    from paper_2106_06695_gb300 import SGPError
    from paper_2106_06695_gb300.lattice import Lattice

    X = synth.gmm_points(2000, 4, 3)
    with pytest.raises(SGPError, match="INVALID_ARG"):
        Lattice(gpu(X), 1.0, precond_rank=129)
    lat = Lattice(gpu(X), 1.0, precond_rank=32)
    B = gpu(synth.solve_rhs(X, 3, probes=1))
    # noise 0: no Woodbury form exists, the solve runs unpreconditioned
    _, it, rel = lat.cg(B, noise=0.0, tol=1e-2, max_iter=50)
    assert (it >= 1).all() and np.isfinite(rel).all()
