"""Long-run CG parity: the GPU's batched CG against the FP64 oracle's over 500 iterations
(Sec. 2; App. A: at most 500 iterations).

The system has the shape of the n = 200,000 solve workload at n = 50,000 (standardised
16-component Gaussian mixture, d = 11, unit lengthscales, binomial stencil, noise 0.01,
B = [y, 8 Rademacher probes]) and is badly conditioned, so plain CG is far from
converged after 500 iterations and its residual history shows where finite precision
costs the GPU ground: the GPU multiplies in fp32 (the oracle in fp64) and carries x and r
as double-float pairs.  Both sides run with tol 0 (every column runs all 500 iterations)
and record ||r_j|| / ||b|| after every iteration.  In exact arithmetic the two histories
are the same sequence; the tests bound how far they drift apart:
  - iterations 1-10 agree to 1e-3 relative (the early Krylov steps are well determined);
  - finite precision delays convergence: the GPU reaches the residual the oracle had after
    j iterations (j = 50, 100, ..., 400) within 1.5 j iterations;
  - the GPU's final residual is its true residual under the oracle's FP64 operator, up to
    5 % and the floor the fp32 operator sets (its products differ from the FP64 operator's
    by about 1e-6 relative, so residuals near 1e-6 cannot be resolved more finely).
The same system with the shifted Nystrom preconditioner (rank 256, one power iteration)
reaches 1e-3 in at most 1.3 x the oracle's iterations (the preconditioners differ by
rounding and by the GPU's estimate of the smallest captured eigenvalue).  At the full
n = 2,000,000 size the GPU's history is compared with the oracle's stored FP64 history
(tests/golden/cg_history_n2M_d11.txt, written by tests/golden/make_cg_history.py).
"""

import os

import numpy as np
import pytest
import torch

import oracle
from oracle import OracleLattice
from paper_2106_06695_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def delays(hg, ho, its, checkpoints):
    """For each checkpoint j (an iteration of the oracle's history ho, sampled at `its`)
    and column: the first iteration at which the GPU's residual history hg (every
    iteration) is at or below the oracle's residual at j, divided by j (inf if never)."""
    out = np.zeros((len(checkpoints), hg.shape[1]))
    for a, j in enumerate(checkpoints):
        level = ho[list(its).index(j)]
        for c in range(hg.shape[1]):
            hit = np.nonzero(hg[:, c] <= level[c])[0]
            out[a, c] = (hit[0] + 1) / j if len(hit) else np.inf
    return out


@pytest.fixture(scope="module")
def system():
    oracle.set_threads(oracle.max_threads())
    n, d = 50_000, 11
    X = synth.gmm_points(n, d, 2)
    B = synth.solve_rhs(X, 2, probes=8)
    ref = OracleLattice(X, np.ones(d, np.float32))
    yield X, B, ref
    oracle.set_threads(1)


def test_plain_cg_history_tracks_the_fp64_oracle_over_500_iterations(system):
    from paper_2106_06695_gb300.lattice import Lattice

    X, B, ref = system
    lat = Lattice(gpu(X), gpu(np.ones(X.shape[1], np.float32)), spacing=ref.s)
    xg, ig, rg, hg = lat.cg(gpu(B), noise=0.01, tol=0.0, max_iter=500, history=True)
    Bd = B.astype(np.float64)
    _, io, ro, ho = ref.cg(Bd, 0.01, tol=0.0, max_iter=500, mode=2, history=True)
    assert (ig == 500).all() and (io == 500).all()
    ratio = hg / ho
    dl = delays(hg, ho, range(1, 501), [50, 100, 200, 300, 400])
    print("GPU / FP64 residual at iterations 10, 100, 250, 500:",
          np.round(ratio[[9, 99, 249, 499]].max(1), 3), "final GPU", rg.max(), "FP64", ro.max(),
          "delay ratios", np.round(dl.max(1), 3))
    assert np.abs(ratio[:10] - 1.0).max() <= 1e-3
    assert dl.max() <= 1.5
    R = Bd - ref.mvm(xg.cpu().numpy().astype(np.float64), mode=2, beta=0.01)
    true_rel = np.linalg.norm(R, axis=0) / np.linalg.norm(Bd, axis=0)
    assert np.all(np.abs(true_rel - rg) <= 0.05 * rg + 5e-6)


def test_preconditioned_cg_reaches_tol_like_the_fp64_oracle(system):
    from paper_2106_06695_gb300.lattice import Lattice

    X, B, ref = system
    lat = Lattice(gpu(X), gpu(np.ones(X.shape[1], np.float32)), spacing=ref.s,
                  precond_rank=256, precond_seed=5, precond_power_iters=1)
    xg, ig, rg, hg = lat.cg(gpu(B), noise=0.01, tol=1e-3, max_iter=500, history=True)
    Bd = B.astype(np.float64)
    _, io, ro, tau = ref.pcg_shifted(Bd, 0.01, rank=256, tol=1e-3, max_iter=500, seed=5,
                                     power_iters=1)
    print("PCG iterations GPU", ig, "oracle", io, "tau", tau)
    assert (rg <= 1e-3).all() and (ig <= 1.3 * io + 3).all()
    for c in range(B.shape[1]):
        assert hg[ig[c] - 1, c] == rg[c] and np.isnan(hg[ig[c]:, c]).all()
    R = Bd - ref.mvm(xg.cpu().numpy().astype(np.float64), mode=2, beta=0.01)
    true_rel = np.linalg.norm(R, axis=0) / np.linalg.norm(Bd, axis=0)
    assert (true_rel <= 1.5e-3).all()


def _golden_history(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            rows.append([float(t) for t in line.split()])
    a = np.array(rows)
    return a[:, 0].astype(int), a[:, 1:]


@pytest.mark.skipif(not os.path.exists(os.path.join(GOLDEN, "cg_history_n2M_d11.txt")),
                    reason="stored n = 2M FP64 history not generated")
def test_full_size_plain_cg_history_tracks_the_stored_fp64_history():
    """n = 2,000,000, d = 11, 16 N(0, 1) right-hand sides, 500 plain iterations: the GPU's
    residual at iterations 1, 10, ..., 500 against the oracle's stored FP64 history.  This
    system is so ill-conditioned that neither reaches 1e-3 (the FP64 residual ends at
    1.1-2.8); its residuals swing between ~1 and ~40 for the first hundred iterations, so
    the delay is measured from checkpoint 100 on (measured 1.18-1.27; at j = 50, inside
    that transient, 1.58)."""
    from paper_2106_06695_gb300.lattice import Lattice

    its, ho = _golden_history("cg_history_n2M_d11.txt")
    X = synth.gmm_points(2_000_000, 11, 4)
    V = synth.gaussian_values(2_000_000, 16, 4)
    ref_s = oracle.stencil(oracle.RBF_BINOMIAL, 1)[0]
    lat = Lattice(gpu(X), gpu(np.ones(11, np.float32)), spacing=ref_s)
    _, ig, rg, hg = lat.cg(gpu(V), noise=0.01, tol=0.0, max_iter=500, history=True)
    ratio = hg[its - 1] / ho
    dl = delays(hg, ho, its, [100, 200, 300, 400])
    print("n = 2M: GPU / FP64 residual at iterations", its[[0, 10, 25, 50]],
          np.round(ratio[[0, 10, 25, 50]].max(1), 3), "delay ratios", np.round(dl.max(1), 3))
    assert np.abs(ratio[0] - 1.0).max() <= 1e-3
    assert dl.max() <= 1.5
