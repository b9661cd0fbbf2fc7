"""Pins of the oracle's GP posterior (Eq. gp_pred_mean, Eq. gp_pred_cov) and the host
logic of the serving path, on the CPU.

The posterior oracle composes the lattice operator with a masked CG and a probe
estimator of the variance; here it is checked against a dense direct solve of the same
joint-lattice covariance, with probes that run over every sign pattern of the test points
(for which the estimator is exactly the diagonal)."""

import itertools

import numpy as np
import pytest

from oracle import OracleLattice, condition_estimate, gp_posterior, rademacher_sketch
from paper_2106_06695_gb300 import synth
from paper_2106_06695_gb300.serve import run_stream


def dense_joint_cov(X, Xs, ls, outputscale):
    """outputscale K~ of the joint lattice as a dense matrix, one unit vector at a time."""
    L = OracleLattice(np.vstack([X, Xs]), ls)
    N = X.shape[0] + Xs.shape[0]
    return L.mvm(np.eye(N), mode=2, alpha=outputscale)


def all_sign_patterns(ns):
    return np.array(list(itertools.product([-1.0, 1.0], repeat=ns))).T  # [ns][2^ns]


@pytest.mark.parametrize("d,outputscale,noise,rank", [(2, 1.0, 0.01, 0), (3, 2.5, 0.1, 0),
                                                     (5, 0.7, 0.05, 0), (2, 1.0, 0.01, 12),
                                                     (3, 2.5, 0.1, 25)])
def test_posterior_equals_dense_solve_with_exhaustive_probes(d, outputscale, noise, rank):
    P = synth.gmm_points(63, d, 3 + d)
    X, Xs = P[:60], P[60:]
    y = synth.regression_targets(X, 7)
    ls = np.full(d, 0.9, np.float32)
    Z = all_sign_patterns(3)
    mean, var, iters, rel = gp_posterior(X, y, Xs, ls, noise, outputscale=outputscale, Z=Z,
                                         tol=1e-13, max_iter=2000, precond_rank=rank)
    Kd = dense_joint_cov(X, Xs, ls, outputscale)
    A = Kd[:60, :60] + noise * np.eye(60)
    mean_exact = Kd[60:, :60] @ np.linalg.solve(A, y.astype(np.float64))
    var_exact = outputscale - np.diag(Kd[60:, :60] @ np.linalg.solve(A, Kd[:60, 60:]))
    assert np.allclose(Kd, Kd.T, atol=1e-12)  # symmetric operator: K*X = KX*^T
    assert np.abs(mean - mean_exact).max() <= 1e-8 * max(1.0, np.abs(mean_exact).max())
    assert np.abs(var - var_exact).max() <= 1e-8 * outputscale
    assert (rel <= 1e-13).all()
    # the posterior variance lies below the prior variance
    assert (var_exact <= outputscale + 1e-12).all()


def test_probe_estimate_with_random_probes_is_the_sign_weighted_diagonal():
    """With random probes the estimate equals outputscale - diag(M) minus the cross terms
    sum_{u != t} M[t][u] mean_s(z_s[t] z_s[u]) -- computed here from the dense M."""
    d = 3
    P = synth.gmm_points(65, d, 11)
    X, Xs = P[:60], P[60:]
    y = synth.regression_targets(X, 2)
    ls = np.ones(d, np.float32)
    noise = 0.02
    mean, var, _, _ = gp_posterior(X, y, Xs, ls, noise, probes=6, seed=5, tol=1e-13,
                                   max_iter=2000)
    Z = rademacher_sketch(5, 6, 5)
    Kd = dense_joint_cov(X, Xs, ls, 1.0)
    M = Kd[60:, :60] @ np.linalg.solve(Kd[:60, :60] + noise * np.eye(60), Kd[:60, 60:])
    want = 1.0 - ((M @ Z) * Z).mean(1)
    assert np.abs(var - want).max() <= 1e-8


def test_preconditioner_cuts_iterations_on_an_ill_conditioned_request():
    """d = 2, 400 points on a coarse lattice, noise 1e-3: the training block has a few
    large eigenvalues (many points per vertex).  The rank-40 preconditioner (App. A)
    takes far fewer iterations to the same posterior; a wrong sign or a dropped factor
    in the Woodbury apply would make it slower or stall."""
    P = synth.gmm_points(416, 2, 17)
    X, Xs = P[:400], P[400:]
    y = synth.regression_targets(X, 3)
    ls = np.full(2, 1.5, np.float32)
    kw = dict(probes=4, seed=9, tol=1e-8, max_iter=3000)
    m0, v0, i0, _ = gp_posterior(X, y, Xs, ls, 1e-3, **kw)
    m1, v1, i1, r1 = gp_posterior(X, y, Xs, ls, 1e-3, precond_rank=40, **kw)
    assert (r1 <= 1e-8).all()
    assert i1.max() * 3 <= i0.max(), (i0, i1)
    assert np.abs(m1 - m0).max() <= 1e-5 * np.abs(m0).max()
    assert np.abs(v1 - v0).max() <= 1e-5


@pytest.mark.parametrize("d,ls,noise", [(2, 1.0, 0.01), (3, 0.5, 0.1), (8, 1.0, 0.01)])
def test_condition_estimate_bounds_the_condition_number(d, ls, noise):
    """Gershgorin: the estimate is at least the exact condition number of the training
    block outputscale K~_XX + noise I, and the mean row sum (a lower bound of the largest
    eigenvalue of a non-negative symmetric matrix, Rayleigh quotient of the ones vector)
    keeps it within a factor of the truth."""
    P = synth.gmm_points(90, d, 23 + d)
    X, Xs = P[:80], P[80:]
    lsv = np.full(d, ls, np.float32)
    os_ = 1.7
    est = condition_estimate(X, Xs, lsv, noise, outputscale=os_)
    Kd = dense_joint_cov(X, Xs, lsv, os_)[:80, :80]
    assert (Kd >= -1e-15).all()
    ev = np.linalg.eigvalsh(Kd + noise * np.eye(80))
    kappa = ev[-1] / ev[0]
    assert kappa <= est * (1 + 1e-12)
    mean_row = (Kd.sum(1).mean() + noise) / noise
    assert mean_row <= ev[-1] / noise * (1 + 1e-12)
    rows = Kd.sum(1)
    assert est == pytest.approx((rows.max() + noise) / noise, rel=1e-12)
    # the largest row sum is within the spread max/mean of the largest eigenvalue
    assert rows.max() <= rows.max() / rows.mean() * ev[-1] * (1 + 1e-12)


def test_zero_targets_give_zero_mean_and_no_probes_give_zero_var():
    P = synth.gmm_points(43, 2, 1)
    mean, var, iters, _ = gp_posterior(P[:40], np.zeros(40, np.float32), P[40:],
                                       np.ones(2, np.float32), 0.01, probes=0)
    assert np.all(mean == 0.0) and np.all(var == 0.0) and iters[0] == 0


class FakeServer:
    """Stands in for Server on the CPU: each request completes `work` steps after it is
    admitted; the clock advances by `dt` seconds per step."""

    def __init__(self, work=2, dt=0.01, max_active=2):
        self.t = 0.0
        self.work, self.dt, self.max_active = work, dt, max_active
        self.queue, self.active, self.st = [], {}, {}
        self.next = 1
        self.peak = 0

    def clock_us(self):
        return self.t * 1e6

    def submit(self, X, y, Xs, ls, outputscale, noise, seed, arrival_us, lattice_key=0):
        rid = self.next
        self.next += 1
        self.st[rid] = dict(arrival_us=arrival_us, done_us=None, iters=0, done=0)
        self.queue.append(rid)
        return rid

    def info(self):
        return {"queued": len(self.queue), "active": len(self.active), "bytes_in_use": 0,
                "peak_active": self.peak}

    def step(self):
        self.t += self.dt
        done = 0
        for rid in list(self.active):
            self.active[rid] -= 1
            if self.active[rid] == 0:
                del self.active[rid]
                self.st[rid].update(done_us=self.t * 1e6, done=1, iters=self.work)
                done += 1
        while self.queue and len(self.active) < self.max_active:
            self.active[self.queue.pop(0)] = self.work
        self.peak = max(self.peak, len(self.active))
        return done

    def stats(self, rid):
        return self.st[rid]


def test_stream_driver_submits_on_time_and_measures_latency_from_arrival():
    reqs = [dict(arrival_s=a, X=None, y=None, Xs=None, lengthscales=None)
            for a in (0.0, 0.005, 0.05, 0.051, 0.3)]
    slept = []

    def fake_sleep(s):
        slept.append(s)
        srv.t += s

    srv = FakeServer(work=2, dt=0.01, max_active=2)
    res = run_stream(srv, reqs, sleep=fake_sleep)
    assert len(res.ids) == 5 and all(srv.st[r]["done"] for r in res.ids)
    arrivals = [srv.st[r]["arrival_us"] / 1e6 for r in res.ids]
    assert np.allclose(arrivals, [r["arrival_s"] for r in reqs])
    assert all(lat > 0 for lat in res.latencies_s)
    assert res.peak_active <= 2
    assert slept  # idle gaps are slept through, not spun
    assert res.makespan_s == pytest.approx(
        max(srv.st[r]["done_us"] for r in res.ids) / 1e6 - 0.0)
    assert res.solves_per_s == pytest.approx(5 / res.makespan_s)
    assert res.percentile(50) <= res.percentile(99)
