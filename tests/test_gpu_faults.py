"""Failure detection without a GPU fault: host-injected faults (SGP_FAULT) take the
library's error paths and leave the context usable, a request past its deadline is
cancelled with SGP_ERR_TIMEOUT without disturbing the others, and a build whose hash
table runs out of bounded probes reports SGP_ERR_HASH_FULL."""

import numpy as np
import pytest
import torch

from paper_2106_06695_gb300 import SGPError, synth
from paper_2106_06695_gb300.lattice import Lattice
from paper_2106_06695_gb300.serve import Server

pytestmark = pytest.mark.gpu


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("fault,status", [("oom", 2), ("cuda_err", 6), ("hash_full", 4),
                                          ("nan_input", 5)])
def test_injected_faults_return_their_status(monkeypatch, fault, status):
    X = synth.gmm_points(3000, 4, 1)  # at lengthscale 0.3: m = 8556 > the 1024-slot table
    monkeypatch.setenv("SGP_FAULT", fault)
    with pytest.raises(SGPError) as e:
        Lattice(gpu(X), 0.3)
    assert e.value.status == status
    monkeypatch.delenv("SGP_FAULT")
    lat = Lattice(gpu(X), 0.3)  # the context is still usable
    out = lat.mvm(gpu(np.ones((3000, 2))))
    assert torch.isfinite(out).all()


def test_request_past_its_deadline_is_cancelled():
    reqs = synth.serving_stream(3, 4, n_range=(3000, 6000), dims=(3, 8), test_points=32)
    # tol 0: every request runs all 4000 iterations unless cancelled
    with Server(max_active=4, tol=0.0, max_iter=4000) as srv:
        slow = srv.submit(reqs[0]["X"], reqs[0]["y"], reqs[0]["Xs"], reqs[0]["lengthscales"],
                          seed=reqs[0]["seed"], timeout_s=0.05)
        srv.run_until_idle()
        st = srv.stats(slow)
        assert st["done"] == 1 and st["status"] == 7
        assert srv.info()["bytes_in_use"] == 0
        with pytest.raises(SGPError):
            srv.result(slow)
    # a queued request whose deadline has passed before admission
    with Server(max_active=1, tol=1e-3) as srv:
        a = srv.submit(reqs[1]["X"], reqs[1]["y"], reqs[1]["Xs"], reqs[1]["lengthscales"],
                       seed=reqs[1]["seed"])
        b = srv.submit(reqs[2]["X"], reqs[2]["y"], reqs[2]["Xs"], reqs[2]["lengthscales"],
                       seed=reqs[2]["seed"], arrival_us=0.0, timeout_s=1e-6)
        srv.run_until_idle()
        assert srv.stats(a)["status"] == 0 and srv.stats(b)["status"] == 7
        mean_a, _ = srv.result(a)
    with Server(max_active=1, tol=1e-3) as srv:  # the survivor is unaffected
        a2 = srv.submit(reqs[1]["X"], reqs[1]["y"], reqs[1]["Xs"], reqs[1]["lengthscales"],
                        seed=reqs[1]["seed"])
        srv.run_until_idle()
        assert np.array_equal(srv.result(a2)[0], mean_a)


def test_served_preconditioner_wait_that_gives_up_voids_only_its_round(monkeypatch):
    """The bounded bulk-copy waits of the serving preconditioner's ring kernels, made to give
    up: SGP_FAULT=ring_wait (read when the server is created) runs the first lane round that
    applies a preconditioner with a wait limit of 0 polls.  Its first chunk wait gives up at
    once; the block waits (bounded, at the normal limit) for its copies in flight and
    returns.  The round's requests complete with SGP_ERR_CUDA, the lane's error word is
    cleared (the next rounds complete normally), and the same requests submitted again on
    that server give results bitwise equal to a fresh server's.  Nothing faults or hangs:
    every copy that was issued lands before its block exits."""
    from oracle import gp_posterior

    reqs = synth.serving_stream(3, 77, n_range=(8000, 12000), dims=(3,), test_points=32)
    kw = dict(max_active=4, tol=1e-5, max_iter=2000)

    def run(srv):
        ids = [srv.submit(r["X"], r["y"], r["Xs"], r["lengthscales"], seed=r["seed"])
               for r in reqs]
        srv.run_until_idle()
        return ids

    with Server(**kw) as fresh:
        ids = run(fresh)
        want = [tuple(a.copy() for a in fresh.result(i)) for i in ids]
        ranks = [fresh.stats(i)["precond_rank"] for i in ids]
    assert all(r > 0 for r in ranks)  # d = 3, n ~ 1e4: condition estimates far above 1e3
    monkeypatch.setenv("SGP_FAULT", "ring_wait")
    srv = Server(**kw)
    monkeypatch.delenv("SGP_FAULT")
    with srv:
        ids = run(srv)
        status = [srv.stats(i)["status"] for i in ids]
        assert 6 in status and set(status) <= {0, 6}, status
        for i, s, w in zip(ids, status, want):
            if s == 0:  # joined the lane after the injected round
                got = srv.result(i)
                assert all(np.array_equal(g, v) for g, v in zip(got, w))
        ids = run(srv)
        for i, w in zip(ids, want):
            assert srv.stats(i)["status"] == 0
            got = srv.result(i)
            assert all(np.array_equal(g, v) for g, v in zip(got, w))
        assert srv.info()["bytes_in_use"] == 0
    r = reqs[0]
    m_ref, _, _, _ = gp_posterior(r["X"], r["y"], r["Xs"], r["lengthscales"], r["noise"],
                                  probes=8, seed=r["seed"], tol=1e-5, max_iter=2000,
                                  precond_rank=ranks[0])
    assert np.linalg.norm(want[0][0] - m_ref) / np.linalg.norm(m_ref) <= 1e-3
