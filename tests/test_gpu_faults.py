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
