"""Host-side logic that needs no GPU: the library's stencil solve (Sec. 4.1) against the
oracle and the closed forms, and the bench's replica aggregation over two gloo ranks."""

import ctypes
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2106_06695_gb300 import _lib, build_lib


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return _lib.load()


def lib_stencil(lib, kernel, r, spacing=0.0):
    s = ctypes.c_double()
    c = np.zeros(r + 1)
    g = np.zeros(r + 1)
    _lib.check(lib.sgp_stencil(kernel, r, spacing, ctypes.byref(s), c.ctypes.data, g.ctypes.data))
    return s.value, c, g


@pytest.mark.parametrize("kernel", [0, 1, 2])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_library_stencil_matches_oracle(lib, kernel, r):
    s, c, g = lib_stencil(lib, kernel, r)
    so, co, go = oracle.stencil(kernel, r)
    # the library integrates numerically, the oracle uses closed-form integrals
    assert abs(s - so) < 1e-7
    assert np.allclose(c, co, atol=1e-7) and np.allclose(g, go, atol=1e-7)
    s2, c2, g2 = lib_stencil(lib, kernel, r, spacing=so)
    assert s2 == so
    assert np.allclose(c2, co, rtol=0, atol=1e-15) and np.allclose(g2, go, rtol=0, atol=1e-15)


def test_library_gaussian_coverage_closed_form(lib):
    for r in (1, 2, 3):
        s, _, _ = lib_stencil(lib, 1, r)
        assert abs(s - math.sqrt(2 * math.pi / (2 * r + 1))) < 1e-7


def test_library_binomial_default(lib, golden):
    s, c, _ = lib_stencil(lib, 0, 1)
    assert np.allclose([c[1], c[0], c[1]], golden("binomial_stencil.txt")[0], atol=1e-15)


def test_stencil_rejects_bad_arguments(lib):
    s = ctypes.c_double()
    assert lib.sgp_stencil(7, 1, 0.0, ctypes.byref(s), None, None) == 1
    assert lib.sgp_stencil(0, 5, 0.0, ctypes.byref(s), None, None) == 1


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    bench.init_dist(world, "gloo")
    elapsed = 100.0 + 50.0 * rank
    units = 1000.0 * (rank + 1)
    results[rank] = bench.aggregate(elapsed, units, world)
    bench.barrier(world)
    import torch.distributed as dist

    dist.destroy_process_group()


def test_bench_replica_aggregation_two_ranks():
    with socket.socket() as sock:
        sock.bind(("127.0.0.1", 0))
        port = sock.getsockname()[1]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, results)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            assert results[r] == (150.0, 3000.0)


def test_mvm_bytes_matches_a_case_worked_by_hand():
    """The roofline's algorithmic bytes per MVM (16 n D ids and weights, 8 n k for V and
    out, 8 m k for the splatted and sliced rows, m (8 r + 8 k) per blur pass, 4 (m + 1)
    offsets), checked against n = 2M, D = 12, k = 16, r = 1, m = 1e6 worked by hand with
    one pass per direction: 0.384 + 0.256 + 0.128 + 1.632 GB + 4 MB."""
    import bench

    got = bench.mvm_bytes(2_000_000, 12, 16, 1_000_000, 1, 12)
    assert got == 384_000_000 + 256_000_000 + 128_000_000 + 1_632_000_000 + 4_000_004
    # the symmetric operator runs twice the passes; only the blur term doubles
    sym = bench.mvm_bytes(2_000_000, 12, 16, 1_000_000, 1, 24)
    assert sym - got == 1_632_000_000
