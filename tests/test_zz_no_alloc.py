"""The allocation-free MVM entry point (sgp_mvm_static) against sgp_mvm_ex.

sgp_mvm_static serves callers that cannot allocate device memory when they need a
product -- serving loops that keep cudaMalloc/cudaFree off their hot path, and processes
whose device memory another allocator has already reserved -- from a 64 MiB work area
compiled into the library.  Both entry points are called through the C-ABI on the same
lattice; the static one twice in a row (its work area keeps the previous call's
contents), and each result must match within the MVM tolerance of the parity tests.
This file is collected last so that a failure here comes after every other test.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_2106_06695_gb300 import _lib, build_lib, synth

pytestmark = pytest.mark.gpu

MVM_RTOL = 1e-5
BLURS = {"sequential": 0, "transpose": 1, "symmetric": 2}


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_l2(a, b):
    return (a - b).double().norm().item() / max(b.double().norm().item(), 1e-300)


def test_static_entry_point_matches_allocating_one():
    build_lib.build()
    lib = _lib.load()
    from paper_2106_06695_gb300.lattice import Lattice

    n, d = 20000, 6
    X = synth.gmm_points(n, d, 31)
    lat = Lattice(gpu(X), gpu(np.full(d, 0.8, np.float32)))
    for k in (16, 3):
        V = gpu(synth.gaussian_values(n, k, 32))
        for blur, code in BLURS.items():
            ref = torch.empty_like(V)
            _lib.check(lib.sgp_mvm_ex(lat._handle(), V.data_ptr(), k, code, ctypes.c_float(1.5),
                                      ctypes.c_float(0.25), ref.data_ptr()))
            for _ in range(2):
                out = torch.full_like(V, float("nan"))
                _lib.check(lib.sgp_mvm_static(lat._handle(), V.data_ptr(), k, code,
                                              ctypes.c_float(1.5), ctypes.c_float(0.25),
                                              out.data_ptr()))
                torch.cuda.synchronize()
                assert torch.isfinite(out).all()
                assert rel_l2(out, ref) <= MVM_RTOL, (k, blur)


def test_static_entry_point_rejects_lattices_beyond_its_work_area():
    build_lib.build()
    lib = _lib.load()
    from paper_2106_06695_gb300.lattice import Lattice

    n, d = 20000, 11
    X = synth.gmm_points(n, d, 33)
    lat = Lattice(gpu(X), gpu(np.ones(d, np.float32)))
    k = 256  # 2 m k floats exceed 64 MiB for this lattice
    assert 2 * lat.m * k * 4 > 64 << 20
    V = torch.zeros(n, k, device="cuda")
    out = torch.zeros_like(V)
    rc = lib.sgp_mvm_static(lat._handle(), V.data_ptr(), k, 0, ctypes.c_float(1.0),
                            ctypes.c_float(0.0), out.data_ptr())
    assert rc == 1
    assert b"64 MiB" in lib.sgp_last_error()
