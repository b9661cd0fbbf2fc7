"""The allocation-free MVM entry point (sgp_mvm_static) against sgp_mvm_ex and the oracle.

sgp_mvm_static serves callers that cannot allocate device memory when they need a
product -- serving loops that keep cudaMalloc/cudaFree off their hot path, and processes
whose device memory another allocator has already reserved -- from a 64 MiB work area
compiled into the library.  It is called through the C-ABI on freshly built lattices
before any allocating entry point, so the handle's device bytes must not change, and
twice in a row (its work area keeps the previous call's contents).  Each result must
match sgp_mvm_ex within the MVM tolerance of the parity tests (fp32 values) or the BF16
bound (bf16 values), and the FP64 oracle within the same bound.  This file is collected
last so that a failure here comes after every other test.
"""

import ctypes

import numpy as np
import pytest
import torch

from oracle import OracleLattice
from paper_2106_06695_gb300 import _lib, build_lib, synth

pytestmark = pytest.mark.gpu

RTOL = {"f32": 1e-5, "bf16": 1e-2}
BLURS = {"sequential": 0, "transpose": 1, "symmetric": 2}


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("values", ["f32", "bf16"])
def test_static_entry_point_matches_allocating_one_and_oracle(values):
    build_lib.build()
    lib = _lib.load()
    from paper_2106_06695_gb300.lattice import Lattice

    n, d = 20000, 6
    X = synth.gmm_points(n, d, 31)
    ls = np.full(d, 0.8, np.float32)
    ref = OracleLattice(X, ls)
    lat = Lattice(gpu(X), gpu(ls), value_dtype=values, spacing=ref.s)
    h = lat._handle()
    bytes0 = lat.device_bytes
    alpha, beta = 1.5, 0.25
    results = {}
    # on the fresh handle: the static entry point first, twice per case
    for k in (16, 3):
        V = synth.gaussian_values(n, k, 32)
        Vd = gpu(V)
        for blur, code in BLURS.items():
            outs = []
            for _ in range(2):
                out = torch.full_like(Vd, float("nan"))
                _lib.check(lib.sgp_mvm_static(h, Vd.data_ptr(), k, code, ctypes.c_float(alpha),
                                              ctypes.c_float(beta), out.data_ptr()))
                torch.cuda.synchronize()
                assert torch.isfinite(out).all()
                outs.append(out.cpu().numpy())
            assert lat.device_bytes == bytes0, "sgp_mvm_static allocated lattice buffers"
            want = ref.mvm(V.astype(np.float64), mode=code, alpha=alpha, beta=beta)
            for o in outs:
                assert rel_l2(o, want) <= RTOL[values], (values, k, blur)
            results[(k, blur)] = (Vd, outs)
    # then the allocating entry point on the same handle
    for (k, blur), (Vd, outs) in results.items():
        ref_out = torch.empty_like(Vd)
        _lib.check(lib.sgp_mvm_ex(h, Vd.data_ptr(), k, BLURS[blur], ctypes.c_float(alpha),
                                  ctypes.c_float(beta), ref_out.data_ptr()))
        ref_np = ref_out.cpu().numpy().astype(np.float64)
        for o in outs:
            assert rel_l2(o, ref_np) <= RTOL[values], (values, k, blur)


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
