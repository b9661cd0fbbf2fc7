"""The hand-written MVM backward on the GPU against the oracle (through the C-ABI):
dV (the transpose product), dX and dls by the exact lattice derivative and by the
Sec. 4.2 filter, the torch.autograd.Function, BF16 storage, and the n = 500k, d = 20
workload (correlated Gaussian points, ARD lengthscales, k = 8)."""

import numpy as np
import pytest
import torch

from oracle import OracleLattice
from oracle.oracle import filter_gradient
from paper_2106_06695_gb300 import SGPError, synth
from paper_2106_06695_gb300.lattice import Lattice, lattice_mvm

pytestmark = pytest.mark.gpu

MODE = {"sequential": 0, "transpose": 1, "symmetric": 2}
# fp32 products (~1e-6 relative) enter dw; dy takes differences of dw over a point's
# vertices and dz sums d of them: 1e-4 relative L2 leaves an order of magnitude margin
# over the measured errors.
DV_TOL, DX_TOL = 1e-5, 1e-4
# The Sec. 4.2 filter subtracts filtered columns that all carry each point's own (large)
# self-contribution, e.g. z_n (g_n . (K v)_n) - g_n . (K (v z))_n; where the operator is
# nearly diagonal (d = 20 here) those terms exceed their difference by ~1e3, which turns
# the fp32 rounding of the filtered columns (~1e-7) into ~1e-4 of the result.
FILTER_TOL = 1e-3

CASES = [(3000, 3, 1, "sequential"), (4000, 8, 8, "symmetric"), (2500, 20, 12, "transpose"),
         (2000, 5, 3, "symmetric"), (1500, 11, 16, "sequential")]


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problem(n, d, k, seed=7):
    X, ls = synth.correlated_points(n, d, seed)
    V = synth.gaussian_values(n, k, seed + 1)
    G = synth.gaussian_values(n, k, seed + 2)
    return X, ls, V, G


@pytest.mark.parametrize("n,d,k,blur", CASES)
def test_lattice_gradient_matches_oracle(n, d, k, blur):
    X, ls, V, G = problem(n, d, k)
    lat = Lattice(gpu(X), gpu(ls))
    dV, dX, dls = lat.mvm_backward(gpu(X), gpu(ls), gpu(V), gpu(G), blur=blur, alpha=1.3)
    ref = OracleLattice(X, ls)
    rdV, rdX, rdls = ref.mvm_backward(V.astype(np.float64), G.astype(np.float64),
                                      mode=MODE[blur], alpha=1.3)
    e = (rel(dV, rdV), rel(dX, rdX), rel(dls, rdls))
    print("n=%d d=%d k=%d %s: dV %.1e dX %.1e dls %.1e" % ((n, d, k, blur) + e))
    assert e[0] <= DV_TOL and e[1] <= DX_TOL and e[2] <= DX_TOL


@pytest.mark.parametrize("n,d,k,blur", CASES[:4])
def test_filter_gradient_matches_oracle(n, d, k, blur):
    X, ls, V, G = problem(n, d, k, seed=11)
    lat = Lattice(gpu(X), gpu(ls))
    dV, dX, dls = lat.mvm_backward(gpu(X), gpu(ls), gpu(V), gpu(G), blur=blur, alpha=0.8,
                                   grad="filter")
    ref = OracleLattice(X, ls)
    rdX, rdls = filter_gradient(lambda M: ref.mvm(M, mode=MODE[blur]), X, ls, V, G, alpha=0.8)
    rdV = ref.mvm(G.astype(np.float64), mode=MODE[blur] if blur == "symmetric"
                  else 1 - MODE[blur], alpha=0.8)
    e = (rel(dV, rdV), rel(dX, rdX), rel(dls, rdls))
    print("filter n=%d d=%d k=%d %s: dV %.1e dX %.1e dls %.1e" % ((n, d, k, blur) + e))
    assert e[0] <= DV_TOL and e[1] <= FILTER_TOL and e[2] <= FILTER_TOL


def test_autograd_function_uses_the_library_backward():
    X, ls, V, G = problem(3000, 6, 4, seed=3)
    Xt, lt, Vt = gpu(X).requires_grad_(), gpu(ls).requires_grad_(), gpu(V).requires_grad_()
    out = lattice_mvm(Xt, lt, Vt, blur="symmetric", alpha=0.9)
    (out * gpu(G)).sum().backward()
    lat = Lattice(gpu(X), gpu(ls))
    assert torch.equal(out.detach(), lat.mvm(gpu(V), blur="symmetric", alpha=0.9))
    dV, dX, dls = lat.mvm_backward(gpu(X), gpu(ls), gpu(V), gpu(G), blur="symmetric", alpha=0.9)
    assert torch.equal(Vt.grad, dV) and torch.equal(Xt.grad, dX) and torch.equal(lt.grad, dls)
    # only the requested gradients: V alone
    Vt2 = gpu(V).requires_grad_()
    (lattice_mvm(gpu(X), gpu(ls), Vt2) * gpu(G)).sum().backward()
    assert Vt2.grad is not None


def test_bf16_values_backward_error():
    X, ls, V, G = problem(4000, 8, 8, seed=5)
    outs = []
    for dt in ("f32", "bf16"):
        lat = Lattice(gpu(X), gpu(ls), value_dtype=dt)
        outs.append(lat.mvm_backward(gpu(X), gpu(ls), gpu(V), gpu(G), blur="symmetric"))
    for name, a, b in zip(("dV", "dX", "dls"), outs[1], outs[0]):
        err = rel(a, b.cpu().numpy())
        print("bf16 lattice values: %s rel L2 %.2e vs fp32" % (name, err))
        assert err <= 3e-2


def test_filter_is_rejected_for_matern():
    X, ls, V, G = problem(500, 3, 2)
    lat = Lattice(gpu(X), gpu(ls), kernel="matern32_coverage")
    with pytest.raises(SGPError):
        lat.mvm_backward(gpu(X), gpu(ls), gpu(V), gpu(G), grad="filter")
    dV, dX, dls = lat.mvm_backward(gpu(X), gpu(ls), gpu(V), gpu(G))  # the exact one works
    assert torch.isfinite(dX).all()


def test_full_size_c3_backward():
    """n = 500,000, d = 20: <dV, V> = <G, out> (the transpose identity, any size), finite
    input gradients, and the timing of forward + backward."""
    n, d, k = 500_000, 20, 8
    X, ls, V, G = problem(n, d, k, seed=17)
    Xd, ld, Vd, Gd = gpu(X), gpu(ls), gpu(V), gpu(G)
    lat = Lattice(Xd, ld)
    out = lat.mvm(Vd, blur="symmetric")
    dV, dX, dls = lat.mvm_backward(Xd, ld, Vd, Gd, blur="symmetric")
    lhs = (dV.double() * Vd.double()).sum().item()
    rhs = (Gd.double() * out.double()).sum().item()
    assert abs(lhs - rhs) <= 1e-5 * abs(rhs)
    assert torch.isfinite(dX).all() and torch.isfinite(dls).all()
    for grad in ("lattice", "filter"):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lat.mvm_backward(Xd, ld, Vd, Gd, blur="symmetric", grad=grad)
        e1.record()
        torch.cuda.synchronize()
        print("n=%d d=%d k=%d m=%d: backward (%s) %.1f ms" % (n, d, k, lat.m, grad,
                                                           e0.elapsed_time(e1)))
