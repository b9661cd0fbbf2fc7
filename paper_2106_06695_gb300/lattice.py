"""Python handle for the sm_103a Simplex-GP lattice (Sec. 3.2; Eq. ski_to_bf).

Argument marshalling only: tensors are passed to libsgp.so as device pointers, with the
current torch CUDA stream, and every step of the path runs in the library's kernels.
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import BLURS, GRADS, KERNELS, VALUE_DTYPES, check


def _f32_cuda(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float32:
        raise TypeError("%s must be float32" % name)
    return t.contiguous()


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class Lattice:
    """Permutohedral lattice of the rows of X (n x d) scaled by ARD lengthscales.

    kernel: "rbf_binomial" (default; stencil [.5, 1, .5] at order 1), "rbf_coverage" or
    "matern32_coverage" (spacing from Eq. balance_coverage); order: stencil order r;
    precond_rank: rank of the CG's Nystrom preconditioner (0 = plain CG; App. A uses 100);
    precond_power_iters: subspace iterations of its sketch (0 or 1).
    """

    def __init__(self, X: torch.Tensor, lengthscales, order: int = 1,
                 kernel: str = "rbf_binomial", spacing: float = 0.0, outputscale: float = 1.0,
                 value_dtype: str = "f32", check_every: int = 8, precond_rank: int = 0,
                 precond_seed: int = 0, precond_power_iters: int = 1):
        self._lib = _lib.load()
        X = _f32_cuda(X, "X")
        if X.dim() != 2:
            raise ValueError("X must be [n, d]")
        n, d = X.shape
        if not isinstance(lengthscales, torch.Tensor):
            lengthscales = torch.full((d,), float(lengthscales), dtype=torch.float32)
        ls = lengthscales.to(device=X.device, dtype=torch.float32).reshape(-1)
        if ls.numel() == 1:
            ls = ls.expand(d)
        ls = ls.contiguous()
        self.device = X.device
        self.n, self.d = int(n), int(d)
        opts = _lib.sgp_opts()
        self._lib.sgp_opts_init(ctypes.byref(opts))
        opts.order_r = int(order)
        opts.kernel = KERNELS[kernel]
        opts.spacing_s = float(spacing)
        opts.outputscale = float(outputscale)
        opts.value_dtype = VALUE_DTYPES[value_dtype]
        opts.check_every = int(check_every)
        opts.precond_rank = int(precond_rank)
        opts.precond_seed = int(precond_seed)
        opts.precond_power_iters = int(precond_power_iters)
        opts.stream = _stream_ptr(self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self._lib.sgp_lattice_build(X.data_ptr(), ls.data_ptr(), self.n, self.d,
                                              ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        m = ctypes.c_int64()
        nbytes = ctypes.c_size_t()
        check(self._lib.sgp_lattice_info(h, ctypes.byref(m), ctypes.byref(nbytes)))
        self.m = int(m.value)
        self.order = int(order)

    # -- lifetime ---------------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.sgp_lattice_free(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _handle(self):
        if self._h is None:
            raise RuntimeError("lattice was closed")
        check(self._lib.sgp_set_stream(self._h, _stream_ptr(self.device)))
        return self._h

    # -- queries ----------------------------------------------------------------
    @property
    def device_bytes(self) -> int:
        nbytes = ctypes.c_size_t()
        check(self._lib.sgp_lattice_info(self._h, None, ctypes.byref(nbytes)))
        return int(nbytes.value)

    @property
    def sparse_blur(self) -> bool:
        """True when the blur runs on per-direction vertex lists (sgp_lattice_blur_lists)."""
        sp = ctypes.c_int()
        check(self._lib.sgp_lattice_blur_lists(self._h, ctypes.byref(sp), None))
        return bool(sp.value)

    def stencil(self):
        """(s, c[0..r], g[0..r]): spacing, paper taps and symmetric-blur taps."""
        r = ctypes.c_int()
        s = ctypes.c_double()
        c = np.zeros(8, np.float64)
        g = np.zeros(8, np.float64)
        check(self._lib.sgp_lattice_stencil(self._h, ctypes.byref(r), ctypes.byref(s),
                                            c.ctypes.data, g.ctypes.data))
        return s.value, c[: r.value + 1].copy(), g[: r.value + 1].copy()

    def export(self):
        """Host copies: keys [m][d+1] int16, idx [n][d+1] int32, w [n][d+1] float32."""
        D = self.d + 1
        keys = np.zeros((self.m, D), np.int16)
        idx = np.zeros((self.n, D), np.int32)
        w = np.zeros((self.n, D), np.float32)
        check(self._lib.sgp_lattice_export(self._handle(), keys.ctypes.data, idx.ctypes.data,
                                           w.ctypes.data))
        return dict(keys=keys, idx=idx, w=w)

    # -- operators ----------------------------------------------------------------
    def _rhs(self, V: torch.Tensor, name: str):
        V = _f32_cuda(V, name)
        squeeze = V.dim() == 1
        if squeeze:
            V = V.unsqueeze(1)
        if V.dim() != 2 or V.shape[0] != self.n:
            raise ValueError("%s must be [n] or [n, k]" % name)
        return V.contiguous(), squeeze

    def mvm(self, V: torch.Tensor, blur: str = "sequential", alpha: float = 1.0,
            beta: float = 0.0, out: torch.Tensor | None = None) -> torch.Tensor:
        """alpha * W B W^T V + beta * V (B per `blur`: sequential / transpose / symmetric)."""
        V2, squeeze = self._rhs(V, "V")
        k = V2.shape[1]
        if out is None:
            out = torch.empty_like(V2)
        check(self._lib.sgp_mvm_ex(self._handle(), V2.data_ptr(), k, BLURS[blur], float(alpha),
                                   float(beta), out.data_ptr()))
        return out.squeeze(1) if squeeze else out

    def mvm_backward(self, X: torch.Tensor, lengthscales, V: torch.Tensor, G: torch.Tensor,
                     blur: str = "sequential", alpha: float = 1.0, grad: str = "lattice",
                     want=("V", "X", "ls")):
        """(dV, dX, dls) of <G, alpha W B W^T V>: dV = alpha W B^T W^T G, and the input
        gradients through the lattice (grad="lattice": exact derivative of the product;
        grad="filter": Sec. 4.2 k'-filter estimate).  X and lengthscales are the build's."""
        G2, squeeze = self._rhs(G, "G")
        V2, _ = self._rhs(V, "V")
        k = G2.shape[1]
        X = _f32_cuda(X, "X")
        ls = lengthscales
        if not isinstance(ls, torch.Tensor):
            ls = torch.full((self.d,), float(ls), dtype=torch.float32)
        ls = ls.to(device=X.device, dtype=torch.float32).reshape(-1).expand(self.d).contiguous()
        dV = torch.empty_like(G2) if "V" in want else None
        dX = torch.empty_like(X) if "X" in want else None
        dls = torch.empty(self.d, dtype=torch.float32, device=X.device) if "ls" in want else None
        ptr = lambda t: t.data_ptr() if t is not None else None  # noqa: E731
        check(self._lib.sgp_mvm_backward(self._handle(), X.data_ptr(), ls.data_ptr(),
                                         V2.data_ptr(), G2.data_ptr(), k, BLURS[blur],
                                         float(alpha), GRADS[grad], ptr(dV), ptr(dX), ptr(dls)))
        if dV is not None and squeeze:
            dV = dV.squeeze(1)
        return dV, dX, dls

    def logdet(self, Z: torch.Tensor, noise: float, max_lanczos: int = 100, tol: float = 1e-6):
        """Stochastic Lanczos quadrature estimate of log det(outputscale K~ + noise I) with
        the probe columns Z ([n, s]); returns (estimate, per-probe quadratures)."""
        Z2, _ = self._rhs(Z, "Z")
        s = Z2.shape[1]
        quad = np.zeros(s, np.float64)
        out = ctypes.c_double()
        check(self._lib.sgp_logdet(self._handle(), Z2.data_ptr(), s, float(noise),
                                   int(max_lanczos), float(tol), ctypes.byref(out),
                                   quad.ctypes.data))
        return out.value, quad

    def cg(self, B: torch.Tensor, noise: float, tol: float = 1e-3, max_iter: int = 500,
           blur: str = "symmetric", out: torch.Tensor | None = None, history: bool = False):
        """Batched CG on (outputscale K~ + noise I) X = B; returns (X, iters, rel_res), and
        with history=True also the [max_iter, k] relative residual after every iteration
        (NaN where a column had stopped)."""
        B2, squeeze = self._rhs(B, "B")
        k = B2.shape[1]
        if out is None:
            out = torch.empty_like(B2)
        iters = np.zeros(k, np.int32)
        rel = np.zeros(k, np.float64)
        if history:
            hist = np.zeros((max(int(max_iter), 1), k), np.float64)
            check(self._lib.sgp_cg_solve_history(
                self._handle(), B2.data_ptr(), k, BLURS[blur], float(noise), float(tol),
                int(max_iter), out.data_ptr(), iters.ctypes.data, rel.ctypes.data,
                hist.ctypes.data))
            return (out.squeeze(1) if squeeze else out), iters, rel, hist[:int(max_iter)]
        check(self._lib.sgp_cg_solve_ex(self._handle(), B2.data_ptr(), k, BLURS[blur],
                                        float(noise), float(tol), int(max_iter), out.data_ptr(),
                                        iters.ctypes.data, rel.ctypes.data))
        return (out.squeeze(1) if squeeze else out), iters, rel


class _LatticeMVM(torch.autograd.Function):
    """out = alpha W B W^T V on the lattice of (X, lengthscales), with the hand-written
    backward of sgp_mvm_backward for V, X and the lengthscales."""

    @staticmethod
    def forward(ctx, X, lengthscales, V, order, kernel, blur, alpha, grad, value_dtype):
        lat = Lattice(X.detach(), lengthscales.detach(), order=order, kernel=kernel,
                      value_dtype=value_dtype)
        out = lat.mvm(V.detach(), blur=blur, alpha=alpha)
        ctx.lat, ctx.blur, ctx.alpha, ctx.grad = lat, blur, alpha, grad
        ctx.save_for_backward(X, lengthscales, V)
        return out

    @staticmethod
    def backward(ctx, gout):
        X, ls, V = ctx.saved_tensors
        want = tuple(name for name, need in zip(("X", "ls", "V"), ctx.needs_input_grad[:3])
                     if need)
        dV, dX, dls = ctx.lat.mvm_backward(X.detach(), ls.detach(), V.detach(),
                                           gout.contiguous(), blur=ctx.blur, alpha=ctx.alpha,
                                           grad=ctx.grad, want=want)
        ctx.lat.close()
        if dls is not None:
            dls = dls.reshape(ls.shape) if ls.numel() == dls.numel() else dls.sum().reshape(ls.shape)
        return dX, dls, dV, None, None, None, None, None, None


def lattice_mvm(X: torch.Tensor, lengthscales: torch.Tensor, V: torch.Tensor, order: int = 1,
                kernel: str = "rbf_binomial", blur: str = "symmetric", alpha: float = 1.0,
                grad: str = "lattice", value_dtype: str = "f32") -> torch.Tensor:
    """Differentiable lattice MVM alpha K~(X / lengthscales) V (Sec. 3.2) for fp32 CUDA
    tensors; gradients flow to X, lengthscales and V through the library's backward."""
    if not isinstance(lengthscales, torch.Tensor):
        lengthscales = torch.full((X.shape[1],), float(lengthscales), dtype=torch.float32,
                                  device=X.device)
    return _LatticeMVM.apply(X, lengthscales, V, order, kernel, blur, alpha, grad, value_dtype)


def trim_memory() -> None:
    """Return the library's unused pooled device blocks on the current device to the driver
    (sgp_trim_memory; the pool otherwise keeps freed blocks mapped for the next call)."""
    check(_lib.load().sgp_trim_memory())
