"""ctypes wrapper of the FP64 C++ oracle (``sgp_oracle.cpp``).

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference legs use it.  Each wrapper states the paper passage its C++
function follows; the C++ file header lists the readings and the pins.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgp_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

RBF_BINOMIAL, RBF_COVERAGE, MATERN32_COVERAGE = 0, 1, 2

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_float_p = ctypes.POINTER(ctypes.c_float)
_c_int_p = ctypes.POINTER(ctypes.c_int)


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no FMA contraction, no fast-math), with OpenMP
    when the compiler supports it (else the thread count stays 1)."""
    with _lock:
        stale = not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + ".%d.tmp" % os.getpid()
            cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
                   "-fPIC", "-shared", "-o", tmp, _SRC]
            if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:],
                              stderr=subprocess.DEVNULL).returncode != 0:
                subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = ctypes.CDLL(_LIB)
        lib.orc_stencil.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _c_double_p,
                                    _c_double_p, _c_double_p]
        lib.orc_stencil.restype = ctypes.c_int
        lib.orc_spatial_coverage.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.orc_spatial_coverage.restype = ctypes.c_double
        lib.orc_fourier_coverage.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.orc_fourier_coverage.restype = ctypes.c_double
        lib.orc_build.argtypes = [_c_float_p, _c_float_p, ctypes.c_int64, ctypes.c_int,
                                  ctypes.c_int, _c_double_p, _c_double_p, ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_void_p)]
        lib.orc_build.restype = ctypes.c_int
        lib.orc_m.argtypes = [ctypes.c_void_p]
        lib.orc_m.restype = ctypes.c_int64
        lib.orc_export.argtypes = [ctypes.c_void_p, _c_double_p, _c_int_p, _c_int_p,
                                   _c_double_p, _c_int_p, _c_int_p]
        lib.orc_export.restype = None
        lib.orc_find.argtypes = [ctypes.c_void_p, _c_int_p]
        lib.orc_find.restype = ctypes.c_int
        lib.orc_splat.argtypes = [ctypes.c_void_p, _c_double_p, ctypes.c_int, _c_double_p]
        lib.orc_splat.restype = None
        lib.orc_blur.argtypes = [ctypes.c_void_p, _c_double_p, ctypes.c_int, ctypes.c_int]
        lib.orc_blur.restype = None
        lib.orc_slice.argtypes = [ctypes.c_void_p, _c_double_p, ctypes.c_int, _c_double_p]
        lib.orc_slice.restype = None
        lib.orc_mvm.argtypes = [ctypes.c_void_p, _c_double_p, ctypes.c_int, ctypes.c_int,
                                ctypes.c_double, ctypes.c_double, _c_double_p]
        lib.orc_mvm.restype = ctypes.c_int
        lib.orc_mvm_backward.argtypes = [ctypes.c_void_p, _c_double_p, _c_double_p, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_double, _c_double_p,
                                         _c_double_p, _c_double_p]
        lib.orc_mvm_backward.restype = ctypes.c_int
        lib.orc_cg.argtypes = [ctypes.c_void_p, _c_double_p, ctypes.c_int, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                               _c_double_p, _c_int_p, _c_double_p]
        lib.orc_cg.restype = ctypes.c_int
        lib.orc_cg_history.argtypes = lib.orc_cg.argtypes + [_c_double_p]
        lib.orc_cg_history.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = ctypes.c_int
        lib.orc_max_threads.argtypes = []
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_dense_rbf.argtypes = [_c_float_p, _c_float_p, ctypes.c_int64, ctypes.c_int,
                                      _c_double_p, ctypes.c_int, _c_double_p]
        lib.orc_dense_rbf.restype = None
        lib.orc_simplex.argtypes = [_c_double_p, ctypes.c_int, _c_int_p, _c_int_p, _c_double_p,
                                    _c_int_p]
        lib.orc_simplex.restype = None
        lib.orc_elevate.argtypes = [_c_double_p, ctypes.c_int, ctypes.c_double, _c_double_p]
        lib.orc_elevate.restype = None
        lib.orc_free.argtypes = [ctypes.c_void_p]
        lib.orc_free.restype = None
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def set_threads(t: int) -> int:
    """Threads of the oracle's parallel loops (results are bit-identical for any count);
    returns the count in effect (1 when the library was built without OpenMP)."""
    return _load().orc_set_threads(int(t))


def max_threads() -> int:
    """Processors the oracle's parallel loops can use."""
    return _load().orc_max_threads()


def stencil(kind: int = RBF_BINOMIAL, r: int = 1, spacing: float = 0.0):
    """(s, c, g): spacing, the paper's taps c_t = k(t s) (Sec. 4.1, Eq. balance_coverage)
    and the symmetric-blur taps g_t of the half kernel, t = 0..r."""
    lib = _load()
    s = ctypes.c_double()
    coef = np.zeros(r + 1, np.float64)
    half = np.zeros(r + 1, np.float64)
    rc = lib.orc_stencil(kind, r, spacing, ctypes.byref(s), _p(coef, ctypes.c_double),
                         _p(half, ctypes.c_double))
    if rc != 0:
        raise ValueError("orc_stencil: invalid arguments")
    return s.value, coef, half


def splitmix64(counter, seed: int = 0) -> np.ndarray:
    """SplitMix64 (Steele, Lea & Flood 2014) output at the given counters (uint64 array):
    the mixing function applied to seed + counter * 0x9e3779b97f4a7c15."""
    c = np.asarray(counter, np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + c * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def rademacher_sketch(n: int, l: int, seed: int = 0) -> np.ndarray:
    """Omega[i][j] = -1 if the top bit of SplitMix64 at counter i l + j + 1 is set, else +1."""
    c = (np.arange(n, dtype=np.uint64)[:, None] * np.uint64(l)
         + np.arange(l, dtype=np.uint64)[None, :] + np.uint64(1))
    return np.where(splitmix64(c, seed) >> np.uint64(63), -1.0, 1.0)


def simplex(y):
    """Enclosing simplex of one elevated point y (Sec. 3.2 "Splat"): dict of rem0,
    rank, w ([D]) and keys ([D][D], vertex k in row k)."""
    y = np.ascontiguousarray(y, np.float64)
    D = y.shape[0]
    rem0 = np.zeros(D, np.int32)
    rank = np.zeros(D, np.int32)
    w = np.zeros(D, np.float64)
    keys = np.zeros((D, D), np.int32)
    _load().orc_simplex(_p(y, ctypes.c_double), D - 1, _p(rem0, ctypes.c_int),
                        _p(rank, ctypes.c_int), _p(w, ctypes.c_double), _p(keys, ctypes.c_int))
    return dict(rem0=rem0, rank=rank, w=w, keys=keys)


def elevate(z, s: float) -> np.ndarray:
    """Elevation of one normalised point z into H_d for spacing s (Sec. 3.2 "Splat")."""
    z = np.ascontiguousarray(z, np.float64)
    y = np.zeros(z.shape[0] + 1, np.float64)
    _load().orc_elevate(_p(z, ctypes.c_double), z.shape[0], s, _p(y, ctypes.c_double))
    return y


def spatial_coverage(kind: int, a: float) -> float:
    return _load().orc_spatial_coverage(kind, a)


def fourier_coverage(kind: int, w: float) -> float:
    return _load().orc_fourier_coverage(kind, w)


def dense_rbf(X: np.ndarray, ls: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Exact RBF kernel MVM (Sec. 3.1), O(n^2): for the approximation report only."""
    X = np.ascontiguousarray(X, np.float32)
    ls = np.ascontiguousarray(ls, np.float32)
    V2 = np.ascontiguousarray(V.reshape(V.shape[0], -1), np.float64)
    out = np.zeros_like(V2)
    _load().orc_dense_rbf(_p(X, ctypes.c_float), _p(ls, ctypes.c_float), X.shape[0],
                          X.shape[1], _p(V2, ctypes.c_double), V2.shape[1],
                          _p(out, ctypes.c_double))
    return out.reshape(V.shape)


class OracleLattice:
    """Permutohedral lattice of n points (Sec. 3.2) built by the FP64 oracle."""

    def __init__(self, X, ls, kind: int = RBF_BINOMIAL, r: int = 1, spacing: float = 0.0):
        lib = _load()
        self.X = np.ascontiguousarray(X, np.float32)
        self.ls = np.ascontiguousarray(np.broadcast_to(np.asarray(ls, np.float32),
                                                       (self.X.shape[1],)))
        self.n, self.d = self.X.shape
        self.D = self.d + 1
        self.r = r
        self.s, self.coef, self.half = stencil(kind, r, spacing)
        h = ctypes.c_void_p()
        rc = lib.orc_build(_p(self.X, ctypes.c_float), _p(self.ls, ctypes.c_float), self.n,
                           self.d, r, _p(self.coef, ctypes.c_double),
                           _p(self.half, ctypes.c_double), self.s, ctypes.byref(h))
        if rc != 0:
            raise ValueError("orc_build: invalid arguments")
        self._h = h
        self.m = lib.orc_m(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_free(h)
            self._h = None

    def export(self):
        """Dict of y, rem0, rank, w, idx ([n][D]) and keys ([m][D])."""
        n, D, m = self.n, self.D, self.m
        y = np.zeros((n, D), np.float64)
        rem0 = np.zeros((n, D), np.int32)
        rank = np.zeros((n, D), np.int32)
        w = np.zeros((n, D), np.float64)
        idx = np.zeros((n, D), np.int32)
        keys = np.zeros((m, D), np.int32)
        _lib.orc_export(self._h, _p(y, ctypes.c_double), _p(rem0, ctypes.c_int),
                        _p(rank, ctypes.c_int), _p(w, ctypes.c_double), _p(idx, ctypes.c_int),
                        _p(keys, ctypes.c_int))
        return dict(y=y, rem0=rem0, rank=rank, w=w, idx=idx, keys=keys)

    def find(self, key) -> int:
        key = np.ascontiguousarray(key, np.int32)
        assert key.shape == (self.D,)
        return _lib.orc_find(self._h, _p(key, ctypes.c_int))

    @staticmethod
    def _as2d(V):
        V = np.asarray(V, np.float64)
        return np.ascontiguousarray(V.reshape(V.shape[0], -1)), V.shape

    def splat(self, V):
        V2, _ = self._as2d(V)
        lat = np.zeros((self.m, V2.shape[1]), np.float64)
        _lib.orc_splat(self._h, _p(V2, ctypes.c_double), V2.shape[1], _p(lat, ctypes.c_double))
        return lat

    def blur(self, lat, transpose: bool = False):
        lat = np.array(lat, np.float64, copy=True, order="C").reshape(self.m, -1)
        _lib.orc_blur(self._h, _p(lat, ctypes.c_double), lat.shape[1], int(transpose))
        return lat

    def slice(self, lat):
        lat = np.ascontiguousarray(lat, np.float64).reshape(self.m, -1)
        out = np.zeros((self.n, lat.shape[1]), np.float64)
        _lib.orc_slice(self._h, _p(lat, ctypes.c_double), lat.shape[1], _p(out, ctypes.c_double))
        return out

    def mvm_backward(self, V, G, mode: int = 0, alpha: float = 1.0):
        """Gradients of <G, alpha K~ V> w.r.t. V ([n][k]), the points X ([n][d]) and the
        lengthscales ([d]) through the barycentric weights (Sec. 3.2)."""
        V2, _ = self._as2d(V)
        G2, _ = self._as2d(G)
        k = V2.shape[1]
        dV = np.zeros_like(V2)
        dX = np.zeros((self.n, self.d))
        dls = np.zeros(self.d)
        rc = _lib.orc_mvm_backward(self._h, _p(V2, ctypes.c_double), _p(G2, ctypes.c_double),
                                   k, mode, alpha, _p(dV, ctypes.c_double),
                                   _p(dX, ctypes.c_double), _p(dls, ctypes.c_double))
        if rc != 0:
            raise ValueError("orc_mvm_backward: invalid arguments")
        return dV, dX, dls

    def mvm(self, V, mode: int = 0, alpha: float = 1.0, beta: float = 0.0):
        """alpha K~ V + beta V; mode 0 sequential blur, 1 its transpose, 2 symmetric."""
        V2, shape = self._as2d(V)
        out = np.zeros_like(V2)
        rc = _lib.orc_mvm(self._h, _p(V2, ctypes.c_double), V2.shape[1], mode, alpha, beta,
                          _p(out, ctypes.c_double))
        if rc != 0:
            raise ValueError("orc_mvm: invalid arguments")
        return out.reshape(shape)

    def nystrom(self, rank: int, noise: float, seed: int = 0, outputscale: float = 1.0,
                mode: int = 2):
        """nystrom_factor of A = outputscale K~ on this lattice (App. A: preconditioner
        rank).  Returns B and the lower Cholesky factor Q of noise I + B^T B."""
        return nystrom_factor(lambda V: self.mvm(V, mode=mode, alpha=outputscale), self.n,
                              rank, noise, seed)

    @staticmethod
    def nystrom_apply(Bm, Q, noise: float, r):
        """P^-1 r = (r - B (noise I + B^T B)^-1 B^T r) / noise (Woodbury)."""
        return nystrom_apply(Bm, Q, noise, r)

    def pcg_shifted(self, B, noise: float, rank: int, tol: float = 1e-3, max_iter: int = 500,
                    seed: int = 0, outputscale: float = 1.0, power_iters: int = 1):
        """Preconditioned CG with the nystrom_shifted preconditioner of outputscale K~
        (symmetric blur) on (outputscale K~ + noise I) X = B, every column independent,
        stopping on ||r|| / ||b|| <= tol.  Returns X, iterations, rel. residuals, tau."""
        B2, shape = self._as2d(B)
        Bm, tau, Minv = nystrom_shifted(lambda V: self.mvm(V, mode=2, alpha=outputscale),
                                        self.n, rank, noise, seed, power_iters)
        X, iters, rel = _pcg_columns(
            lambda P: self.mvm(P, mode=2, alpha=outputscale, beta=noise), B2,
            lambda R: nystrom_shifted_apply(Bm, tau, Minv, R), tol, max_iter)
        return X.reshape(shape), iters, rel, tau

    def pcg(self, B, noise: float, rank: int, tol: float = 1e-3, max_iter: int = 500,
            seed: int = 0, outputscale: float = 1.0, mode: int = 2):
        """Preconditioned CG (P = B B^T + noise I from nystrom) on (outputscale K~ + noise I)
        X = B, every column independent, stopping on ||r|| / ||b|| <= tol."""
        B2, shape = self._as2d(B)
        Bm, Q = self.nystrom(rank, noise, seed, outputscale, mode)
        X, iters, rel = _pcg_columns(
            lambda P: self.mvm(P, mode=mode, alpha=outputscale, beta=noise), B2,
            lambda R: nystrom_apply(Bm, Q, noise, R), tol, max_iter)
        return X.reshape(shape), iters, rel

    def logdet(self, Z, noise: float, outputscale: float = 1.0, max_lanczos: int = 100,
               tol: float = 0.0):
        """lanczos_quadrature on A = outputscale K~ + noise I (symmetric blur)."""
        return lanczos_quadrature(lambda P: self.mvm(P, mode=2, alpha=outputscale, beta=noise),
                                  Z, max_lanczos, tol)

    def cg(self, B, noise: float, tol: float = 1e-3, max_iter: int = 500,
           outputscale: float = 1.0, mode: int = 0, history: bool = False):
        """CG on (outputscale K~ + noise I) X = B; returns X, iterations, rel. residuals
        (and, with history=True, the [max_iter][k] relative residual after every iteration,
        NaN where a column had stopped)."""
        B2, shape = self._as2d(B)
        k = B2.shape[1]
        X = np.zeros_like(B2)
        iters = np.zeros(k, np.int32)
        rel = np.zeros(k, np.float64)
        hist = np.full((max(max_iter, 1), k), np.nan) if history else None
        rc = _lib.orc_cg_history(self._h, _p(B2, ctypes.c_double), k, outputscale, noise, tol,
                                 max_iter, mode, _p(X, ctypes.c_double),
                                 _p(iters, ctypes.c_int), _p(rel, ctypes.c_double),
                                 _p(hist, ctypes.c_double) if history else None)
        if rc != 0:
            raise ValueError("orc_cg: invalid arguments")
        if history:
            return X.reshape(shape), iters, rel, hist[:max_iter]
        return X.reshape(shape), iters, rel


def nystrom_factor(apply_K, n: int, rank: int, noise: float, seed: int = 0):
    """Rank-l randomized Nystrom factor B of a symmetric positive semi-definite A (App. A:
    CG preconditioner of rank 100), built from products with A only: Omega = the n x l
    rademacher_sketch(n, l, seed), Y = A Omega + nu Omega (nu = 1e-3 noise keeps C
    positive definite when A Omega is rank deficient), C = Omega^T Y = R R^T,
    B = Y R^-T, so that B B^T = Y C^-1 Y^T.  apply_K maps an [n][c] array to A times it.
    Returns B and the lower Cholesky factor Q of noise I + B^T B; the preconditioner is
    P = B B^T + noise I."""
    from scipy.linalg import cholesky, solve_triangular

    om = rademacher_sketch(n, rank, seed)
    Y = apply_K(om) + 1e-3 * noise * om
    C = om.T @ Y
    R = cholesky(0.5 * (C + C.T), lower=True)
    Bm = solve_triangular(R, Y.T, lower=True).T
    Q = cholesky(noise * np.eye(rank) + Bm.T @ Bm, lower=True)
    return Bm, Q


def nystrom_shifted(apply_K, n: int, rank: int, noise: float, seed: int = 0,
                    power_iters: int = 1, rel_shift: float = 1e-6):
    """Randomized Nystrom preconditioner of large rank for A = K + noise I (App. A: CG
    pre-conditioner; the rank grows with the system's conditioning), built from products
    with the symmetric positive semi-definite K only:
      Omega   the n x l rademacher_sketch(n, l, seed);
      Q       Omega, or after `power_iters` subspace iterations an orthonormal basis of
              K^q Omega (numpy QR of each product; the approximation depends only on the
              subspace);
      Y       = K Q;  C = (Q^T Y + Y^T Q) / 2 + eps I,  eps = rel_shift max_j C_jj;
      B       = Y R^-T with C = R R^T, so that B B^T = Y C^-1 Y^T ~ K;
      tau     = lambda_min(B^T B) + noise (the smallest retained eigenvalue of the
              approximation, plus the noise);
      P       = B B^T + tau I, applied as P^-1 r = (r - B (tau I + B^T B)^-1 B^T r) / tau.
    On the captured subspace P ~ K + tau I and elsewhere P = tau I, so P^-1 A has its
    spectrum in [noise / tau, ~1]: the condition number is about tau / noise.  Returns
    (B, tau, Minv) with Minv = (tau I + B^T B)^-1."""
    from scipy.linalg import cholesky, solve_triangular

    Q = rademacher_sketch(n, rank, seed)
    for _ in range(power_iters):
        Q, _ = np.linalg.qr(apply_K(Q))
    Y = apply_K(Q)
    C = Q.T @ Y
    C = 0.5 * (C + C.T)
    C += rel_shift * np.max(np.diag(C)) * np.eye(rank)
    R = cholesky(C, lower=True)
    Bm = solve_triangular(R, Y.T, lower=True).T
    G = Bm.T @ Bm
    tau = float(np.linalg.eigvalsh(G)[0]) + noise
    Minv = np.linalg.inv(tau * np.eye(rank) + G)
    return Bm, tau, Minv


def nystrom_shifted_apply(Bm, tau: float, Minv, r):
    """P^-1 r for P = B B^T + tau I (Woodbury identity)."""
    return (r - Bm @ (Minv @ (Bm.T @ r))) / tau


def nystrom_apply(Bm, Q, noise: float, r):
    """P^-1 r = (r - B (noise I + B^T B)^-1 B^T r) / noise (Woodbury identity)."""
    from scipy.linalg import cho_solve

    return (r - Bm @ cho_solve((Q, True), Bm.T @ r)) / noise


def _pcg_columns(apply_A, B, apply_Pinv, tol: float, max_iter: int):
    """Preconditioned CG, one independent iteration per column of B: x_0 = 0, r_0 = b,
    z_0 = P^-1 r_0, p_0 = z_0; each step alpha = <r, z> / <p, A p>, x += alpha p,
    r -= alpha A p; a column stops when ||r|| / ||b|| <= tol (the unpreconditioned
    residual) or after max_iter iterations; otherwise z = P^-1 r, beta = <r, z>_new /
    <r, z>_old, p = z + beta p.  b = 0 gives x = 0."""
    n, k = B.shape
    X = np.zeros((n, k))
    r = np.array(B, np.float64, copy=True)
    z = apply_Pinv(r)
    p = z.copy()
    rho = (r * z).sum(0)
    bnorm = np.linalg.norm(B, axis=0)
    active = (bnorm > 0) & (1.0 > tol) & (max_iter > 0)
    rel = np.where(bnorm > 0, 1.0, 0.0)
    iters = np.zeros(k, np.int32)
    while active.any():
        q = apply_A(p)
        pq = (p * q).sum(0)
        for c in np.nonzero(active)[0]:
            if not pq[c] > 0:
                active[c] = False
                continue
            a = rho[c] / pq[c]
            X[:, c] += a * p[:, c]
            r[:, c] -= a * q[:, c]
            iters[c] += 1
            rel[c] = np.linalg.norm(r[:, c]) / bnorm[c]
            if rel[c] <= tol or iters[c] >= max_iter:
                active[c] = False
        if not active.any():
            break
        z = apply_Pinv(r)
        rz = (r * z).sum(0)
        for c in np.nonzero(active)[0]:
            p[:, c] = z[:, c] + (rz[c] / rho[c]) * p[:, c]
            rho[c] = rz[c]
    return X, iters, rel


def _cg_columns(apply_A, B, tol: float, max_iter: int, history=None):
    """Textbook CG (Sec. 2), one independent iteration per column of B: x_0 = 0, stop a
    column when ||r|| / ||b|| <= tol or after max_iter iterations; b = 0 gives x = 0.
    history: optional dict that receives per column the lists of step sizes alpha_j and
    ratios beta_j = <r_j+1, r_j+1> / <r_j, r_j> (the latter only while iterating on)."""
    n, k = B.shape
    X = np.zeros((n, k))
    R = B.copy()
    P = R.copy()
    bnorm = np.linalg.norm(B, axis=0)
    rho = (R * R).sum(0)
    iters = np.zeros(k, np.int32)
    rel = np.where(bnorm > 0, 1.0, 0.0)
    active = (bnorm > 0) & (1.0 > tol) & (max_iter > 0)
    if history is not None:
        history["alpha"] = [[] for _ in range(k)]
        history["beta"] = [[] for _ in range(k)]
    while active.any():
        AP = apply_A(P)
        for c in np.nonzero(active)[0]:
            pap = P[:, c] @ AP[:, c]
            if not pap > 0:
                active[c] = False
                continue
            a = rho[c] / pap
            if history is not None:
                history["alpha"][c].append(a)
            X[:, c] += a * P[:, c]
            R[:, c] -= a * AP[:, c]
            iters[c] += 1
            rr = R[:, c] @ R[:, c]
            rel[c] = np.sqrt(rr) / bnorm[c]
            if rel[c] <= tol or iters[c] >= max_iter:
                active[c] = False
                continue
            if history is not None:
                history["beta"][c].append(rr / rho[c])
            P[:, c] = R[:, c] + (rr / rho[c]) * P[:, c]
            rho[c] = rr
    return X, iters, rel


def lanczos_quadrature(apply_A, Z, max_iter: int = 100, tol: float = 0.0):
    """Stochastic Lanczos quadrature of log det A (the log-det term of Eq. gp_mll): for each
    probe z (a column of Z), CG on A x = z yields the Lanczos tridiagonal T of the Krylov
    space of z (diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal
    sqrt(beta_j)/alpha_j), and z^T log(A) z ~ ||z||^2 e1^T log(T) e1 from T's eigenvalues
    and the first components of its eigenvectors.  Returns (mean over probes, per-probe
    values)."""
    from scipy.linalg import eigh_tridiagonal

    Z = np.asarray(Z, np.float64)
    hist = {}
    _, iters, _ = _cg_columns(apply_A, Z, tol, max_iter, history=hist)
    quads = np.zeros(Z.shape[1])
    for c in range(Z.shape[1]):
        m = int(iters[c])
        if m == 0:
            continue
        a = np.asarray(hist["alpha"][c][:m])
        b = np.asarray(hist["beta"][c][:m - 1])
        diag = 1.0 / a
        diag[1:] += b / a[:-1]
        off = np.sqrt(b) / a[:-1]
        lam, Q = eigh_tridiagonal(diag, off)
        quads[c] = (Z[:, c] @ Z[:, c]) * float((Q[0] ** 2) @ np.log(lam))
    return float(quads.mean()), quads


PRECOND_SEED_XOR = 0x6A09E667F3BCC909  # sketch seed of a request = its seed XOR this


def gp_posterior(X, y, Xs, ls, noise: float, outputscale: float = 1.0, probes: int = 8,
                 seed: int = 0, tol: float = 1e-3, max_iter: int = 500,
                 kind: int = RBF_BINOMIAL, r: int = 1, Z=None, precond_rank: int = 0):
    """Posterior mean and probe-estimated variance at the test inputs Xs.

    Eq. gp_pred_mean with a zero prior mean: mean = K*X (K_XX + noise I)^-1 y, and the
    diagonal of Eq. gp_pred_cov: var = k(x, x) - diag(K*X (K_XX + noise I)^-1 KX*),
    with k(x, x) = outputscale and the second term estimated from probe vectors z_s over
    the test points, diag(M) ~ (1/S) sum_s z_s * (M z_s) (its expectation is diag(M) for
    independent +-1 entries; exact when the z_s run over all sign patterns).  Every
    covariance is the lattice operator outputscale K~ (symmetric blur) of ONE lattice
    built over the joint point set [X; Xs]: K_XX, KX* and K*X are its blocks.  Default
    probes: Z[t][s] from rademacher_sketch(ns, probes, seed).  Returns (mean, var,
    iterations per column, final relative residual per column); column 0 is y, columns
    1..S the probes.  precond_rank = l > 0 solves with _pcg_columns and the nystrom_factor
    of the training block outputscale K~_XX (App. A), its sketch over the n training rows
    drawn with seed XOR PRECOND_SEED_XOR.
    """
    X = np.asarray(X, np.float32)
    Xs = np.asarray(Xs, np.float32)
    n, ns = X.shape[0], Xs.shape[0]
    L = OracleLattice(np.vstack([X, Xs]), ls, kind=kind, r=r)
    Z = rademacher_sketch(ns, probes, seed) if Z is None else np.asarray(Z, np.float64)
    S = Z.shape[1]

    def K(V):  # outputscale K~ V on the joint point set
        return L.mvm(V, mode=2, alpha=outputscale)

    def pad(V):  # training-row vector -> joint vector with zero test rows
        full = np.zeros((n + ns, V.shape[1]))
        full[:n] = V
        return full

    B = np.asarray(y, np.float64)[:, None]
    if S > 0:
        Vz = np.zeros((n + ns, S))
        Vz[n:] = Z
        B = np.concatenate([B, K(Vz)[:n]], 1)
    def A(V):  # (outputscale K~ + noise I) on the training rows
        return K(pad(V))[:n] + noise * V

    if precond_rank > 0:
        Bm, Q = nystrom_factor(lambda V: K(pad(V))[:n], n, precond_rank, noise,
                               int(seed) ^ PRECOND_SEED_XOR)
        W, iters, rel = _pcg_columns(A, B, lambda R: nystrom_apply(Bm, Q, noise, R), tol,
                                     max_iter)
    else:
        W, iters, rel = _cg_columns(A, B, tol, max_iter)
    P = K(pad(W))[n:]
    mean = P[:, 0]
    var = outputscale - (Z * P[:, 1:]).mean(1) if S > 0 else np.zeros(ns)
    return mean, var, iters, rel


def condition_estimate(X, Xs, ls, noise: float, outputscale: float = 1.0,
                       kind: int = RBF_BINOMIAL, r: int = 1) -> float:
    """Upper estimate of the condition number of A = outputscale K~_XX + noise I (the
    training block of the joint lattice operator): K~ has non-negative entries, so by
    Gershgorin's theorem its largest eigenvalue is at most its largest row sum, and the
    smallest eigenvalue of A is at least noise; returns
    (outputscale max_i (K~_XX 1)_i + noise) / noise."""
    X = np.asarray(X, np.float32)
    Xs = np.asarray(Xs, np.float32)
    n, ns = X.shape[0], Xs.shape[0]
    L = OracleLattice(np.vstack([X, Xs]), ls, kind=kind, r=r)
    ones = np.zeros((n + ns, 1))
    ones[:n] = 1.0
    rows = L.mvm(ones, mode=2, alpha=outputscale)[:n, 0]
    return float((rows.max() + noise) / noise)


def filter_gradient(apply_K, X, ls, V, G, alpha: float = 1.0, kprime_ratio: float = -0.5):
    """Sec. 4.2: gradient of L = <G, alpha K V> with respect to the inputs from ONE filtering
    call.  With k_ij = k(d_ij^2) on z = x / l and k' its derivative in d^2,
        dL/dz_n = 2 sum_j k'_nj [ (g_n . v_j)(z_n - z_j) + (g_j . v_n)(z_n - z_j) ],
    which splits into filtering the columns [z (.) g, g, z (.) v, v] with k' and combining
    the outputs at each point.  For the RBF k(d^2) = exp(-d^2 / 2), k' = -k / 2, so the
    filter is the kernel operator itself (kprime_ratio = -1/2).  apply_K maps an [n][c]
    array to K times it.  Returns (dX [n][d], dls [d])."""
    X = np.asarray(X, np.float64)
    ls = np.asarray(ls, np.float64)
    V = np.asarray(V, np.float64)
    G = np.asarray(G, np.float64)
    Z = X / ls
    n, d = Z.shape
    k = V.shape[1]
    ZG = (G[:, :, None] * Z[:, None, :]).reshape(n, k * d)  # column c d + t: g_c z_t
    ZV = (V[:, :, None] * Z[:, None, :]).reshape(n, k * d)
    F = apply_K(np.concatenate([ZG, G, ZV, V], 1))
    FZG = F[:, :k * d].reshape(n, k, d)
    FG = F[:, k * d:k * d + k]
    FZV = F[:, k * d + k:2 * k * d + k].reshape(n, k, d)
    FV = F[:, 2 * k * d + k:]
    dZ = 2.0 * alpha * kprime_ratio * (
        Z * (G * FV).sum(1)[:, None] - (G[:, :, None] * FZV).sum(1)
        + Z * (V * FG).sum(1)[:, None] - (V[:, :, None] * FZG).sum(1))
    return dZ / ls, -(dZ * Z).sum(0) / ls
