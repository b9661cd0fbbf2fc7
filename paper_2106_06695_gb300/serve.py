"""Python handle of the continuous-batching GP posterior server (C-ABI in
include/sgp_serve.h) and a driver that replays a request stream against it.

Argument marshalling only: requests are host numpy arrays handed to libsgp.so, which
uploads them, builds each request's lattice, runs the batched CG and writes the
posterior mean and variance back into host arrays owned by this object.
"""

from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass, field

import numpy as np

from . import _lib
from ._lib import KERNELS, VALUE_DTYPES, check


def _host_f32(a, name: str, ndim: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != ndim:
        raise ValueError("%s must have %d dimensions" % (name, ndim))
    return a


class Server:
    """GP posterior requests (Eq. gp_pred_mean, gp_pred_cov) solved in one batch.

    max_active = 1 is the plain one-request-at-a-time path (same kernels); probes is the
    number S of Rademacher probes of the variance estimate (k = 1 + S right-hand sides).
    precond_rank: rank of the Nystrom CG preconditioner (App. A; 0 = none), used for the
    requests whose condition estimate reaches precond_min_kappa.
    """

    def __init__(self, max_active: int = 16, probes: int = 8, hbm_budget: int | None = None,
                 order: int = 1, kernel: str = "rbf_binomial", value_dtype: str = "f32",
                 tol: float = 1e-3, max_iter: int = 1000, check_every: int = 8,
                 precond_rank: int = 100, precond_min_kappa: float = 1e3,
                 lane_classes: bool = True):
        self._lib = _lib.load()
        o = _lib.sgp_server_opts()
        self._lib.sgp_server_opts_init(ctypes.byref(o))
        if hbm_budget is not None:
            o.hbm_budget = int(hbm_budget)
        o.max_active = int(max_active)
        o.probes = int(probes)
        o.order_r = int(order)
        o.kernel = KERNELS[kernel]
        o.value_dtype = VALUE_DTYPES[value_dtype]
        o.tol = float(tol)
        o.max_iter = int(max_iter)
        o.check_every = int(check_every)
        o.precond_rank = int(precond_rank)
        o.precond_min_kappa = float(precond_min_kappa)
        o.lane_classes = 1 if lane_classes else 0
        self.opts = o
        h = ctypes.c_void_p()
        check(self._lib.sgp_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    # -- lifetime -------------------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.sgp_server_destroy(h)
        self._h = None
        self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- requests ---------------------------------------------------------------------
    def submit(self, X, y, Xs, lengthscales, outputscale: float = 1.0, noise: float = 0.01,
               seed: int = 0, arrival_us: float | None = None,
               timeout_s: float | None = None, lattice_key: int = 0) -> int:
        X = _host_f32(X, "X", 2)
        Xs = _host_f32(Xs, "Xs", 2)
        y = _host_f32(y, "y", 1)
        d = X.shape[1]
        ls = np.ascontiguousarray(np.broadcast_to(np.asarray(lengthscales, np.float32), (d,)))
        mean = np.zeros(Xs.shape[0], np.float32)
        var = np.zeros(Xs.shape[0], np.float32)
        r = _lib.sgp_request()
        r.X, r.y, r.n = X.ctypes.data, y.ctypes.data, X.shape[0]
        r.Xs, r.ns, r.d = Xs.ctypes.data, Xs.shape[0], d
        r.lengthscales = ls.ctypes.data
        r.outputscale, r.noise, r.seed = float(outputscale), float(noise), int(seed)
        r.mean, r.var = mean.ctypes.data, var.ctypes.data
        r.arrival_us = -1.0 if arrival_us is None else float(arrival_us)
        r.timeout_us = 0.0 if timeout_s is None else 1e6 * float(timeout_s)
        r.lattice_key = int(lattice_key)
        rid = ctypes.c_longlong()
        check(self._lib.sgp_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)))
        self._keep[rid.value] = (X, y, Xs, ls, mean, var)
        return rid.value

    def step(self) -> int:
        done = ctypes.c_int()
        check(self._lib.sgp_server_step(self._h, ctypes.byref(done)))
        return done.value

    def stats(self, rid: int) -> dict:
        s = _lib.sgp_request_stats()
        check(self._lib.sgp_server_stats(self._h, int(rid), ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def result(self, rid: int):
        """(mean, var) host arrays of a completed request."""
        st = self.stats(rid)
        if not st["done"]:
            raise RuntimeError("request %d has not completed" % rid)
        check(st["status"])
        _, _, _, _, mean, var = self._keep[rid]
        return mean, var

    def info(self) -> dict:
        q, a, peak = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        b = ctypes.c_ulonglong()
        check(self._lib.sgp_server_info(self._h, ctypes.byref(q), ctypes.byref(a),
                                        ctypes.byref(b), ctypes.byref(peak)))
        return {"queued": q.value, "active": a.value, "bytes_in_use": b.value,
                "peak_active": peak.value}

    def cache_info(self) -> dict:
        n, b = ctypes.c_int(), ctypes.c_ulonglong()
        check(self._lib.sgp_server_cache_info(self._h, ctypes.byref(n), ctypes.byref(b)))
        return {"lattices": n.value, "bytes": b.value}

    def clock_us(self) -> float:
        return float(self._lib.sgp_server_clock_us(self._h))

    def run_until_idle(self) -> None:
        while True:
            i = self.info()
            if i["queued"] + i["active"] == 0:
                return
            self.step()


def request_bytes_bound(n_points: int, d: int, order: int = 1, k: int = 10,
                        value_dtype: str = "f32", precond_rank: int = 100) -> int:
    """Upper bound of one request's device bytes (sgp_request_bytes_bound); k = 1 + probes
    + 1 columns, precond_rank as the server's option."""
    return int(_lib.load().sgp_request_bytes_bound(int(n_points), int(d), int(order), int(k),
                                                  VALUE_DTYPES[value_dtype],
                                                  int(precond_rank)))


@dataclass
class StreamResult:
    latencies_s: list = field(default_factory=list)  # per request, completion - arrival
    solves_per_s: float = 0.0
    makespan_s: float = 0.0
    ids: list = field(default_factory=list)
    iters: list = field(default_factory=list)
    peak_active: int = 0

    def percentile(self, q: float) -> float:
        return float(np.percentile(np.asarray(self.latencies_s), q))


def run_stream(server, requests, sleep=time.sleep) -> StreamResult:
    """Submit each request at its arrival time and step the server until all complete.

    requests: sequence of dicts with "arrival_s" (seconds after the start, ascending),
    "X", "y", "Xs", "lengthscales", "outputscale", "noise", "seed".  A request is
    submitted with its scheduled arrival time on the server clock, so the time it waits
    while the host is inside a step counts towards its latency.
    """
    reqs = sorted(requests, key=lambda r: r["arrival_s"])
    t0 = server.clock_us()
    ids = []
    i = 0
    while True:
        now = (server.clock_us() - t0) / 1e6
        while i < len(reqs) and reqs[i]["arrival_s"] <= now:
            r = reqs[i]
            ids.append(server.submit(r["X"], r["y"], r["Xs"], r["lengthscales"],
                                     r.get("outputscale", 1.0), r.get("noise", 0.01),
                                     r.get("seed", 0), t0 + 1e6 * r["arrival_s"],
                                     lattice_key=r.get("lattice_key", 0)))
            i += 1
        info = server.info()
        if info["queued"] + info["active"] > 0:
            server.step()
        elif i < len(reqs):
            sleep(max(0.0, reqs[i]["arrival_s"] - now))
        else:
            break
    res = StreamResult(ids=ids, peak_active=server.info()["peak_active"])
    first = min(server.stats(r)["arrival_us"] for r in ids)
    last = max(server.stats(r)["done_us"] for r in ids)
    for rid in ids:
        st = server.stats(rid)
        res.latencies_s.append((st["done_us"] - st["arrival_us"]) / 1e6)
        res.iters.append(st["iters"])
    res.makespan_s = (last - first) / 1e6
    res.solves_per_s = len(ids) / res.makespan_s if res.makespan_s > 0 else 0.0
    return res
