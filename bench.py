#!/usr/bin/env python
"""Throughput of the Simplex-GP hot path on one GB300 (or N independent replicas).

One step = the whole path over one batch of synthetic input, run to the solver's
tolerance:
  build the permutohedral lattice of X (elevate, enclosing simplex, barycentric
  weights, hash insert, vertex numbering, neighbour table, splat lists; Sec. 3.2), build
  the rank-1024 Nystrom preconditioner of the CG (App. A; one power iteration: two
  1024-column lattice products, tensor-core Grams, fp64 factorizations), then solve
  (K~ + noise I) X = V for all k right-hand sides with batched preconditioned CG to
  ||r|| / ||b|| <= 1e-3 (Sec. 2); each CG iteration is one lattice MVM (splat, 2(d+1)
  blur passes of the symmetric operator, slice) and one preconditioner apply.
Metric: lattice MVM Mpoint/s = n * (k-column MVMs in the step) / step time, whole job,
iterations counted as the max over columns and each sketch product of l columns counted as
l / k MVMs; the step time is the time to tolerance.  Reported beside it: the graph-replayed
MVM alone, the per-stage rooflines (splat, blur, slice, preconditioner), the plain CG of
500 iterations on the same system, and the time to tolerance of the n = 200,000 solve
workload.  `--precond-rank 0` makes plain CG the timed step.

Workload (default): n = 2,000,000 points, d = 11, standardised 16-component Gaussian
mixture (the shape of Houseelectric, n=2,049,280 d=11, Sec. 5 Table n_lattice), unit ARD
lengthscales, binomial stencil r = 1, k = 16 right-hand sides ~ N(0, 1), noise 0.01,
CG tolerance 1e-3, at most 500 iterations.

Serving (`serving` in the JSON line): a Poisson stream of GP posterior requests through the
continuous-batching server and through the plain one-at-a-time path, solves/s and p50/p99.

`--impl reference` times the FP64 CPU oracle (the reference for this path) on a bounded
sample of the same workload, on this host's cores.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

# The CPU legs time the oracle on one core: keep numpy's BLAS pools single-threaded
# (set before numpy loads; the GPU arm does no BLAS work).
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "lattice MVM Mpoint/s at n=2M,d=11 (%HBM peak)"
UNIT = "Mpoint/s"
WORKLOAD = dict(n=2_000_000, d=11, k=16, seed=4, lengthscale=1.0, noise=0.01, tol=1e-3,
                max_iter=500, kernel="rbf_binomial", order=1, blur="symmetric",
                precond_rank=1024, precond_power_iters=1)
# the n = 200,000, d = 11 solve workload: y plus 8 Rademacher probes, noise 0.01
C2 = dict(n=200_000, d=11, seed=2, probes=8, noise=0.01, tol=1e-3, max_iter=500,
          precond_rank=256, precond_power_iters=1)
SERVING = dict(requests=256, rate_per_s=50.0, seed=5, max_active=16, test_points=256)
CPU_SAMPLE = dict(n=200_000, iters=100)  # oracle sample of the cpu_baseline leg, all cores
CPU_SAMPLE_1T = dict(n=100_000, iters=4)  # the same on one thread (a smaller sample)
REF_SAMPLE = dict(n=100_000, iters=20)   # oracle sample per step for --impl reference


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=WORKLOAD["n"], help="points (default 2,000,000)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precond-rank", type=int, default=WORKLOAD["precond_rank"],
                    help="rank of the CG preconditioner in the timed step (default 1024; "
                         "0 = plain CG)")
    ap.add_argument("--max-iter", type=int, default=WORKLOAD["max_iter"],
                    help="CG iteration cap (default 500; lower only for profiling runs)")
    ap.add_argument("--serving-requests", type=int, default=SERVING["requests"],
                    help="requests in the serving stream (0 = skip the serving comparison)")
    ap.add_argument("--no-backward", action="store_true",
                    help="skip the backward (n=500k, d=20) and log-det (n=200k) timings")
    ap.add_argument("--mvm-only", type=int, default=0, metavar="R",
                    help="profiling aid: build once, run R symmetric MVMs, print their time")
    ap.add_argument("--serve-single", action="store_true",
                    help="profiling aid: serve two ill-conditioned requests (d = 3, n = 240k "
                         "and d = 8, n = 100k) one at a time and print their statistics")
    ap.add_argument("--oracle-full", action="store_true",
                    help="time the FP64 oracle on the whole workload (build + one symmetric "
                         "MVM at n = 2M, all host cores and one thread; about 1.5 min of CPU "
                         "work) and print one JSON line; no GPU work")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------------------
# distributed plumbing (replicas only: the only collectives are the timing barrier/max)
# ---------------------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world, backend):
    if world > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def aggregate(elapsed_ms: float, units: float, world: int):
    """Max of the elapsed time over ranks and sum of the work units over ranks."""
    if world == 1:
        return elapsed_ms, units
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def blur_traffic_per_launch(m: int, k: int):
    """DRAM bytes per blur launch from the committed ncu summary, scaled to this m, if the
    blur kernel's source has not changed since it was captured; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))["blur_pass"]
    except (OSError, KeyError, ValueError):
        return None
    src = open(os.path.join(ROOT, "paper_2106_06695_gb300", "csrc", "mvm.cu")).read()
    body = re.search(r"template <class S>\n__global__ void __launch_bounds__\(kThreads\) "
                     r"k_blur_pipe\(.*?\n}\n", src, re.S)
    if (body is None or hashlib.sha1(body.group(0).encode()).hexdigest() != rec.get("src_sha1")
            or rec.get("k") != k):
        return None
    return float(rec["bytes_per_vertex"]) * m


def stage_traffic(stage: str):
    """DRAM bytes per launch of a stage's kernel from the committed ncu summary
    (profiles/traffic.json), if recorded for this workload and kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[stage]
    except (OSError, KeyError, ValueError):
        return None
    src_file = os.path.join(ROOT, "paper_2106_06695_gb300", "csrc", rec.get("file", ""))
    try:
        src = open(src_file).read()
    except OSError:
        return None
    body = re.search(rec["pattern"], src, re.S) if "pattern" in rec else None
    if body is None or hashlib.sha1(body.group(0).encode()).hexdigest() != rec.get("src_sha1"):
        return None
    return float(rec["bytes_per_launch"])


def run_solve_c2():
    """Time to tolerance of the n = 200,000, d = 11 solve workload (GMM seed 2, unit
    lengthscales, noise 0.01, B = [y, 8 Rademacher probes], tol 1e-3): lattice build +
    rank-256 Nystrom preconditioner with one power iteration + preconditioned CG, median of
    3 after a warm-up, wall clock around the whole call (host timers, synchronised); plus
    the plain CG of the same system for comparison."""
    import torch

    from paper_2106_06695_gb300 import synth
    from paper_2106_06695_gb300.lattice import Lattice

    C = C2
    X = torch.from_numpy(synth.gmm_points(C["n"], C["d"], C["seed"])).cuda()
    B = torch.from_numpy(synth.solve_rhs(X.cpu().numpy(), C["seed"], probes=C["probes"])).cuda()
    ls = torch.ones(C["d"], device="cuda")
    out = torch.empty_like(B)

    def solve(rank):
        lat = Lattice(X, ls, precond_rank=rank, precond_seed=C["seed"],
                      precond_power_iters=C["precond_power_iters"])
        _, it, rel = lat.cg(B, noise=C["noise"], tol=C["tol"], max_iter=C["max_iter"], out=out)
        torch.cuda.synchronize()
        true = None
        if rank:
            r = B.double() - lat.mvm(out, blur="symmetric", beta=C["noise"]).double()
            true = (r.norm(dim=0) / B.double().norm(dim=0)).max().item()
        lat.close()
        return it, rel, true

    solve(C["precond_rank"])
    ts = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, rel, true = solve(C["precond_rank"])
        ts.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    pit, prel, _ = solve(0)
    plain_s = time.perf_counter() - t0
    return {"workload": "n=%d d=%d k=%d (y + %d probes), noise %g, tol %g, rank-%d "
                        "preconditioner with %d power iteration"
                        % (C["n"], C["d"], C["probes"] + 1, C["probes"], C["noise"], C["tol"],
                           C["precond_rank"], C["precond_power_iters"]),
            "time_to_tol_s": float(np.median(ts)), "cg_iters": int(it.max()),
            "rel_res_max": float(rel.max()), "true_rel_res_max": true,
            "plain_cg": {"s": plain_s, "cg_iters": int(pit.max()),
                         "rel_res_max": float(prel.max())}}


def run_approximation_c1():
    """Approximation error of the lattice operator against the exact RBF kernel (Sec. 5.1)
    on the n = 4096, d = 3 workload (X ~ U[0,1]^3, lengthscale 0.3, outputscale 1, binomial
    stencil r = 1, one right-hand side V ~ N(0, 1)): 1 - cosine and relative L2 of K~V
    against the dense K V (computed in float64 with numpy), for the paper's sequential
    blur and the symmetric blur the CG uses."""
    import torch

    from paper_2106_06695_gb300 import synth
    from paper_2106_06695_gb300.lattice import Lattice

    X = synth.uniform_points(4096, 3, 1)
    V = synth.gaussian_values(4096, 1, 1).astype(np.float64)
    Z = X.astype(np.float64) / 0.3
    sq = (Z * Z).sum(1)
    K = np.exp(-0.5 * np.maximum(sq[:, None] + sq[None, :] - 2.0 * Z @ Z.T, 0.0))
    exact = (K @ V)[:, 0]
    lat = Lattice(torch.from_numpy(X).cuda(), 0.3)
    out = {"workload": "n=4096 d=3 X~U[0,1]^3, lengthscale 0.3, binomial r=1, k=1", "m": lat.m}
    for blur in ("sequential", "symmetric"):
        got = lat.mvm(torch.from_numpy(V.astype(np.float32)).cuda(), blur=blur).cpu().numpy()
        got = got.astype(np.float64)[:, 0]
        cos = float(got @ exact / (np.linalg.norm(got) * np.linalg.norm(exact)))
        out[blur] = {"one_minus_cosine": 1.0 - cos,
                     "rel_l2": float(np.linalg.norm(got - exact) / np.linalg.norm(exact))}
    lat.close()
    return out


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def run_ours(args, world, rank, local):
    import torch

    from paper_2106_06695_gb300 import _lib, build_lib, synth
    from paper_2106_06695_gb300.lattice import Lattice

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the lattice library has no CPU path)")
    torch.cuda.set_device(local)
    init_dist(world, "nccl")
    build_lib.build()
    lib = _lib.load()
    W = dict(WORKLOAD, n=args.n, max_iter=args.max_iter, precond_rank=args.precond_rank)
    n, d, k = W["n"], W["d"], W["k"]
    Xh = torch.from_numpy(synth.gmm_points(n, d, W["seed"])).pin_memory()
    Vh = torch.from_numpy(synth.gaussian_values(n, k, W["seed"])).pin_memory()
    lsh = torch.full((d,), W["lengthscale"], dtype=torch.float32).pin_memory()
    dev = torch.device("cuda", local)
    Xd, Vd, lsd = Xh.to(dev), Vh.to(dev), lsh.to(dev)
    out = torch.empty_like(Vd)
    if args.mvm_only:
        lat = Lattice(Xd, lsd, order=W["order"], kernel=W["kernel"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.mvm_only):
            lat.mvm(Vd, blur=W["blur"], out=out)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"mvm_only": True, "n": n, "m": lat.m, "reps": args.mvm_only,
                          "ms_per_mvm": e0.elapsed_time(e1) / args.mvm_only}), flush=True)
        return
    prof = {"ms": 0.0, "passes": 0, "m": 0, "iters": [], "build_ms": [], "rel": [],
            "stages": np.zeros(5), "samples": 0}
    sketch_mvms = (1 + W["precond_power_iters"]) * W["precond_rank"] / k

    def make_lattice(Xdev, ls_dev, rank=None):
        r = W["precond_rank"] if rank is None else rank
        return Lattice(Xdev, ls_dev, order=W["order"], kernel=W["kernel"], precond_rank=r,
                       precond_seed=W["seed"], precond_power_iters=W["precond_power_iters"])

    def step(Xdev, Vdev, ls_dev, profile=False):
        t0 = time.perf_counter()
        lat = make_lattice(Xdev, ls_dev)
        prof["build_ms"].append(1e3 * (time.perf_counter() - t0))
        if profile:
            _lib.check(lib.sgp_profile_blur(lat._h, 1))
        _, iters, rel = lat.cg(Vdev, noise=W["noise"], tol=W["tol"], max_iter=W["max_iter"],
                               blur=W["blur"], out=out)
        if profile:
            import ctypes

            ms, passes = ctypes.c_double(), ctypes.c_int64()
            _lib.check(lib.sgp_profile_read(lat._h, ctypes.byref(ms), ctypes.byref(passes)))
            prof["ms"] += ms.value
            prof["passes"] += passes.value
            st = np.zeros(5, np.float64)
            nsamp = ctypes.c_int64()
            _lib.check(lib.sgp_profile_read_stages(lat._h, st.ctypes.data, ctypes.byref(nsamp)))
            prof["stages"] += st
            prof["samples"] += nsamp.value
        prof["m"] = lat.m
        prof["iters"].append(int(iters.max()))
        prof["rel"].append(float(rel.max()))
        lat.close()
        print("step: m=%d build %.1f ms, cg iters %d, rel %.2e, %.1f ms total" % (
            lat.m, prof["build_ms"][-1], int(iters.max()), float(rel.max()),
            1e3 * (time.perf_counter() - t0)), file=sys.stderr, flush=True)
        return int(iters.max()) + sketch_mvms, rel

    for _ in range(args.warmup):
        step(Xd, Vd, lsd)
    prof.update(ms=0.0, passes=0, iters=[], build_ms=[], rel=[], stages=np.zeros(5), samples=0)
    torch.cuda.synchronize()
    barrier(world)
    launches0 = lib.sgp_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mvms = 0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(args.steps):
            it, rel = step(Xd, Vd, lsd, profile=True)
            mvms += it
        ev1.record()
        torch.cuda.synchronize()
    barrier(world)
    launches = lib.sgp_kernel_launches() - launches0
    elapsed_ms = ev0.elapsed_time(ev1)
    max_ms, units = aggregate(elapsed_ms, float(n) * mvms, world)
    value = units / (max_ms / 1e3) / 1e6
    m = prof["m"]

    # rooflines from the live samples (CUDA events around each stage of one sampled
    # iteration per flag check, recorded inside the CG graph on the solve's stream)
    peak, peak_kind = measured_peak_gbs()
    samples = max(prof["samples"], 1)
    r_, D = W["order"], d + 1
    ld = -(-W["precond_rank"] // 128) * 128
    stage_bytes = {  # algorithmic bytes per launch (per sampled iteration for splat, slice)
        "blur_pass": m * (8 * k + 8 * r_),
        "splat": 8 * n * D + 4 * n * k + 4 * m * k,
        "slice_dot": 8 * n * D + 4 * m * k + 8 * n * k,
        "precond_bt": 2 * n * ld + 128 * n,   # bf16 B once, the split r ([n][64] bf16) once
        "precond_z": 2 * n * ld + 8 * n * min(k, 16),   # bf16 B once, r (fp32) read, z written
    }
    stage_ms = {  # average duration of one launch
        "blur_pass": prof["ms"] / max(prof["passes"], 1),
        "splat": prof["stages"][0] / samples,
        "slice_dot": prof["stages"][2] / samples,
        "precond_bt": prof["stages"][3] / samples,
        "precond_z": prof["stages"][4] / samples,
    }
    stages = {}
    for name, b in stage_bytes.items():
        t = stage_ms[name]
        if t > 0:
            ach = b / (t / 1e3) / 1e9
            stages[name] = {"avg_launch_ms": t, "algorithmic_bytes": b, "achieved_gbs": ach,
                            "frac": ach / peak}
    per_iter_ms = {"blur": prof["ms"] / samples, "splat": stage_ms["splat"],
                   "slice_dot": stage_ms["slice_dot"], "precond_bt": stage_ms["precond_bt"],
                   "precond_z": stage_ms["precond_z"]}
    # the dominant kernel: the largest time per iteration among the single kernels
    dom = max(("precond_bt", "precond_z", "splat", "slice_dot"),
              key=lambda s: per_iter_ms[s] if s in stages else 0.0)
    if per_iter_ms[dom] < per_iter_ms["blur"] or dom not in stages:
        dom = "blur_pass"
    names = {"blur_pass": "k_blur_pipe<float> (one lattice direction)",
             "splat": "k_splat<4,float> (+ fix-ups)", "slice_dot": "k_slice_dot<4,float>",
             "precond_bt": "k_bt_tc (preconditioner B^T r, tcgen05 bf16, TMA)",
             "precond_z": "k_z_tc (preconditioner z = (r - B u)/tau, tcgen05 bf16, TMA)"}
    ds = stages.get(dom, {})
    traffic = blur_traffic_per_launch(m, k) if dom == "blur_pass" else stage_traffic(dom)
    roofline = {"kernel": names[dom], "bound": "hbm",
                "achieved": ds.get("achieved_gbs"), "peak": peak, "unit": "GB/s",
                "frac": ds.get("frac"), "traffic": traffic,
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": ds.get("algorithmic_bytes"),
                "avg_launch_ms": ds.get("avg_launch_ms"), "sampled_iterations": prof["samples"],
                "per_iteration_ms": per_iter_ms, "stages": stages}

    # the preconditioner's set-up alone (a solve with max_iter 0), the true residual of the
    # timed solve's answer, the graph-replayed MVM, and the plain CG of 500 iterations
    lat = make_lattice(Xd, lsd)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.cg(Vd, noise=W["noise"], tol=W["tol"], max_iter=0, blur=W["blur"], out=out)
    torch.cuda.synchronize()
    setup_ms = 1e3 * (time.perf_counter() - t0)
    _, it_last, rel_last = lat.cg(Vd, noise=W["noise"], tol=W["tol"], max_iter=W["max_iter"],
                                  blur=W["blur"], out=out)
    resid = Vd.double() - lat.mvm(out, blur=W["blur"], beta=W["noise"]).double()
    true_rel = (resid.norm(dim=0) / Vd.double().norm(dim=0)).max().item()
    mvm_ms = graph_replay_median_ms(lat, Vd, out, W["blur"])
    mvm_seq_ms = graph_replay_median_ms(lat, Vd, out, "sequential")
    ref_out = lat.mvm(Vd, blur=W["blur"]).double()
    lat.close()
    lat = make_lattice(Xd, lsd, rank=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, p_iters, p_rel = lat.cg(Vd, noise=W["noise"], tol=W["tol"], max_iter=W["max_iter"],
                               blur=W["blur"], out=out)
    torch.cuda.synchronize()
    plain_ms = 1e3 * (time.perf_counter() - t0)
    lat.close()
    plain = {"ms": plain_ms, "cg_iters": int(p_iters.max()), "rel_res_max": float(p_rel.max()),
             "mpoint_s": n * int(p_iters.max()) / (plain_ms / 1e3) / 1e6,
             "note": "plain CG (no preconditioner) on the same system, build included"}
    # the same product with the lattice values stored in bf16 (fp32 sums)
    lat = Lattice(Xd, lsd, order=W["order"], kernel=W["kernel"], value_dtype="bf16")
    mvm_bf16_ms = graph_replay_median_ms(lat, Vd, out, W["blur"])
    bf16_rel_err = ((out.double() - ref_out).norm() / ref_out.norm()).item()
    lat.close()

    c2 = run_solve_c2() if rank == 0 else None
    approx = run_approximation_c1() if rank == 0 else None

    e2e = None
    if not args.no_e2e:
        Xs_host = torch.empty(n, k, dtype=torch.float32).pin_memory()
        e2e_mvms = 0
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            Xdev = Xh.to(dev, non_blocking=True)
            Vdev = Vh.to(dev, non_blocking=True)
            ls_dev = lsh.to(dev, non_blocking=True)
            it, _ = step(Xdev, Vdev, ls_dev)
            Xs_host.copy_(out, non_blocking=True)
            torch.cuda.synchronize()
            e2e_mvms += it
        barrier(world)
        e2e_ms, e2e_units = aggregate(1e3 * (time.perf_counter() - t0), float(n) * e2e_mvms, world)
        e2e = {"value": e2e_units / (e2e_ms / 1e3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(Xh.numel() * 4 + Vh.numel() * 4 + lsh.numel() * 4),
               "d2h_bytes_per_step": int(n * k * 4)}

    backward = run_backward_c3() if rank == 0 and not args.no_backward else None
    logdet = run_logdet_c2() if rank == 0 and not args.no_backward else None

    serving = None
    if rank == 0 and args.serving_requests > 0:
        serving = run_serving(args.serving_requests)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(W)

    if rank == 0:
        steps_ms = max_ms / args.steps
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": steps_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: standardised 16-component Gaussian mixture (seeded), "
                    "V ~ N(0,1); stands in for the paper's UCI datasets",
            "config": {"workload": "GP solve n=%d d=%d k=%d to rel. residual %g: lattice build "
                                   "+ rank-%d Nystrom preconditioner (%d power iteration) + "
                                   "batched preconditioned CG (max %d) on the symmetric "
                                   "lattice operator"
                                   % (n, d, k, W["tol"], W["precond_rank"],
                                      W["precond_power_iters"], W["max_iter"]),
                       "n": n, "d": d, "k": k, "m": m, "m_over_L": m / (n * (d + 1)),
                       "kernel": "%s r=%d" % (W["kernel"], W["order"]), "noise": W["noise"],
                       "precond_rank": W["precond_rank"],
                       "precond_power_iters": W["precond_power_iters"],
                       "cg_iters_per_step": prof["iters"],
                       "cg_rel_res_per_step": prof["rel"],
                       "mvms_per_step_counted": float(mvms / max(args.steps, 1)),
                       "time_to_tol_s": steps_ms / 1e3,
                       "precond_setup_ms": setup_ms,
                       "build_ms_median": float(np.median(prof["build_ms"])),
                       "plain_cg_500": plain,
                       "solve_n200k": c2,
                       "mvm_symmetric_ms": mvm_ms,
                       "mvm_symmetric_ms_note": "median of 50 graph-replayed MVMs",
                       "mvm_symmetric_mpoint_s": n / (mvm_ms / 1e3) / 1e6,
                       "mvm_symmetric_mpoint_columns_s": n * k / (mvm_ms / 1e3) / 1e6,
                       "mvm_symmetric_hbm_frac": mvm_bytes(n, d + 1, k, m, W["order"], 2 * (d + 1))
                                                 / (mvm_ms / 1e3) / 1e9 / peak,
                       "mvm_sequential_ms": mvm_seq_ms,
                       "mvm_sequential_mpoint_s": n / (mvm_seq_ms / 1e3) / 1e6,
                       "mvm_sequential_hbm_frac": mvm_bytes(n, d + 1, k, m, W["order"], d + 1)
                                                  / (mvm_seq_ms / 1e3) / 1e9 / peak,
                       "mvm_hbm_frac_note": "algorithmic bytes of one MVM, 16 n D + 8 n k + "
                                            "8 m k + P m (8 r + 8 k) + 4 (m + 1) for P blur "
                                            "passes, over the graph-replayed time and the "
                                            "measured HBM peak",
                       "mvm_symmetric_bf16_values_ms": mvm_bf16_ms,
                       "bf16_values_rel_l2_vs_fp32": bf16_rel_err,
                       "approximation_n4096": approx,
                       "l2": "no flush: every step's working set (X 88 MB, V 128 MB, "
                             "lattice values 2 x m x k x 4 B, the 8 GB preconditioner factor) "
                             "exceeds the 129 MB L2",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "serving": serving,
            "backward": backward, "logdet": logdet,
            "gpu_launches": int(launches), "clocks": clk.summary(),
            "cg_final_rel_res_max": float(np.max(rel_last)), "cg_true_rel_res_max": true_rel,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def mvm_bytes(n, D, k, m, r, passes):
    """Algorithmic bytes of one lattice MVM: ids and weights read by splat and slice, V
    read and out written, the splatted and sliced lattice rows, and per blur pass each
    vertex's row read and written plus its 2r neighbour ids."""
    return 16 * n * D + 8 * n * k + 8 * m * k + passes * m * (8 * r + 8 * k) + 4 * (m + 1)


def graph_replay_median_ms(lat, V, out, blur, replays=50, warmup=5):
    """Median time of one MVM captured as a CUDA graph and replayed (events around each
    replay, on the replaying stream)."""
    import torch

    lat.mvm(V, blur=blur, out=out)  # buffers allocated outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lat.mvm(V, blur=blur, out=out)
    for _ in range(warmup):
        g.replay()
    times = []
    for _ in range(replays):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.median(times))


def run_backward_c3():
    """Forward MVM and hand-written backward on n = 500,000, d = 20 (correlated Gaussian
    points, ARD lengthscales log-uniform [0.5, 2], k = 8, symmetric blur): median of 5 of
    each, after a warm-up, with CUDA events on the current stream."""
    import torch

    from paper_2106_06695_gb300 import synth
    from paper_2106_06695_gb300.lattice import Lattice

    n, d, k = 500_000, 20, 8
    X, ls = synth.correlated_points(n, d, 3)
    Xd = torch.from_numpy(X).cuda()
    ld = torch.from_numpy(ls).cuda()
    Vd = torch.from_numpy(synth.gaussian_values(n, k, 4)).cuda()
    Gd = torch.from_numpy(synth.gaussian_values(n, k, 5)).cuda()
    lat = Lattice(Xd, ld)
    out = torch.empty_like(Vd)

    def timed(fn, reps=5):
        fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    fwd = timed(lambda: lat.mvm(Vd, blur="symmetric", out=out))
    bwd = timed(lambda: lat.mvm_backward(Xd, ld, Vd, Gd, blur="symmetric"))
    bwd_f = timed(lambda: lat.mvm_backward(Xd, ld, Vd, Gd, blur="symmetric", grad="filter"))
    res = {"workload": "n=%d d=%d k=%d correlated Gaussian, ARD lengthscales, symmetric blur"
                       % (n, d, k), "m": lat.m, "sparse_blur": lat.sparse_blur,
           "forward_ms": fwd, "backward_lattice_ms": bwd, "backward_filter_ms": bwd_f,
           "backward_over_forward": bwd / fwd,
           "forward_backward_mpoint_s": n / ((fwd + bwd) / 1e3) / 1e6}
    lat.close()
    # both input gradients against the exact RBF gradient on a seeded n = 2,000 subsample
    # (dense numpy float64): d/dx_i of <G, K V>, K_ij = exp(-|z_i - z_j|^2 / 2), z = x / l
    rows = synth.subsample(n, 2000, 3)
    Xs, Vs, Gs = X[rows], synth.gaussian_values(n, k, 4)[rows], synth.gaussian_values(n, k, 5)[rows]
    Z = Xs.astype(np.float64) / ls.astype(np.float64)
    diff = Z[:, None, :] - Z[None, :, :]
    Kd = np.exp(-0.5 * (diff ** 2).sum(-1))
    Wd = (Gs.astype(np.float64) @ Vs.astype(np.float64).T) * Kd
    dX_dense = -((Wd + Wd.T)[:, :, None] * diff).sum(1) / ls.astype(np.float64)
    sub_lat = Lattice(torch.from_numpy(Xs).cuda(), ld)
    cosines = {}
    for grad in ("lattice", "filter"):
        _, dX, _ = sub_lat.mvm_backward(torch.from_numpy(Xs).cuda(), ld, torch.from_numpy(Vs).cuda(),
                                        torch.from_numpy(Gs).cuda(), blur="symmetric", grad=grad,
                                        want=("X",))
        g = dX.cpu().numpy().astype(np.float64).ravel()
        cosines[grad] = float(g @ dX_dense.ravel() / (np.linalg.norm(g) * np.linalg.norm(dX_dense)))
    sub_lat.close()
    res["dX_cosine_vs_dense_rbf_n2000"] = cosines
    res["dX_cosine_note"] = ("cosine of the GPU's dX (exact lattice derivative; Sec. 4.2 filter) "
                             "against the exact RBF kernel's gradient on a seeded 2,000-point "
                             "subsample at d = 20, where the lattice barely resolves the "
                             "off-diagonal kernel")
    return res


def run_logdet_c2():
    """log det(K~ + noise I) by stochastic Lanczos quadrature on n = 200,000, d = 11 (the
    GMM solve workload, noise 0.01): 8 Rademacher probes, 100 Lanczos steps (App. A),
    median of 3 after a warm-up; Mpoint/s counts n x Lanczos steps x probes / time."""
    import torch

    from paper_2106_06695_gb300 import synth
    from paper_2106_06695_gb300.lattice import Lattice

    n, d, probes, steps = 200_000, 11, 8, 100
    X = torch.from_numpy(synth.gmm_points(n, d, 2)).cuda()
    Z = torch.from_numpy(synth.rademacher(n, probes, 2)).cuda()
    lat = Lattice(X, 1.0)
    lat.logdet(Z, noise=0.01, max_lanczos=steps, tol=0.0)
    ts, est = [], None
    for _ in range(3):
        t0 = time.perf_counter()
        est, quad = lat.logdet(Z, noise=0.01, max_lanczos=steps, tol=0.0)
        ts.append(time.perf_counter() - t0)
    t = float(np.median(ts))
    lat.close()
    return {"workload": "n=%d d=%d, %d probes, %d Lanczos steps, noise 0.01"
                        % (n, d, probes, steps), "ms": 1e3 * t, "logdet": est,
            "probe_quadrature_sd": float(np.std(quad, ddof=1)),
            "mpoint_s": n * steps / t / 1e6}


# ---------------------------------------------------------------------------------------
# serving: the same request stream through the batched server and the plain path
# ---------------------------------------------------------------------------------------
def run_serving(count: int):
    """GP posterior requests (mean and probe variance, k = 1 + 8) with Poisson arrivals,
    replayed in real time through the continuous-batching server and through the plain
    one-request-at-a-time path (the same server with one slot); latency is completion
    minus scheduled arrival, solves/s = requests / (last completion - first arrival)."""
    from paper_2106_06695_gb300 import synth
    from paper_2106_06695_gb300.serve import Server, run_stream

    t0 = time.perf_counter()
    reqs = synth.serving_stream(count, SERVING["seed"], rate_per_s=SERVING["rate_per_s"],
                                test_points=SERVING["test_points"])
    gen_s = time.perf_counter() - t0
    out, results = {}, {}
    for name, slots in (("batched", SERVING["max_active"]), ("plain", 1)):
        with Server(max_active=slots) as srv:
            res = run_stream(srv, reqs)
            results[name] = [tuple(a.copy() for a in srv.result(i)) for i in res.ids]
            stats = [srv.stats(i) for i in res.ids]
        rel = [st["rel_res"] for st in stats]
        setup_s = sum(st["setup_us"] for st in stats) / 1e6
        dims = [r["X"].shape[1] for r in sorted(reqs, key=lambda r: r["arrival_s"])]
        by_d = {str(d): float(np.mean([st["iters"] for st, dd in zip(stats, dims) if dd == d]))
                for d in sorted(set(dims))}
        out[name] = {"solves_per_s": res.solves_per_s, "p50_s": res.percentile(50),
                     "p99_s": res.percentile(99), "makespan_s": res.makespan_s,
                     "max_active": slots, "peak_active": res.peak_active,
                     "cg_iters_mean": float(np.mean(res.iters)),
                     "cg_iters_max": int(np.max(res.iters)),
                     "cg_iters_mean_by_d": by_d,
                     "preconditioned": int(sum(1 for st in stats if st["precond_rank"] > 0)),
                     "converged_fraction": float(np.mean([r_ <= 1e-3 for r_ in rel])),
                     "rel_res_max": float(np.max(rel)), "setup_s_total": setup_s}
        print("serving %s: %.2f solves/s p50 %.3f s p99 %.3f s" % (
            name, res.solves_per_s, res.percentile(50), res.percentile(99)),
            file=sys.stderr, flush=True)
    same = all(np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
               for a, b in zip(results["batched"], results["plain"]))
    # the same stream with BF16 lattice values (batched), kept for requests whose condition
    # estimate is at most 100 (the others are solved with fp32 values)
    with Server(max_active=SERVING["max_active"], value_dtype="bf16") as srv:
        res = run_stream(srv, reqs)
        bf = [tuple(a.copy() for a in srv.result(i)) for i in res.ids]
        kept = [srv.stats(i)["value_dtype"] == 1 for i in res.ids]
    errs = [np.linalg.norm(b[0] - a[0]) / max(np.linalg.norm(a[0]), 1e-30)
            for a, b in zip(results["batched"], bf)]
    out["batched_bf16"] = {"solves_per_s": res.solves_per_s, "p50_s": res.percentile(50),
                           "p99_s": res.percentile(99),
                           "requests_with_bf16_values": int(sum(kept)),
                           "mean_rel_l2_vs_fp32_median": float(np.median(errs)),
                           "mean_rel_l2_vs_fp32_max": float(np.max(errs)),
                           "mean_rel_l2_vs_fp32_max_bf16_requests":
                               float(max([e for e, k_ in zip(errs, kept) if k_] or [0.0]))}
    # the same stream through one lane for all requests (lane_classes off): every round then
    # runs the blur passes of the largest active d for every request
    with Server(max_active=SERVING["max_active"], lane_classes=False) as srv:
        res = run_stream(srv, reqs)
        one = [tuple(a.copy() for a in srv.result(i)) for i in res.ids]
        iters_one = [srv.stats(i)["iters"] for i in res.ids]
    out["batched_one_lane"] = {
        "solves_per_s": res.solves_per_s, "p50_s": res.percentile(50),
        "p99_s": res.percentile(99), "makespan_s": res.makespan_s,
        "cg_iters_mean": float(np.mean(iters_one)),
        "identical_results_vs_lanes": bool(all(
            np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
            for a, b in zip(results["batched"], one)))}
    # a stream the GPU keeps up with: 64 requests arriving at 5/s, so that p50/p99 measure
    # a request's own latency rather than queueing
    light = synth.serving_stream(64, SERVING["seed"] + 2, rate_per_s=5.0,
                                 test_points=SERVING["test_points"])
    for name, slots in (("light_batched", SERVING["max_active"]), ("light_plain", 1)):
        with Server(max_active=slots) as srv:
            res = run_stream(srv, light)
            rel_l = [srv.stats(i)["rel_res"] for i in res.ids]
        out[name] = {"requests": len(light), "arrival_rate_per_s": 5.0,
                     "solves_per_s": res.solves_per_s, "p50_s": res.percentile(50),
                     "p99_s": res.percentile(99),
                     "converged_fraction": float(np.mean([r_ <= 1e-3 for r_ in rel_l]))}
    # repeated solves on resident lattices: 64 requests over 8 point sets, with and
    # without lattice keys (batched server both times)
    rep = synth.repeated_stream(64, 8, SERVING["seed"] + 1, rate_per_s=SERVING["rate_per_s"],
                                test_points=SERVING["test_points"])
    reuse = {"requests": len(rep), "datasets": 8}
    for name, keyed in (("with_keys", True), ("without_keys", False)):
        stream = [dict(r, lattice_key=(r["dataset"] + 1) if keyed else 0) for r in rep]
        with Server(max_active=SERVING["max_active"]) as srv:
            res = run_stream(srv, stream)
            reused = sum(srv.stats(i)["lattice_reused"] for i in res.ids)
        reuse[name] = {"solves_per_s": res.solves_per_s, "p50_s": res.percentile(50),
                       "p99_s": res.percentile(99), "lattices_reused": int(reused)}
    out["reuse"] = reuse
    out.update({"requests": count, "arrival_rate_per_s": SERVING["rate_per_s"],
                "identical_results_batched_vs_plain": bool(same),
                "stream": "n log-uniform [5e3, 5e5], d uniform over {3, 8, 20, 50, 90}, "
                          "standardised 16-component GMM, y = sum sin(2 x) + N(0, 0.01), "
                          "%d test points, unit lengthscales, noise 0.01, k = 1 + 8 probes, "
                          "tol 1e-3, max 1000 iterations, rank-100 Nystrom preconditioner "
                          "(App. A) where the condition estimate is >= 1e3; generated in %.1f s"
                          % (SERVING["test_points"], gen_s),
                "solves_per_s_ratio": out["batched"]["solves_per_s"] / out["plain"]["solves_per_s"],
                "p99_ratio": out["batched"]["p99_s"] / out["plain"]["p99_s"]})
    return out


# ---------------------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------------------
def oracle_sample(W, n_sample, iters, threads=1):
    """Oracle build + plain CG stopped after `iters` iterations (the lattice MVMs the metric
    counts), on a seeded n_sample-row subsample of the workload, with `threads` threads
    (results are bit-identical for any count); returns (seconds, point-MVMs done, threads
    in effect)."""
    import oracle
    from oracle import OracleLattice
    from paper_2106_06695_gb300 import synth

    used = oracle.set_threads(threads)
    X = synth.gmm_points(W["n"], W["d"], W["seed"])
    V = synth.gaussian_values(W["n"], W["k"], W["seed"])
    rows = synth.subsample(W["n"], n_sample, W["seed"])
    Xs, Vs = X[rows], V[rows].astype(np.float64)
    t0 = time.perf_counter()
    L = OracleLattice(Xs, np.full(W["d"], W["lengthscale"], np.float32), r=W["order"])
    _, it, _ = L.cg(Vs, W["noise"], tol=0.0, max_iter=iters, mode=2)
    secs = time.perf_counter() - t0
    oracle.set_threads(1)
    return secs, float(n_sample) * int(it.max()), used


def cpu_baseline(W):
    import oracle

    cores = oracle.max_threads()
    secs1, units1, _ = oracle_sample(W, CPU_SAMPLE_1T["n"], CPU_SAMPLE_1T["iters"], 1)
    secs, units, used = oracle_sample(W, CPU_SAMPLE["n"], CPU_SAMPLE["iters"], cores)

    def what(smp):
        return ("FP64 oracle: lattice build (vertex insertion sequential) + %d plain CG "
                "iterations (symmetric operator, k=%d) on a seeded %d-row subsample of the "
                "workload" % (smp["iters"], W["k"], smp["n"]))
    return {"value": units / secs / 1e6, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": "%s, %d threads; %.1f s" % (what(CPU_SAMPLE), used, secs),
            "single_thread": {"value": units1 / secs1 / 1e6, "unit": UNIT, "cores": 1,
                              "sample": "%s, 1 thread; %.1f s" % (what(CPU_SAMPLE_1T), secs1)}}


def run_oracle_full(args):
    """The FP64 oracle on the whole workload: the lattice build (sequential vertex
    insertion) and one symmetric-operator MVM with k columns, once with every host core and
    once with one thread (results are bit-identical for any thread count).  Mpoint/s is
    n / MVM seconds, the unit of the metric."""
    import oracle
    from oracle import OracleLattice
    from paper_2106_06695_gb300 import synth

    W = dict(WORKLOAD, n=args.n)
    X = synth.gmm_points(W["n"], W["d"], W["seed"])
    V = synth.gaussian_values(W["n"], W["k"], W["seed"]).astype(np.float64)
    ls = np.full(W["d"], W["lengthscale"], np.float32)
    modes = []
    for threads in (oracle.max_threads(), 1):
        used = oracle.set_threads(threads)
        t0 = time.perf_counter()
        L = OracleLattice(X, ls, r=W["order"])
        build_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        L.mvm(V, mode=2)
        mvm_s = time.perf_counter() - t0
        modes.append({"threads": used, "build_s": build_s, "mvm_s": mvm_s,
                      "mvm_mpoint_s": W["n"] / mvm_s / 1e6, "m": int(L.m)})
        del L
    oracle.set_threads(1)
    print(json.dumps({"oracle_full": {"workload": "n=%d d=%d k=%d, symmetric operator"
                                                  % (W["n"], W["d"], W["k"]),
                                      "modes": modes}}), flush=True)


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle

    W = dict(WORKLOAD, n=args.n, precond_rank=args.precond_rank)
    cores = oracle.max_threads()
    for _ in range(args.warmup):
        oracle_sample(W, REF_SAMPLE["n"], REF_SAMPLE["iters"], cores)
    secs, units, used = 0.0, 0.0, 1
    for _ in range(args.steps):
        s, u, used = oracle_sample(W, REF_SAMPLE["n"], REF_SAMPLE["iters"], cores)
        secs += s
        units += u
    value = units / secs / 1e6
    sample = ("FP64 oracle, %d threads, per step: lattice build + %d plain CG iterations "
              "(symmetric operator, k=%d) on a seeded %d-row subsample of the workload"
              % (used, REF_SAMPLE["iters"], W["k"], REF_SAMPLE["n"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "GP solve n=%d d=%d k=%d (oracle sample of %d rows)"
                                   % (W["n"], W["d"], W["k"], REF_SAMPLE["n"])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serve_single():
    """Two preconditioned requests served alone (one slot), for the launch list and the
    counters of the preconditioner's kernels: d = 3 with n = 240k (363 vertices, condition
    estimate ~1e7) and d = 8 with n = 100k; 256 test points each, k = 1 + 8."""
    from paper_2106_06695_gb300 import synth
    from paper_2106_06695_gb300.serve import Server

    reqs = (synth.serving_stream(1, 901, n_range=(240_000, 240_001), dims=(3,))
            + synth.serving_stream(1, 902, n_range=(100_000, 100_001), dims=(8,)))
    out = []
    for r in reqs:
        with Server(max_active=1) as srv:
            rid = srv.submit(r["X"], r["y"], r["Xs"], r["lengthscales"], r["outputscale"],
                             r["noise"], r["seed"])
            srv.run_until_idle()
            st = srv.stats(rid)
        out.append({"d": r["X"].shape[1], "n": len(r["X"]), "m": st["m"],
                    "kappa_est": st["kappa_est"], "precond_rank": st["precond_rank"],
                    "iters": st["iters"], "rel_res": st["rel_res"],
                    "setup_ms": st["setup_us"] / 1e3,
                    "total_ms": (st["done_us"] - st["arrival_us"]) / 1e3})
    print(json.dumps({"serve_single": out}), flush=True)


def main(argv=None):
    args = parse_args(argv)
    world, rank, local = dist_env()
    if args.serve_single:
        run_serve_single()
        return
    if args.oracle_full:
        if rank == 0:
            run_oracle_full(args)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
