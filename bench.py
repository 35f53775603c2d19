"""Benchmark: k-eigenpair solves/sec of ARRABIT-MPM (Algorithm 8) on one GB300.

Workload (default): 3D 7-point Dirichlet Laplacian on a 128^3 grid (n = 2,097,152,
nnz = 14,581,760), k = 200 smallest eigenpairs (largest of 12 I - A), block p = 240,
Chebyshev-interpolant degree d = 20, q = 2 augmentation blocks, relative residual 1e-8.
Default precision: mixed_df (FP32 filter and FP32 block-Krylov Rayleigh-Ritz, then a
refinement phase to the same tolerance whose filter runs in double-float arithmetic and
whose Rayleigh-Ritz runs in FP64); --precision mixed refines with an FP64 filter,
--precision fp64 runs the plain FP64 path.
One step = one whole solve (every step of the hot path) with A and the Gaussian start block
already resident in HBM.

Printed JSON line: value (solves/s, device-timed), e2e (same metric through the C ABI with
host buffers: A and X0 uploaded from pinned host memory, eigenpairs read back), roofline of
the dominant kernel (the fused filter SpMM), the CPU oracle baseline, clocks, launches.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1507_06078_gb300 import inputs as I  # noqa: E402

METRIC = "k-eigenpair solves/sec at rel. residual 1e-8"
UNIT = "solves/s"
# Work counts of one solve of the 128^3 workload by the CUDA path at this commit (the bench
# line's solve.spmm_cols and solve.outer_iters, recorded in
# profiles/solve_counts_laplace3d_128.md).  The reference arm runs before the GPU arm and
# cannot read them live; it scales its oracle sample with these, and the GPU arm's
# cpu_baseline scales the same sample with the live counts.
SOLVE_COUNTS = {128: {"spmm_cols": 508266, "outer_iters": 4}}


def laplacian_3d_closed_form(m: int) -> np.ndarray:
    """Eigenvalues of the m^3 7-point Dirichlet Laplacian, ascending: sums of three 1D
    terms 2 - 2 cos(pi i / (m + 1))."""
    c = 2.0 - 2.0 * np.cos(np.pi * np.arange(1, m + 1) / (m + 1))
    return np.sort((c[:, None, None] + c[None, :, None] + c[None, None, :]).ravel())


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=128, help="3D grid side (128 = the benchmark workload)")
    ap.add_argument("--precision", default="mixed_df", choices=["mixed", "mixed_df", "fp64"])
    ap.add_argument("--b-update", default="every_arr", choices=["continuation", "every_arr"],
                    help="when b = mu_{k+q} is refreshed: at continuation steps (Algorithm 8) or after "
                         "every ARR (Section 5)")
    ap.add_argument("--no-compare-fp64", dest="compare_fp64", action="store_false",
                    help="skip the plain FP64 solve of the same workload (timed by default)")
    ap.add_argument("--no-serve-mix", dest="serve_mix", action="store_false",
                    help="skip the bounded served mix (p50/p99 latency, mixed and plain FP64) of the default run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the batched workload (256 diffusion instances in one lock-step solve)")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched workload: --instances instances, --precision, graph/autotune flags")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--c0", action="store_true", help="the 2D 64^2 workload: milliseconds per solve, FP64 and mixed")
    ap.add_argument("--batched-filter", action="store_true",
                    help="one batched filter call over --instances diffusion instances against per-instance calls")
    ap.add_argument("--c2", action="store_true", help="the full-size Chung-Lu workload (k = 500, p = 600)")
    ap.add_argument("--k", type=int, default=0)
    ap.add_argument("--c2-precisions", default="fp64,mixed")
    ap.add_argument("--ablations", action="store_true", help="RR vs ARR, degree, filter kind and k sweeps")
    ap.add_argument("--max-side", type=int, default=512, help="batched workload: largest grid side")
    ap.add_argument("--adapt-degree", action="store_true", help="batched workload: the paper's degree rule")
    ap.add_argument("--batch-flags", type=int, default=3, help="lock-step flags: 1 graphs, 2 autotune")
    ap.add_argument("--no-strict", dest="strict", action="store_false",
                    help="skip the tol 1e-9 solve whose residuals are all strictly within 1e-8")
    ap.add_argument("--filter-only", action="store_true",
                    help="only apply the filter (--reps times) to an n x --ncols block: for profiling")
    ap.add_argument("--dense-only", action="store_true",
                    help="only time the dense building blocks of one ARR at the workload's sizes: for profiling")
    ap.add_argument("--serve", action="store_true",
                    help="served mix: a seeded Poisson stream of solve requests against one server; "
                         "prints p50/p99 latency and solves/s")
    ap.add_argument("--rate", type=float, default=8.0, help="served mix: arrivals per second")
    ap.add_argument("--requests", type=int, default=36, help="served mix: number of requests")
    ap.add_argument("--slots", type=int, default=4, help="--serve: concurrent solves of the server")
    ap.add_argument("--ncols", type=int, default=0)
    ap.add_argument("--chung-lu", type=int, default=0,
                    help="filter-only: the Chung-Lu normalised graph Laplacian with this many rows instead")
    ap.add_argument("--sell", default="",
                    help="filter-only: give the matrix a SELL-C-sigma copy, 'C,sigma' (e.g. 32,1024)")
    ap.add_argument("--degree", type=int, default=0)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tol-switch", type=float, default=0.0,
                    help="mixed paths: residual at which the FP32 phase hands over (0: library default)")
    return ap.parse_args()


def workload(m):
    if m == 128:
        return I.workload_3d128()
    k = max(8, int(round(200 * (m / 128) ** 3)))
    p = int(round(1.2 * k))
    return I.workload_3d(m, k, p)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        # the raw samples go to $ARB_BENCH_OUT (default: the system temp directory)
        out = os.environ.get("ARB_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_dev{device}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sms if s > 0.5 * max(sms)] or sms
        return {"sm_mhz": float(np.median(busy)), "sm_max_mhz": float(max(maxs)), "reasons": sorted(reasons),
                "samples": len(sms)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def filter_algorithmic_bytes(n, nnz, p, d, s=8, z=8):
    """Algorithmic HBM bytes of one Clenshaw filter application (d fused SpMM passes):
    every pass reads A once (nnz*(8+4) + 4(n+1)); the block traffic is 2 n p s for the
    first pass (read X, write b_{d-1}), 3 n p s for the second (read b_{d-1}, X; write) and
    4 n p s for every later pass (read b_{j+1}, b_{j+2}, X; write b_j)."""
    a_bytes = nnz * (z + 4) + 4 * (n + 1)
    blocks = 2 + (3 if d >= 2 else 0) + 4 * max(d - 2, 0)
    return d * a_bytes + blocks * n * p * s


class RowBlockOperator:
    """B @ Y computed as independent products of row blocks of B on a thread pool (scipy's
    sparse products release the GIL): every row is computed exactly as B @ Y computes it,
    only different rows run on different cores.  Lets the oracle's unchanged filter run
    on all host cores."""

    def __init__(self, B, threads):
        from concurrent.futures import ThreadPoolExecutor
        self.B = B
        self.shape = B.shape
        cuts = np.linspace(0, B.shape[0], threads + 1).astype(np.int64)
        self.blocks = [(int(a), int(b), B[a:b]) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
        self.pool = ThreadPoolExecutor(threads)

    def __matmul__(self, Y):
        out = np.empty((self.shape[0],) + Y.shape[1:], dtype=np.result_type(self.B.dtype, Y.dtype))

        def part(blk):
            a, b, Bb = blk
            out[a:b] = Bb @ Y

        list(self.pool.map(part, self.blocks))
        return out


def cpu_oracle_sample(W, counts, budget_s=20.0, degree=2):
    """Extrapolated oracle time per solve: the oracle's own Clenshaw filter
    (oracle.poly_clenshaw, FP64, unchanged) applied to the full workload block on all host
    cores (row blocks of B on a thread pool) for about budget_s seconds; its time per
    SpMV-equivalent column times the solve's count of such columns.  The oracle's dense
    Rayleigh-Ritz work is left out, so this is a lower bound on the oracle's time per solve."""
    import scipy.sparse as sp
    from oracle import arrabit_oracle as O
    A = O.csr_to_scipy(W.A.n, W.A.rowptr, W.A.col, W.A.val)
    sigma = O.gershgorin_bounds(A)[1]
    threads = os.cpu_count() or 1
    B = RowBlockOperator((sigma * sp.identity(W.A.n, format="csr") - A).tocsr(), threads)
    X = I.gaussian_block(W.A.n, W.p, W.seed)
    coef = O.interpolant_cheb_coeffs(degree)
    t0 = time.perf_counter()
    calls = 0
    while True:
        O.poly_clenshaw(B, X, 0.0, 0.99 * sigma, coef)
        calls += 1
        if time.perf_counter() - t0 > budget_s:
            break
    B.pool.shutdown()
    t_col = (time.perf_counter() - t0) / (calls * degree * W.p)
    cols = int(counts["spmm_cols"])
    solve_s = t_col * cols
    return {"value": 1.0 / solve_s, "unit": UNIT, "cores": threads, "kind": "oracle",
            "extrapolated": True,
            "sample": f"{calls} calls of oracle.poly_clenshaw (degree {degree}: {calls * degree} full-size SpMM "
                      f"steps of width {W.p}, {t_col * W.p:.3f} s per step on {threads} threads) scaled by "
                      f"{cols} SpMV-equivalent columns per solve; dense Rayleigh-Ritz work excluded "
                      "(a lower bound on the oracle's time)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    W = workload(args.grid)
    counts = SOLVE_COUNTS.get(args.grid)
    if counts is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no recorded solve counts for grid {args.grid}"}))
        return
    samples = []
    r = None
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_sample(W, counts, budget_s=4.0)
        if i >= args.warmup:
            samples.append(r["value"])
    v = float(np.mean(samples))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W.name, "n": W.A.n, "nnz": W.A.nnz, "k": W.k, "p": W.p, "q": W.q,
                       "degree": W.degree, "tol": W.tol},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "extrapolated": True, "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1507_06078_gb300 import arrabit as arb
    from paper_1507_06078_gb300 import build

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    build.build()
    W = workload(args.grid)
    ctx = arb.Context(local)
    stream = ctx.stream
    mat = arb.Matrix.from_csr(ctx, W.A)
    X0h = I.gaussian_block(W.A.n, W.p, W.seed + rank)
    X0 = torch.from_numpy(X0h).cuda(local)
    opts = arb.arb_options_default(W.k)
    opts.p, opts.q, opts.degree = W.p, W.q, W.degree
    opts.precision = {"mixed": arb.ARB_MIXED, "mixed_df": arb.ARB_MIXED_DF, "fp64": arb.ARB_FP64}[args.precision]
    opts.b_update = 1 if args.b_update == "every_arr" else 0
    opts.tol_switch = args.tol_switch

    def step():
        return arb.arb_solve(ctx, mat, W.k, arb.ARB_SMALLEST, W.tol, opts, x0=X0, evecs="device")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        r = step()
    barrier()
    launches0 = ctx.launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    infos = []
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            r = step()
            infos.append(r.info)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    launches = (ctx.launches() - launches0) // max(args.steps, 1)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per = ms / args.steps
    value = world * args.steps / (ms * 1e-3)
    # correctness of the timed solves: closed-form spectrum and residuals
    lam = laplacian_3d_closed_form(args.grid)[:W.k]  # closed form, no oracle involved
    eig_err = float(np.max(np.abs(r.evals - lam) / np.maximum(1.0, np.abs(lam))))

    # dominant kernel: the fused filter SpMM (one filter = W.degree launches), timed live
    # with CUDA events on the context's stream, on the full n x p block of the workload
    coef = arb.arb_filter_coefficients(arb.ARB_FILTER_CHEBINTERP, W.degree)
    if args.precision in ("mixed", "mixed_df"):
        Xf = X0.float()
        run_filter = lambda Y: arb.arb_filter_f32(ctx, mat, -1.0, 12.0, 0.0, 11.9, coef, Xf, Y=Y)  # noqa: E731
        s_bytes, z_bytes, kname = 4, 4, "spmm_fused_kernel<float,4> (Clenshaw filter pass, FP32)"
    else:
        Xf = X0
        run_filter = lambda Y: arb.arb_filter(ctx, mat, -1.0, 12.0, 0.0, 11.9, coef, Xf, Y=Y)  # noqa: E731
        s_bytes, z_bytes, kname = 8, 8, "spmm_fused_kernel<double,2> (Clenshaw filter pass, FP64)"
    Yf = torch.empty_like(Xf)
    run_filter(Yf)
    barrier()
    nrep = 3
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(nrep):
        run_filter(Yf)
    e1.record(stream)
    barrier()
    f_ms = e0.elapsed_time(e1) / nrep
    del Yf
    fbytes = filter_algorithmic_bytes(W.A.n, W.A.nnz, W.p, W.degree, s=s_bytes, z=z_bytes)
    fflops = W.degree * (2.0 * W.A.nnz * W.p + 6.0 * W.A.n * W.p)
    peak, peak_src = measured_peaks()
    achieved = fbytes / (f_ms * 1e-3) / 1e9
    # DRAM bytes per launch: ncu's dram__bytes_read.sum + dram__bytes_write.sum on a
    # 100^3 x 240 FP32 filter pass of this kernel came to 1.000 x its algorithmic bytes
    # (2.9399 GB vs 2.9395 GB); scaled to the full launch by the same ratio (the FP32 kernel only)
    traffic = 1.000 * fbytes / W.degree if s_bytes == 4 else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kname, "launch_ms": f_ms / W.degree,
            "algorithmic_bytes_per_launch": fbytes / W.degree, "flops_per_launch": fflops / W.degree,
            "peak_source": peak_src + " hbm_gbs (STREAM-style copy)"}

    fp64_cmp = None
    if args.compare_fp64 and args.precision != "fp64":
        o64 = arb.arb_options_default(W.k)
        o64.p, o64.q, o64.degree, o64.precision = W.p, W.q, W.degree, arb.ARB_FP64
        o64.b_update = opts.b_update
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        r64 = arb.arb_solve(ctx, mat, W.k, arb.ARB_SMALLEST, W.tol, o64, x0=X0, evecs="device")
        t1.record(stream)
        barrier()
        ms64 = t0.elapsed_time(t1)
        fp64_cmp = {"solves_per_s": 1e3 / ms64, "ms_per_solve": ms64, "speedup_mixed_vs_fp64": ms64 / ms_per,
                    "maxres": r64.info["maxres"], "outer_iters": r64.info["outer_iters"],
                    "eig_rel_err_vs_closed_form": float(np.max(np.abs(r64.evals - lam) / np.maximum(1.0, np.abs(lam)))),
                    "max_eig_diff_vs_mixed": float(np.max(np.abs(r64.evals - r.evals) / np.maximum(1.0, np.abs(lam))))}

    # the same workload run to tol 1e-9: the paper's near-tolerance rule (iii) then stops at
    # maxres < (1 + 9h/k) 1e-9 <= 1e-8 at the latest, so every residual is strictly within
    # the metric's 1e-8 (the headline solve at tol 1e-8 may end up to (1 + 9h/k) 1e-8)
    strict = None
    if args.strict:
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        rs = arb.arb_solve(ctx, mat, W.k, arb.ARB_SMALLEST, 1e-9, opts, x0=X0, evecs="device")
        t1.record(stream)
        barrier()
        ms_s = t0.elapsed_time(t1)
        strict = {"tol": 1e-9, "solves_per_s": 1e3 / ms_s, "ms_per_solve": ms_s, "maxres": rs.info["maxres"],
                  "stop": rs.info["stop_reason"], "outer_iters": rs.info["outer_iters"],
                  "eig_rel_err_vs_closed_form": float(np.max(np.abs(rs.evals - lam) / np.maximum(1.0, np.abs(lam))))}
        if fp64_cmp is not None:
            o64s = arb.arb_options_default(W.k)
            o64s.p, o64s.q, o64s.degree, o64s.precision = W.p, W.q, W.degree, arb.ARB_FP64
            o64s.b_update = opts.b_update
            barrier()
            t0.record(stream)
            r64s = arb.arb_solve(ctx, mat, W.k, arb.ARB_SMALLEST, 1e-9, o64s, x0=X0, evecs="device")
            t1.record(stream)
            barrier()
            ms64s = t0.elapsed_time(t1)
            strict["fp64_solves_per_s"] = 1e3 / ms64s
            strict["fp64_maxres"] = r64s.info["maxres"]
            strict["speedup_vs_fp64"] = ms64s / ms_s

    e2e = None
    if not args.no_e2e:
        pin_rowptr = torch.from_numpy(W.A.rowptr).pin_memory()
        pin_col = torch.from_numpy(W.A.col).pin_memory()
        pin_val = torch.from_numpy(W.A.val).pin_memory()
        pin_x0 = torch.from_numpy(X0h).pin_memory()
        out_vecs = torch.empty((W.k, W.A.n), dtype=torch.float64).pin_memory()
        import ctypes as C
        lib = arb.load()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            h = C.c_void_p()
            st = lib.arb_matrix_create_csr(ctx.handle, W.A.n, W.A.nnz, pin_rowptr.data_ptr(), pin_col.data_ptr(),
                                           pin_val.data_ptr(), 0, C.byref(h))
            assert st == 0
            ev = np.zeros(W.k)
            info = arb.arb_info()
            st = lib.arb_solve(ctx.handle, h, W.k, arb.ARB_SMALLEST, W.tol, C.byref(opts), pin_x0.data_ptr(), 0,
                               ev.ctypes.data, out_vecs.data_ptr(), W.A.n, 0, C.byref(info))
            lib.arb_matrix_destroy(h)
            assert st in (0, 1)
        barrier()
        t_e2e = (time.perf_counter() - t0) / args.steps
        h2d = W.A.rowptr.nbytes + W.A.col.nbytes + W.A.val.nbytes + X0h.nbytes
        d2h = W.k * W.A.n * 8 + W.k * 8
        e2e = {"value": world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # the workload's ~76 GB of workspaces go back before the served mix and the batch
    mat.close()
    ctx.close()
    torch.cuda.empty_cache()

    batched = None
    if rank == 0 and world == 1 and args.batched:
        from paper_1507_06078_gb300 import arrabit as arbm
        # 256 instances at the small end of the batched workload's sides (32-128): the full
        # range (sides to 512) takes ~750 s, most of it in instances that reach maxit
        batched = batched_c3(256, arbm.ARB_MIXED, arbm.ARB_BATCH_GRAPHS | arbm.ARB_BATCH_AUTOTUNE, sides=(32, 128))

    served = None
    if rank == 0 and world == 1 and args.serve_mix:
        # the mixed form with an FP64 refinement: on the 125k-row Chung-Lu kind the
        # double-float refinement stalls near 1e-7 where FP64 converges
        mix = served_mix(arb.ARB_MIXED, args.rate, args.requests, args.slots)
        mix64 = served_mix(arb.ARB_FP64, args.rate, args.requests, args.slots)
        served = {"mixed": mix, "fp64": mix64,
                  "p99_speedup_vs_fp64": mix64["p99_s"] / mix["p99_s"],
                  "solves_per_s_speedup_vs_fp64": mix["solves_per_s"] / max(mix64["solves_per_s"], 1e-30)}

    small = None
    if rank == 0 and world == 1:
        small = _guarded(lambda: c0_timings(steps=5, warmup=2))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_sample(W, {"spmm_cols": int(np.mean([i["spmm_cols"] for i in infos]))})
        cpu["full_solves"] = _guarded(lambda: cpu_full_solves(budget_s=20.0))

    if rank == 0:
        info = infos[-1]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"mixed": "f32+f64", "mixed_df": "f32+f32x2+f64", "fp64": "f64"}[args.precision],
                "data": "synthetic",
                "config": {"workload": W.name, "n": W.A.n, "nnz": W.A.nnz, "k": W.k, "p": W.p, "q": W.q,
                           "degree": W.degree, "tol": W.tol, "precision": args.precision,
                           "b_update": args.b_update,
                           "l2": "inputs larger than L2 (A 175 MB, X0 4 GB, work blocks ~50 GB)",
                           "parallelism": "replicas" if world > 1 else "single"},
                "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "clocks": clk.summary(),
                "gpu_launches": int(launches), "fp64_path": fp64_cmp, "strict_1e-8": strict, "served": served,
                "batched_c3": batched, "small_c0": small,
                "solve": {"eig_rel_err_vs_closed_form": eig_err, "maxres": info["maxres"],
                          "outer_iters": info["outer_iters"], "n_filters": info["n_filters"],
                          "spmm_cols": info["spmm_cols"], "t_filter_s": info["t_filter"],
                          "t_arr_s": info["t_arr"], "stop": info["stop_reason"],
                          "outer_iters_fp32": info["outer_iters_fp32"]}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_dense_only(args):
    """Time (CUDA events, context stream, after one warm-up call) the dense products of the
    Rayleigh-Ritz steps at the workload's sizes: FP32 Grams (tensor cores), FP64 and
    double-float Grams, and the Jacobi eigensolver at m = p and m = (q+1) p."""
    import torch

    from paper_1507_06078_gb300 import arrabit as arb
    from paper_1507_06078_gb300 import build
    build.build()
    W = workload(args.grid)
    p = args.ncols or W.p
    n, m = W.A.n, (W.q + 1) * p
    ctx = arb.Context(0)
    ctx_df = arb.Context(0)
    ctx_df.set_dense_df(True)

    def timed(f, reps=3, c=ctx):
        f()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(c.stream)
        for _ in range(reps):
            f()
        e1.record(c.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"dense_only": True, "n": n, "p": p, "m": m}
    X32 = torch.randn((n, p), dtype=torch.float32, device="cuda")
    out["gram_f32_pxp_sym_ms"] = timed(lambda: arb.arb_gram_f32(ctx, X32, X32))
    U32 = torch.randn((n, m), dtype=torch.float32, device="cuda")
    AU32 = torch.randn((n, m), dtype=torch.float32, device="cuda")
    out["gram_f32_mxm_ms"] = timed(lambda: arb.arb_gram_f32(ctx, U32, AU32), reps=1)
    # the FP32 phase's Ritz rotation U V (n x (q+1)p times (q+1)p x p): tensor cores, and the
    # CUDA-core kernel on the same data with an odd leading dimension
    Vr = torch.randn((m, p), dtype=torch.float64, device="cuda")
    R32 = torch.empty((n, p), dtype=torch.float32, device="cuda")
    out["gemm_tc_mxp_ms"] = timed(lambda: arb.arb_gemm_tall_f32(ctx, U32, Vr, 1.0, 0.0, R32), reps=2)
    del AU32
    Uo = torch.empty((n, m + 1), dtype=torch.float32, device="cuda")[:, :m]
    Uo.copy_(U32)
    del U32
    out["gemm_cuda_core_mxp_ms"] = timed(lambda: arb.arb_gemm_tall_f32(ctx, Uo, Vr, 1.0, 0.0, R32), reps=1)
    del Uo, R32
    X64 = torch.randn((n, p), dtype=torch.float64, device="cuda")
    out["gram_f64_pxp_sym_ms"] = timed(lambda: arb.arb_gram(ctx, X64, X64), reps=1)
    out["gram_df_pxp_sym_ms"] = timed(lambda: arb.arb_gram(ctx_df, X64, X64), reps=2, c=ctx_df)
    for mm in (p, m):
        H = torch.randn((mm, mm), dtype=torch.float64, device="cuda")
        H = 0.5 * (H + H.T)
        out[f"syevj_{mm}_ms"] = timed(lambda: arb.arb_syevj(ctx, H), reps=2)
        out[f"syevj_df_{mm}_ms"] = timed(lambda: arb.arb_syevj(ctx_df, H), reps=2, c=ctx_df)
    print(json.dumps(out))


def run_filter_only(args):
    """Apply the Chebyshev-interpolant filter to a Gaussian block of the workload matrix and
    print the per-pass time (CUDA events on the context's stream)."""
    import torch

    from paper_1507_06078_gb300 import arrabit as arb
    from paper_1507_06078_gb300 import build
    build.build()
    W = workload(args.grid)
    A, shift, b = W.A, 12.0, 11.9  # S = 12 I - A maps the 3D Laplacian's spectrum into [0, 12]
    if args.chung_lu:
        A, _ = I.chung_lu_laplacian(args.chung_lu, seed=1507)
        shift, b = 2.0, 1.9  # a normalised Laplacian's spectrum lies in [0, 2]
    ncols = args.ncols or W.p
    d = args.degree or W.degree
    ctx = arb.Context(0)
    mat = arb.Matrix.from_csr(ctx, A)
    if args.sell:
        c_, s_ = (int(v) for v in args.sell.split(","))
        mat.set_sell(c_, s_)
    X = arb.arb_gaussian_block(ctx, A.n, ncols, W.seed)
    if args.precision == "mixed":
        X = X.float()
        f = arb.arb_filter_f32
        s = 4
    elif args.precision == "mixed_df":  # double-float passes (plus one conversion each way per filter)
        f = arb.arb_filter_df
        s = 8
    else:
        f = arb.arb_filter
        s = 8
    Y = torch.empty_like(X)
    coef = arb.arb_filter_coefficients(arb.ARB_FILTER_CHEBINTERP, d)
    f(ctx, mat, -1.0, shift, 0.0, b, coef, X, Y=Y)  # warm-up: workspaces, kernel attributes
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(args.reps):
        f(ctx, mat, -1.0, shift, 0.0, b, coef, X, Y=Y)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (args.reps * d)
    nb = filter_algorithmic_bytes(A.n, A.nnz, ncols, d, s=s, z=s) / d
    print(json.dumps({"filter_only": True, "n": A.n, "nnz": A.nnz, "ncols": ncols, "degree": d,
                      "precision": args.precision, "layout": ("sell " + args.sell) if args.sell else "csr",
                      "ms_per_pass": ms, "algorithmic_GBps": nb / ms / 1e6}))


def served_mix(precision, rate, requests, slots, seed=4242):
    """Served mix, bounded: a seeded Poisson stream of solve requests in equal thirds of 2D
    64^2 Laplacian problems (k = 20, p = 30, d = 10), variable-coefficient diffusion
    instances (sides 32-256, k 8-64, p = 1.5k, d = 20) and a 1/8-scale Chung-Lu graph
    Laplacian (n ~ 125k, k 10-60, p = 1.2k, d = 15), all with q = 1, b refreshed after every
    ARR (Section 5) and relative residual 1e-8 in the given precision (arb_precision),
    against one server with `slots` concurrent solves.  Latency is the library's
    submit-to-completion wall time; p50/p99 are over the requests that converged (the others
    are counted per kind); solves/s counts converged requests over first submission to last
    completion."""
    from paper_1507_06078_gb300 import arrabit as arb
    ctx = arb.Context(0)
    rng = np.random.Generator(np.random.Philox(seed))
    w0 = I.workload_2d64()
    lap2d = arb.Matrix.from_csr(ctx, w0.A)
    diff = I.batched_diffusion_instances(count=4, base_seed=42420, side_range=(32, 256))
    diff_m = [arb.Matrix.from_csr(ctx, w.A) for w in diff]
    cl, _ = I.chung_lu_laplacian(125000, seed=4242)
    cl_m = arb.Matrix.from_csr(ctx, cl)
    reqs = []
    for _ in range(requests):
        kind = int(rng.integers(0, 3))
        if kind == 0:
            reqs.append(("laplace2d_64", lap2d, 20, 30, 10))
        elif kind == 1:
            j = int(rng.integers(0, len(diff)))
            reqs.append((diff[j].name, diff_m[j], diff[j].k, diff[j].p, 20))
        else:
            k = int(rng.integers(10, 61))
            reqs.append(("chung_lu_125k", cl_m, k, int(round(1.2 * k)), 15))
    gaps = rng.exponential(1.0 / rate, size=requests)
    srv = arb.Server(0, hbm_budget_bytes=64 << 30, max_slots=slots)
    tickets, t_sub = [], []
    t0 = time.perf_counter()
    t_next = t0
    for (name, mat, k, p, d), g in zip(reqs, gaps):
        t_next += g
        delay = t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        o = arb.arb_options_default(k)
        o.p, o.q, o.degree, o.precision, o.b_update = p, 1, d, precision, 1
        t_sub.append(time.perf_counter())
        tickets.append(srv.submit(mat, k, arb.ARB_SMALLEST, 1e-8, o, want_evecs=False))
    lat, conv, worst = [], [], 0.0
    per_kind = {}
    for (name, *_), t in zip(reqs, tickets):
        r = srv.wait(t)
        lat.append(r.info["latency_s"])
        conv.append(r.status == arb.ARB_OK)
        worst = max(worst, r.info["maxres"])
        kd = per_kind.setdefault(name, {"requests": 0, "converged": 0, "max_maxres": 0.0, "stops": {}})
        kd["requests"] += 1
        kd["converged"] += int(r.status == arb.ARB_OK)
        kd["max_maxres"] = max(kd["max_maxres"], r.info["maxres"])
        kd["stops"][r.info["stop_reason"]] = kd["stops"].get(r.info["stop_reason"], 0) + 1
        kd.setdefault("latencies_s", []).append(r.info["latency_s"])
        kd.setdefault("solve_s", []).append(r.info["t_total"])
    for kd in per_kind.values():
        kd["mean_latency_s"] = float(np.mean(kd.pop("latencies_s")))
        kd["mean_solve_s"] = float(np.mean(kd.pop("solve_s")))
    srv.close()
    done = max(ts + lt for ts, lt in zip(t_sub, lat))
    lat = np.array(lat)
    conv = np.array(conv)
    lc = lat[conv] if conv.any() else np.array([np.nan])
    return {"precision": {0: "fp64", 1: "mixed", 2: "mixed_df"}[precision], "rate_per_s": rate,
            "requests": requests, "slots": slots, "converged": int(conv.sum()), "max_maxres": worst,
            "p50_s": float(np.percentile(lc, 50)), "p99_s": float(np.percentile(lc, 99)),
            "mean_s": float(lc.mean()), "p99_all_s": float(np.percentile(lat, 99)),
            "solves_per_s": float(conv.sum()) / (done - t_sub[0]), "by_kind": per_kind, "tol": 1e-8}


def batched_c3(instances, precision, flags, sides=(32, 512), degree=20, adapt_degree=False, compare_slots=True):
    """Batched workload: `instances` 2D variable-coefficient diffusion operators (5-point,
    lognormal edge coefficients, seeds 30000 + i, sides uniform in `sides`, k uniform in
    8..64, p = 1.5 k), smallest pairs to relative residual 1e-8, q = 1, b refreshed after
    every ARR, degree 20 (or the paper's adaptive rule from `degree`, cap 20), solved together by
    arb_solve_lockstep (one batched filter launch per round, rounds replayed from CUDA
    graphs, SpMM layout autotuned per matrix).  Returns the whole batch's solves/s (CUDA
    events around the call), convergence, launch statistics and a dense-eigenvalue check of
    the two smallest instances."""
    import torch
    from paper_1507_06078_gb300 import arrabit as arb
    ctx = arb.Context(0)
    ws = I.batched_diffusion_instances(count=instances, base_seed=30000, side_range=sides)
    probs = []
    for w in ws:
        o = arb.arb_options_default(w.k)
        o.p, o.q, o.degree, o.precision, o.b_update = w.p, 1, degree, precision, 1
        if adapt_degree:
            o.adapt, o.d_max = arb.ARB_ADAPT_DEGREE, 20
        probs.append(dict(mat=arb.Matrix.from_csr(ctx, w.A), k=w.k, which=arb.ARB_SMALLEST, tol=1e-8, opts=o,
                          x0=I.gaussian_block(w.A.n, w.p, w.seed)))
    # every instance of a lock-step call holds its workspaces for the whole call: the batch
    # goes in chunks whose summed footprints stay within a budget of HBM
    chunks, cur, used = [], [], 0
    budget = 100 << 30
    for pr, w in zip(probs, ws):
        f = arb.arb_server_footprint(w.A.n, w.A.nnz, w.p, 1, precision) + 8 * w.A.n * ((w.p + 3) // 4 * 4)
        if cur and used + f > budget:
            chunks.append(cur)
            cur, used = [], 0
        cur.append(pr)
        used += f
    chunks.append(cur)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(ctx.stream)
    res, st, stats = [], arb.ARB_OK, {}
    for ch in chunks:
        st_c, res_c, stats_c = arb.arb_solve_lockstep(ctx, ch, flags=flags, evecs=False)
        res += res_c
        st = st if st != arb.ARB_OK else st_c
        for key, v in stats_c.items():
            stats[key] = stats.get(key, 0) + v
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    conv = sum(r.info["stop_reason"] in ("converged", "near_tol") for r in res)
    # the same problems through arb_solve_batched (independent solves on 8 concurrent
    # streams, no batched filter), for comparison
    slots = None
    if compare_slots:
        e0.record(ctx.stream)
        t1 = time.perf_counter()
        for ch in chunks:
            arb.arb_solve_batched(ctx, ch, max_concurrent=8, evecs=False)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        slots = {"solves_per_s": instances / (e0.elapsed_time(e1) * 1e-3), "wall_s": time.perf_counter() - t1}
    small = sorted(range(len(ws)), key=lambda i: ws[i].A.n)[:2]
    err = 0.0
    for i in small:
        lam = np.linalg.eigvalsh(ws[i].A.to_dense())[:ws[i].k]
        err = max(err, float(np.max(np.abs(res[i].evals - lam) / np.maximum(1.0, np.abs(lam)))))
    return {"instances": instances, "precision": {0: "fp64", 1: "mixed", 2: "mixed_df"}[precision],
            "solves_per_s": instances / (ms * 1e-3), "ms": ms, "wall_s": wall, "converged": int(conv),
            "max_maxres": float(max(r.info["maxres"] for r in res)),
            "n_total": int(sum(w.A.n for w in ws)), "k_total": int(sum(w.k for w in ws)),
            "final_degrees": sorted({r.info["final_d"] for r in res}),
            "eig_rel_err_two_smallest_vs_dense": err, "stats": stats, "status": st, "chunks": len(chunks),
            "sides": list(sides), "degree": degree, "adaptive_degree": adapt_degree, "concurrent_streams": slots}


def run_serve(args):
    """--serve: the served mix at --rate / --requests / --slots in the chosen precision."""
    from paper_1507_06078_gb300 import build
    build.build()
    prec = {"mixed": 1, "mixed_df": 2, "fp64": 0}[args.precision]
    out = served_mix(prec, args.rate, args.requests, args.slots)
    out["serve"] = True
    print(json.dumps(out))


def _solve_timed(arb, ctx, mat, k, o, x0, tol=1e-8, which=None):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    r = arb.arb_solve(ctx, mat, k, arb.ARB_SMALLEST if which is None else which, tol, o, x0=x0, evecs="device")
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    return r, e0.elapsed_time(e1) * 1e-3


def run_c2(args):
    """The Chung-Lu workload at full size: normalised Laplacian of the largest component of
    a Chung-Lu graph with n = 1e6 (power-law expected degrees, exponent 2.5, mean 16, max
    5000; seed 1507), k = 500 smallest pairs, p = 600, degree 15, q = 1, relative residual
    1e-8, b refreshed after every ARR; the matrix in its original order and after a reverse
    Cuthill-McKee reordering (SELL-C-sigma C = 32, sigma = 1024 when --sell).  Prints one
    filter pass per layout and the solve in the chosen precisions."""
    import torch
    from paper_1507_06078_gb300 import arrabit as arb
    from paper_1507_06078_gb300 import build
    build.build()
    t0 = time.perf_counter()
    A, _ = I.chung_lu_laplacian(args.chung_lu or 1_000_000, seed=1507)
    t_gen = time.perf_counter() - t0
    R, perm = I.rcm_permuted(A)
    k, p = args.k or 500, int(round(1.2 * (args.k or 500)))
    ctx = arb.Context(0)
    out = {"c2": True, "n": A.n, "nnz": A.nnz, "k": k, "p": p, "t_generate_s": t_gen}
    coef = arb.arb_filter_coefficients(arb.ARB_FILTER_CHEBINTERP, 15)
    passes = {}
    for name, M, sell in (("csr", A, None), ("sell32", A, (32, 1024)), ("rcm_csr", R, None), ("rcm_sell32", R, (32, 1024))):
        mat = arb.Matrix.from_csr(ctx, M)
        if sell:
            mat.set_sell(*sell)
        X = arb.arb_gaussian_block(ctx, M.n, p, 5).float()
        Y = torch.empty_like(X)
        arb.arb_filter_f32(ctx, mat, -1.0, 2.0, 0.0, 1.9, coef, X, Y=Y)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        arb.arb_filter_f32(ctx, mat, -1.0, 2.0, 0.0, 1.9, coef, X, Y=Y)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 15
        passes[name] = {"ms_per_pass": ms, "algorithmic_GBps": filter_algorithmic_bytes(M.n, M.nnz, p, 15, 4, 4) / 15 / ms / 1e6}
        del X, Y
        mat.close()
    out["filter_pass_fp32"] = passes
    mat = arb.Matrix.from_csr(ctx, R)
    mat.set_sell(32, 1024)
    x0 = I.gaussian_block(R.n, p, 20150724)
    solves = {}
    for prec in args.c2_precisions.split(","):
        o = arb.arb_options_default(k)
        o.p, o.q, o.degree, o.b_update = p, 1, 15, 1
        o.precision = {"fp64": arb.ARB_FP64, "mixed": arb.ARB_MIXED, "mixed_df": arb.ARB_MIXED_DF}[prec]
        r, sec = _solve_timed(arb, ctx, mat, k, o, x0)
        solves[prec] = {"seconds": sec, "status": r.status, "maxres": r.info["maxres"], "stop": r.info["stop_reason"],
                        "outer_iters": r.info["outer_iters"], "n_filters": r.info["n_filters"],
                        "lambda_1": float(r.evals[0]), "lambda_k": float(r.evals[-1])}
        print(json.dumps({"c2_solve": prec, **solves[prec]}), flush=True)
    out["solves"] = solves
    print(json.dumps(out))


def run_ablations(args):
    """Synthetic analogues of the paper's ablations and k sweep (Tables ARR, polydeg,
    comp-cheby, and the k-scaling runs of Section 6.4) on the GPU path: one solve per
    setting, CUDA-event time, outer iterations and SpMV-equivalent columns.
    * RR vs ARR: q = 0, 1, 2 and the adaptive rule (eq. block), 3D 48^3 Laplacian, k = 50.
    * degree: d = 5, 10, 15, 20 and the adaptive rule (eqs. hat-d, degree) from d = 3.
    * filter: Chebyshev interpolant of max(0,t)^(10d) vs the plain Chebyshev T_d, d = 10, 20.
    * k sweep: k = 25, 50, 100, 200 on the 3D 64^3 Laplacian (p = 1.2 k, d = 20, q = 2).
    All smallest pairs to relative residual 1e-8 in FP64 except the k sweep (mixed_df)."""
    from paper_1507_06078_gb300 import arrabit as arb
    from paper_1507_06078_gb300 import build
    build.build()
    ctx = arb.Context(0)
    A = I.laplacian_3d(48)
    mat = arb.Matrix.from_csr(ctx, A)
    k, p = 50, 60
    x0 = I.gaussian_block(A.n, p, 77)
    lam = laplacian_3d_closed_form(48)[:k]
    rows = []

    def one(group, setting, o, M=mat, kk=k, xx=x0, ll=lam):
        r, sec = _solve_timed(arb, ctx, M, kk, o, xx)
        err = float(np.max(np.abs(r.evals - ll) / np.maximum(1.0, np.abs(ll))))
        row = {"group": group, "setting": setting, "seconds": sec, "outer_iters": r.info["outer_iters"],
               "spmm_cols": r.info["spmm_cols"], "stop": r.info["stop_reason"], "maxres": r.info["maxres"],
               "final_q": r.info["final_q"], "final_d": r.info["final_d"], "eig_err": err}
        rows.append(row)
        print(json.dumps(row), flush=True)

    def opts(q=1, d=15, filt=arb.ARB_FILTER_CHEBINTERP, adapt=0, prec=arb.ARB_FP64, kk=k, pp=p):
        o = arb.arb_options_default(kk)
        o.p, o.q, o.degree, o.filter, o.adapt, o.precision, o.b_update = pp, q, d, filt, adapt, prec, 1
        return o

    for q in (0, 1, 2):
        one("rr_vs_arr", f"q={q}", opts(q=q))
    one("rr_vs_arr", "adaptive q", opts(q=1, adapt=arb.ARB_ADAPT_Q))
    for d in (5, 10, 15, 20):
        one("degree", f"d={d}", opts(d=d))
    one("degree", "adaptive d from 3", opts(d=3, adapt=arb.ARB_ADAPT_DEGREE))
    for d in (10, 20):
        one("filter", f"interpolant d={d}", opts(d=d))
        one("filter", f"chebyshev T_d d={d}", opts(d=d, filt=arb.ARB_FILTER_CHEBYSHEV))
    A64 = I.laplacian_3d(64)
    m64 = arb.Matrix.from_csr(ctx, A64)
    lam64 = laplacian_3d_closed_form(64)
    for kk in (25, 50, 100, 200):
        pp = int(round(1.2 * kk))
        one("k_sweep", f"k={kk}", opts(q=2, d=20, prec=arb.ARB_MIXED_DF, kk=kk, pp=pp), M=m64, kk=kk,
            xx=I.gaussian_block(A64.n, pp, 78), ll=lam64[:kk])
    print(json.dumps({"ablations": True, "rows": rows}))


def run_batched_only(args):
    from paper_1507_06078_gb300 import build
    build.build()
    prec = {"mixed": 1, "mixed_df": 2, "fp64": 0}[args.precision]
    out = batched_c3(args.instances, prec, args.batch_flags, sides=(32, args.max_side), degree=args.degree or 20,
                     adapt_degree=args.adapt_degree)
    out["batched_only"] = True
    print(json.dumps(out))


def run_batched_filter(args):
    """--batched-filter: one degree-20 FP32 filter of --instances diffusion instances (sides
    32..--max-side, p = 1.5 k rounded up to 4 columns) as one arb_filter_batched call
    against one arb_filter_f32 call per instance, best of 5 after 2 warm-ups; wall time with
    a device synchronisation on both sides."""
    import torch
    from paper_1507_06078_gb300 import arrabit as arb, build
    build.build()
    ctx = arb.Context(0)
    ws = I.batched_diffusion_instances(count=args.instances, base_seed=30000, side_range=(32, args.max_side))
    d = args.degree or 20
    coef = arb.arb_filter_coefficients(arb.ARB_FILTER_CHEBINTERP, d)
    jobs, alg = [], 0
    for w in ws:
        mat = arb.Matrix.from_csr(ctx, w.A)
        hi = arb.arb_matrix_gershgorin(ctx, mat)[1]
        pc = (w.p + 3) // 4 * 4
        X = torch.from_numpy(I.gaussian_block(w.A.n, pc, w.seed).astype(np.float32)).cuda()
        jobs.append(dict(mat=mat, op_scale=-1.0, op_shift=hi, a=0.0, b=0.5 * hi, coef=coef, X=X,
                         colss=torch.zeros(pc, dtype=torch.float64, device="cuda")))
        alg += filter_algorithmic_bytes(w.A.n, w.A.nnz, pc, d, s=4, z=4)

    def timed(f):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    batched = lambda: arb.arb_filter_batched(ctx, jobs)  # noqa: E731
    single = lambda: [arb.arb_filter_f32(ctx, j["mat"], -1.0, j["op_shift"], 0.0, j["b"], coef, j["X"])  # noqa: E731
                      for j in jobs]
    for _ in range(2):
        timed(batched)
        timed(single)
    tb = min(timed(batched) for _ in range(5))
    ts = min(timed(single) for _ in range(5))
    print(json.dumps({"batched_filter": True, "instances": len(ws), "rows": int(sum(w.A.n for w in ws)),
                      "degree": d, "batched_ms": tb * 1e3, "per_instance_calls_ms": ts * 1e3,
                      "algorithmic_GB": alg / 1e9, "batched_alg_GBps": alg / tb / 1e9,
                      "per_instance_alg_GBps": alg / ts / 1e9}))


def c0_timings(steps=5, warmup=2):
    """The 2D 64^2 workload (k = 20, p = 30, d = 10, q = 1, b after every ARR) solved to its
    relative residual 1e-10 in FP64 and in mixed precision: milliseconds per solve (wall
    time around each arb_solve with a device synchronisation, `warmup` untimed solves, then
    `steps` timed ones), kernel launches per solve and the work counts.  Problems of this
    size are latency bound: the metric is the time per solve."""
    import torch
    from paper_1507_06078_gb300 import arrabit as arb
    ctx = arb.Context(0)
    w = I.workload_2d64()
    mat = arb.Matrix.from_csr(ctx, w.A)
    X0 = I.gaussian_block(w.A.n, w.p, 20150722)
    out = {"workload": w.name, "tol": w.tol}
    c = 2.0 - 2.0 * np.cos(np.pi * np.arange(1, 65) / 65.0)
    lam = np.sort((c[:, None] + c[None, :]).ravel())[:w.k]
    for name, prec in (("fp64", arb.ARB_FP64), ("mixed", arb.ARB_MIXED)):
        o = arb.arb_options_default(w.k)
        o.p, o.q, o.degree, o.precision, o.b_update = w.p, 1, 10, prec, 1
        for _ in range(warmup):
            arb.arb_solve(ctx, mat, w.k, arb.ARB_SMALLEST, w.tol, o, x0=X0)
        ts, r, l0 = [], None, ctx.launches()
        for _ in range(max(steps, 1)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = arb.arb_solve(ctx, mat, w.k, arb.ARB_SMALLEST, w.tol, o, x0=X0)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        out[name] = {"ms_per_solve": 1e3 * float(np.median(ts)), "ms_min": 1e3 * min(ts),
                     "launches_per_solve": (ctx.launches() - l0) // max(steps, 1),
                     "outer_iters": r.info["outer_iters"], "n_filters": r.info["n_filters"],
                     "maxres": r.info["maxres"], "stop": r.info["stop_reason"],
                     "t_filter_s": r.info["t_filter"], "t_arr_s": r.info["t_arr"],
                     "eig_err_vs_closed_form": float(np.max(np.abs(r.evals - lam)))}
    mat.close()
    ctx.close()
    return out


def cpu_full_solves(budget_s=20.0):
    """The oracle (oracle.arrabit_mpm, FP64, unchanged) solving whole problems end to end on
    the host: the 2D 64^2 workload (k = 20, tol 1e-10) and the smallest instances of the
    batched diffusion family (seeds 30000 + i, sides 32-128, q = 1, d = 20, tol 1e-8), each
    with the same options as the GPU runs, until about budget_s seconds are spent.  Seconds
    per solve, measured, not extrapolated."""
    from oracle import arrabit_oracle as O
    t_start = time.perf_counter()
    out = []
    w = I.workload_2d64()
    probs = [(w.name, w.A, w.k, I.gaussian_block(w.A.n, w.p, 20150722), w.tol, 10)]
    for inst in sorted(I.batched_diffusion_instances(count=8, base_seed=30000, side_range=(32, 128)),
                       key=lambda v: v.A.n)[:3]:
        probs.append((inst.name, inst.A, inst.k, I.gaussian_block(inst.A.n, inst.p, inst.seed), 1e-8, 20))
    for name, A, k, X0, tol, d in probs:
        if time.perf_counter() - t_start > budget_s:
            break
        B = O.csr_to_scipy(A.n, A.rowptr, A.col, A.val)
        t0 = time.perf_counter()
        r = O.arrabit_mpm(B, k, X0, which="smallest", tol=tol, q=1, degree=d, b_update="every_arr")
        out.append({"problem": name, "n": int(A.n), "k": int(k), "seconds": time.perf_counter() - t0,
                    "converged": bool(r.converged), "outer_iters": int(r.outer_iters)})
    return out


def _guarded(f):
    """Run one optional part of the bench line; an exception becomes an error entry."""
    try:
        return f()
    except Exception as e:  # noqa: BLE001 - the line must still be printed
        return {"error": repr(e)[:300]}


def run_c0(args):
    """--c0: the small workload's time per solve (c0_timings), FP64 and mixed."""
    from paper_1507_06078_gb300 import build
    build.build()
    out = c0_timings(args.steps, args.warmup)
    out["c0"] = True
    print(json.dumps(out))


def main():
    args = parse()
    if args.c0:
        run_c0(args)
        return
    if args.batched_filter:
        run_batched_filter(args)
        return
    if args.c2:
        run_c2(args)
        return
    if args.ablations:
        run_ablations(args)
        return
    if args.batched_only:
        run_batched_only(args)
        return
    if args.filter_only:
        run_filter_only(args)
        return
    if args.serve:
        run_serve(args)
        return
    if args.dense_only:
        run_dense_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
