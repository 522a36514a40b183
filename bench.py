"""Benchmark of the GB300 sketch-and-project ridge solver.

Workload (default): dense primal ridge, X 100000 x 4096 = U diag(sigma) V^T with
Haar U, V and sigma geometric from 1 to 1e-3 (float32 storage), y = X w* + 0.01 noise,
lambda = 1e-2, count sketch tau = 256 with the heuristic momentum, to relative
residual 1e-6 in mixed precision: X^T X on the tensor cores (TF32 in, FP32
accumulation), S^T A and the iterations in FP32, the small system S^T A S factored
by FP64 Cholesky and its pseudo-inverse applied in FP64, and the FP64 true residual
through X every 50 iterations. Beside it: the plain FP64 GPU path on the same
problem (count and subsample sketches, with its per-kernel profile), the same mixed
path with an FP32 small solve and a 400-iteration refresh period, the subsample
sketch in mixed precision, and the small dense case (X 2000 x 500, plain FP64,
subsample tau = 50, no momentum).

A step is one full solve through the C ABI: rs_create (copies X, y; forms A, b on
the device) + rs_solve to 1e-6 + the weights back. ``value`` is the iteration
throughput of the solve phase (iterations per second); time to tolerance of the
whole step is ``ms_per_step``. With --gpus N (torchrun) every rank solves its own
replica of the workload (different data seed); no data moves between GPUs.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-6 rel. residual & iters/s, chosen form vs plain FP64, one GB300"
N_ROWS, N_COLS, TAU, LAM, TOL, MAX_IT = 100000, 4096, 256, 1e-2, 1e-6, 30000
REFRESH = 50
WORKLOAD = ("dense primal ridge X 100000x4096 (Haar U,V; sigma geometric 1..1e-3; fp32), "
            "lambda 1e-2, count sketch tau 256, heuristic momentum, mixed: TF32 X^T X, FP32 "
            "S^T A and iterations, FP64 Cholesky small solve, FP64 true residual every 50 "
            "iterations, tol 1e-6")
# the small dense case: X 2000 x 500 iid N(0, 1), y = X w* + 0.1 noise, lambda 1e-3,
# plain FP64, subsample tau = 50, no momentum, seed 0
SMALL = dict(n=2000, d=500, lam=1e-3, tau=50)
# FP64 FMA throughput of one GB300 from its unit counts (the recipe's nominal
# 1.25 TFLOP/s dense FP64); no measured FP64 figure is provided with the peaks
FP64_PEAK_TFLOPS = 1.25


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while active."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._th = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._th = threading.Thread(target=self._run, daemon=True)
        self._th.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._th.join(timeout=10)

    def summary(self):
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def make_problem(seed, device, n_rows=N_ROWS):
    from synth import geometric_sigma, spectrum_problem_torch

    return spectrum_problem_torch(n_rows, N_COLS, geometric_sigma(N_COLS, 1e-3), seed=seed,
                                  noise=0.01, device=device)


def one_solve(rs, X, y, precision, sketch, device, w_out, on_host=False, chol_fp64=True,
              refresh=REFRESH, method="snp"):
    """One step: create (copy X, y; form A, b), solve to TOL (sketch-and-project, or
    method="cg": Conjugate Gradients on the same system), weights out, destroy.
    Returns dict of times (ms), iteration count and the chunking."""
    import torch

    st = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    e0.record(st)
    with rs.Solver(X, y, LAM, sketch=sketch, tau=TAU, momentum="heuristic", seed=0,
                   precision=precision, refresh_every=refresh, device=device.index or 0,
                   stream=st.cuda_stream, chol_fp64=chol_fp64) as s:
        solve = s.solve_cg if method == "cg" else s.solve
        w, hist, iters, conv = solve(TOL, MAX_IT, w_out=None if on_host else w_out)
        setup_ms, solve_ms = s.timings()
        chunk, ref, fused = s.chunking()
    e1.record(st)
    torch.cuda.synchronize(device)
    w = w.detach().cpu().numpy() if hasattr(w, "detach") else np.array(w)
    return {"ms": e0.elapsed_time(e1), "iters": iters, "conv": bool(conv), "setup_ms": setup_ms,
            "solve_ms": solve_ms, "final_rel": float(hist[-1]), "w": w, "chunk": chunk,
            "refresh": ref, "fused_potri": fused}


def launches_per_step(iters, chunk, refresh, fused=True, chunks_per_graph=4):
    """Kernels one mixed step launches: per chunk the chunk start, the sketch plans, the
    row -> bucket map, S^T A with S^T A S, M^+ (the fused kernel in its two forms, of
    which the active slot count runs one; else factor and product), and per refresh
    period the persistent iteration kernel and the FP64
    refresh (float-pair X^T X w, its sum, the finish); chunks are replayed four per
    CUDA graph until the solve stops; per step 7 more for the setup (transposed copy,
    tensor-core X^T X, mirror, b = X^T y in three launches, initial state)."""
    per_chunk = 6 + 4 * (chunk // refresh)  # M^+: two launches either way
    replays = max(1, ((iters + chunk - 1) // chunk + chunks_per_graph - 1) // chunks_per_graph)
    return replays * chunks_per_graph * per_chunk + 7


def aggregate_replicas(dist, solve_s, step_ms, iters, device):
    """Replicas (one independent problem per rank): the slowest rank's solve and step
    times, the iterations of all ranks, and every rank's own (iterations, solve s,
    step ms) so that a slow or long-running rank is visible."""
    import torch

    t = torch.tensor([solve_s, step_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    it = torch.tensor([float(iters)], device=device, dtype=torch.float64)
    dist.all_reduce(it)
    mine = torch.tensor([float(iters), solve_s, step_ms], device=device, dtype=torch.float64)
    every = [torch.zeros_like(mine) for _ in range(dist.get_world_size())]
    dist.all_gather(every, mine)
    s, m = t.tolist()
    per_rank = [{"rank": r, "iters": int(v[0].item()), "solve_s": float(v[1].item()),
                 "step_ms": float(v[2].item())} for r, v in enumerate(every)]
    return s, m, int(it.item()), per_rank


def profile_kernels(rs, X, y, device, precision="mixed", chol_fp64=True, refresh=REFRESH,
                    reps=1200):
    """Per-kernel mean device time (CUDA events on the solver's stream), continuing
    from the first iterations of a solve."""
    import torch

    st = torch.cuda.current_stream(device)
    with rs.Solver(X, y, LAM, sketch="count", tau=TAU, momentum="heuristic", seed=0,
                   precision=precision, refresh_every=refresh, device=device.index or 0,
                   stream=st.cuda_stream, chol_fp64=chol_fp64) as s:
        s.solve(TOL, 60)
        return s.profile_iteration(reps)


def roofline(stats, pk):
    """Dominant kernel of the iteration and its achieved fraction of its peak: HBM
    bytes against the measured copy bandwidth, or (the FP64 factor, inverse and
    product of the small systems) FP64 FLOP/s against the FP64 FMA peak."""
    name, (ms, n, nbytes, flops, _its) = max(stats.items(), key=lambda kv: kv[1][0] * kv[1][1])
    hbm = pk.get("hbm_gbs", 6800.0)
    if name in ("potri", "factor", "pinv", "chol"):
        achieved = flops / (ms * 1e-3) / 1e12
        return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": PROFILED_TRAFFIC[name](_its / n) if name in PROFILED_TRAFFIC else None,
                "peak_source": "FP64 FMA peak from the unit counts (nominal 1.25 TFLOP/s dense "
                               "FP64 of one GB300)"}
    achieved = nbytes / (ms * 1e-3) / 1e9
    traffic = None
    if name in PROFILED_TRAFFIC and n > 0:
        traffic = PROFILED_TRAFFIC[name](_its / n)  # per launch
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic, "peak_source": "MEASURED_PEAKS.json hbm_gbs"}


def h2d_gbs(xh, device):
    """GB/s of one copy of the pinned host tensor xh to the device (CUDA events)."""
    import torch

    xd = torch.empty(xh.shape, dtype=xh.dtype, device=device)
    st = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    e0.record(st)
    xd.copy_(xh, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize(device)
    return xh.numel() * xh.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9


def dgemm_tflops(device, n=4096, reps=5):
    """FP64 GEMM throughput of this GPU through cuBLAS (torch.mm on float64, n^3 with
    2 n^3 flops, CUDA events, after one warm-up): the measured counterpart of the FP64
    peak derived from the unit counts, reported beside it."""
    import torch

    g = torch.Generator(device=device).manual_seed(0)
    a = torch.randn(n, n, dtype=torch.float64, device=device, generator=g)
    b = torch.randn(n, n, dtype=torch.float64, device=device, generator=g)
    torch.mm(a, b)
    st = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    e0.record(st)
    for _ in range(reps):
        torch.mm(a, b)
    e1.record(st)
    torch.cuda.synchronize(device)
    return 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12


def cpu_baseline(X, y, iters_ref, sample_iters=4):
    """The FP64 oracle on the host cores: A = X^T X + lambda I from the full X
    (setup), then `sample_iters` count-sketch iterations; iters/s of its loop. Also
    returns the FP64 solution w* = A^{-1} b of that A (the reference the GPU results are checked against),
    and the small dense case run by the oracle to tolerance."""
    import oracle
    from synth import gaussian_problem

    cores = os.cpu_count()
    Xh = X.detach().cpu().double().numpy()
    yh = y.detach().cpu().numpy()
    t0 = time.perf_counter()
    A, b = oracle.form_system(Xh, yh, LAM, "primal")
    t_setup = time.perf_counter() - t0
    t1 = time.perf_counter()
    oracle.sketch_and_project(A, b, "count", TAU, 0, 0.0, sample_iters,
                              mom={"kind": "heuristic"})
    t_it = (time.perf_counter() - t1) / sample_iters
    one = single_thread_iters(A, b)
    w_star = np.linalg.solve(A, b)
    del A
    Xs, ys, _ = gaussian_problem(SMALL["n"], SMALL["d"], seed=0)
    t2 = time.perf_counter()
    ref = oracle.solve_ridge(Xs, ys, SMALL["lam"], "primal", "subsample", SMALL["tau"], seed=0,
                             tol=TOL, max_iters=100000, mom={"kind": "none"})
    t_small = time.perf_counter() - t2
    out = {"value": 1.0 / t_it, "unit": "iters/s", "cores": cores, "kind": "oracle",
           "sample": (f"numpy FP64 oracle: setup X^T X on the full 100000x4096 X ({t_setup:.1f} s), "
                      f"then {sample_iters} count-sketch iterations ({t_it * 1e3:.0f} ms each); "
                      f"time to 1e-6 extrapolated with {iters_ref} iterations = "
                      f"{t_setup + iters_ref * t_it:.1f} s; on one thread the iterations take "
                      f"{one if one is None else round(one * 1e3)} ms each"),
           "setup_s": t_setup, "s_per_iter": t_it, "s_per_iter_1_thread": one,
           "small_case": {"iters": int(ref["iters"]), "s": t_small}}
    return out, w_star, ref


def single_thread_iters(A, b, iters=2):
    """Seconds per iteration of the oracle's count-sketch loop on one host thread: a
    child process with the BLAS thread pools set to one thread (they are fixed when
    numpy loads) runs `iters` iterations on the same A, b."""
    import tempfile

    with tempfile.TemporaryDirectory() as d:
        np.save(os.path.join(d, "A.npy"), A)
        np.save(os.path.join(d, "b.npy"), b)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
                   MKL_NUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
        code = ("import sys, time, numpy as np; sys.path.insert(0, sys.argv[1]); import oracle; "
                "A = np.load(sys.argv[2]); b = np.load(sys.argv[3]); t = time.perf_counter(); "
                f"oracle.sketch_and_project(A, b, 'count', {TAU}, 0, 0.0, {iters}, "
                "mom={'kind': 'heuristic'}); print((time.perf_counter() - t) / " + str(iters) + ")")
        try:
            out = subprocess.run([sys.executable, "-c", code, ROOT, os.path.join(d, "A.npy"),
                                  os.path.join(d, "b.npy")], env=env, capture_output=True,
                                 text=True, timeout=600)
            return float(out.stdout.strip().splitlines()[-1])
        except Exception:
            return None


def run_reference(args):
    """--impl reference: the FP64 oracle as it stands, on the host cores, on this
    workload; each step a bounded sample (setup once, 3 iterations per step)."""
    import torch

    import oracle

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else torch.device("cpu")
    X, y, _ = make_problem(1234, dev)
    Xh = X.detach().cpu().double().numpy()
    yh = y.detach().cpu().numpy()
    del X, y
    A, b = oracle.form_system(Xh, yh, LAM, "primal")
    per_step = 3
    for _ in range(args.warmup):
        oracle.sketch_and_project(A, b, "count", TAU, 0, 0.0, 1, mom={"kind": "heuristic"})
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sketch_and_project(A, b, "count", TAU, 0, 0.0, per_step, mom={"kind": "heuristic"})
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": "iters/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": args.gpus,
                       "parallelism": "replicas" if args.gpus > 1 else "single"},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{per_step} oracle iterations per step after one setup"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ncu DRAM traffic (read + write) per launch, taken on the X 20000 x 4096 profiling
# case (profiles/): the iteration kernel does not touch X, so its bytes do not depend
# on n (1799.5 MB read + 3.3 MB written by a launch of 400 iterations, scaled to the
# launch's iterations); the refresh product reads X once, so its traffic scales with
# n (327.8 MB read + 2.9 MB written at n = 20000, times 5)
PROFILED_TRAFFIC = {"iterate": lambda its_per_launch: 228.7e6 * its_per_launch / 50.0,
                    # the tile work space of k_potri: 1819.1 MB read + 1415.4 MB written
                    # per launch of 600 slots (the bench's chunk), independent of n
                    "potri": lambda _unused: 3234.5e6,
                    "refresh": lambda its_per_launch: 330.7e6 * N_ROWS / 20000.0}


def bench_batched(args, rs, dev):
    """256 uneven problems (d log-uniform in [256, 4096], n = 4 d, lambda log-uniform in
    [1e-4, 1]), 4 right-hand sides each, count sketch tau = min(128, d / 8), heuristic
    momentum, mixed precision to 1e-6 per pair; the plain FP64 batch timed over a
    bounded number of iterations beside it."""
    import torch

    from synth import batched_problem_torch, batched_specs

    P = 256
    d, n, lam = batched_specs(P, 4)
    taus = [min(128, int(v) // 8) for v in d]

    def make(prec):
        Xs, Ys = [], []
        for p in range(P):
            X, Y = batched_problem_torch(int(n[p]), int(d[p]), 4, 10000 + p, device=dev)
            Xs.append(X if prec == "mixed" else X.double())
            Ys.append(Y)
        return Xs, Ys

    Xs, Ys = make("mixed")
    torch.cuda.synchronize(dev)
    # the problems' generation leaves torch's allocator holding cached blocks that the
    # library's own pool cannot use
    torch.cuda.empty_cache()
    with ClockSampler(dev.index or 0) as clk:
        with rs.Batch(Xs, Ys, list(lam), sketch="count", taus=taus, momentum="heuristic", seed=0,
                      precision="mixed") as b:
            W, iters, resid, conv = b.solve(tol=TOL, max_iters=400000)
            info = b.info()
            parts = b.profile(2)
    solve_s = info["solve_ms"] / 1e3
    it_p = iters.max(axis=1).astype(np.float64)
    a_bytes = float(np.sum(it_p * d.astype(np.float64) ** 2 * 4))
    out = {"workload": "batched", "converged": bool(conv), "time_to_tol_ms": info["solve_ms"],
           "setup_ms": info["setup_ms"], "tune_ms": info["tune_ms"],
           "iter_threads": info["iter_threads"], "phase1_streams": info["phase1_streams"],
           "problem_iters_per_s": float(it_p.sum() / solve_s), "max_iters": int(iters.max()),
           "mean_iters": float(iters.mean()), "max_resid": float(resid.max()),
           "a_bytes_per_s_gbs": a_bytes / solve_s / 1e9, "chunk_profile_all_running_ms": parts,
           "clocks": clk.summary()}
    del Xs
    torch.cuda.empty_cache()
    Xd, Yd = make("fp64")
    torch.cuda.empty_cache()
    with rs.Batch(Xd, Yd, list(lam), sketch="count", taus=taus, momentum="heuristic", seed=0,
                  precision="fp64") as b:
        K = 2000
        _, pit, _, _ = b.solve(tol=0.0, max_iters=K)
        pinfo = b.info()
    out["plain_fp64_problem_iters_per_s"] = float(pit.max(axis=1).sum() / (pinfo["solve_ms"] / 1e3))
    out["plain_fp64_time_to_tol_ms_extrapolated"] = pinfo["solve_ms"] / K * int(iters.max())
    out["speedup_vs_plain_fp64"] = out["plain_fp64_time_to_tol_ms_extrapolated"] / info["solve_ms"]
    print(json.dumps(out), flush=True)


def bench_sparse(args, rs, dev):
    """Zipf-sparse X 1e6 x 5e4 (about 5e6 entries, bfloat16 values), lambda 0.1, SubCount
    s = 4096 -> tau = 512, heuristic momentum, matrix-free: the mixed solve to 1e-6
    (at most 30000 iterations; time to tolerance when reached, else the FP64 residual
    reached: 60000 iterations reach 1.0e-5), the plain FP64 rate over 2000 iterations,
    and Conjugate Gradients on the
    same matrix-free system to 1e-6 (the comparison of Section 8.3 on RCV1)."""
    from synth import sparse_problem

    n, d = 1_000_000, 50_000
    rowptr, colidx, vals, y, _ = sparse_problem(n, d, 5_000_000, 3000, bf16=True)
    out = {"workload": "sparse", "n": n, "d": d, "nnz": int(len(vals))}
    for prec, bf, K in (("mixed", True, 30000), ("fp64", False, 2000)):
        X = rs.CSR(rowptr, colidx, vals, (n, d), bf16=bf)
        with rs.Solver(X, y, 0.1, sketch="subcount", tau=512, momentum="heuristic", seed=0,
                       precision=prec, sub_s=4096) as s:
            w, hist, iters, conv = s.solve(tol=TOL, max_iters=K)
            setup_ms, solve_ms = s.timings()
            out[prec] = {"iters_per_s": iters / (solve_ms / 1e3), "setup_ms": setup_ms,
                         "solve_ms": solve_ms, "iters": iters, "converged": bool(conv),
                         "final_rel": float(hist[-1]), "true_rel": s.true_residual(w)}
            if prec == "mixed":
                wc, hc, itc, cvc = s.solve_cg(tol=TOL, max_iters=20000)
                _, cg_ms = s.timings()
                out["cg"] = {"iters": itc, "converged": bool(cvc), "solve_ms": cg_ms,
                             "final_rel": float(hc[-1]), "true_rel": s.true_residual(wc)}
                # per-group device time of the mixed iterations (CUDA events)
                out["mixed_kernels"] = {
                    k: {"ms": v[0], "launches": v[1]} for k, v in s.profile_iteration(600).items()}
    out["iters_per_s_mixed_vs_plain_fp64"] = out["mixed"]["iters_per_s"] / out["fp64"]["iters_per_s"]
    print(json.dumps(out), flush=True)


def bench_kernel(args, rs, dev):
    """Kernel ridge with the Gaussian kernel (Section 2.2), California-Housing-shaped
    synthetic data: n = 20640 points in d = 8 standardised features (a mixture of
    three Gaussian clusters), y = sin(x_1) + x_2 x_3 / 2 + 0.1 noise, sigma = 1,
    lambda = 1e-2; count sketch tau = 256 with the heuristic momentum, plain FP64 and
    mixed (kernel matrix and A on the tensor cores), and CG on the same system; time to
    1e-4 (the tolerance of the paper's Experiment 1, at most 60000 iterations) and to
    1e-6 (at most 20000 iterations: the system's conditioning keeps every method far
    from it within a bench-sized run)."""
    n, d, sigma, lam = 20640, 8, 1.0, 1e-2
    g = np.random.default_rng(4321)
    centers = g.standard_normal((3, d)) * 1.5
    P = centers[g.integers(0, 3, n)] + g.standard_normal((n, d))
    P = (P - P.mean(axis=0)) / P.std(axis=0)
    y = np.sin(P[:, 0]) + 0.5 * P[:, 1] * P[:, 2] + 0.1 * g.standard_normal(n)
    out = {"workload": "kernel ridge RBF", "n": n, "d": d, "sigma": sigma, "lambda": lam}
    for prec in ("mixed", "fp64"):
        Pp = P.astype(np.float32) if prec == "mixed" else P
        with rs.Solver(Pp, y, lam, sketch="count", tau=256, momentum="heuristic", seed=0,
                       precision=prec, kernel_sigma=sigma) as s:
            setup_ms, _ = s.timings()
            row = {"setup_ms": setup_ms}
            for tol, cap in ((1e-4, 60000), (1e-6, 20000)):
                _, hist, iters, conv = s.solve(tol=tol, max_iters=cap)
                _, solve_ms = s.timings()
                _, hc, itc, cvc = s.solve_cg(tol=tol, max_iters=cap)
                _, cg_ms = s.timings()
                row[f"snp_{tol:g}"] = {"iters": iters, "converged": bool(conv), "solve_ms": solve_ms,
                                       "final_rel": float(hist[-1])}
                row[f"cg_{tol:g}"] = {"iters": itc, "converged": bool(cvc), "solve_ms": cg_ms,
                                      "final_rel": float(hc[-1])}
            out[prec] = row
    print(json.dumps(out), flush=True)


def profile_case(workload, rs, dev):
    """Short cases of the other workloads for ncu captures (mixed precision):
    batched: the first 32 problems of the batched recipe, 50 iterations, 256 threads
    per CTA, one phase-1 stream; sparse: the sparse recipe, 100 iterations in chunks
    of 50; plain: the dense recipe at 20000 x 4096 in plain FP64 (count sketch tau = 256,
    heuristic momentum) to 1e-6; gaussian: the dense recipe at 20000 x 4096 with the
    Gaussian sketch tau = 256
    in mixed precision (S^T A on the tensor cores), one chunk of 64 slots;
    kernel: kernel ridge on 8192 random points in 256 dimensions (mixed: the
    tensor-core kernel matrix, then K^T K), 50 iterations; learned: X = U diag(i^-0.8)
    V^T at 16384 x 8192, lambda 1e-3, an untrained network (synth.mlp_init(4) rounded
    to bfloat16), eps 0.1, 60 iterations in chunks of 20, then three training steps of
    the network on 65536 random rows (the gradient kernel). Prints one line with the
    iteration count."""
    import torch

    if workload == "batched":
        from synth import batched_problem_torch, batched_specs

        P = 32
        d, n, lam = batched_specs(P, 4)
        Xs, Ys = [], []
        for p in range(P):
            X, Y = batched_problem_torch(int(n[p]), int(d[p]), 4, 10000 + p, device=dev)
            Xs.append(X)
            Ys.append(Y)
        torch.cuda.synchronize(dev)
        taus = [min(128, int(v) // 8) for v in d]
        with rs.Batch(Xs, Ys, list(lam), sketch="count", taus=taus, momentum="heuristic", seed=0,
                      precision="mixed") as b:
            b.set_launch(256, 1)
            _, iters, _, _ = b.solve(tol=0.0, max_iters=50)
        out = int(iters.max())
    elif workload == "sparse":
        from synth import sparse_problem

        n, d = 1_000_000, 50_000
        rowptr, colidx, vals, y, _ = sparse_problem(n, d, 5_000_000, 3000, bf16=True)
        X = rs.CSR(rowptr, colidx, vals, (n, d), bf16=True)
        with rs.Solver(X, y, 0.1, sketch="subcount", tau=512, momentum="heuristic", seed=0,
                       precision="mixed", sub_s=4096, refresh_every=50) as s:
            _, _, out, _ = s.solve(tol=0.0, max_iters=100)
    elif workload == "plain":
        X, y, _ = make_problem(1234, dev, 20000)
        with rs.Solver(X.double(), y, LAM, sketch="count", tau=TAU, momentum="heuristic", seed=0,
                       precision="fp64") as s:
            _, _, out, _ = s.solve(tol=TOL, max_iters=MAX_IT)
    elif workload == "gaussian":
        from synth import geometric_sigma, spectrum_problem_torch

        X, y, _ = spectrum_problem_torch(20000, 4096, geometric_sigma(4096, 1e-3), seed=1234,
                                         noise=0.01, device=dev)
        with rs.Solver(X, y, LAM, sketch="gaussian", tau=TAU, momentum="heuristic", seed=0,
                       precision="mixed", chunk=64) as s:
            _, _, out, _ = s.solve(tol=0.0, max_iters=64)
    elif workload == "kernel":
        g = np.random.default_rng(4321)
        P = g.standard_normal((8192, 256)).astype(np.float32)
        y = np.sin(P[:, 0].astype(np.float64))
        with rs.Solver(P, y, 1e-2, sketch="count", tau=256, momentum="heuristic", seed=0,
                       precision="mixed", kernel_sigma=16.0) as s:
            _, _, out, _ = s.solve(tol=0.0, max_iters=50)
    else:
        from synth import mlp_init, power_sigma, spectrum_problem_torch

        X, y, _ = spectrum_problem_torch(16384, 8192, power_sigma(8192, 0.8), 999, device=dev)
        f = np.ascontiguousarray(mlp_init(4), np.float32).view(np.uint32).astype(np.uint64)
        wb = (((f + 0x7FFF + ((f >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)
        with rs.Solver(X, y, 1e-3, sketch="subsample", tau=256, momentum="none", seed=5,
                       precision="mixed", chunk=20, refresh_every=20) as s:
            s.set_proposal(wb, 0.1)
            _, _, out, _ = s.solve(tol=0.0, max_iters=60)
        # training steps of the network (the gradient kernel's tensor-core products)
        g = np.random.default_rng(0)
        Z = torch.as_tensor(g.standard_normal((65536, 4)), dtype=torch.float32, device=dev)
        t = torch.as_tensor(g.standard_normal(65536), dtype=torch.float32, device=dev)
        with rs.MLP(mlp_init(4)) as net:
            for _ in range(3):
                net.step(Z, t, 1e-3)
    print(json.dumps({"profile_case": workload, "iters": out}), flush=True)


def bench_learned(args, rs, dev):
    """X 65536 x 8192 = U diag(i^-0.8) V^T (Haar U, V), lambda 1e-3, subsample tau 256,
    no momentum, to 1e-6. Training: plain FP64 trajectories of the uniform proposal on
    64 seeds of the same recipe (700..763): trajectories of 60 of them (1500 iterations
    each, labels formed on the device by rs_collect; w* of each seed from a mixed solve
    to 1e-11), 3000 Adam steps of the library's kernels; the uniform mixture weight eps
    of the proposal chosen among 0.1, 0.25, 0.5, 0.75 by the mean plain FP64 iteration
    count on the other 4 seeds. Evaluation on 16 held-out seeds (900..915): uniform
    draws, the learned proposal and the A_jj proposal of Section 7, plain FP64 (one
    context per seed, the samplers switched on it) and mixed; the mean and quartiles of
    the iteration and time ratios against uniform."""
    import torch

    from paper_2105_05565_gb300 import learned
    from synth import power_sigma, spectrum_problem_torch

    n, m, tau, lam, chunk = 65536, 8192, 256, 1e-3, 20
    n_pool = 6 if args.small else 64
    n_val = 2 if args.small else 4
    n_train = n_pool - n_val
    n_eval = 2 if args.small else 16
    eps_grid = (0.1, 0.25, 0.5, 0.75)
    out = {"workload": "learned", "n": n, "m": m, "tau": tau, "chunk": chunk,
           "train_seeds": n_train, "validation_seeds": n_val, "eval_seeds": n_eval}
    t0 = time.perf_counter()
    Zs, Ys = [], []
    for sd in range(n_train):
        X, y, _ = spectrum_problem_torch(n, m, power_sigma(m, 0.8), 700 + sd, device=dev)
        torch.cuda.synchronize(dev)
        with rs.Solver(X, y, lam, sketch="subsample", tau=tau, momentum="heuristic", seed=sd,
                       precision="mixed") as s:
            w_star, _, _, _ = s.solve(tol=1e-11, max_iters=200000)
        Xd = X.double()
        del X
        b = (Xd.T @ y.double()).cpu().numpy()  # the collection starts from w = 0, r = -b
        torch.cuda.synchronize(dev)
        with rs.Solver(Xd, y, lam, sketch="subsample", tau=tau, momentum="none", seed=sd,
                       chunk=1) as s:
            s.set_proposal(None, 0.1)
            s.set_state(np.zeros(m), np.zeros(m), -b, -b, 0)
            Z, t = learned.collect(s, w_star, 1500, tol=1e-6)
        del Xd
        Zs.append(Z)
        Ys.append(t)
    out["collect_s"] = time.perf_counter() - t0
    t1 = time.perf_counter()
    wb, _, losses = learned.train(np.concatenate(Zs), np.concatenate(Ys), steps=3000, batch=2048,
                                  lr=3e-3, seed=0)
    out["train_s"] = time.perf_counter() - t1
    out["train_rows"] = int(sum(len(t) for t in Ys))
    out["train_loss_first_last"] = [float(losses[:50].mean()), float(losses[-200:].mean())]
    del Zs, Ys
    # eps on the validation seeds (plain FP64 iterations to tolerance)
    val = {e: [] for e in eps_grid}
    for sd in range(n_train, n_pool):
        X, y, _ = spectrum_problem_torch(n, m, power_sigma(m, 0.8), 700 + sd, device=dev)
        Xd = X.double()
        del X
        torch.cuda.synchronize(dev)
        with rs.Solver(Xd, y, lam, sketch="subsample", tau=tau, momentum="none", seed=5 + sd,
                       chunk=chunk) as s:
            for e in eps_grid:
                s.set_proposal(wb, e)
                _, _, iters, _ = s.solve(tol=TOL, max_iters=100000)
                val[e].append(iters)
        del Xd
    eps = min(eps_grid, key=lambda e: float(np.mean(val[e])))
    out["validation_iters_by_eps"] = {str(e): float(np.mean(v)) for e, v in val.items()}
    out["eps"] = eps
    arms = {"uniform": lambda s: s.set_sampling("uniform"),
            "learned": lambda s: s.set_proposal(wb, eps),
            "diag": lambda s: s.set_sampling("diag")}
    res = {f"{p}_{a}": [] for p in ("fp64", "mixed") for a in arms}
    for sd in range(n_eval):
        X, y, _ = spectrum_problem_torch(n, m, power_sigma(m, 0.8), 900 + sd, device=dev)
        for prec in ("fp64", "mixed"):
            Xp = X.double() if prec == "fp64" else X
            torch.cuda.synchronize(dev)
            with rs.Solver(Xp, y, lam, sketch="subsample", tau=tau, momentum="none", seed=5 + sd,
                           precision=prec, chunk=chunk) as s:
                for name, setter in arms.items():
                    setter(s)
                    w, hist, iters, conv = s.solve(tol=TOL, max_iters=100000)
                    setup_ms, solve_ms = s.timings()
                    res[f"{prec}_{name}"].append((iters, solve_ms, bool(conv), float(hist[-1]),
                                                  setup_ms))
            del Xp
        del X

    def q(v):
        v = np.asarray(v, dtype=np.float64)
        return {"mean": float(v.mean()), "q25": float(np.quantile(v, 0.25)),
                "median": float(np.median(v)), "q75": float(np.quantile(v, 0.75))}

    for key, rows in res.items():
        its = [r[0] for r in rows]
        out[key] = {"iters": q(its), "solve_ms": q([r[1] for r in rows]),
                    "all_converged": all(r[2] for r in rows),
                    "max_final_rel": max(r[3] for r in rows),
                    "setup_ms": q([r[4] for r in rows])}
    for prec in ("fp64", "mixed"):
        u = res[f"{prec}_uniform"]
        for name in ("learned", "diag"):
            a = res[f"{prec}_{name}"]
            out[f"{prec}_{name}_vs_uniform_iters_ratio"] = q([x[0] / y[0] for x, y in zip(a, u)])
            out[f"{prec}_{name}_vs_uniform_time_ratio"] = q([x[1] / y[1] for x, y in zip(a, u)])
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--small", action="store_true",
                    help="profiling case: dense X 20000 x 4096 (328 MB, larger than L2), same "
                         "sketch and schedule, prints the line of that case; with --workload "
                         "batched / sparse / learned the short case of that workload for ncu "
                         "(profile_case)")
    ap.add_argument("--workload", default="dense",
                    choices=["dense", "batched", "sparse", "learned", "kernel", "gaussian",
                             "plain"],
                    help="dense: the benchmark line; batched / sparse: measurement lines of the "
                         "256-problem batch and the Zipf-sparse matrix-free solve")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "dense":
        import torch

        import paper_2105_05565_gb300 as rs

        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        rs.lib()
        if args.small:
            return profile_case(args.workload, rs, dev)
        if args.workload in ("gaussian", "plain"):
            raise SystemExit(f"--workload {args.workload} is a profiling case: use it with --small")
        fn = {"batched": bench_batched, "sparse": bench_sparse, "learned": bench_learned,
              "kernel": bench_kernel}[args.workload]
        return fn(args, rs, dev)

    import torch

    import paper_2105_05565_gb300 as rs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    rs.lib()
    X, y, _ = make_problem(1234 + rank, dev, 20000 if args.small else N_ROWS)
    w_out = torch.empty(N_COLS, dtype=torch.float64, device=dev)

    for _ in range(max(args.warmup, 3)):
        r = one_solve(rs, X, y, "mixed", "count", dev, w_out)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    runs = []
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            runs.append(one_solve(rs, X, y, "mixed", "count", dev, w_out))
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    iters = sum(r["iters"] for r in runs)
    solve_s = sum(r["solve_ms"] for r in runs) / 1e3
    step_ms = sum(r["ms"] for r in runs) / len(runs)
    per_rank = None
    if dist:
        solve_s, step_ms, iters, per_rank = aggregate_replicas(dist, solve_s, step_ms, iters, dev)
    value = iters / solve_s
    if rank != 0:
        dist.destroy_process_group()
        return

    # end to end: host inputs in pinned memory, weights back to the host
    Xh = X.cpu().pin_memory()
    yh = y.cpu().pin_memory()
    # one untimed warm-up of this path (the library's memory pool takes its block sizes)
    one_solve(rs, Xh, yh, "mixed", "count", dev, None, on_host=True)
    e2e_runs = [one_solve(rs, Xh, yh, "mixed", "count", dev, None, on_host=True)
                for _ in range(2)]
    e2e_iters = sum(r["iters"] for r in e2e_runs)
    e2e_ms = sum(r["ms"] for r in e2e_runs)
    e2e = {"value": e2e_iters / (e2e_ms / 1e3), "unit": "iters/s",
           "h2d_bytes_per_step": int(Xh.numel() * 4 + yh.numel() * 8),
           "d2h_bytes_per_step": int(N_COLS * 8 + (MAX_IT + 1) * 8),
           "ms_per_step": e2e_ms / len(e2e_runs),
           # this box's pinned host -> device rate for the same bytes (one copy of X)
           "h2d_gbs_measured": h2d_gbs(Xh, dev),
           # each timed run: step, setup (upload overlapped with the Gram) and solve
           "runs_ms": [[round(r["ms"], 3), round(r["setup_ms"], 3), round(r["solve_ms"], 3)]
                       for r in e2e_runs]}

    # roofline of the dominant kernel (CUDA events inside the library, same stream)
    stats = profile_kernels(rs, X, y, dev)
    pk = peaks()
    roof = roofline(stats, pk)
    if roof["bound"] == "alu":
        roof["dgemm_tflops_measured"] = dgemm_tflops(dev)

    def keep(r):
        return {k: r[k] for k in ("ms", "iters", "conv", "setup_ms", "solve_ms", "final_rel")}

    extra = {}
    last = runs[-1]
    ws = {"mixed": last["w"]}
    if not args.no_plain:
        plain = one_solve(rs, X, y, "fp64", "count", dev, w_out)
        ws["plain_fp64"] = plain["w"]
        extra["plain_fp64_count"] = keep(plain)
        extra["plain_fp64_count"]["iters_per_s"] = plain["iters"] / (plain["solve_ms"] / 1e3)
        extra["speedup_time_to_tol_vs_plain_fp64"] = plain["ms"] / step_ms
        extra["speedup_solve_vs_plain_fp64"] = plain["solve_ms"] / last["solve_ms"]
        Xd = X.double()
        extra["plain_fp64_kernels"] = {
            k: {"ms": v[0], "launches": v[1], "bytes": v[2], "flops": v[3], "iters": v[4]}
            for k, v in profile_kernels(rs, Xd, y, dev, precision="fp64", reps=384).items()}
        del Xd
        f32 = one_solve(rs, X, y, "mixed", "count", dev, w_out, chol_fp64=False, refresh=400)
        extra["mixed_count_fp32_small_solve_refresh400"] = keep(f32)
        # Conjugate Gradients on the same system (the competitor of Section 8.3)
        for prec in ("fp64", "mixed"):
            cg = one_solve(rs, X, y, prec, "count", dev, w_out, method="cg")
            extra[f"cg_{'plain_fp64' if prec == 'fp64' else 'mixed'}"] = keep(cg)
            ws[f"cg_{prec}"] = cg["w"]
        for prec in ("mixed", "fp64"):
            sub = one_solve(rs, X, y, prec, "subsample", dev, w_out)
            extra[f"{'plain_fp64' if prec == 'fp64' else 'mixed'}_subsample"] = keep(sub)
        # the small dense case: plain FP64, subsample tau 50, no momentum, to 1e-6
        from synth import gaussian_problem

        Xs, ys, _ = gaussian_problem(SMALL["n"], SMALL["d"], seed=0)
        Xs_d, ys_d = torch.from_numpy(Xs).to(dev), torch.from_numpy(ys).to(dev)
        small = []
        for _ in range(4):
            st = torch.cuda.current_stream(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            with rs.Solver(Xs_d, ys_d, SMALL["lam"], sketch="subsample", tau=SMALL["tau"],
                           momentum="none", seed=0, stream=st.cuda_stream) as sm:
                wsm, hsm, itsm, cvsm = sm.solve(TOL, 100000)
                sms = sm.timings()
            e1.record(st)
            torch.cuda.synchronize(dev)
            small.append((e0.elapsed_time(e1), itsm, cvsm, sms, float(hsm[-1]), wsm))
        ms_s, it_s, cv_s, (su_s, so_s), fin_s, w_small = small[-1]
        extra["small_dense_plain_fp64_subsample50"] = {
            "workload": "X 2000x500 iid N(0,1), y = X w* + 0.1 noise, lambda 1e-3, plain FP64, "
                        "subsample tau 50, no momentum, seed 0, tol 1e-6",
            "ms": ms_s, "iters": int(it_s), "conv": bool(cv_s), "setup_ms": su_s,
            "solve_ms": so_s, "iters_per_s": it_s / (so_s / 1e3), "final_rel": fin_s}
    cpu = None
    if not args.no_cpu:
        cpu, w_star, small_ref = cpu_baseline(X, y, last["iters"])
        nrm = float(np.linalg.norm(w_star))
        extra["rel_err_vs_fp64_solution"] = {k: float(np.linalg.norm(v - w_star) / nrm)
                                             for k, v in ws.items()}
        if "small_dense_plain_fp64_subsample50" in extra:
            sd = extra["small_dense_plain_fp64_subsample50"]
            sd["oracle_iters"] = int(small_ref["iters"])
            sd["rel_err_w_vs_oracle"] = float(np.linalg.norm(w_small - small_ref["w"]) /
                                              np.linalg.norm(small_ref["w"]))
            sd["oracle_s"] = cpu["small_case"]["s"]
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("100000x4096", "20000x4096") if args.small else WORKLOAD,
                   "global_batch": world, "seq_len": None,
                   "parallelism": "replicas" if world > 1 else "single",
                   "small_solve": "fp64", "refresh_every": last["refresh"], "chunk": last["chunk"],
                   "l2": "inputs larger than L2 (X = 1.64 GB re-read every step)"},
        "time_to_tol_ms": step_ms, "iters_to_tol": last["iters"], "converged": last["conv"],
        "final_true_rel_residual": last["final_rel"], "setup_ms": last["setup_ms"],
        "solve_ms": last["solve_ms"],
        "gpu_launches": None, "kernels": {k: {"ms": v[0], "launches": v[1], "bytes": v[2],
                                              "flops": v[3], "iters": v[4]}
                                          for k, v in stats.items()},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
        "wall_s_timed": wall,
    }
    if per_rank is not None:
        line["per_rank"] = per_rank
    line.update(extra)
    line["gpu_launches"] = int(sum(launches_per_step(r["iters"], r["chunk"], r["refresh"],
                                                     bool(r["fused_potri"])) for r in runs))
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
