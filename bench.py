#!/usr/bin/env python
"""Benchmark: time to relative residual 1e-10 and DOF/s of the RRE-accelerated
geometric-multigrid solver for the 2D IGA Poisson problem on 1024 x 1024
elements (about 1M unknowns), FP32 V-cycles in FP64 iterative refinement
(the mixed form) with the plain FP64 form timed beside it.

One step = one complete solve from s_0 = 0 to ||b - A x|| / ||b|| <= 1e-10
(restarted RRE, k = 5, multicolour Gauss-Seidel V(1,1)-cycles), inputs
resident in HBM, L2 flushed between steps.  value = DOF / time-to-tolerance,
summed over ranks (each rank solves its own independent problem: weak
scaling, no collective on the data path).

  python bench.py [--steps K] [--warmup W] [--p 3] [--k 5] [--method rre]
  python bench.py --impl reference      # the CPU oracle on a bounded sample
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to rel. residual 1e-10 and DOF/s: FP64 GMG+RRE vs mixed/learned form"
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# FP32 GS row-phase kernel on the finest level, from the ncu capture summarised
# in profiles/k_gs_phase_2d_1024_p3_fp32.md; keyed by (dim, n, p).
GS_TRAFFIC = {(2, 1024, 3): 11.77e6}


# FP64 pipe: the nominal GB300 rate of the profiling recipe (1.25 TFLOP/s;
# an FMA-throughput loop measured 1.20 on this machine's GB300).
FP64_PEAK_GFLOPS = 1250.0


def kernel_models(a, p, k):
    """Algorithmic bytes and FP64 flops per unknown of one launch of the
    streaming kernels of a 2D mixed-precision solve, by kernel name prefix.
    GS row phase: the 12 B/DOF of a sweep (read x, b; write x) over the phase's
    rows; residual + restriction and prolongation + correction: 9 B/DOF (FP32);
    float-pair refinement kernels: four float-pair row-sum arrays (16 B) with r
    or the iterates (20 B); CholeskyQR2 passes: the q+2 iterates (8(q+2) B),
    (q+1)(q+3) and 2(q+1)(q+2) flops; combination x-pass: the iterates read and
    x, T_M, T_K written, 2(q+2) + 4(2p+1) flops; FP64 residual: b, T_M, T_K
    read, r in FP32 and FP64 written, 4(2p+1) flops."""
    q = k
    return {
        "k_gs_phase2<float": (12.0, 0.0),
        "k_residual_restrict_x<float": (9.0, 0.0),
        "k_prolong_fused2<float": (9.0, 0.0),
        "k_xpass_df<": (36.0, 0.0),
        "k_residual_df<": (36.0, 0.0),
        "k_gram_partial<": (8.0 * (q + 2), float((q + 1) * (q + 3))),
        "k_gram2_partial<": (8.0 * (q + 2), float(2 * (q + 1) * (q + 2))),
        "k_xpass<double, double": (8.0 * (q + 2) + 24.0, float(2 * (q + 2) + 4 * (2 * p + 1))),
        "k_residual<double, float": (36.0, float(4 * (2 * p + 1))),
    }


def kernel_table(pkg, s, b, a, peak_hbm):
    """One mixed-precision solve enqueued kernel by kernel (no graph) with
    every launch timed by CUDA events on its own stream (igamg_profile_*).
    Per kernel: launches, total time and share, average launch time; for the
    streaming kernels also the finest-level launches' algorithmic bytes and
    FP64 flops per launch and their fractions of the measured HBM copy rate
    and of the FP64 peak.  Finest-level launches are those with the largest
    grid of their kernel (row kernels: one CTA per row; the Gram passes run
    on the finest level only)."""
    import numpy as np
    pkg.igamg_profile_start()
    s.solve(b, tol=1e-10, method=a.method, k=a.k, prec="fp32_ir", max_cycles=200, graph=False, host_loop=True)
    recs = pkg.igamg_profile_stop()
    mx, my = s.levels[-1][0], s.levels[-1][1] * s.levels[-1][2]
    models = kernel_models(a, a.p, a.k)
    total = sum(r[1] for r in recs)
    by = {}
    for name, us, grid in recs:
        by.setdefault(name, []).append((us, grid))
    rows = []
    for name, lst in sorted(by.items(), key=lambda kv: -sum(u for u, _ in kv[1])):
        t = sum(u for u, _ in lst)
        e = {"kernel": name, "launches": len(lst), "total_us": round(t, 1), "share": round(t / total, 4),
             "avg_us": round(t / len(lst), 3)}
        model = next((v for key, v in models.items() if name.startswith(key)), None)
        if model is not None:
            gmax = max(g for _, g in lst)
            fin = [u for u, g in lst if g == gmax]
            us = float(np.mean(fin))
            if name.startswith(("k_gs_phase2", "k_residual_restrict_x", "k_prolong_fused2", "k_xpass_df",
                                "k_residual_df", "k_xpass<", "k_residual<")):
                dofs = gmax * mx                    # one CTA per row of mx unknowns
            else:
                dofs = s.N                          # the Gram passes: the finest vectors
            bts, fl = model[0] * dofs, model[1] * dofs
            e.update({"finest_launches": len(fin), "finest_avg_us": round(us, 3), "algorithmic_bytes": bts,
                      "hbm_gbs": round(bts / (us * 1e3), 1), "hbm_frac": round(bts / (us * 1e3) / peak_hbm, 4)})
            if fl > 0:
                e.update({"fp64_flops": fl, "fp64_gflops": round(fl / (us * 1e3), 1),
                          "fp64_frac": round(fl / (us * 1e3) / FP64_PEAK_GFLOPS, 4)})
        rows.append(e)
    return {"how": "one FP32-IR solve enqueued without the graph, every launch between CUDA events on its "
                   "stream (launch overlap lost); fractions of measured HBM copy rate (MEASURED_PEAKS.json) "
                   "and of the FP64 peak (1.25 TFLOP/s nominal)",
            "total_us": round(total, 1), "kernels": rows[:16]}


def measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError):
        return fallback


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "batch256"],
                    help="c2: one 1024^2 solve (default); batch256: 256 uneven problems solved together")
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--method", default="rre", choices=["rre", "mpe"])
    ap.add_argument("--prec", default="fp32_ir", choices=["fp32_ir", "fp64"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-count", type=int, default=256, help="problems in --workload batch256")
    ap.add_argument("--tail-ctas", type=int, default=0, choices=[0, 1, 8, 16],
                    help="with --no-autotune: coarse tail on one CTA or a cluster of 8 or 16 CTAs, deepest level "
                         "(0: the default schedule)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch schedule (profiling runs: timings under a profiler mislead the autotuner)")
    ap.add_argument("--host-loop", action="store_true",
                    help="restart loop driven from the host (one graph launch per restart cycle): for profilers "
                         "that do not follow kernels inside conditional graph nodes")
    ap.add_argument("--no-extra-forms", action="store_true",
                    help="skip the 3D 128^3 and 256-problem batch forms of the default line")
    return ap.parse_args()


def workload_config(a):
    return {"workload": f"{a.dim}D IGA Poisson, {a.n}^{a.dim} elements, p={a.p}, "
                        f"{a.method.upper()}(k={a.k}) V(1,1) multicolour GS, tol 1e-10",
            "dim": a.dim, "n_elements": a.n, "p": a.p, "method": a.method, "k": a.k,
            "rhs": "random sine series, 16 modes/direction, N(0,1), seed = rank",
            "l2": "flushed between steps (256 MiB write)"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, nm in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def host_info():
    """Host CPU model and core count (the oracle's baseline runs here)."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_model": model or platform.processor() or platform.machine(),
            "host_cores": os.cpu_count(), "arch": platform.machine()}


def _memory_limit_bytes():
    """Smallest of MemAvailable and the cgroup memory limit."""
    lim = []
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    lim.append(int(line.split()[1]) * 1024)
    except OSError:
        pass
    for path in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            with open(path) as f:
                v = f.read().strip()
            if v.isdigit():
                lim.append(int(v))
        except OSError:
            pass
    return min(lim) if lim else 8 << 30


def _oracle_worker(jobs, barrier, queue):
    """One oracle process: build its problems (set-up, untimed), wait for the
    others, then solve each completely to 1e-10 and report the wall times
    (time.time(): one clock for every process on the host).  jobs: list of
    (dim, n, p, method, k, seed)."""
    import workloads
    from oracle import solver
    probs = [(solver.Problem(d, n, p, workloads.random_sine_coeffs(d, seed=sd, modes=16)), m, k)
             for (d, n, p, m, k, sd) in jobs]
    barrier.wait(timeout=1800)
    for prob, method, k in probs:
        t0 = time.time()
        out = solver.solve(prob, method, k=k, tol=1e-10, max_cycles=200)
        t1 = time.time()
        queue.put((t0, t1, out["cycles"], prob.H.finest.N, bool(out["converged"])))


def oracle_bytes_per_dof(dim, p):
    """Peak RSS of one oracle solve per unknown: its sparse operator and the
    per-colour row slices hold about 2 x 24 B per non-zero, (2p+1)^dim per row
    (measured 2D p = 3: 2.75 GB at 1.05 M unknowns)."""
    return 50.0 * (2 * p + 1) ** dim + 400.0


def oracle_run(jobs_per_worker):
    """Complete oracle solves (the CPU oracle as it stands, FP64, one thread
    per process), one spawned process per entry of jobs_per_worker, all at
    once.  Returns the aggregate DOF/s (every solve's N over the wall time
    from the first start to the last end), the per-solve times and cycles."""
    import multiprocessing as mp
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"                       # one thread per process: cores = processes
    ctx = mp.get_context("spawn")                 # never fork a process that has touched CUDA
    workers = len(jobs_per_worker)
    barrier, queue = ctx.Barrier(workers), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(jobs, barrier, queue)) for jobs in jobs_per_worker]
    total = sum(len(j) for j in jobs_per_worker)
    try:
        for pr in procs:
            pr.start()
        res = [queue.get(timeout=3600) for _ in range(total)]
        for pr in procs:
            pr.join(timeout=60)
    finally:
        for pr in procs:
            if pr.is_alive():
                pr.terminate()
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    t0 = min(r[0] for r in res)
    t1 = max(r[1] for r in res)
    per = sorted(r[1] - r[0] for r in res)
    return {"value": sum(r[3] for r in res) / (t1 - t0), "wall_s": t1 - t0, "solve_s": per,
            "dof": sum(r[3] for r in res), "cycles": sorted({r[2] for r in res}),
            "converged": all(r[4] for r in res)}


def all_core_workers(a, want):
    """Concurrent oracle processes: one per host core, at most `want`, and as
    many as the host memory (MemAvailable / cgroup limit) holds with room to spare."""
    N = (oracle_n(a) + a.p - 2) ** a.dim
    fit = int(0.5 * _memory_limit_bytes() / (oracle_bytes_per_dof(a.dim, a.p) * N))
    return max(1, min(os.cpu_count() or 1, want, fit))


def oracle_n(a):
    """Elements per direction of the oracle's sample: the workload's own, except
    that 3D problems above 64^3 are sampled at 64^3 (same p and k; the oracle's
    sparse operator holds (2p+1)^3 = 343 non-zeros per row at p = 3, 37 GB at
    128^3).  Multigrid work is linear in N, so DOF/s carries over."""
    return min(a.n, 64) if a.dim == 3 else a.n


def _job(a, seed):
    return (a.dim, oracle_n(a), a.p, a.method, a.k, seed)


def cpu_baseline(a):
    """The oracle timed on this host: one complete solve single-threaded, then
    one complete solve per process on all cores at once."""
    one = oracle_run([[_job(a, a.seed)]])
    P = all_core_workers(a, 64)
    many = oracle_run([[_job(a, a.seed + i)] for i in range(P)]) if P > 1 else one
    info = host_info()
    return {"value": many["value"], "unit": "DOF/s", "cores": P, "kind": "oracle",
            "sample": f"{P} complete solves to 1e-10 of the same workload at {oracle_n(a)}^{a.dim} elements "
                      f"(seeds {a.seed}..{a.seed + P - 1}), "
                      f"one per process on {P} cores at once, wall {many['wall_s']:.1f} s; set-up excluded",
            "time_to_tol_s": {"single_thread": one["solve_s"][0],
                              "all_cores_median": many["solve_s"][len(many["solve_s"]) // 2]},
            "single_thread": {"value": one["value"], "unit": "DOF/s", "cores": 1,
                              "sample": "one complete solve to 1e-10, seed %d" % a.seed},
            "cycles": many["cycles"], "converged": many["converged"], **info}


def run_reference(a, rank, world):
    """The oracle as the reference arm: `steps` complete solves of this arm's
    workload, run as concurrent single-threaded processes on the host cores
    (as many at once as cores and memory allow, in waves); value = DOF of all
    solves / wall time.  The oracle keeps no state between solves, so the
    warm-up is its set-up (hierarchy and factors), built before the timed region."""
    if rank != 0:
        return
    steps = max(1, a.steps)
    P = all_core_workers(a, steps)
    per_worker = (steps + P - 1) // P
    r = oracle_run([[_job(a, a.seed + i * per_worker + j) for j in range(per_worker)] for i in range(P)])
    nsolves = P * per_worker
    ms = 1e3 * r["wall_s"] / nsolves
    info = host_info()
    line = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": "DOF/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(a),
            "time_to_tol_ms": 1e3 * r["solve_s"][len(r["solve_s"]) // 2], "cycles": r["cycles"],
            "converged": r["converged"],
            "cpu_baseline": {"kind": "oracle", "cores": P, "value": r["value"], "unit": "DOF/s",
                             "sample": f"{nsolves} complete solves to 1e-10 at {oracle_n(a)}^{a.dim} elements "
                                       f"({P} processes x {per_worker}, one "
                                       f"thread each), wall {r['wall_s']:.1f} s; set-up excluded", **info},
            "e2e": {"value": r["value"], "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_ours(a, rank, world, local):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2412_20205_gb300 as pkg
    import workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    s = pkg.Solver(a.dim, a.p, a.n, k=a.k)
    # launch schedule of the FP32 cycles, picked by timing
    if a.no_autotune and a.tail_ctas:
        pkg.igamg_set_tail_ctas(s.ctx, a.tail_ctas)
        pkg.igamg_set_schedule(s.ctx, 0, 99)
    schedule = pkg.igamg_get_schedule(s.ctx) if a.no_autotune else s.autotune()
    coeffs = workloads.random_sine_coeffs(a.dim, seed=a.seed + rank, modes=16)
    b = s.rhs_sine(coeffs)
    x = torch.zeros(s.N, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def solve(prec):
        return s.solve(b, x=x, tol=1e-10, method=a.method, k=a.k, prec=prec, max_cycles=200, host_loop=a.host_loop)

    def timed(prec, steps):
        times = []
        out = None
        for _ in range(steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = solve(prec)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return times, out

    for _ in range(a.warmup):
        torch.cuda.nvtx.range_push("warmup_solve")          # marks the solves for profiler filters
        solve(a.prec)
        torch.cuda.nvtx.range_pop()
        solve("fp64")
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = pkg.igamg_launch_count()
    times, out = timed(a.prec, a.steps)
    launches = pkg.igamg_launch_count() - l0
    barrier(world)
    torch.cuda.synchronize()
    clk = clocks.stop()
    times64, out64 = timed("fp64", a.steps)

    # end to end through the public API: pinned host b in, host x out, per step
    hb = torch.empty(s.N, dtype=torch.float64, pin_memory=True)
    hb.copy_(b.cpu())
    hx = torch.empty(s.N, dtype=torch.float64, pin_memory=True)
    db = torch.empty_like(b)
    e2e_times = []
    for _ in range(a.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        db.copy_(hb, non_blocking=True)
        o = s.solve(db, x=x, tol=1e-10, method=a.method, k=a.k, prec=a.prec, max_cycles=200)
        hx.copy_(o["x"], non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append((time.perf_counter() - t0) * 1e3)

    # learned form (2D): the stored network as finest post-smoother
    learned = None
    if a.dim == 2:
        wfile = os.path.join(ROOT, "paper_2412_20205_gb300", "weights", "smoother_2d_n256_p3.npy")
        wnet = torch.tensor(np.load(wfile), dtype=torch.float32, device=dev)
        s.set_smoother(wnet)
        for _ in range(a.warmup):
            solve("fp32_ir_learned")
        tl, outl = timed("fp32_ir_learned", a.steps)
        learned = {"ms": float(np.mean(tl)), "cycles": outl["cycles"], "fell_back": outl["fell_back"],
                   "final_rel_residual": float(outl["history"][-1])}

    jacobi = None
    if a.dim == 2:     # the weighted-Jacobi cycle with omega = 2/3 stagnates in 3D (128^3, p = 3: 1.6e-3 after 200 restarts)
        # the paper's own smoother (Sec. 4): weighted Jacobi, omega = 2/3, same V(1,1)-cycle
        pkg.igamg_set_cycle(s.ctx, "jacobi", 1, 2.0 / 3.0)
        for _ in range(a.warmup):
            torch.cuda.nvtx.range_push("jacobi_warmup_solve")   # marks the solves for profiler filters
            solve(a.prec)
            torch.cuda.nvtx.range_pop()
            solve("fp64")
        tj, outj = timed(a.prec, a.steps)
        tj64, outj64 = timed("fp64", a.steps)
        pkg.igamg_set_cycle(s.ctx, "gs", 1)
        jacobi = {"ms": float(np.mean(tj)), "cycles": outj["cycles"], "ms64": float(np.mean(tj64)),
                  "cycles64": outj64["cycles"], "final_rel_residual": float(outj["history"][-1])}

    # Dominant kernel (ncu launch list of this workload): the FP32 row-phase
    # Gauss-Seidel kernel.  Timed here on the finest level, same launch
    # configuration as inside the solve, with CUDA events over `reps` sweeps
    # ((p+1)^(dim-1) launches each) on this stream.  Algorithmic bytes of a
    # sweep: read x, b and write x in FP32 = 12 B per DOF; one launch does its
    # share, 12 N / (p+1)^(dim-1) bytes.
    top = len(s.levels) - 1
    xg = torch.randn(s.N, dtype=torch.float32, device=dev)
    bg = torch.randn(s.N, dtype=torch.float32, device=dev)
    pkg.igamg_smooth_f32(s.ctx, top, xg, bg, 0, s.ws)
    for _ in range(3):
        pkg.igamg_smooth_f32(s.ctx, top, xg, bg, 0, s.ws, sums_current=True)
    reps = 50
    launches_per_sweep = (a.p + 1) ** (a.dim - 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        pkg.igamg_smooth_f32(s.ctx, top, xg, bg, 0, s.ws, sums_current=True, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    launch_ms = e0.elapsed_time(e1) / (reps * launches_per_sweep)
    bytes_per_launch = 12.0 * s.N / launches_per_sweep
    achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9
    peak_hbm = measured_peak("hbm_gbs", 6800.0)

    if learned is not None:
        learned["ms"] = max_over_ranks(learned["ms"], world)
    if jacobi is not None:
        jacobi["ms"] = max_over_ranks(jacobi["ms"], world)
        jacobi["ms64"] = max_over_ranks(jacobi["ms64"], world)
    t_max = max_over_ranks(float(np.mean(times)), world)
    t64_max = max_over_ranks(float(np.mean(times64)), world)
    e2e_max = max_over_ranks(float(np.mean(e2e_times)), world)
    if rank != 0:
        return
    units = s.N * world
    line = {
        "metric": METRIC, "value": units / (t_max * 1e-3), "unit": "DOF/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if a.prec == "fp32_ir" else "f64",
        "data": "synthetic", "config": dict(workload_config(a), schedule=schedule),
        "time_to_tol_ms": t_max, "cycles": out["cycles"], "vcycles": out["vcycles"],
        "final_rel_residual": float(out["history"][-1]),
        "vcycle_throughput": {"value": units * out["vcycles"] / (t_max * 1e-3), "unit": "DOF x V-cycles/s"},
        "fp64_form": {"ms_per_step": t64_max, "value": units / (t64_max * 1e-3), "unit": "DOF/s",
                      "cycles": out64["cycles"], "final_rel_residual": float(out64["history"][-1])},
        "e2e": {"value": units / (e2e_max * 1e-3), "unit": "DOF/s",
                "h2d_bytes_per_step": s.N * 8, "d2h_bytes_per_step": s.N * 8},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": f"k_gs_phase{a.dim}<float, {a.p}, {str(a.dim == 3 or a.p != 3).lower()}> "
                                                    "(finest level, one row phase)",
                     "achieved": achieved, "peak": peak_hbm, "unit": "GB/s", "frac": achieved / peak_hbm,
                     "traffic": GS_TRAFFIC.get((a.dim, a.n, a.p)),
                     "algorithmic_bytes_per_launch": bytes_per_launch, "launch_us": launch_ms * 1e3,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
        "clocks": clk,
    }
    if learned is not None:
        tl_max = learned["ms"]
        line["learned_form"] = {"ms_per_step": tl_max, "value": units / (tl_max * 1e-3), "unit": "DOF/s",
                                "cycles": learned["cycles"], "fell_back": learned["fell_back"],
                                "final_rel_residual": learned["final_rel_residual"],
                                "network": "3x3 conv 1-16-16-1, BF16/FP32, trained on 257^2 p=3 pairs"}
    if jacobi is not None:
        line["jacobi_form"] = {"ms_per_step": jacobi["ms"], "value": units / (jacobi["ms"] * 1e-3), "unit": "DOF/s",
                               "cycles": jacobi["cycles"], "final_rel_residual": jacobi["final_rel_residual"],
                               "fp64_ms_per_step": jacobi["ms64"], "fp64_cycles": jacobi["cycles64"],
                               "smoother": "weighted Jacobi, omega = 2/3 (the paper's experiments), V(1,1)"}
    if a.dim == 2 and a.prec == "fp32_ir":
        line["kernel_table"] = kernel_table(pkg, s, b, a, peak_hbm)
    if not a.no_extra_forms and a.dim == 2 and world == 1:
        # the other two build workloads, measured in the same run (complete solves)
        sx = min(a.steps, 5)
        line["c3_form"] = c3_form(a, pkg, flush, stream, sx, min(a.warmup, 2))
        line["c4_form"] = c4_form(a, pkg, flush, stream, sx, min(a.warmup, 2))
    if not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a)
    print(json.dumps(line), flush=True)


def _timed_solves(fn, steps, flush, stream):
    """CUDA-event times (ms) of `steps` calls of fn(), L2 flushed before each."""
    import torch
    times, out = [], None
    for _ in range(steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times, out


def c3_form(a, pkg, flush, stream, steps, warmup):
    """3D Poisson, 128^3 elements, p = 3, RRE(10), manufactured right side: the
    mixed and FP64 forms, complete solves to 1e-10."""
    import numpy as np
    import workloads
    s = pkg.Solver(3, 3, 128, k=10)
    b = s.rhs_sine(workloads.manufactured_coeffs(3))
    res = {"workload": "3D IGA Poisson, 128^3 elements, p=3, RRE(k=10), V(1,1) multicolour GS (64 colours), "
                       "f = 3 pi^2 prod sin(pi x_d), tol 1e-10", "dof": s.N}
    for prec in ("fp32_ir", "fp64"):
        fn = lambda: s.solve(b, tol=1e-10, method="rre", k=10, prec=prec, max_cycles=100)
        for _ in range(warmup):
            fn()
        t, out = _timed_solves(fn, steps, flush, stream)
        ms = float(np.mean(t))
        res[prec] = {"ms_per_step": ms, "value": s.N / (ms * 1e-3), "unit": "DOF/s", "cycles": out["cycles"],
                     "vcycles": out["vcycles"], "final_rel_residual": float(out["history"][-1])}
    s.close()
    return res


def c4_form(a, pkg, flush, stream, steps, warmup):
    """256 independent 2D problems, n ~ U{32..512}, p ~ U{2,3,4}, random 16-mode
    right sides, RRE(5): the mixed and FP64 forms of one batched solve."""
    import numpy as np
    import workloads
    probs = workloads.batch_problems(256, seed=0)
    B = pkg.Batch(2, [q["p"] for q in probs], [q["n"] for q in probs], k=5)
    coeffs = np.stack([workloads.random_sine_coeffs(2, seed=q["rhs_seed"], modes=16) for q in probs])
    b = B.rhs_sine(coeffs)
    B.autotune()
    res = {"workload": "256 independent 2D IGA Poisson problems, n ~ U{32..512}, p ~ U{2,3,4}, RRE(k=5), "
                       "tol 1e-10", "dof": B.N}
    for prec in ("fp32_ir", "fp64"):
        fn = lambda: B.solve(b, tol=1e-10, method="rre", k=5, prec=prec)
        for _ in range(warmup):
            fn()
        l0 = pkg.igamg_launch_count()
        t, out = _timed_solves(fn, steps, flush, stream)
        ms = float(np.mean(t))
        res[prec] = {"ms_per_step": ms, "value": B.N / (ms * 1e-3), "unit": "DOF/s",
                     "max_cycles": int(max(out["cycles"])), "converged": bool(out["converged"]),
                     "max_rel_residual": float(max(out["residuals"])),
                     "gpu_launches_per_solve": (pkg.igamg_launch_count() - l0) // max(1, steps)}
    B.close()
    return res


def run_batch(a, rank, world, local):
    """256 independent 2D problems, n ~ U{32..512}, p ~ U{2,3,4}, random 16-mode
    right-hand sides; one step = one batched solve of all of them."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2412_20205_gb300 as pkg
    import workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    probs = workloads.batch_problems(a.batch_count, seed=a.seed + rank)
    ps = [q["p"] for q in probs]
    ns = [q["n"] for q in probs]
    B = pkg.Batch(2, ps, ns, k=a.k)
    coeffs = np.stack([workloads.random_sine_coeffs(2, seed=q["rhs_seed"], modes=16) for q in probs])
    b = B.rhs_sine(coeffs)
    B.autotune()                            # launch schedules of the FP32 cycles, picked by timing
    x = torch.empty(B.N, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(prec, steps):
        times, out = [], None
        for _ in range(steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = B.solve(b, x=x, tol=1e-10, method=a.method, k=a.k, prec=prec)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return times, out

    for _ in range(a.warmup):
        B.solve(b, x=x, tol=1e-10, method=a.method, k=a.k, prec=a.prec)
        B.solve(b, x=x, tol=1e-10, method=a.method, k=a.k, prec="fp64")
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = pkg.igamg_launch_count()
    times, out = timed(a.prec, a.steps)
    launches = pkg.igamg_launch_count() - l0
    clk = clocks.stop()
    times64, out64 = timed("fp64", a.steps)
    hb = b.cpu().pin_memory()
    hx = torch.empty(B.N, dtype=torch.float64, pin_memory=True)
    db = torch.empty_like(b)
    e2e = []
    for _ in range(a.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        db.copy_(hb, non_blocking=True)
        o = B.solve(db, x=x, tol=1e-10, method=a.method, k=a.k, prec=a.prec)
        hx.copy_(o["x"], non_blocking=True)
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    t_max = max_over_ranks(float(np.mean(times)), world)
    t64 = max_over_ranks(float(np.mean(times64)), world)
    te = max_over_ranks(float(np.mean(e2e)), world)
    if rank != 0:
        return
    units = B.N * world
    line = {
        "metric": METRIC, "value": units / (t_max * 1e-3), "unit": "DOF/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if a.prec == "fp32_ir" else "f64", "data": "synthetic",
        "config": {"workload": f"{len(probs)} independent 2D IGA Poisson problems, n ~ U{{32..512}}, p ~ U{{2,3,4}}, "
                               f"{a.method.upper()}(k={a.k}), tol 1e-10, {B.N} unknowns in total",
                   "problems": len(probs), "total_dof": B.N, "method": a.method, "k": a.k,
                   "rhs": "random sine series, 16 modes/direction, N(0,1), seed 1000 + i",
                   "schedule": "autotuned per degree (igamg_batch_autotune)",
                   "l2": "flushed between steps (256 MiB write)"},
        "converged": bool(out["converged"]), "max_cycles": int(max(out["cycles"])),
        "max_rel_residual": float(max(out["residuals"])),
        "fp64_form": {"ms_per_step": t64, "value": units / (t64 * 1e-3), "unit": "DOF/s",
                      "max_cycles": int(max(out64["cycles"]))},
        "e2e": {"value": units / (te * 1e-3), "unit": "DOF/s", "h2d_bytes_per_step": B.N * 8,
                "d2h_bytes_per_step": B.N * 8},
        "gpu_launches": launches, "clocks": clk,
    }
    if not a.no_cpu_baseline:
        # the batch's first members, each solved completely, one per process on
        # all cores at once (every worker gets the same count; memory-bounded)
        P = max(1, min(os.cpu_count() or 1, 16,
                       int(0.5 * _memory_limit_bytes() / (oracle_bytes_per_dof(2, 4) * 513 ** 2))))
        per = 2
        jobs = [[(2, q["n"], q["p"], a.method, a.k, q["rhs_seed"]) for q in probs[i * per:(i + 1) * per]]
                for i in range(P)]
        r = oracle_run(jobs)
        line["cpu_baseline"] = {"value": r["value"], "unit": "DOF/s", "cores": P, "kind": "oracle",
                                "sample": f"batch members 0..{P * per - 1} ({r['dof']} unknowns) solved "
                                          f"completely to 1e-10, {per} per process on {P} cores at once, "
                                          f"wall {r['wall_s']:.1f} s; set-up excluded", **host_info()}
    print(json.dumps(line), flush=True)
    B.close()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"      # gloo (host tests): CPU tensors
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if a.workload == "batch256":
        run_batch(a, rank, world, local)
    else:
        run_ours(a, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
