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


# ---------------------------------------------------------------- CPU oracle sample
def oracle_sample(a, rank_seed=0, restarts=1):
    """Bounded sample of the oracle on the same workload: the restart-cycle count
    to tolerance is taken from the oracle on the 128^dim version of the problem
    (multigrid convergence is mesh independent), and one restart cycle (k+1
    V-cycles, extrapolation, residual) is timed on the full-size problem.
    Returns (dof_per_s, seconds_per_restart, cycles, setup_s)."""
    import numpy as np
    import workloads
    from oracle import extrapolation, solver
    coeffs = workloads.random_sine_coeffs(a.dim, seed=rank_seed, modes=16)
    small = solver.Problem(a.dim, min(a.n, 128), a.p, coeffs)
    cycles = solver.solve(small, a.method, k=a.k, tol=1e-10, max_cycles=100)["cycles"]
    t0 = time.perf_counter()
    prob = solver.Problem(a.dim, a.n, a.p, coeffs)
    setup = time.perf_counter() - t0
    N = prob.H.finest.N
    s = np.zeros(N)
    t0 = time.perf_counter()
    for _ in range(restarts):
        S = [s]
        for _ in range(a.k + 1):
            S.append(prob.cycle(S[-1]))
        s = extrapolation.extrapolate(S, a.method)[0]
        prob.residual(s)
    per = (time.perf_counter() - t0) / restarts
    return N / (per * cycles), per, cycles, setup, N


def run_reference(a, rank, world):
    if rank != 0:
        return
    for _ in range(a.warmup):
        pass                                    # the oracle has no warm-up state
    vals, pers = [], []
    cycles = None
    for _ in range(max(1, a.steps)):
        v, per, cycles, setup, N = oracle_sample(a)
        vals.append(v)
        pers.append(per)
    v = sorted(vals)[len(vals) // 2]
    ms = 1e3 * N / v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DOF/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(a),
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": v, "unit": "DOF/s",
                             "sample": f"one restart cycle ({a.k + 1} V-cycles + extrapolation + residual) "
                                       f"timed at full size x {cycles} cycles (count from the 128^dim problem)"},
            "e2e": {"value": v, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
    schedule = s.autotune()                 # launch schedule of the FP32 cycles, picked by timing
    coeffs = workloads.random_sine_coeffs(a.dim, seed=a.seed + rank, modes=16)
    b = s.rhs_sine(coeffs)
    x = torch.zeros(s.N, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def solve(prec):
        return s.solve(b, x=x, tol=1e-10, method=a.method, k=a.k, prec=prec, max_cycles=200)

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
        "roofline": {"bound": "hbm", "kernel": f"k_gs_phase<float,{a.dim},{a.p}> (finest level, one row phase)",
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
    line["jacobi_form"] = {"ms_per_step": jacobi["ms"], "value": units / (jacobi["ms"] * 1e-3), "unit": "DOF/s",
                           "cycles": jacobi["cycles"], "final_rel_residual": jacobi["final_rel_residual"],
                           "fp64_ms_per_step": jacobi["ms64"], "fp64_cycles": jacobi["cycles64"],
                           "smoother": "weighted Jacobi, omega = 2/3 (the paper's experiments), V(1,1)"}
    if not a.no_cpu_baseline:
        v, per, cycles, setup, N = oracle_sample(a)
        line["cpu_baseline"] = {"value": v, "unit": "DOF/s", "cores": 1, "kind": "oracle",
                                "sample": f"one restart cycle timed at full size ({per:.2f} s) x {cycles} "
                                          f"cycles (count from the 128^dim problem); set-up {setup:.1f} s excluded"}
    print(json.dumps(line), flush=True)


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
    probs = workloads.batch_problems(256, seed=a.seed + rank)
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
    jacobi["ms"] = max_over_ranks(jacobi["ms"], world)
    jacobi["ms64"] = max_over_ranks(jacobi["ms64"], world)
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
        "config": {"workload": f"256 independent 2D IGA Poisson problems, n ~ U{{32..512}}, p ~ U{{2,3,4}}, "
                               f"{a.method.upper()}(k={a.k}), tol 1e-10, {B.N} unknowns in total",
                   "problems": 256, "total_dof": B.N, "method": a.method, "k": a.k,
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
        from oracle import solver
        sample = [q for q in probs if q["n"] <= 96][:6]
        dof = 0
        tsum = 0.0
        for q in sample:
            prob = solver.Problem(2, q["n"], q["p"], workloads.random_sine_coeffs(2, seed=q["rhs_seed"], modes=16))
            t1 = time.perf_counter()
            solver.solve(prob, a.method, k=a.k, tol=1e-10, max_cycles=100)
            tsum += time.perf_counter() - t1
            dof += prob.H.finest.N
        line["cpu_baseline"] = {"value": dof / tsum, "unit": "DOF/s", "cores": 1, "kind": "oracle",
                                "sample": f"{len(sample)} members with n <= 96 solved to 1e-10 "
                                          f"({dof} unknowns, {tsum:.1f} s), set-up excluded"}
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
