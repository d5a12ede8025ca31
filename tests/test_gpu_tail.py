"""The one-CTA coarse tail of FP32 2D V-cycles, through the C ABI.

The tail changes the schedule of Algorithm 2's coarse levels, not its
arithmetic: one FP32 refinement step with the tail agrees with the same step
without it to FP32 round-off (relative 1e-5 on the correction) and with the
FP64 oracle's V-cycle to FP32 accuracy (2e-5, as for the per-level path);
whole solves converge in the same number of restart cycles.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import multigrid as omg  # noqa: E402
from oracle.galerkin import load_vector  # noqa: E402
import workloads  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build_library()
    import paper_2412_20205_gb300 as p
    assert torch.cuda.is_available()
    return p


DEV = "cuda"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n,p", [(64, 3), ((40, 27), 2), (130, 5), (100, 7), (33, 1), (70, 4)])
def test_tail_cycle_matches_per_level_cycle_and_oracle(pkg, n, p):
    ns = list(n) if isinstance(n, tuple) else [n, n]
    ctx = pkg.igamg_setup(2, p, ns, 0)
    pkg.igamg_assemble(ctx)
    assert pkg.igamg_coarse_tail_level(ctx) >= 1
    H = omg.Hierarchy(2, ns, p)
    ws = torch.empty(pkg.igamg_workspace_bytes(ctx, 5, pkg.IGAMG_FP32_IR), dtype=torch.uint8, device=DEV)
    rng = np.random.default_rng(p)
    b = load_vector(H.finest.breaks, p, rng.standard_normal((3, 3)))
    x0 = rng.standard_normal(H.finest.N) * 1e-3
    ref = omg.cycle(H, x0, b)
    out = {}
    for on in (True, False):
        pkg.igamg_set_coarse_tail(ctx, on)
        x = _t(x0)
        pkg.igamg_vcycle(ctx, x, _t(b), pkg.IGAMG_FP32_IR, ws)
        out[on] = _np(x) - x0
    assert pkg.igamg_coarse_tail_level(ctx) == 0          # switched off last
    assert _rel(out[True], out[False]) < 1e-5
    assert _rel(out[True], ref - x0) < 2e-5
    pkg.igamg_destroy(ctx)


def test_tail_levels(pkg):
    # 1024^2, p = 3: levels n = 8, 16, 32, 64 ((n+1)^2 <= 6000 unknowns) form the tail
    ctx = pkg.igamg_setup(2, 3, [1024, 1024], 0)
    pkg.igamg_assemble(ctx)
    assert pkg.igamg_coarse_tail_level(ctx) == 3
    pkg.igamg_destroy(ctx)
    # 3D has no one-CTA tail; its coarse levels run on a 16-CTA cluster by default
    ctx = pkg.igamg_setup(3, 2, [32, 32, 32], 0)
    pkg.igamg_assemble(ctx)
    assert pkg.igamg_tail_levels_available(ctx, 1) == 0
    assert pkg.igamg_get_schedule(ctx)["tail_ctas"] == 16
    assert pkg.igamg_coarse_tail_level(ctx) == pkg.igamg_tail_levels_available(ctx, 16) >= 1
    pkg.igamg_destroy(ctx)


@pytest.mark.parametrize("p", [2, 3, 5])
def test_tail_solves_like_per_level_schedule(pkg, p):
    s = pkg.Solver(2, p, 256, k=5)
    b = s.rhs_sine(workloads.random_sine_coeffs(2, seed=p))
    res = {}
    for on in (False, True):
        pkg.igamg_set_coarse_tail(s.ctx, on)
        res[on] = s.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir", max_cycles=60)
        assert res[on]["converged"]
    assert abs(res[True]["cycles"] - res[False]["cycles"]) <= 1
    ref = s.solve(b, tol=1e-12, method="rre", k=5, prec="fp64", max_cycles=60)["x"]
    assert float((res[True]["x"] - ref).norm() / ref.norm()) < 1e-7
    s.close()


def test_schedules_agree_and_autotune_solves(pkg):
    """Every launch schedule (GS row-CTA cap x tail depth) computes the same
    FP32 cycle up to rounding order; the autotuned one solves to tolerance."""
    s = pkg.Solver(2, 3, 200, k=5)
    H = omg.Hierarchy(2, [200, 200], 3)
    rng = np.random.default_rng(8)
    b = load_vector(H.finest.breaks, 3, rng.standard_normal((4, 4)))
    x0 = rng.standard_normal(H.finest.N) * 1e-3
    ref = omg.cycle(H, x0, b) - x0
    outs = []
    for cap in (128, 256, 512):
        for tail in (0, 1, 99):
            pkg.igamg_set_schedule(s.ctx, cap, tail)
            sch = pkg.igamg_get_schedule(s.ctx)
            assert sch["gs_threads"] == cap and sch["tail_levels"] <= 99
            x = _t(x0)
            pkg.igamg_vcycle(s.ctx, x, _t(b), pkg.IGAMG_FP32_IR, s.ws)
            outs.append(_np(x) - x0)
    for o in outs:
        assert _rel(o, ref) < 2e-5
    sch = s.autotune(reps=2)
    assert sch["gs_threads"] in (128, 256, 512) and sch["tail_levels"] >= 0
    bb = s.rhs_sine(workloads.random_sine_coeffs(2, seed=3))
    out = s.solve(bb, tol=1e-10, method="rre", k=5, prec="fp32_ir")
    assert out["converged"]
    ref64 = s.solve(bb, tol=1e-12, method="rre", k=5, prec="fp64")["x"]
    assert float((out["x"] - ref64).norm() / ref64.norm()) < 1e-7
    with pytest.raises(RuntimeError):
        pkg.igamg_set_schedule(s.ctx, 100, 0)
    s.close()


def test_batch_autotune(pkg):
    ps, ns = [2, 3, 3, 4, 2, 3], [40, 90, 64, 33, 120, 70]
    B = pkg.Batch(2, ps, ns, k=5)
    coeffs = np.stack([workloads.random_sine_coeffs(2, seed=i) for i in range(len(ps))])
    b = B.rhs_sine(coeffs)
    B.autotune(reps=2)
    out = B.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir")
    assert out["converged"], out["statuses"]


@pytest.mark.parametrize("p", [2, 3, 5])
def test_fp32_ir_residual_recurrence_reaches_tight_tolerance(pkg, p):
    """The FP32-IR form carries the FP64 residual by r <- r - A e in
    double-FP32 arithmetic inside a restart; it must not stall above the
    FP64 solve's accuracy: relative residual 1e-12 is reached and the
    solution agrees with an FP64 solve to 1e-10."""
    s = pkg.Solver(2, p, 256, k=5)
    b = s.rhs_sine(workloads.random_sine_coeffs(2, seed=11))
    out = s.solve(b, tol=1e-12, method="rre", k=5, prec="fp32_ir", max_cycles=80)
    assert out["converged"], out["history"][-4:]
    ref = s.solve(b, tol=1e-13, method="rre", k=5, prec="fp64", max_cycles=120)
    assert ref["converged"]
    assert float((out["x"] - ref["x"]).norm() / ref["x"].norm()) < 1e-10
    s.close()


@pytest.mark.parametrize("n,p", [(32, 2), (24, 3), (16, 4)])
def test_fp32_ir_residual_recurrence_3d_reaches_tight_tolerance(pkg, n, p):
    """The 3D recurrence (double-FP32 x pass, y pass and z pass of the
    sum-factorised residual) must not stall either: relative residual 1e-12 is
    reached and the true FP64 residual b - A x of the result (applied
    independently) meets it.  Near 1e-12 the FP32 V-cycles' own rounding can
    cost a few restarts against the FP64 solve (16^3, p = 4: 29 against 27)."""
    s = pkg.Solver(3, p, n, k=10)
    b = s.rhs_sine(workloads.random_sine_coeffs(3, seed=12, modes=6))
    out = s.solve(b, tol=1e-12, method="rre", k=10, prec="fp32_ir", max_cycles=80)
    assert out["converged"], out["history"][-4:]
    y = torch.empty_like(b)
    pkg.igamg_apply(s.ctx, len(s.levels) - 1, out["x"], y, s.ws)
    res = float((b - y).norm() / b.norm())
    assert res <= 1.05e-12, res
    ref = s.solve(b, tol=1e-12, method="rre", k=10, prec="fp64", max_cycles=120)
    assert ref["converged"]
    assert out["cycles"] <= ref["cycles"] + 3 + ref["cycles"] // 10
    # both within 1e-12 in residual: their distance is at most cond(A) times that
    assert float((out["x"] - ref["x"]).norm() / ref["x"].norm()) < 1e-8
    s.close()


def test_launch_overlap_is_bitwise_neutral(pkg):
    """Launch overlap (programmatic dependent launch) changes when a kernel's
    CTAs are scheduled, never what they compute: every precision form, 2D and
    3D, single and batched, gives bit-identical solutions and cycle counts with
    the overlap on and off, inside the restart-cycle graphs and outside them."""
    import os
    wfile = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                         "paper_2412_20205_gb300", "weights", "smoother_2d_n256_p3.npy")
    cases = [(2, 3, 256, ["fp64", "fp32_ir", "fp32_ir_learned"]), (3, 2, 24, ["fp64", "fp32_ir"])]
    assert pkg.igamg_get_launch_overlap()
    try:
        for dim, p, n, precs in cases:
            s = pkg.Solver(dim, p, n, k=5)
            if "fp32_ir_learned" in precs:
                s.set_smoother(torch.tensor(np.load(wfile), dtype=torch.float32, device=DEV))
            b = s.rhs_sine(workloads.random_sine_coeffs(dim, seed=5))
            for prec in precs:
                res = {}
                for ov in (1, 0, 1):
                    pkg.igamg_set_launch_overlap(ov)
                    assert pkg.igamg_get_launch_overlap() == bool(ov)
                    out = s.solve(b, tol=1e-10, method="rre", k=5, prec=prec)
                    assert out["converged"]
                    res.setdefault(ov, []).append((_np(out["x"]).copy(), out["cycles"]))
                x_on, c_on = res[1][0]
                for x, c in res[1][1:] + res[0]:
                    assert c == c_on and np.array_equal(x, x_on), (dim, prec)
            # the component entry points (no graph) as well
            x0 = s.rhs_sine(workloads.random_sine_coeffs(dim, seed=6)) * 1e-3
            outs = []
            for ov in (1, 0):
                pkg.igamg_set_launch_overlap(ov)
                x = x0.clone()
                pkg.igamg_vcycle(s.ctx, x, b, pkg.IGAMG_FP32_IR, s.ws)
                outs.append(_np(x))
            assert np.array_equal(outs[0], outs[1])
            s.close()
        ps, ns = [2, 3, 4, 3], [40, 90, 33, 70]
        B = pkg.Batch(2, ps, ns, k=5)
        bb = B.rhs_sine(np.stack([workloads.random_sine_coeffs(2, seed=i) for i in range(len(ps))]))
        xs = []
        for ov in (1, 0):
            pkg.igamg_set_launch_overlap(ov)
            out = B.solve(bb, tol=1e-10, method="rre", k=5, prec="fp32_ir")
            assert out["converged"]
            xs.append(_np(out["x"]).copy())
        assert np.array_equal(xs[0], xs[1])
    finally:
        pkg.igamg_set_launch_overlap(1)
