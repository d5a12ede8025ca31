"""The coarse tail of FP32 2D V-cycles on a thread-block cluster, through the
C ABI.

Like the one-CTA tail it changes the schedule of Algorithm 2's coarse levels,
not its arithmetic: each CTA of the cluster owns a band of grid rows of every
tail level, and reads its neighbours' rows from their shared memory.  One
FP32 refinement step with the cluster tail agrees with the per-level cycle
and with the one-CTA tail to FP32 round-off (relative 1e-5 on the
correction, 2-norm and max-norm) and with the FP64 oracle's cycle to FP32
accuracy (2e-5), for several depths, both cluster sizes, both smoothers,
square and rectangular grids, p = 1..7 and bands of unequal row counts;
whole solves converge like the per-level schedule.  The 3D form (the default
for 3D cycles) is checked the same way: one cycle against the per-level
cycle and the oracle's, both smoothers, several depths and shapes, and
whole solves.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import multigrid as omg  # noqa: E402
from oracle.galerkin import load_vector  # noqa: E402
import workloads  # noqa: E402

DEV = "cuda"


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build_library()
    import paper_2412_20205_gb300 as p
    assert torch.cuda.is_available()
    return p


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _relmax(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


SHAPES = [(64, 3), ((40, 27), 2), (130, 5), (100, 7), (33, 1), (70, 4), (256, 3), ((300, 77), 2), (150, 6)]


@pytest.mark.parametrize("n,p", SHAPES, ids=lambda c: str(c))
@pytest.mark.parametrize("smoother", ["gs", "jacobi"])
def test_cluster_tail_cycle_matches_oracle_and_other_schedules(pkg, n, p, smoother):
    ns = list(n) if isinstance(n, tuple) else [n, n]
    ctx = pkg.igamg_setup(2, p, ns, 0)
    pkg.igamg_assemble(ctx)
    pkg.igamg_set_cycle(ctx, smoother, 1)
    H = omg.Hierarchy(2, ns, p)
    ws = torch.empty(pkg.igamg_workspace_bytes(ctx, 5, pkg.IGAMG_FP32_IR), dtype=torch.uint8, device=DEV)
    rng = np.random.default_rng(p + 10)
    b = load_vector(H.finest.breaks, p, rng.standard_normal((3, 3)))
    x0 = rng.standard_normal(H.finest.N) * 1e-3
    ref = omg.cycle(H, x0, b, smoother=smoother) - x0

    def cycle():
        x = _t(x0)
        pkg.igamg_vcycle(ctx, x, _t(b), pkg.IGAMG_FP32_IR, ws)
        return _np(x) - x0

    pkg.igamg_set_coarse_tail(ctx, False)
    per_level = cycle()
    pkg.igamg_set_coarse_tail(ctx, True)
    pkg.igamg_set_tail_ctas(ctx, 1)
    one_cta = cycle() if pkg.igamg_coarse_tail_level(ctx) > 0 else per_level
    checked = 0
    for ctas in (8, 16):
        most = pkg.igamg_tail_levels_available(ctx, ctas)
        assert most >= 1, (ctas, ns, p)
        pkg.igamg_set_tail_ctas(ctx, ctas)
        for lc in sorted({1, (most + 1) // 2, most}):
            pkg.igamg_set_schedule(ctx, 0, lc)
            assert pkg.igamg_coarse_tail_level(ctx) == lc
            assert pkg.igamg_get_schedule(ctx)["tail_ctas"] == ctas
            out = cycle()
            for other in (per_level, one_cta):
                assert _rel(out, other) < 1e-5 and _relmax(out, other) < 1e-5, (ctas, lc)
            assert _rel(out, ref) < 2e-5 and _relmax(out, ref) < 2e-5, (ctas, lc)
            checked += 1
    assert checked >= 2
    pkg.igamg_destroy(ctx)


def test_cluster_tail_reaches_the_level_of_257_rows(pkg):
    """1024^2, p = 3: 16 CTAs hold levels up to 256^2 elements (257 rows),
    8 CTAs up to 128^2; the one-CTA tail stops at 64^2."""
    ctx = pkg.igamg_setup(2, 3, [1024, 1024], 0)
    pkg.igamg_assemble(ctx)
    # rows of levels 0..7: 9, 17, 33, 65, 129, 257, 513, 1025
    assert pkg.igamg_tail_levels_available(ctx, 1) == 3
    assert pkg.igamg_tail_levels_available(ctx, 8) == 4
    assert pkg.igamg_tail_levels_available(ctx, 16) == 5
    with pytest.raises(pkg.IgamgError):
        pkg.igamg_set_tail_ctas(ctx, 4)
    pkg.igamg_destroy(ctx)


@pytest.mark.parametrize("p", [2, 3, 5])
def test_cluster_tail_solves_like_per_level_schedule(pkg, p):
    s = pkg.Solver(2, p, 1024, k=5)
    b = s.rhs_sine(workloads.random_sine_coeffs(2, seed=p, modes=16))
    pkg.igamg_set_coarse_tail(s.ctx, False)
    ref32 = s.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir", max_cycles=60)
    assert ref32["converged"]
    pkg.igamg_set_coarse_tail(s.ctx, True)
    pkg.igamg_set_tail_ctas(s.ctx, 16)
    pkg.igamg_set_schedule(s.ctx, 0, 99)
    assert pkg.igamg_coarse_tail_level(s.ctx) == 5
    out = s.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir", max_cycles=60)
    assert out["converged"]
    assert abs(out["cycles"] - ref32["cycles"]) <= 1
    ref = s.solve(b, tol=1e-12, method="rre", k=5, prec="fp64", max_cycles=60)["x"]
    assert float((out["x"] - ref).norm() / ref.norm()) < 1e-7
    # outside the graphs (host loop, no capture) the same
    again = s.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir", max_cycles=60, graph=False, host_loop=True)
    assert again["cycles"] == out["cycles"]
    assert float((again["x"] - out["x"]).norm() / out["x"].norm()) < 1e-12
    s.close()


def test_batch_members_with_cluster_tails(pkg):
    """Members of a batch run concurrently in one graph; each member's cluster
    tail is its own cluster."""
    ps, ns = [2, 3, 3, 4, 2, 3, 3, 2], [256, 300, 128, 200, 512, 90, 256, 33]
    B = pkg.Batch(2, ps, ns, k=5)
    coeffs = np.stack([workloads.random_sine_coeffs(2, seed=i) for i in range(len(ps))])
    b = B.rhs_sine(coeffs)
    base = B.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir")
    assert base["converged"]
    pkg.igamg_batch_set_tail_ctas(B.handle, 16)
    out = B.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir")
    assert out["converged"], out["statuses"]
    assert np.all(np.abs(np.asarray(out["cycles"]) - np.asarray(base["cycles"])) <= 1)
    B.close()


# three or more levels (a tail needs a level between the finest and the coarsest)
SHAPES3 = [(20, 3), (24, 2), ((20, 17, 24), 3), (18, 5), (20, 1), (24, 4), (18, 6)]


@pytest.mark.parametrize("n,p", SHAPES3, ids=lambda c: str(c))
@pytest.mark.parametrize("smoother", ["gs", "jacobi"])
def test_cluster_tail3_cycle_matches_oracle_and_per_level(pkg, n, p, smoother):
    ns = list(n) if isinstance(n, tuple) else [n, n, n]
    ctx = pkg.igamg_setup(3, p, ns, 0)
    pkg.igamg_assemble(ctx)
    pkg.igamg_set_cycle(ctx, smoother, 1)
    H = omg.Hierarchy(3, ns, p)
    ws = torch.empty(pkg.igamg_workspace_bytes(ctx, 5, pkg.IGAMG_FP32_IR), dtype=torch.uint8, device=DEV)
    rng = np.random.default_rng(p + 30)
    b = load_vector(H.finest.breaks, p, rng.standard_normal((2, 2, 2)))
    x0 = rng.standard_normal(H.finest.N) * 1e-3
    ref = omg.cycle(H, x0, b, smoother=smoother) - x0

    def cycle():
        x = _t(x0)
        pkg.igamg_vcycle(ctx, x, _t(b), pkg.IGAMG_FP32_IR, ws)
        return _np(x) - x0

    assert pkg.igamg_get_schedule(ctx)["tail_ctas"] == 16       # the 3D default
    pkg.igamg_set_coarse_tail(ctx, False)
    per_level = cycle()
    assert _rel(per_level, ref) < 2e-5
    pkg.igamg_set_coarse_tail(ctx, True)
    checked = 0
    for ctas in (8, 16):
        most = pkg.igamg_tail_levels_available(ctx, ctas)
        if most < 1:
            continue
        pkg.igamg_set_tail_ctas(ctx, ctas)
        for lc in sorted({1, most}):
            pkg.igamg_set_schedule(ctx, 0, lc)
            assert pkg.igamg_coarse_tail_level(ctx) == lc
            out = cycle()
            assert _rel(out, per_level) < 1e-5 and _relmax(out, per_level) < 1e-5, (ctas, lc)
            assert _rel(out, ref) < 2e-5 and _relmax(out, ref) < 2e-5, (ctas, lc)
            checked += 1
    assert checked >= 1
    pkg.igamg_destroy(ctx)


def test_cluster_tail3_schedule_switches(pkg):
    """3D has no one-CTA tail: asking for it switches the tail off; the cluster
    sizes switch back; the autotuner picks one of the forms and still solves."""
    s = pkg.Solver(3, 3, 32, k=10)
    assert pkg.igamg_get_schedule(s.ctx)["tail_ctas"] == 16
    pkg.igamg_set_tail_ctas(s.ctx, 1)
    assert pkg.igamg_coarse_tail_level(s.ctx) == 0
    pkg.igamg_set_tail_ctas(s.ctx, 8)
    assert pkg.igamg_coarse_tail_level(s.ctx) == pkg.igamg_tail_levels_available(s.ctx, 8) >= 1
    sch = s.autotune(reps=2)
    assert sch["tail_ctas"] in (1, 8, 16)
    b = s.rhs_sine(workloads.random_sine_coeffs(3, seed=9, modes=6))
    out = s.solve(b, tol=1e-10, method="rre", k=10, prec="fp32_ir", max_cycles=60)
    assert out["converged"]
    s.close()


def test_cluster_tail3_depth_at_128(pkg):
    """128^3, p = 3 (levels 9^3 .. 129^3 nodes per direction): 16 CTAs hold
    the levels up to 33^3; the default schedule uses them."""
    ctx = pkg.igamg_setup(3, 3, [128, 128, 128], 0)
    pkg.igamg_assemble(ctx)
    assert pkg.igamg_tail_levels_available(ctx, 16) == 2
    assert pkg.igamg_coarse_tail_level(ctx) == 2
    pkg.igamg_destroy(ctx)


@pytest.mark.parametrize("n,p,k", [(48, 3, 10), (40, 2, 5)])
def test_cluster_tail3_solves_like_per_level_schedule(pkg, n, p, k):
    s = pkg.Solver(3, p, n, k=k)
    b = s.rhs_sine(workloads.random_sine_coeffs(3, seed=p, modes=8))
    pkg.igamg_set_coarse_tail(s.ctx, False)
    ref32 = s.solve(b, tol=1e-10, method="rre", k=k, prec="fp32_ir", max_cycles=60)
    assert ref32["converged"]
    pkg.igamg_set_coarse_tail(s.ctx, True)
    assert pkg.igamg_coarse_tail_level(s.ctx) >= 1
    out = s.solve(b, tol=1e-10, method="rre", k=k, prec="fp32_ir", max_cycles=60)
    assert out["converged"]
    assert abs(out["cycles"] - ref32["cycles"]) <= 1
    ref = s.solve(b, tol=1e-12, method="rre", k=k, prec="fp64", max_cycles=60)["x"]
    assert float((out["x"] - ref).norm() / ref.norm()) < 1e-7
    s.close()
