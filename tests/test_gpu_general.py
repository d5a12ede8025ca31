"""GPU parity of the general operator of Sec. 4.3 (variable-coefficient full
elliptic problem, advection-diffusion, the quarter annulus) against the
oracle (oracle/general.py), through the C ABI.

Each side evaluates the problem's functions at its own quadrature points
(the library returns its points; the oracle builds its own), assembles its own
operator (the library's stencil in C++, the oracle's sparse products) and its
own coarse operators (Galerkin with the knot-insertion P on the GPU side, with
the L2-projection P in the oracle).  Tolerances: operator, load vector,
sweeps and one cycle to round-off (1e-12 relative, 2-norm and max-norm);
whole RRE/MPE solves: stopping cycle within +-1 and, at the oracle's count,
solutions within 1e-9; the annulus solution's L2 error against the exact
solution as the oracle's.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from oracle import extrapolation as oex  # noqa: E402
from oracle import general as og  # noqa: E402
from oracle import multigrid as omg  # noqa: E402

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


def _close(a, b, tol, what=""):
    r2 = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    rm = np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)
    assert r2 < tol and rm < tol, f"{what}: rel 2-norm {r2:.2e}, rel max {rm:.2e} (tol {tol:g})"


def _pair(pkg, name, n, p, k=8):
    pr = workloads.GENERAL_PROBLEMS[name]()
    prob = og.GeneralProblem(n, p, pr["A"], pr["B"], pr["c"], pr["f"], geometry=pr["geometry"])
    s = pkg.GeneralSolver(p, n, pr["A"], pr["B"], pr["c"], geometry=pr["geometry"], k=k)
    return pr, prob, s


CASES = [("full_elliptic", 17, 2), ("full_elliptic", (20, 13), 3), ("advection_diffusion", 24, 1),
         ("advection_diffusion", 19, 4), ("annulus", 16, 3), ("annulus", 12, 5)]


@pytest.mark.parametrize("name,n,p", CASES)
def test_operator_load_vector_sweeps_and_cycle(pkg, name, n, p):
    pr, prob, s = _pair(pkg, name, n, p)
    H = prob.H
    assert [tuple(l.m) + (1,) for l in H.levels] == [tuple(m) for m in s.levels]
    b = s.rhs(pr["f"])
    _close(_np(b), prob.b, 1e-12, "load vector")
    rng = np.random.default_rng(7)
    for l, lev in enumerate(H.levels):
        x = rng.standard_normal(lev.N)
        y = torch.empty(lev.N, dtype=torch.float64, device=DEV)
        pkg.igamg_apply(s.ctx, l, _t(x), y, s.ws)
        # coarse operators: Galerkin with two exact forms of P (knot insertion,
        # L2 projection accurate to about cond(M_f) eps)
        _close(_np(y), lev.A @ x, 1e-12 if l == len(H.levels) - 1 else 1e-11, f"apply level {l}")
        bl = rng.standard_normal(lev.N)
        for desc in (0, 1):
            xs = _t(x)
            pkg.igamg_smooth(s.ctx, l, xs, _t(bl), desc, s.ws)
            _close(_np(xs), omg.gs_sweep(lev, x, bl, descending=bool(desc)), 1e-11, f"sweep level {l} desc={desc}")
    x0 = rng.standard_normal(H.finest.N) * 1e-2
    for smoother, mu in (("gs", 1), ("jacobi", 1), ("gs", 2)):
        pkg.igamg_set_cycle(s.ctx, smoother, mu)
        x = _t(x0)
        pkg.igamg_vcycle(s.ctx, x, _t(prob.b), pkg.IGAMG_FP64, s.ws)
        ref = omg.cycle(H, x0, prob.b, smoother=smoother, mu=mu)
        _close(_np(x), ref, 1e-10, f"cycle {smoother} mu={mu}")
    pkg.igamg_set_cycle(s.ctx, "gs", 1)
    s.close()


SOLVES = [("full_elliptic", 32, 2, "rre"), ("full_elliptic", 64, 4, "rre"), ("advection_diffusion", 64, 3, "rre"),
          ("advection_diffusion", 32, 2, "mpe"), ("annulus", 32, 3, "rre"), ("annulus", 16, 5, "rre")]


@pytest.mark.parametrize("name,n,p,method", SOLVES)
def test_solve_matches_oracle(pkg, name, n, p, method):
    """Restarted RRE(8)/MPE(8) with the paper's absolute test 1e-12 (Sec. 4.3)."""
    k = 8
    pr, prob, s = _pair(pkg, name, n, p, k=k)
    G = lambda x: omg.cycle(prob.H, x, prob.b)
    ref = oex.restarted(G, prob.residual, np.zeros(prob.H.finest.N), k, method, tol=1e-12, max_cycles=80,
                        keep_iterates=True)
    assert ref["converged"]
    b = s.rhs(pr["f"])
    out = s.solve(b, tol=1e-12, method=method, k=k, prec="fp64", max_cycles=80, absolute=True)
    assert out["converged"]
    assert abs(out["cycles"] - ref["cycles"]) <= 1, (out["cycles"], ref["cycles"])
    c = min(out["cycles"], ref["cycles"])
    out_c = s.solve(b, tol=0.0, method=method, k=k, prec="fp64", max_cycles=c, absolute=True)
    _close(_np(out_c["x"]), ref["iterates"][c - 1], 1e-9, f"solution after {c} cycles")
    if name == "annulus":
        bx, by = prob.breaks
        _, _, w = og.parametric_points(bx, by, p)

        def err(uh):
            vals = og.solution_at_points(bx, by, p, uh)
            ue = pr["solution"](prob.x, prob.y)
            return np.sqrt(np.sum(w * prob.det * (vals - ue) ** 2) / np.sum(w * prob.det * ue ** 2))
        e_gpu, e_ref = err(_np(out["x"])), err(ref["x"])
        assert abs(e_gpu - e_ref) <= 1e-3 * e_ref, (e_gpu, e_ref)
    s.close()


def test_general_context_rejects_poisson_only_calls(pkg):
    pr = workloads.full_elliptic_square()
    s = pkg.GeneralSolver(2, 16, pr["A"], pr["B"], pr["c"])
    b = torch.empty(s.N, dtype=torch.float64, device=DEV)
    with pytest.raises(pkg.IgamgError):
        pkg.igamg_rhs_sine(s.ctx, np.ones((2, 2)), b)
    bb = s.rhs(pr["f"])
    with pytest.raises(pkg.IgamgError):
        s.solve(bb, prec="fp32_ir")
    with pytest.raises(pkg.IgamgError):
        pkg.igamg_autotune(s.ctx, s.ws)
    out = s.solve(bb, tol=1e-12, method="rre", k=8, prec="fp64", absolute=True)
    assert out["converged"]
    s.close()
