"""GPU parity at the sizes the product runs at, through the C ABI.

The parity cases in test_gpu_parity.py stay small (rows of <= 65 nodes); the
row kernels take a different path once a row is longer than a CTA's threads
and its shared-memory rows exceed 48 KiB.  These tests run that path:

* the FP64 operator, one FP64 Gauss-Seidel sweep and one FP32 sweep on the
  1024^2 (p = 3) finest level against the oracle, element by element;
* whole FP64 solves against the oracle: 2D 1024^2 with p = 3 and p = 5,
  RRE(5), the benchmark's right-hand side (random 16-mode sine series, seed
  0), 1024^2 with p = 2, MPE(10), manufactured right side, and 3D 48^3,
  p = 3, RRE(10): stopping count within +-1 and, at the oracle's count,
  solutions equal to 1e-9 (relative 2-norm and max-norm);
* the mixed form (FP32 V-cycles inside FP64 refinement) at 1024^2: it reaches
  the oracle's residual test and its distance from the oracle's solution is
  stated;
* 3D 128^3, p = 3, RRE(10) (too large for the oracle's sparse operator, 343
  non-zeros per row): the GPU solution, FP64 and mixed, passes the residual
  test with A applied as the Kronecker sum of the oracle's 1D factors and b
  from the oracle's quadrature.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import bspline as obs  # noqa: E402
from oracle import galerkin as ogk  # noqa: E402
from oracle import multigrid as omg  # noqa: E402
from oracle import solver as osolver  # noqa: E402
import workloads  # noqa: E402

DEV = "cuda"


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build_library()
    import paper_2412_20205_gb300 as p
    assert torch.cuda.is_available()
    return p


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _np(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _assert_close(a, b, tol, what):
    r2, rm = _rel(a, b), _relmax(a, b)
    assert r2 < tol and rm < tol, f"{what}: rel 2-norm {r2:.2e}, rel max {rm:.2e} (tol {tol:g})"


@pytest.fixture(scope="module")
def big2d(pkg):
    """1024^2, p = 3: the oracle's finest level and a GPU context."""
    H = omg.Hierarchy(2, 1024, 3)
    ctx = pkg.igamg_setup(2, 3, [1024, 1024], 0)
    pkg.igamg_assemble(ctx)
    nb = max(pkg.igamg_workspace_bytes(ctx, 5, v) for v in (pkg.IGAMG_FP64, pkg.IGAMG_FP32_IR))
    ws = torch.empty(nb, dtype=torch.uint8, device=DEV)
    yield H, ctx, ws
    pkg.igamg_destroy(ctx)


def test_apply_and_sweeps_1024(pkg, big2d):
    H, ctx, ws = big2d
    lev = H.finest
    top = len(H.levels) - 1
    rng = np.random.default_rng(21)
    x0, b = rng.standard_normal(lev.N), rng.standard_normal(lev.N)
    y = torch.empty(lev.N, dtype=torch.float64, device=DEV)
    pkg.igamg_apply(ctx, top, _t(x0), y, ws)
    _assert_close(_np(y), lev.A @ x0, 1e-13, "apply")
    for desc in (0, 1):
        x = _t(x0)
        pkg.igamg_smooth(ctx, top, x, _t(b), desc, ws)
        _assert_close(_np(x), omg.gs_sweep(lev, x0, b, descending=bool(desc)), 1e-12, f"FP64 sweep desc={desc}")
    ref = omg.gs_sweep(lev, omg.gs_sweep(lev, x0, b), b, descending=True)
    xf, bf = _t(x0, torch.float32), _t(b, torch.float32)
    pkg.igamg_smooth_f32(ctx, top, xf, bf, 0, ws)
    pkg.igamg_smooth_f32(ctx, top, xf, bf, 1, ws, sums_current=True)
    _assert_close(_np(xf), ref, 2e-5, "FP32 sweeps")


def _fp64_vs_oracle(pkg, dim, n, p, k, coeffs, max_cycles=60, method="rre"):
    prob = osolver.Problem(dim, n, p, coeffs)
    ref = osolver.solve(prob, method, k=k, tol=1e-10, max_cycles=max_cycles, keep_iterates=True)
    assert ref["converged"]
    s = pkg.Solver(dim, p, n, k=k)
    b = s.rhs_sine(coeffs)
    _assert_close(_np(b), prob.b, 1e-13, "load vector")
    out = s.solve(b, tol=1e-10, method=method, k=k, prec="fp64", max_cycles=max_cycles)
    assert out["converged"]
    assert abs(out["cycles"] - ref["cycles"]) <= 1, (out["cycles"], ref["cycles"])
    c = min(out["cycles"], ref["cycles"])
    out_c = s.solve(b, tol=0.0, method=method, k=k, prec="fp64", max_cycles=c)
    assert out_c["cycles"] == c
    _assert_close(_np(out_c["x"]), ref["iterates"][c - 1], 1e-9, f"FP64 solve after {c} cycles")
    return prob, ref, s, b


@pytest.mark.parametrize("p", [3, 5])
def test_fp64_solve_1024_matches_oracle(pkg, p):
    coeffs = workloads.random_sine_coeffs(2, seed=0, modes=16)
    prob, ref, s, b = _fp64_vs_oracle(pkg, 2, 1024, p, 5, coeffs)
    # the mixed form on the same problem: the oracle's residual test, and its
    # distance from the oracle's converged solution (both have relative
    # residual <= 1e-10; the solutions differ by at most cond(A) times that)
    out = s.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir", max_cycles=60)
    assert out["converged"]
    x = _np(out["x"])
    res = np.linalg.norm(prob.b - prob.H.finest.A @ x) / prob.bnorm
    assert res <= 1.05e-10, res
    d2, dm = _rel(x, ref["x"]), _relmax(x, ref["x"])
    print(f"p={p}: mixed form vs oracle solution: rel 2-norm {d2:.2e}, rel max {dm:.2e}")
    assert d2 < 1e-7 and dm < 1e-7
    s.close()


def test_fp64_mpe10_1024_matches_oracle(pkg):
    """MPE with restart number 10 at 1024^2, p = 2 (the other extrapolation and
    cycle length of the 1024^2 configuration), manufactured right-hand side."""
    _, _, s, _ = _fp64_vs_oracle(pkg, 2, 1024, 2, 10, workloads.manufactured_coeffs(2), method="mpe")
    s.close()


def test_fp64_solve_3d_48_matches_oracle(pkg):
    coeffs = workloads.random_sine_coeffs(3, seed=0, modes=8)
    _, _, s, _ = _fp64_vs_oracle(pkg, 3, 48, 3, 10, coeffs)
    s.close()


def _kron_apply_3d(F, x):
    """A x with A = K_z (x) M_y (x) M_x + M_z (x) K_y (x) M_x + M_z (x) M_y (x) K_x
    applied axis by axis from the dense 1D factors F = (M, K) (x fastest)."""
    M, K = F
    m = M.shape[0]
    X = x.reshape(m, m, m)                       # [z][y][x]

    def ax(A, X, axis):
        return np.moveaxis(np.tensordot(A, X, axes=([1], [axis])), 0, axis)

    MxX, KxX = ax(M, X, 2), ax(K, X, 2)
    MyMx = ax(M, MxX, 1)
    Y = ax(K, MyMx, 0) + ax(M, ax(K, MxX, 1) + ax(M, KxX, 1), 0)
    return Y.ravel()


def test_c3_128_residual_property(pkg):
    """128^3 elements, p = 3, RRE(10), manufactured f = 3 pi^2 prod sin(pi x_d):
    both GPU forms pass the oracle's residual test at 1e-10."""
    n, p, k = 128, 3, 10
    coeffs = workloads.manufactured_coeffs(3)
    br = obs.uniform_breaks(n)
    F = ogk.factors_1d(br, p)
    bo = ogk.load_vector([br, br, br], p, coeffs)
    s = pkg.Solver(3, p, n, k=k)
    b = s.rhs_sine(coeffs)
    _assert_close(_np(b), bo, 1e-13, "load vector")
    xs = {}
    for prec in ("fp64", "fp32_ir"):
        out = s.solve(b, tol=1e-10, method="rre", k=k, prec=prec, max_cycles=40)
        assert out["converged"], prec
        x = _np(out["x"])
        res = np.linalg.norm(bo - _kron_apply_3d(F, x)) / np.linalg.norm(bo)
        assert res <= 1.05e-10, (prec, res)
        xs[prec] = x
    d = _rel(xs["fp32_ir"], xs["fp64"])
    print(f"128^3: mixed vs FP64 GPU solution rel 2-norm {d:.2e}")
    assert d < 1e-7
    s.close()
