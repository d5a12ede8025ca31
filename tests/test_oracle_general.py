"""Pins of the oracle's general operator (Sec. 4.3, Eq. fullelliptic; oracle/general.py)
against what the mathematics fixes, independently of the Kronecker Poisson path.

* The Poisson operator is the special case A = I, B = 0, c = 0 on the unit
  square; the mass matrix the case c = 1.
* A constant (divergence-free) advection field gives a skew-symmetric
  advection matrix (integration by parts with zero boundary values).
* Brute force: element-by-element assembly with the basis evaluated point by
  point and J inverted explicitly, on a mapped grid.
* The quarter-annulus map: the quadrature of |J| is the exact area.
* Manufactured solutions converge at O(h^{p+1}) in L2 (unit square with the
  paper's coefficients; the quarter annulus of Table 15).
* The manufactured right-hand side of workloads.py against a symbolic one.
* RRE on the non-symmetric V-cycle-preconditioned system is GMRES, restart by
  restart (Algorithm 5 with s_0 := t).
* Iteration counts of Tables 13-15: loose (factor 2, p <= 4; parity unpinned
  by the paper beyond that).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads
from oracle import extrapolation as ex
from oracle import galerkin as gk
from oracle import general as og
from oracle import krylov
from oracle import multigrid as omg
from oracle.bspline import basis, basis_derivative, element_quadrature, open_knot_vector, uniform_breaks


def _coef(n, p, A=None, B=None, c=None, geometry=None, ns=None):
    ns = ns or (n, n)
    bx, by = uniform_breaks(ns[0]), uniform_breaks(ns[1])
    x, y, J = og.geometry_at_points(bx, by, p, geometry)
    nq = x.size
    Av = A(x, y) if A else np.zeros((nq, 2, 2))
    Bv = B(x, y) if B else np.zeros((nq, 2))
    cv = c(x, y) if c else np.zeros(nq)
    Ah, Bh, ch, det = og.transformed_coefficients(J, Av, Bv, cv)
    return bx, by, Ah, Bh, ch


def _eye(x, y):
    A = np.zeros(x.shape + (2, 2))
    A[..., 0, 0] = A[..., 1, 1] = 1.0
    return A


@pytest.mark.parametrize("n,p", [((7, 5), 2), ((6, 6), 3), ((9, 4), 1)])
def test_poisson_and_mass_are_special_cases(n, p):
    bx, by, Ah, Bh, ch = _coef(None, p, A=_eye, ns=n)
    A = og.assemble(bx, by, p, Ah, Bh, ch)
    ref = gk.operator([gk.factors_1d(bx, p), gk.factors_1d(by, p)])
    assert abs(A - ref).max() < 1e-13 * abs(ref).max()
    bx, by, Ah, Bh, ch = _coef(None, p, c=lambda x, y: np.ones_like(x), ns=n)
    M = og.assemble(bx, by, p, Ah, Bh, ch)
    Mref = gk.kron_list([gk.factors_1d(bx, p)[0], gk.factors_1d(by, p)[0]])
    assert abs(M - Mref).max() < 1e-14 * abs(Mref).max() * 10


@pytest.mark.parametrize("p", [1, 2, 4])
def test_constant_advection_is_skew(p):
    bx, by, Ah, Bh, ch = _coef(8, p, B=lambda x, y: np.stack([np.full_like(x, 1.3), np.full_like(x, -0.7)], -1))
    C = og.assemble(bx, by, p, Ah, Bh, ch)
    assert abs(C + C.T).max() < 1e-14 * abs(C).max() * 10
    assert abs(C).max() > 0.01


def _brute(bx, by, p, prob_fn, geometry):
    """Element by element: at every quadrature point of every element, the
    local basis values and parametric gradients (point-wise Cox-de Boor), the
    physical gradient J^{-T} grad^, weight w |J|, and the integrand summed over
    all pairs of interior functions."""
    kx, ky = open_knot_vector(bx, p), open_knot_vector(by, p)
    mx, my = len(bx) - 1 + p - 2, len(by) - 1 + p - 2
    A = np.zeros((mx * my, mx * my))
    gx, wgx = element_quadrature(bx, p + 1)
    gy, wgy = element_quadrature(by, p + 1)
    for qy, wy in zip(gy, wgy):
        for qx, wx in zip(gx, wgx):
            xi, eta = np.array([qx]), np.array([qy])
            x, y, J = geometry(xi, eta)
            J = J[0]
            Nx = basis(kx, p, [qx])[0, 1:-1]
            Ny = basis(ky, p, [qy])[0, 1:-1]
            dNx = basis_derivative(kx, p, [qx])[0, 1:-1]
            dNy = basis_derivative(ky, p, [qy])[0, 1:-1]
            Ji = np.linalg.inv(J)
            det = abs(np.linalg.det(J))
            Ac, Bc, cc = prob_fn["A"](x, y)[0], prob_fn["B"](x, y)[0], prob_fn["c"](x, y)[0]
            for I in range(mx * my):
                i, j = I % mx, I // mx
                vI = Nx[i] * Ny[j]
                gI = Ji.T @ np.array([dNx[i] * Ny[j], Nx[i] * dNy[j]])
                for K in range(mx * my):
                    a, b = K % mx, K // mx
                    vK = Nx[a] * Ny[b]
                    gK = Ji.T @ np.array([dNx[a] * Ny[b], Nx[a] * dNy[b]])
                    A[I, K] += wx * wy * det * (gI @ Ac @ gK + (Bc @ gK) * vI + cc * vI * vK)
    return A


def test_mapped_assembly_equals_brute_force():
    p = 2
    bx, by = uniform_breaks(3), uniform_breaks(2)
    pr = workloads.full_elliptic_annulus()
    x, y, J = og.geometry_at_points(bx, by, p, pr["geometry"])
    Ah, Bh, ch, det = og.transformed_coefficients(J, pr["A"](x, y), pr["B"](x, y), pr["c"](x, y))
    A = og.assemble(bx, by, p, Ah, Bh, ch).toarray()
    ref = _brute(bx, by, p, pr, pr["geometry"])
    assert np.abs(A - ref).max() < 1e-13 * np.abs(ref).max()


def test_annulus_map_area_and_orientation():
    geom = workloads.annulus_map()
    for n, p in [(4, 2), (16, 3)]:
        bx = uniform_breaks(n)
        xi, eta, w = og.parametric_points(bx, bx, p)
        x, y, J = geom(xi, eta)
        det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
        assert np.all(det > 0)
        assert abs(np.sum(w * det) - np.pi * (1.0 - 0.04) / 4) < 1e-13
        r = np.hypot(x, y)
        assert np.all((r > 0.2) & (r < 1.0) & (x > 0) & (y > 0))


def _l2_rel(prob, p, uh, uex):
    bx, by = prob.breaks
    _, _, w = og.parametric_points(bx, by, p)
    vals = og.solution_at_points(bx, by, p, uh)
    ue = uex(prob.x, prob.y)
    return np.sqrt(np.sum(w * prob.det * (vals - ue) ** 2) / np.sum(w * prob.det * ue ** 2))


def _square_manufactured():
    """u = sin(pi x) sin(pi y) with the Table 13 coefficients (c = 1)."""
    base = workloads.full_elliptic_square()

    def u(x, y):
        return np.sin(np.pi * x) * np.sin(np.pi * y)

    def f(x, y):
        A, div = workloads._A_full(x, y)
        s, c_ = np.sin(np.pi * x), np.cos(np.pi * x)
        t, d = np.sin(np.pi * y), np.cos(np.pi * y)
        gu = np.stack([np.pi * c_ * t, np.pi * s * d], -1)
        H = np.empty(x.shape + (2, 2))
        H[..., 0, 0] = H[..., 1, 1] = -np.pi ** 2 * s * t
        H[..., 0, 1] = H[..., 1, 0] = np.pi ** 2 * c_ * d
        return (-(np.einsum("...ab,...ab->...", A, H) + np.einsum("...a,...a->...", div, gu))
                + np.einsum("...a,...a->...", base["B"](x, y), gu) + u(x, y))
    return dict(base, f=f, solution=u)


@pytest.mark.parametrize("which,p", [("square", 2), ("square", 3), ("annulus", 2), ("annulus", 3)])
def test_manufactured_solutions_converge_at_order_p_plus_1(which, p):
    pr = _square_manufactured() if which == "square" else workloads.full_elliptic_annulus()
    errs = []
    for n in (8, 16, 32):
        prob = og.GeneralProblem(n, p, pr["A"], pr["B"], pr["c"], pr["f"], geometry=pr["geometry"])
        uh = spla.spsolve(prob.A_fine.tocsc(), prob.b)
        errs.append(_l2_rel(prob, p, uh, pr["solution"]))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - (p + 1)) < 0.3), (errs, slopes)


def test_annulus_right_hand_side_matches_symbolic():
    sympy = pytest.importorskip("sympy")
    X, Y = sympy.symbols("x y")
    u = (X ** 2 + Y ** 2 - sympy.Rational(1, 25)) * (X ** 2 + Y ** 2 - 1) * sympy.sin(X) * sympy.sin(Y)
    A = sympy.Matrix([[(2 + sympy.cos(X)) * (1 + Y), sympy.cos(X + Y) * sympy.sin(X + Y)],
                      [sympy.cos(X + Y) * sympy.sin(X + Y), (2 + sympy.sin(Y)) * (1 + X)]])
    grad = sympy.Matrix([sympy.diff(u, X), sympy.diff(u, Y)])
    flux = A * grad
    f = -(sympy.diff(flux[0], X) + sympy.diff(flux[1], Y)) + (-5 * Y) * grad[0] + 5 * X * grad[1] + X * Y * u
    fn = sympy.lambdify((X, Y), f, "numpy")
    rng = np.random.default_rng(0)
    x, y = rng.uniform(0, 1, 50), rng.uniform(0, 1, 50)
    ours = workloads.full_elliptic_annulus()["f"](x, y)
    assert np.allclose(ours, fn(x, y), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("q", [2, 4])
def test_restarted_rre_is_restarted_gmres_on_nonsymmetric_system(q):
    pr = workloads.advection_diffusion()
    prob = og.GeneralProblem(12, 3, pr["A"], pr["B"], pr["c"], pr["f"])
    H, b = prob.H, prob.b
    G = lambda x: omg.cycle(H, x, b)
    N = H.finest.N
    c = G(np.zeros(N))
    F = lambda v: v - (G(v) - c)
    out = ex.restarted(G, prob.residual, np.zeros(N), q, "rre", tol=0.0, max_cycles=3, keep_iterates=True)
    x = np.zeros(N)
    for cyc in range(3):
        x = krylov.gmres(F, c, x, q)
        assert np.linalg.norm(out["iterates"][cyc] - x) < 1e-10 * np.linalg.norm(x), cyc


# Tables 13-15 (RRE(8)-V-cycle, absolute residual 1e-12, zero start): restart counts
PAPER_COUNTS = {
    "full_elliptic": {16: [2, 3, 4, 6, 9], 32: [3, 3, 4, 8, 9]},
    "advection_diffusion": {16: [2, 2, 4, 6], 32: [2, 2, 4, 5]},
    "annulus": {16: [2, 2, 2, 4, 9], 32: [2, 2, 2, 4, 7]},
}


@pytest.mark.parametrize("name", sorted(PAPER_COUNTS))
def test_iteration_counts_near_tables_13_to_15(name):
    """Loose: multicolour Gauss-Seidel V(1,1)-cycles (the build's smoother) on
    the paper's level hierarchy reading (coarsest 8 elements), within a factor
    of two of the printed counts for p <= 4."""
    pr = workloads.GENERAL_PROBLEMS[name]()
    for n, row in PAPER_COUNTS[name].items():
        for p, ref in zip(range(1, 5), row):
            prob = og.GeneralProblem(n, p, pr["A"], pr["B"], pr["c"], pr["f"], geometry=pr["geometry"])
            G = lambda x: omg.cycle(prob.H, x, prob.b)
            out = ex.restarted(G, prob.residual, np.zeros(prob.H.finest.N), 8, "rre", tol=1e-12, max_cycles=60)
            assert out["converged"]
            assert ref / 2 <= out["cycles"] <= 2 * ref, (n, p, out["cycles"], ref)
