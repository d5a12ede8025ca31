"""Pins of the oracle's discretisation (Sec. 2, Eq. 1-4; Sec. 2.3; Sec. 4)."""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bspline as bs
from oracle import galerkin as gk
from tests.test_oracle_bspline import cardinal_bspline

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return rows


def test_p1_closed_form():
    n = 10
    h = 1.0 / n
    M, K = gk.factors_1d(bs.uniform_breaks(n), 1)
    m = n - 1
    T = np.diag(np.full(m, 2.0)) - np.diag(np.ones(m - 1), 1) - np.diag(np.ones(m - 1), -1)
    assert np.allclose(K, T / h, atol=1e-12)
    S = np.diag(np.full(m, 4.0)) + np.diag(np.ones(m - 1), 1) + np.diag(np.ones(m - 1), -1)
    assert np.allclose(M, S * h / 6, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 7))
def test_interior_rows_are_cardinal_autocorrelations(p):
    """Interior (Toeplitz) rows: M = h B_{2p+1}(p+1+k), K = -(1/h) B''_{2p+1}(p+1+k),
    B'' by the second difference of B_{2p-1} (truncated-power formula)."""
    n = 4 * p + 6
    h = 1.0 / n
    M, K = gk.factors_1d(bs.uniform_breaks(n), p)
    i = 2 * p + 1                                   # an interior row
    k = np.arange(-p, p + 1)
    m_ref = h * cardinal_bspline(2 * p + 1, p + 1 + k)
    b = lambda x: cardinal_bspline(2 * p - 1, x) if p > 1 else np.where(np.isclose(x, 1.0), 1.0, 0.0)
    k_ref = -(b(p + 1 + k) - 2 * b(p + k) + b(p - 1 + k)) / h
    assert np.allclose(M[i, i - p:i + p + 1], m_ref, rtol=1e-12, atol=1e-17)
    assert np.allclose(K[i, i - p:i + p + 1], k_ref, rtol=1e-11, atol=1e-12)


def test_p2_p3_printed_stencils():
    n = 20
    h = 1.0 / n
    M, K = gk.factors_1d(bs.uniform_breaks(n), 2)
    assert np.allclose(M[8, 6:11] * 120 / h, [1, 26, 66, 26, 1], atol=1e-11)
    assert np.allclose(K[8, 6:11] * h, [-1 / 6, -1 / 3, 1, -1 / 3, -1 / 6], atol=1e-12)
    M, K = gk.factors_1d(bs.uniform_breaks(n), 3)
    assert np.allclose(M[9, 6:13] * 5040 / h, [1, 120, 1191, 2416, 1191, 120, 1], atol=1e-9)
    assert np.allclose(K[9, 6:13] * 120 * h, [-1, -24, -15, 80, -15, -24, -1], atol=1e-10)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_full_basis_row_sums(p):
    """Full (boundary-included) K annihilates constants; M row sums = int N_i."""
    br = np.concatenate([[0.0], np.sort(np.random.default_rng(p).uniform(0.1, 0.9, 6)), [1.0]])
    knots = bs.open_knot_vector(br, p)
    pts, wts = bs.element_quadrature(br, p + 1)
    B = bs.basis(knots, p, pts)
    D = bs.basis_derivative(knots, p, pts)
    Mf = B.T @ (wts[:, None] * B)
    Kf = D.T @ (wts[:, None] * D)
    assert np.allclose(Kf.sum(axis=1), 0.0, atol=1e-12)
    integ = (knots[p + 1:] - knots[:-(p + 1)]) / (p + 1)
    assert np.allclose(Mf.sum(axis=1), integ, atol=1e-15)


@pytest.mark.parametrize("dim,n,p", [(2, 3, 1), (2, 4, 2), (2, 3, 3), (2, 5, 2), (3, 3, 1), (3, 3, 2)])
def test_kronecker_form_equals_direct_assembly(dim, n, p):
    rng = np.random.default_rng(dim * 10 + n + p)
    brs = []
    for d in range(dim):
        nd = n + d            # rectangular grids catch axis-order mistakes
        inner = np.sort(rng.uniform(0.1, 0.9, nd - 1))
        brs.append(np.concatenate([[0.0], inner, [1.0]]))
    A = gk.operator([gk.factors_1d(b, p) for b in brs]).toarray()
    Ad = gk.assemble_direct(brs, p)
    assert np.allclose(A, Ad, rtol=0, atol=1e-13 * np.abs(Ad).max())
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0


def test_2d_p1_interior_stencil():
    n = 8
    f = gk.factors_1d(bs.uniform_breaks(n), 1)
    A = gk.operator([f, f]).toarray()
    m = n - 1
    c = 3 * m + 3
    st = A[c].reshape(m, m)[2:5, 2:5]
    assert np.allclose(st * 3, [[-1, -1, -1], [-1, 8, -1], [-1, -1, -1]], atol=1e-12)


def test_load_vector_separable_mode_matches_1d_products():
    """For one sine mode the dim-D quadrature sum factorises into 1D sums."""
    p, brx, bry = 3, bs.uniform_breaks(6), bs.uniform_breaks(9)
    c = np.zeros((3, 2))
    c[2, 1] = 1.7                                  # sin(2 pi x) sin(3 pi y)
    b = gk.load_vector([brx, bry], p, c)
    g = []
    for br, kx in [(brx, 2), (bry, 3)]:
        knots = bs.open_knot_vector(br, p)
        x, w = bs.element_quadrature(br, p + 1)
        g.append((w * np.sin(kx * np.pi * x)) @ bs.basis(knots, p, x)[:, 1:-1])
    assert np.allclose(b, 1.7 * np.outer(g[1], g[0]).ravel(), rtol=1e-13, atol=1e-17)


def test_table1_l2_errors_1d():
    """Paper Table 1: the discrete solution's L2 error, with the norm taken by the
    assembly's own (p+1)-point Gauss rule, matches every printed value >= 1e-12."""
    c = np.zeros(2)
    c[1] = 4 * np.pi ** 2
    cu = gk.poisson_solution_coeffs(c)
    for N, p, ref in _load("table1_l2err.txt"):
        if ref < 1e-12:
            continue
        br = bs.uniform_breaks(int(N))
        M, K = gk.factors_1d(br, int(p))
        u = np.linalg.solve(K, gk.load_vector([br], int(p), c))
        err = gk.l2_error([br], int(p), u, cu, extra=0)
        assert abs(err / ref - 1) < 0.015, (N, p, err, ref)


def test_table11_l2_errors_2d():
    c = np.zeros((2, 2))
    c[1, 1] = 8 * np.pi ** 2
    cu = gk.poisson_solution_coeffs(c)
    br = bs.uniform_breaks(64)
    for p, ref in _load("table11_l2err.txt"):
        p = int(p)
        f = gk.factors_1d(br, p)
        A = gk.operator([f, f]).tocsc()
        u = spla.spsolve(A, gk.load_vector([br, br], p, c))
        err = gk.l2_error([br, br], p, u, cu, extra=0)
        assert abs(err / ref - 1) < 0.01, (p, err, ref)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_l2_convergence_order_manufactured(p):
    """||u - u_h|| = O(h^{p+1}) for u = sin(pi x) sin(pi y) (accurate error rule)."""
    c = np.zeros((1, 1))
    c[0, 0] = 2 * np.pi ** 2
    cu = gk.poisson_solution_coeffs(c)
    errs = []
    ns = [8, 16, 32]
    for n in ns:
        br = bs.uniform_breaks(n)
        f = gk.factors_1d(br, p)
        u = spla.spsolve(gk.operator([f, f]).tocsc(), gk.load_vector([br, br], p, c))
        errs.append(gk.l2_error([br, br], p, u, cu, extra=3))
    slope = np.log2(errs[-2] / errs[-1])
    assert abs(slope - (p + 1)) < 0.2, (p, errs, slope)


@pytest.mark.parametrize("p", range(1, 7))
def test_prolongation_knot_insertion_mask_and_partition(p):
    n = 16
    bf = bs.uniform_breaks(n)
    bc = bs.coarsen_breaks(bf)
    Pfull, P = gk.prolongation_1d(bf, bc, p)
    assert np.allclose(Pfull.sum(axis=1), 1.0, atol=1e-13)       # P 1 = 1
    J = Pfull.shape[1] // 2                                       # an interior coarse column
    col = Pfull[:, J]
    nz = np.flatnonzero(np.abs(col) > 1e-12)
    mask = np.array([math.comb(p + 1, j) for j in range(p + 2)]) / 2 ** p
    assert len(nz) == p + 2
    assert np.allclose(col[nz], mask, atol=1e-13)


@pytest.mark.parametrize("n,p", [(16, 2), (9, 3), (13, 1), (10, 5)])
def test_galerkin_identity_and_exact_representation(n, p):
    """P^T K_f P = K_c and P^T M_f P = M_c (Eq. 4 coincides with re-discretisation),
    and the coarse B-splines equal the fine ones combined with P."""
    bf = bs.uniform_breaks(n)
    bc = bs.coarsen_breaks(bf)
    Pfull, P = gk.prolongation_1d(bf, bc, p)
    Mf, Kf = gk.factors_1d(bf, p)
    Mc, Kc = gk.factors_1d(bc, p)
    assert np.allclose(P.T @ Kf @ P, Kc, atol=1e-12 * np.abs(Kc).max())
    assert np.allclose(P.T @ Mf @ P, Mc, atol=1e-13 * np.abs(Mc).max())
    t = np.random.default_rng(n).uniform(0, 1, 200)
    Bf = bs.basis(bs.open_knot_vector(bf, p), p, t)
    Bc = bs.basis(bs.open_knot_vector(bc, p), p, t)
    assert np.allclose(Bf @ Pfull, Bc, atol=1e-13)
    # 2D Galerkin identity
    P2 = gk.kron_list([P, P])
    A_f = gk.operator([(Mf, Kf), (Mf, Kf)])
    A_c = gk.operator([(Mc, Kc), (Mc, Kc)]).toarray()
    assert np.allclose((P2.T @ A_f @ P2).toarray(), A_c, atol=1e-12 * np.abs(A_c).max())
