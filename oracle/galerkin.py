"""Galerkin discretisation of -Laplace(u) = f with homogeneous Dirichlet data (oracle).

Test infrastructure only.  Sec. 2, Eq. (1)-(2): the IGA discretisation of the
model problem on the unit square (cube) yields the SPD system A^h u^h = b^h.
On a tensor-product B-spline space the Galerkin stiffness matrix of the
Laplacian is the Kronecker sum
    A = sum_d  K_d (x) prod_{e != d} M_e ,
with the 1D Galerkin mass M_ij = int N_i N_j and stiffness K_ij = int N_i' N_j'.
Homogeneous Dirichlet data removes the first and last B-spline of every open
knot vector (the only ones non-zero on the boundary), leaving m = n + p - 2
unknowns per direction.  Grid vectors are stored C-order with x fastest:
index = i_0 + m_0 (i_1 + m_1 i_2).

Quadrature: p+1 Gauss points per element and direction (exact for M and K,
whose integrands have degree <= 2p on every element).

Prolongation P_{2h}^h (Sec. 2) is the exact representation of the coarse
B-splines in the fine basis; here it is obtained by L2 projection onto the fine
space, P = M_f^{-1} int N^f N^c, which is exact because the spaces are nested.
"""
import itertools

import numpy as np
import scipy.sparse as sp

from .bspline import (basis, basis_derivative, element_quadrature, gauss_legendre,
                      open_knot_vector)


def n_interior(breaks, p):
    """Interior unknowns per direction: (n + p) basis functions minus the two end ones."""
    return len(breaks) - 1 + p - 2


def factors_1d(breaks, p):
    """Interior 1D Galerkin mass M and stiffness K (dense m x m) on the open
    knot vector over ``breaks``, by (p+1)-point Gauss quadrature per element."""
    knots = open_knot_vector(breaks, p)
    pts, wts = element_quadrature(breaks, p + 1)
    B = basis(knots, p, pts)
    D = basis_derivative(knots, p, pts)
    M = B.T @ (wts[:, None] * B)
    K = D.T @ (wts[:, None] * D)
    return M[1:-1, 1:-1].copy(), K[1:-1, 1:-1].copy()


def kron_list(mats):
    """Kronecker product with the LAST list entry varying fastest, i.e.
    kron_list([F_0, F_1, F_2]) = F_2 (x) F_1 (x) F_0 for x-fastest ordering."""
    out = sp.csr_matrix(mats[0])
    for F in mats[1:]:
        out = sp.kron(sp.csr_matrix(F), out, format="csr")
    return out


def operator(factors):
    """A = sum_d K_d (x) prod_{e!=d} M_e for factors = [(M_0, K_0), ..., ] where
    direction 0 is x (fastest).  Returns a scipy CSR matrix."""
    dim = len(factors)
    A = None
    for d in range(dim):
        mats = [factors[e][1] if e == d else factors[e][0] for e in range(dim)]
        term = kron_list(mats)
        A = term if A is None else A + term
    A = sp.csr_matrix(A)
    A.eliminate_zeros()
    A.sort_indices()
    return A


def assemble_direct(breaks_list, p):
    """Dense A assembled directly by dim-D Gauss quadrature of grad(phi_I).grad(phi_J)
    over every element, with phi_I the tensor-product B-spline (brute force; only
    for tiny grids).  Independent of the Kronecker form above."""
    dim = len(breaks_list)
    knots = [open_knot_vector(b, p) for b in breaks_list]
    m = [n_interior(b, p) for b in breaks_list]
    Ntot = int(np.prod(m))
    A = np.zeros((Ntot, Ntot))
    xg, wg = gauss_legendre(p + 1)
    elems = [range(len(b) - 1) for b in breaks_list]
    for el in itertools.product(*elems):
        for q in itertools.product(range(p + 1), repeat=dim):
            pt, w = [], 1.0
            for d in range(dim):
                a, b = breaks_list[d][el[d]], breaks_list[d][el[d] + 1]
                pt.append(a + 0.5 * (xg[q[d]] + 1.0) * (b - a))
                w *= 0.5 * wg[q[d]] * (b - a)
            val = [basis(knots[d], p, [pt[d]])[0, 1:-1] for d in range(dim)]
            der = [basis_derivative(knots[d], p, [pt[d]])[0, 1:-1] for d in range(dim)]
            for d in range(dim):
                # gradient component d of every tensor-product function, x fastest
                g = np.ones(1)
                for e in range(dim):
                    g = np.multiply.outer(der[e] if e == d else val[e], g).ravel()
                A += w * np.outer(g, g)
    return A


def sine_series_on_grid(coeffs, points):
    """Evaluate f = sum_k c[k_{D-1},...,k_0] prod_d sin((k_d+1) pi x_d) on the
    tensor grid points[0] x ... (returned with x fastest, shape (n_{D-1},...,n_0))."""
    c = np.asarray(coeffs, dtype=np.float64)
    dim = c.ndim
    F = c
    for d in range(dim):
        axis = dim - 1 - d                     # array axis of direction d
        k = np.arange(1, c.shape[axis] + 1)
        S = np.sin(np.pi * np.outer(k, points[d]))          # (K, n_d)
        F = np.moveaxis(np.tensordot(F, S, axes=([axis], [0])), -1, axis)
    return F


def load_vector(breaks_list, p, coeffs):
    """b_I = int f phi_I with (p+1)^dim Gauss points per element, f a sine
    series.  f is evaluated at every tensor quadrature point, then the weighted
    sum over points is taken axis by axis.  Returns a flat x-fastest vector."""
    dim = len(breaks_list)
    pts, wts, Bs = [], [], []
    for d in range(dim):
        knots = open_knot_vector(breaks_list[d], p)
        x, w = element_quadrature(breaks_list[d], p + 1)
        pts.append(x)
        wts.append(w)
        Bs.append(basis(knots, p, x)[:, 1:-1])
    F = sine_series_on_grid(coeffs, pts)
    for d in range(dim):
        axis = dim - 1 - d
        W = wts[d][:, None] * Bs[d]                      # (n_pts, m_d)
        F = np.moveaxis(np.tensordot(F, W, axes=([axis], [0])), -1, axis)
    return F.ravel()


def poisson_solution_coeffs(coeffs_f):
    """For -Laplace(u) = sum c_k prod sin((k_d+1) pi x_d) with zero Dirichlet data
    the exact solution is the sine series with c_k / (pi^2 sum_d (k_d+1)^2)."""
    c = np.asarray(coeffs_f, dtype=np.float64)
    grids = np.meshgrid(*[np.arange(1, s + 1) for s in c.shape], indexing="ij")
    lam = np.pi ** 2 * sum(g.astype(np.float64) ** 2 for g in grids)
    return c / lam


def l2_error(breaks_list, p, u_h, coeffs_u, extra=2):
    """Continuous ||u - u_h||_{L2(Omega)} with (p+1+extra) Gauss points per
    element and direction; u is the sine series with coefficients coeffs_u."""
    dim = len(breaks_list)
    m = [n_interior(b, p) for b in breaks_list]
    U = np.asarray(u_h, dtype=np.float64).reshape(m[::-1])
    pts, wts = [], []
    for d in range(dim):
        knots = open_knot_vector(breaks_list[d], p)
        x, w = element_quadrature(breaks_list[d], p + 1 + extra)
        pts.append(x)
        wts.append(w)
        B = basis(knots, p, x)[:, 1:-1]                  # (n_pts, m_d)
        axis = dim - 1 - d
        U = np.moveaxis(np.tensordot(U, B, axes=([axis], [1])), -1, axis)
    E = U - sine_series_on_grid(coeffs_u, pts)
    s = E * E
    for d in range(dim):          # the last array axis is always the next direction
        s = s @ wts[d]
    return float(np.sqrt(s))


def prolongation_1d(breaks_fine, breaks_coarse, p):
    """Interior prolongation P (m_f x m_c): coarse B-splines written in the fine
    basis, by L2 projection P = M_f^{-1} G with G_iJ = int N^f_i N^c_J over the
    full bases, then restricted to interior rows and columns (coarse interior
    functions vanish at both ends, so their end coefficients are zero)."""
    kf = open_knot_vector(breaks_fine, p)
    kc = open_knot_vector(breaks_coarse, p)
    pts, wts = element_quadrature(breaks_fine, p + 1)
    Bf = basis(kf, p, pts)
    Bc = basis(kc, p, pts)
    Mf = Bf.T @ (wts[:, None] * Bf)
    G = Bf.T @ (wts[:, None] * Bc)
    P = np.linalg.solve(Mf, G)
    # Compact support (Prop. 3): coarse function J is a combination of the fine
    # functions overlapping its support only; entries elsewhere are exact zeros
    # that the dense solve returns as rounding noise.
    P[np.abs(P) < 1e-13 * np.abs(P).max()] = 0.0
    return P, P[1:-1, 1:-1].copy()
