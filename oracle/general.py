"""General second-order operator on a 2D (possibly mapped) B-spline domain (oracle).

Test infrastructure only.  Sec. 4.3, Eq. (fullelliptic):

    -div(A grad u) + B . grad u + c u = f  in Omega,   u = 0 on the boundary,

with A(x) SPD, B a vector field and c >= 0.  The Galerkin form on the
tensor-product B-spline space (homogeneous Dirichlet data removes the first
and last function per direction, as for the Poisson problem) is

    a(u, v) = int grad v . A grad u + (B . grad u) v + c u v,   l(v) = int f v.

Omega is the image of the unit square under a map F(xi, eta); with J = DF,
the substitution x = F(xi) turns every integral into one over the unit square
with the transformed coefficients

    A^ = |J| J^{-1} A J^{-T},   B^ = |J| J^{-1} B,   c^ = |J| c,   f^ = |J| f,

evaluated at the mapped points (J^{-T} grad^ = grad).  The unit square itself is
F = identity.  Quadrature: p+1 Gauss points per element and direction, the
rule of the Poisson path.

The map F is given as a function of the parameter point returning the
physical point and J (the quarter annulus of Sec. 4.3 uses its polar map).

Coarse operators: the Galerkin product A_{2h} = P^T A_h P of Eq. (4) with the
oracle's L2-projection P (the coefficients vary, so re-discretisation is no
longer the same operator).  The smoothers and the mu-cycle are those of
multigrid.py; the coarsest solve is a dense LU solve (A is not symmetric).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .bspline import basis, basis_derivative, coarsen_breaks, element_quadrature, open_knot_vector, uniform_breaks
from .galerkin import kron_list, n_interior, prolongation_1d


def quadrature_1d(breaks, p):
    """Gauss points, weights, interior basis values and derivatives (p+1 points per element)."""
    knots = open_knot_vector(breaks, p)
    x, w = element_quadrature(breaks, p + 1)
    return x, w, basis(knots, p, x)[:, 1:-1], basis_derivative(knots, p, x)[:, 1:-1]


def parametric_points(breaks_x, breaks_y, p):
    """The tensor quadrature points (xi, eta), weights w (x fastest, flat)."""
    xq, wx, _, _ = quadrature_1d(breaks_x, p)
    yq, wy, _, _ = quadrature_1d(breaks_y, p)
    XI, ETA = np.meshgrid(xq, yq)                     # [eta][xi]
    return XI.ravel(), ETA.ravel(), np.outer(wy, wx).ravel()


def geometry_at_points(breaks_x, breaks_y, p, geometry):
    """Physical points and Jacobian J = DF at the quadrature points of the unit
    square for the map geometry(xi, eta) -> (x, y, J) (J: nq x 2 x 2,
    J[q, a, b] = d F_a / d xi_b); geometry = None is the identity."""
    xi, eta, _ = parametric_points(breaks_x, breaks_y, p)
    if geometry is None:
        J = np.zeros((xi.size, 2, 2))
        J[:, 0, 0] = J[:, 1, 1] = 1.0
        return xi, eta, J
    return geometry(xi, eta)


def transformed_coefficients(J, A, B, c):
    """A^ = |J| J^{-1} A J^{-T}, B^ = |J| J^{-1} B, c^ = |J| c at every point
    (A: nq x 2 x 2, B: nq x 2, c: nq).  Returns (A^, B^, c^, |J|)."""
    det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    Ji = np.linalg.inv(J)
    Ah = det[:, None, None] * np.einsum("qab,qbc,qdc->qad", Ji, A, Ji)
    Bh = det[:, None] * np.einsum("qab,qb->qa", Ji, B)
    return Ah, Bh, det * c, det


def assemble(breaks_x, breaks_y, p, Ah, Bh, ch):
    """Galerkin matrix of a(u, v) on the unit square with the (transformed)
    coefficients at the quadrature points: for basis functions phi_I (rows,
    test) and phi_J (columns, trial),
        A_IJ = sum_q w_q [ grad phi_I . Ah grad phi_J + (Bh . grad phi_J) phi_I + ch phi_I phi_J ].
    The 2D values and derivatives at the points are Kronecker products of the
    1D ones (x fastest)."""
    _, wx, Bx, Dx = quadrature_1d(breaks_x, p)
    _, wy, By, Dy = quadrature_1d(breaks_y, p)
    w = np.outer(wy, wx).ravel()
    V = sp.csr_matrix(sp.kron(sp.csr_matrix(By), sp.csr_matrix(Bx)))                # phi at points
    GX = sp.csr_matrix(sp.kron(sp.csr_matrix(By), sp.csr_matrix(Dx)))               # d phi / d xi
    GY = sp.csr_matrix(sp.kron(sp.csr_matrix(Dy), sp.csr_matrix(Bx)))               # d phi / d eta
    G = [GX, GY]

    def wdiag(v):
        return sp.diags(w * v)

    A = None
    for a in range(2):
        for b in range(2):
            term = G[a].T @ wdiag(Ah[:, a, b]) @ G[b]
            A = term if A is None else A + term
    for b in range(2):
        A = A + V.T @ wdiag(Bh[:, b]) @ G[b]
    A = A + V.T @ wdiag(ch) @ V
    A = sp.csr_matrix(A)
    A.eliminate_zeros()
    A.sort_indices()
    return A


def load_vector(breaks_x, breaks_y, p, fh):
    """l_I = sum_q w_q fh_q phi_I(q)."""
    _, wx, Bx, _ = quadrature_1d(breaks_x, p)
    _, wy, By, _ = quadrature_1d(breaks_y, p)
    w = np.outer(wy, wx).ravel()
    return sp.csr_matrix(sp.kron(sp.csr_matrix(By), sp.csr_matrix(Bx))).T @ (w * fh)


class GeneralLevel:
    """One grid of the hierarchy with an assembled (possibly non-symmetric)
    operator, with the attributes the smoothers of multigrid.py use."""

    def __init__(self, A, m, p):
        self.p = p
        self.dim = 2
        self.m = list(m)
        self.N = int(np.prod(m))
        self.A = sp.csr_matrix(A)
        self.diag = self.A.diagonal().copy()
        idx = np.indices(self.m[::-1]).reshape(2, -1)
        colour = (idx[1] % (p + 1)) + (p + 1) * (idx[0] % (p + 1))
        self.n_colours = (p + 1) ** 2
        self.colour_rows = [np.flatnonzero(colour == c) for c in range(self.n_colours)]
        self.colour_A = [self.A[rows] for rows in self.colour_rows]


class GeneralHierarchy:
    """Levels 0 (coarsest) .. L-1 (finest): the finest operator assembled by
    quadrature, coarse ones by the Galerkin product P^T A P (Eq. (4))."""

    def __init__(self, n, p, A_fine, coarsest=8, n_levels=None):
        ns = list(n) if np.ndim(n) else [int(n)] * 2
        chain = [[uniform_breaks(k) for k in ns]]
        if n_levels is None:
            while max(len(b) - 1 for b in chain[-1]) > coarsest:
                chain.append([coarsen_breaks(b) for b in chain[-1]])
        else:
            for _ in range(n_levels - 1):
                chain.append([coarsen_breaks(b) for b in chain[-1]])
        chain = chain[::-1]
        self.p, self.dim = p, 2
        self.P = [None]
        for l in range(1, len(chain)):
            P1 = [prolongation_1d(chain[l][d], chain[l - 1][d], p)[1] for d in range(2)]
            self.P.append(sp.csr_matrix(kron_list(P1)))
        ops = [sp.csr_matrix(A_fine)]
        for l in range(len(chain) - 1, 0, -1):
            ops.append(sp.csr_matrix(self.P[l].T @ ops[-1] @ self.P[l]))
        ops = ops[::-1]
        self.levels = [GeneralLevel(ops[l], [n_interior(b, p) for b in chain[l]], p) for l in range(len(chain))]
        self.coarse_lu = sla.lu_factor(self.levels[0].A.toarray())

    @property
    def finest(self):
        return self.levels[-1]

    def solve_coarsest(self, b):
        return sla.lu_solve(self.coarse_lu, b)


class GeneralProblem:
    """Hierarchy + load vector of one problem: coefficient functions of the
    physical point, A(x, y) -> (nq, 2, 2), B(x, y) -> (nq, 2), c(x, y), f(x, y),
    on the unit square or the image of geometry(xi, eta) -> (x, y, J)."""

    def __init__(self, n, p, A, B, c, f, geometry=None, coarsest=8):
        ns = list(n) if np.ndim(n) else [int(n)] * 2
        bx, by = uniform_breaks(ns[0]), uniform_breaks(ns[1])
        x, y, J = geometry_at_points(bx, by, p, geometry)
        self.x, self.y, self.J = x, y, J
        Ah, Bh, ch, det = transformed_coefficients(J, A(x, y), B(x, y), c(x, y))
        self.det = det
        self.A_fine = assemble(bx, by, p, Ah, Bh, ch)
        self.b = load_vector(bx, by, p, det * f(x, y))
        self.bnorm = float(np.linalg.norm(self.b))
        self.H = GeneralHierarchy(ns, p, self.A_fine, coarsest=coarsest)
        self.breaks = (bx, by)

    def residual(self, x):
        return float(np.linalg.norm(self.b - self.A_fine @ x))


def solution_at_points(breaks_x, breaks_y, p, u_h):
    """u_h (interior coefficients, x fastest) at the quadrature points."""
    _, _, Bx, _ = quadrature_1d(breaks_x, p)
    _, _, By, _ = quadrature_1d(breaks_y, p)
    U = np.asarray(u_h).reshape(By.shape[1], Bx.shape[1])
    return (By @ U @ Bx.T).ravel()
