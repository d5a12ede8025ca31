"""Geometric multigrid on tensor-product B-spline spaces (oracle; test infrastructure only).

Sec. 2 and Algorithm 2 (mu-cycle; mu = 1 is the V-cycle, mu = 2 the W-cycle):
pre-smooth, residual, restriction R = P^T, zero coarse initial guess, mu
recursive calls, prolongation and correction, post-smooth; a direct solve on
the coarsest grid.  Coarse operators come from re-discretisation on the coarse
knot vector (equal to the Galerkin product R A P of Eq. (4) for nested spaces
with exact quadrature; a test checks this).

Smoothers:
* multicolour Gauss-Seidel: node colour c = sum_d (i_d mod (p+1)) (p+1)^d;
  two nodes of the same colour never couple (the stencil reaches p nodes in
  each direction), so updating one colour at once is exact Gauss-Seidel in
  colour order.  Pre-smoothing visits colours in ascending order and
  post-smoothing in descending order (this makes the cycle symmetric).  The
  paper notes Gauss-Seidel behaves like its Jacobi runs (Sec. 2.4).
* weighted Jacobi with omega = 2/3, the paper's smoother in Sec. 4.

Parity unpinned: nothing in the paper fixes GS-smoothed iteration counts; the
Jacobi-smoothed counts are checked loosely against Tables 4, 11 and the
RRE(8)/MPE(8) tables.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .bspline import coarsen_breaks, uniform_breaks
from .galerkin import factors_1d, kron_list, n_interior, operator, prolongation_1d


class Level:
    """One grid: 1D factors per direction, the operator A, its diagonal and
    the row sets of the multicolour ordering."""

    def __init__(self, breaks_list, p):
        self.p = p
        self.dim = len(breaks_list)
        self.breaks = [np.asarray(b, dtype=np.float64) for b in breaks_list]
        self.m = [n_interior(b, p) for b in self.breaks]
        self.N = int(np.prod(self.m))
        self.factors = [factors_1d(b, p) for b in self.breaks]
        self.A = operator(self.factors)
        self.diag = self.A.diagonal().copy()
        idx = np.indices(self.m[::-1]).reshape(self.dim, -1)   # idx[0] = slowest axis
        colour = np.zeros(self.N, dtype=np.int64)
        for d in range(self.dim):
            colour += (idx[self.dim - 1 - d] % (p + 1)) * (p + 1) ** d
        self.n_colours = (p + 1) ** self.dim
        self.colour_rows = [np.flatnonzero(colour == c) for c in range(self.n_colours)]
        self.colour_A = [self.A[rows] for rows in self.colour_rows]


class Hierarchy:
    """Levels 0 (coarsest) .. L-1 (finest) and prolongations P[l]: level l-1 -> l."""

    def __init__(self, dim, n, p, n_levels=None, coarsest=8):
        ns = list(n) if np.ndim(n) else [int(n)] * dim
        breaks = [uniform_breaks(k) for k in ns]
        chain = [breaks]
        if n_levels is None:
            while max(len(b) - 1 for b in chain[-1]) > coarsest:
                chain.append([coarsen_breaks(b) for b in chain[-1]])
        else:
            for _ in range(n_levels - 1):
                chain.append([coarsen_breaks(b) for b in chain[-1]])
        chain = chain[::-1]
        self.p = p
        self.dim = dim
        self.levels = [Level(b, p) for b in chain]
        self.P = [None]
        for l in range(1, len(self.levels)):
            P1 = [prolongation_1d(chain[l][d], chain[l - 1][d], p)[1] for d in range(dim)]
            self.P.append(kron_list(P1))
        self.coarse_chol = sla.cho_factor(self.levels[0].A.toarray(), lower=True)

    @property
    def finest(self):
        return self.levels[-1]

    def solve_coarsest(self, b):
        """A_0^{-1} b by the Cholesky factor (A_0 is SPD)."""
        return sla.cho_solve(self.coarse_chol, b)


def gs_sweep(level, x, b, descending=False):
    """One multicolour Gauss-Seidel sweep: for each colour c in order,
    x_i += (b_i - (A x)_i) / A_ii for every node i of colour c, all with the
    x values left by the previous colours."""
    order = range(level.n_colours - 1, -1, -1) if descending else range(level.n_colours)
    x = x.copy()
    for c in order:
        rows = level.colour_rows[c]
        x[rows] += (b[rows] - level.colour_A[c] @ x) / level.diag[rows]
    return x


def jacobi_sweep(level, x, b, omega=2.0 / 3.0):
    """Weighted Jacobi: x += omega D^{-1} (b - A x)."""
    return x + omega * (b - level.A @ x) / level.diag


def smooth(level, x, b, nu, smoother, pre, omega=2.0 / 3.0):
    for _ in range(nu):
        if smoother == "gs":
            x = gs_sweep(level, x, b, descending=not pre)
        elif smoother == "jacobi":
            x = jacobi_sweep(level, x, b, omega)
        else:
            raise ValueError(smoother)
    return x


def mu_cycle(H, l, x, b, mu=1, nu1=1, nu2=1, smoother="gs", omega=2.0 / 3.0):
    """Algorithm 2 on level l (0 = coarsest) with initial guess x and right side b."""
    if l == 0:
        return H.solve_coarsest(b)                              # direct coarsest solve
    lev = H.levels[l]
    u = smooth(lev, x, b, nu1, smoother, pre=True, omega=omega)  # pre-smooth
    r = b - lev.A @ u                                           # residual
    rc = H.P[l].T @ r                                           # restriction R = P^T
    ec = np.zeros(H.levels[l - 1].N)                            # coarse error := 0
    for _ in range(mu):
        ec = mu_cycle(H, l - 1, ec, rc, mu, nu1, nu2, smoother, omega)
    u = u + H.P[l] @ ec                                         # correction
    return smooth(lev, u, b, nu2, smoother, pre=False, omega=omega)  # post-smooth


def cycle(H, x, b, **kw):
    """The multigrid fixed-point map G of Eq. (fixedpoint): s_{k+1} = G(s_k)."""
    return mu_cycle(H, len(H.levels) - 1, x, b, **kw)


def residual_norm(H, x, b):
    return float(np.linalg.norm(b - H.finest.A @ x))
