"""Whole-solve driver of the oracle: the restarted RRE/MPE-accelerated mu-cycle
(Algorithm 5 around Algorithm 2) on -Laplace(u) = f, f a sine series (Sec. 4).

Test infrastructure only.  The iteration starts from s_0 = 0 (Sec. 4.1) and,
with the relative accuracy test, stops once ||b - A t|| / ||b|| <= tol.
"""
import numpy as np

from . import extrapolation, multigrid
from .galerkin import load_vector


class Problem:
    """Hierarchy + load vector for one (dim, n, p, f) problem."""

    def __init__(self, dim, n, p, coeffs, n_levels=None, coarsest=8):
        self.H = multigrid.Hierarchy(dim, n, p, n_levels=n_levels, coarsest=coarsest)
        self.b = load_vector(self.H.finest.breaks, p, coeffs)
        self.bnorm = float(np.linalg.norm(self.b))

    def cycle(self, x, **kw):
        return multigrid.cycle(self.H, x, self.b, **kw)

    def residual(self, x):
        return float(np.linalg.norm(self.b - self.H.finest.A @ x))


def solve(prob, method="rre", k=5, tol=1e-10, max_cycles=100, relative=True,
          mu=1, smoother="gs", keep_iterates=False, s0=None):
    """Restarted extrapolation (method 'rre' / 'mpe') with restart number k, or
    the plain mu-cycle (method 'none'; then one 'cycle' is one mu-cycle)."""
    G = lambda x: prob.cycle(x, mu=mu, smoother=smoother)
    bnorm = prob.bnorm if relative else 1.0
    s0 = np.zeros(prob.H.finest.N) if s0 is None else s0
    if method == "none":
        x = s0.copy()
        hist = [prob.residual(x) / bnorm]
        its = []
        for c in range(1, max_cycles + 1):
            x = G(x)
            hist.append(prob.residual(x) / bnorm)
            if keep_iterates:
                its.append(x.copy())
            if hist[-1] <= tol:
                return dict(x=x, history=hist, cycles=c, vcycles=c, converged=True, iterates=its)
        return dict(x=x, history=hist, cycles=max_cycles, vcycles=max_cycles,
                    converged=False, iterates=its)
    return extrapolation.restarted(G, prob.residual, s0, k, method, tol, max_cycles,
                                   bnorm, keep_iterates=keep_iterates)
