"""B-spline bases on open knot vectors (oracle; test infrastructure only).

Sec. 2.3: a knot vector is a non-decreasing sequence; it is *open* when its
first and last entries are repeated p+1 times, and *uniform* when the distinct
knots are equidistant.  The B-splines follow the Cox-de Boor recurrence
(Eq. moneq) with the convention 0/0 := 0, starting from indicator functions of
the half-open knot spans (the last non-empty span is closed at its right end so
that the basis is a partition of unity on the whole closed interval, Prop. 3).
"""
import numpy as np


def uniform_breaks(n):
    """n+1 equidistant breakpoints of [0, 1] (n elements of size h = 1/n)."""
    return np.linspace(0.0, 1.0, n + 1)


def coarsen_breaks(breaks):
    """Breakpoints of the coarse grid Omega^{2h} (Sec. 2): every other fine
    breakpoint, plus the last one when the fine element count is odd, so the
    coarse spline space is nested in the fine one."""
    breaks = np.asarray(breaks, dtype=np.float64)
    coarse = breaks[::2]
    if (len(breaks) - 1) % 2 == 1:
        coarse = np.append(coarse, breaks[-1])
    return coarse


def open_knot_vector(breaks, p):
    """Open knot vector (Sec. 2.3): end breakpoints repeated p+1 times, every
    interior breakpoint once.  Gives len(breaks)-1+p basis functions."""
    breaks = np.asarray(breaks, dtype=np.float64)
    return np.concatenate([np.full(p + 1, breaks[0]), breaks[1:-1],
                           np.full(p + 1, breaks[-1])])


def _degree_zero(knots, t):
    """N_j^0 = indicator of [t_j, t_{j+1}); the last non-empty span is closed."""
    nk = len(knots)
    lo = knots[:-1][None, :]
    hi = knots[1:][None, :]
    N = ((t[:, None] >= lo) & (t[:, None] < hi)).astype(np.float64)
    last = max(j for j in range(nk - 1) if knots[j] < knots[j + 1])
    N[t == knots[last + 1], last] = 1.0
    return N


def _raise_degree(knots, q, t, N):
    """One step of Eq. (moneq): degree q-1 -> q for every j, with 0/0 := 0."""
    nb = N.shape[1] - 1
    j = np.arange(nb)
    d1 = knots[j + q] - knots[j]
    d2 = knots[j + q + 1] - knots[j + 1]
    w1 = np.where(d1 > 0, (t[:, None] - knots[j][None, :]) / np.where(d1 > 0, d1, 1.0), 0.0)
    w2 = np.where(d2 > 0, (knots[j + q + 1][None, :] - t[:, None]) / np.where(d2 > 0, d2, 1.0), 0.0)
    return w1 * N[:, :-1] + w2 * N[:, 1:]


def basis(knots, p, t):
    """Values of all B-splines N_j^p(t_a); array of shape (len(t), len(knots)-p-1)."""
    knots = np.asarray(knots, dtype=np.float64)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    N = _degree_zero(knots, t)
    for q in range(1, p + 1):
        N = _raise_degree(knots, q, t, N)
    return N


def basis_derivative(knots, p, t):
    """Derivatives dN_j^p/dt at t, from the degree p-1 basis:
    N'_j = p [N_j^{p-1}/(t_{j+p}-t_j) - N_{j+1}^{p-1}/(t_{j+p+1}-t_{j+1})], 0/0 := 0."""
    knots = np.asarray(knots, dtype=np.float64)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    if p == 0:
        return np.zeros((len(t), len(knots) - 1))
    Nm = basis(knots, p - 1, t)
    nb = len(knots) - p - 1
    j = np.arange(nb)
    d1 = knots[j + p] - knots[j]
    d2 = knots[j + p + 1] - knots[j + 1]
    a = np.where(d1 > 0, Nm[:, :-1] / np.where(d1 > 0, d1, 1.0), 0.0)
    b = np.where(d2 > 0, Nm[:, 1:] / np.where(d2 > 0, d2, 1.0), 0.0)
    return p * (a - b)


def gauss_legendre(npts):
    """npts-point Gauss-Legendre rule on [-1, 1]: nodes are the roots of the
    Legendre polynomial P_npts, found by Newton's method from the Chebyshev-like
    guesses cos(pi (i - 1/4) / (npts + 1/2)); weights 2 / ((1 - x^2) P'(x)^2)."""
    i = np.arange(1, npts + 1)
    x = np.cos(np.pi * (i - 0.25) / (npts + 0.5))
    for _ in range(100):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for k in range(2, npts + 1):            # Bonnet recurrence
            p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        dp = npts * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p0 = np.ones_like(x)
    p1 = x.copy()
    for k in range(2, npts + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    dp = npts * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def element_quadrature(breaks, npts):
    """Tensor-free 1D quadrature: npts Gauss points mapped into every element
    [breaks[e], breaks[e+1]]; returns (points, weights) of length n*npts."""
    breaks = np.asarray(breaks, dtype=np.float64)
    xg, wg = gauss_legendre(npts)
    a = breaks[:-1][:, None]
    h = (breaks[1:] - breaks[:-1])[:, None]
    pts = a + 0.5 * (xg[None, :] + 1.0) * h
    wts = 0.5 * wg[None, :] * h
    return pts.ravel(), wts.ravel()
