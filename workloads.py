"""Seeded synthetic inputs for the extrapolated-multigrid IGA solver.

This module holds the problem definitions only -- sizes, degrees, solver
settings and the sine-series coefficients of the right-hand side f -- and none
of the method's arithmetic.  Both the CPU oracle's callers and the CUDA path's
callers draw their inputs from here, so the two sides see identical inputs.

A right-hand side is the sine series
    f(x) = sum_k c[k_{D-1}, ..., k_0] prod_d sin((k_d + 1) pi x_d)
on the unit square (cube); ``c`` is an array of shape (K,)*dim indexed with
the x mode last.  The paper's experiments (Sec. 4) use manufactured sine
solutions; the random fields stand in for "seeded random smooth Fourier
fields" (16 modes per direction, N(0,1) coefficients).
"""
import math

import numpy as np


def manufactured_coeffs(dim, freq=1):
    """-Laplace(u) = f for u = prod_d sin(freq pi x_d): one mode, c = dim (freq pi)^2."""
    c = np.zeros((freq,) * dim)
    c[(freq - 1,) * dim] = dim * (freq * math.pi) ** 2
    return c


def random_sine_coeffs(dim, seed, modes=16):
    """N(0,1) coefficients of the first ``modes`` sine modes per direction."""
    return np.random.default_rng(seed).standard_normal((modes,) * dim)


# The five workloads: (dim, n elements per direction, degree p, solver settings).
CONFIGS = {
    "c1_2d_64_p2": dict(dim=2, n=64, p=2, method="rre", k=5, tol=1e-10, rhs="manufactured"),
    "c2_2d_1024": dict(dim=2, n=1024, p=(2, 3, 4, 5), method=("rre", "mpe"), k=(5, 10),
                       tol=1e-10, rhs=("manufactured", "random")),
    "c3_3d_128_p3": dict(dim=3, n=128, p=3, method="rre", k=10, tol=1e-10, rhs="manufactured"),
    "c4_batch_256": dict(dim=2, count=256, n_range=(32, 512), p_set=(2, 3, 4), method="rre",
                         k=5, tol=1e-10, rhs="random"),
    "c5_learned": dict(dim=2, train_n=256, train_p=3, eval_n=1024, eval_p=(3, 4), method="rre",
                       k=5, tol=1e-10, rhs="random"),
}


def batch_problems(count=256, seed=0, n_range=(32, 512), p_set=(2, 3, 4)):
    """Uneven batch: n ~ U{n_range}, p ~ U(p_set), RHS seed 1000 + i per problem."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    ps = rng.choice(np.asarray(p_set), size=count)
    return [dict(n=int(ns[i]), p=int(ps[i]), rhs_seed=1000 + i) for i in range(count)]


# ----------------------------------------------------------------------------
# Sec. 4.3: the full elliptic problem -div(A grad u) + B . grad u + c u = f
# with homogeneous Dirichlet data.  Coefficient functions take arrays of
# physical points and return A: (n, 2, 2), B: (n, 2), c: (n,), f: (n,).

def _A_full(x, y):
    """The SPD diffusion tensor of Sec. 4.3 and its divergence (d_x A_11 + d_y A_12,
    d_x A_12 + d_y A_22), for manufactured right-hand sides."""
    A = np.empty(x.shape + (2, 2))
    A[..., 0, 0] = (2.0 + np.cos(x)) * (1.0 + y)
    A[..., 1, 1] = (2.0 + np.sin(y)) * (1.0 + x)
    A[..., 0, 1] = A[..., 1, 0] = np.cos(x + y) * np.sin(x + y)
    c2 = np.cos(2.0 * (x + y))                       # d/dx and d/dy of cos(s) sin(s) = cos(2s)
    div = np.stack([-np.sin(x) * (1.0 + y) + c2, c2 + (1.0 + x) * np.cos(y)], axis=-1)
    return A, div


def full_elliptic_square():
    """Table 13: the unit square, A as above,
    B = (11 + sin x + y sin x - 2 cos^2(x+y), -9 - cos y - x cos y - 2 cos^2(x+y)), c = f = 1."""
    def B(x, y):
        k = 2.0 * np.cos(x + y) ** 2
        return np.stack([11.0 + np.sin(x) + y * np.sin(x) - k, -9.0 - np.cos(y) - x * np.cos(y) - k], axis=-1)
    return dict(A=lambda x, y: _A_full(x, y)[0], B=B, c=lambda x, y: np.ones_like(x),
                f=lambda x, y: np.ones_like(x), geometry=None)


def advection_diffusion(eps=0.1, b=(1.0, 1.0)):
    """Table 14: -eps Laplace(u) + (1, 1) . grad u = f on the unit square,
    eps = 0.1; the paper gives no f, f = 1 is taken."""
    def A(x, y):
        out = np.zeros(x.shape + (2, 2))
        out[..., 0, 0] = out[..., 1, 1] = eps
        return out
    return dict(A=A, B=lambda x, y: np.stack([np.full_like(x, b[0]), np.full_like(x, b[1])], axis=-1),
                c=lambda x, y: np.zeros_like(x), f=lambda x, y: np.ones_like(x), geometry=None)


def annulus_map(r0=0.2, r1=1.0):
    """The quarter annulus r0 < |x| < r1, x, y > 0 as the polar map
    F(xi, eta) = (r cos t, r sin t), r = r0 + (r1 - r0) xi, t = pi/2 eta;
    returns geometry(xi, eta) -> (x, y, J), J[q, a, b] = d F_a / d xi_b."""
    def geometry(xi, eta):
        r = r0 + (r1 - r0) * xi
        t = 0.5 * np.pi * eta
        ct, st = np.cos(t), np.sin(t)
        J = np.empty(xi.shape + (2, 2))
        J[..., 0, 0] = (r1 - r0) * ct
        J[..., 1, 0] = (r1 - r0) * st
        J[..., 0, 1] = -0.5 * np.pi * r * st
        J[..., 1, 1] = 0.5 * np.pi * r * ct
        return r * ct, r * st, J
    return geometry


def annulus_solution(x, y, r0=0.2, r1=1.0):
    """u = (x^2+y^2-r0^2)(x^2+y^2-r1^2) sin x sin y: value, gradient and Hessian."""
    s = x * x + y * y
    g, h = s - r0 * r0, s - r1 * r1
    sx, sy, cx, cy = np.sin(x), np.sin(y), np.cos(x), np.cos(y)
    P = g * h                                         # radial factor and its derivatives
    Px, Py = 2 * x * (g + h), 2 * y * (g + h)
    Pxx = 2 * (g + h) + 8 * x * x
    Pyy = 2 * (g + h) + 8 * y * y
    Pxy = 8 * x * y
    S = sx * sy
    Sx, Sy = cx * sy, sx * cy
    Sxx, Syy, Sxy = -S, -S, cx * cy
    u = P * S
    ux, uy = Px * S + P * Sx, Py * S + P * Sy
    uxx = Pxx * S + 2 * Px * Sx + P * Sxx
    uyy = Pyy * S + 2 * Py * Sy + P * Syy
    uxy = Pxy * S + Px * Sy + Py * Sx + P * Sxy
    return u, np.stack([ux, uy], -1), np.stack([np.stack([uxx, uxy], -1), np.stack([uxy, uyy], -1)], -2)


def full_elliptic_annulus():
    """Table 15: the quarter annulus (r = 0.2, R = 1), A as above, B = (-5y, 5x),
    c = xy, f manufactured from u = (x^2+y^2-0.04)(x^2+y^2-1) sin x sin y:
    f = -(A : Hess u + div(A) . grad u) + B . grad u + c u."""
    def B(x, y):
        return np.stack([-5.0 * y, 5.0 * x], axis=-1)

    def f(x, y):
        u, gu, Hu = annulus_solution(x, y)
        A, div = _A_full(x, y)
        return (-(np.einsum("...ab,...ab->...", A, Hu) + np.einsum("...a,...a->...", div, gu))
                + np.einsum("...a,...a->...", B(x, y), gu) + x * y * u)
    return dict(A=lambda x, y: _A_full(x, y)[0], B=B, c=lambda x, y: x * y, f=f, geometry=annulus_map(),
                solution=lambda x, y: annulus_solution(x, y)[0])


GENERAL_PROBLEMS = {"full_elliptic": full_elliptic_square, "advection_diffusion": advection_diffusion,
                    "annulus": full_elliptic_annulus}
