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
