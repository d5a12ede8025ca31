"""Pins of the oracle's B-spline layer (Sec. 2.3, Eq. moneq, Prop. 3)."""
import math

import numpy as np
import pytest

from oracle import bspline as bs


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_legendre_matches_library_rule(n):
    x, w = bs.gauss_legendre(n)
    X, W = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, X, atol=1e-15, rtol=0)
    assert np.allclose(w, W, atol=1e-14, rtol=0)


@pytest.mark.parametrize("n", [1, 3, 6])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = bs.gauss_legendre(n)
    for k in range(2 * n):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


def _breaks(kind, n):
    if kind == "uniform":
        return bs.uniform_breaks(n)
    rng = np.random.default_rng(n)
    inner = np.sort(rng.uniform(0.05, 0.95, n - 1))
    return np.concatenate([[0.0], inner, [1.0]])


@pytest.mark.parametrize("p", range(0, 7))
@pytest.mark.parametrize("kind", ["uniform", "random"])
def test_partition_of_unity_nonnegativity_support(p, kind):
    br = _breaks(kind, 7)
    k = bs.open_knot_vector(br, p)
    t = np.concatenate([np.random.default_rng(0).uniform(0, 1, 400), br])
    N = bs.basis(k, p, t)
    assert N.shape[1] == len(br) - 1 + p
    assert np.allclose(N.sum(axis=1), 1.0, atol=1e-14)          # partition of unity
    assert N.min() >= -1e-15                                     # non-negativity
    for j in range(N.shape[1]):                                  # compact support
        outside = (t < k[j]) | (t > k[j + p + 1])
        assert np.all(N[outside, j] == 0.0)
    assert np.all((N > 0).sum(axis=1) <= p + 1)                  # at most p+1 non-zero


@pytest.mark.parametrize("p", range(1, 7))
def test_derivative_matches_central_differences(p):
    k = bs.open_knot_vector(_breaks("random", 6), p)
    t = np.random.default_rng(1).uniform(0.01, 0.99, 50)
    eps = 1e-6
    fd = (bs.basis(k, p, t + eps) - bs.basis(k, p, t - eps)) / (2 * eps)
    D = bs.basis_derivative(k, p, t)
    # skip points within eps of a knot (one-sided kinks for p = 1)
    near = np.min(np.abs(t[:, None] - k[None, :]), axis=1) < 1e-4
    assert np.allclose(D[~near], fd[~near], atol=1e-6 * max(1, np.abs(D).max()))


def cardinal_bspline(r, x):
    """Cardinal B-spline of degree r on [0, r+1] by the truncated-power sum
    (1/r!) sum_k (-1)^k C(r+1,k) (x-k)_+^r -- independent of Cox-de Boor."""
    x = np.asarray(x, dtype=np.float64)
    s = np.zeros_like(x)
    for kk in range(r + 2):
        s += (-1) ** kk * math.comb(r + 1, kk) * np.where(x > kk, (x - kk) ** r, 0.0)
    return s / math.factorial(r)


@pytest.mark.parametrize("p", range(1, 7))
def test_interior_basis_is_cardinal_bspline(p):
    n = 3 * p + 4
    k = bs.open_knot_vector(bs.uniform_breaks(n), p)
    h = 1.0 / n
    j = p + 1                                      # support [t_j, t_{j+p+1}] all interior
    t = np.linspace(k[j], k[j + p + 1], 97)
    assert np.allclose(bs.basis(k, p, t)[:, j], cardinal_bspline(p, (t - k[j]) / h), atol=1e-13)


def test_coarsening_nested_and_odd_counts():
    for n in [8, 9, 33, 512]:
        b = bs.uniform_breaks(n)
        c = bs.coarsen_breaks(b)
        assert len(c) - 1 == (n + 1) // 2
        assert set(np.round(c, 15)).issubset(set(np.round(b, 15)))
        assert c[0] == 0.0 and c[-1] == 1.0
