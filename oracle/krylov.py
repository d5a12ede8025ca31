"""Textbook Arnoldi-based GMRES and FOM (oracle; test infrastructure only).

Used only to pin RRE and MPE: for a linear fixed-point map G(x) = B x + c,
the q-th RRE extrapolant from s_0 is the GMRES iterate after q Arnoldi steps
on (I - B) x = c from x_0 = s_0, and the MPE extrapolant is the FOM (Arnoldi
Galerkin) iterate (Sec. 3 defines both through sum_j gamma_j Delta s_j, which is
exactly the residual c - (I - B) t of the extrapolant t).
"""
import numpy as np


def arnoldi(F, r0, q):
    """q steps of Arnoldi with modified Gram-Schmidt on the operator F."""
    beta = np.linalg.norm(r0)
    V = [r0 / beta]
    H = np.zeros((q + 1, q))
    for j in range(q):
        w = F(V[j])
        for i in range(j + 1):
            H[i, j] = np.dot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else np.zeros_like(w))
    return np.column_stack(V), H, beta


def gmres(F, c, x0, q):
    """x in x0 + K_q(F, r0) minimising ||c - F x||_2 (r0 = c - F x0)."""
    r0 = c - F(x0)
    V, H, beta = arnoldi(F, r0, q)
    rhs = np.zeros(q + 1)
    rhs[0] = beta
    y = np.linalg.lstsq(H, rhs, rcond=None)[0]
    return x0 + V[:, :q] @ y


def fom(F, c, x0, q):
    """x in x0 + K_q(F, r0) with residual orthogonal to K_q (Galerkin)."""
    r0 = c - F(x0)
    V, H, beta = arnoldi(F, r0, q)
    rhs = np.zeros(q)
    rhs[0] = beta
    y = np.linalg.solve(H[:q, :q], rhs)
    return x0 + V[:, :q] @ y
