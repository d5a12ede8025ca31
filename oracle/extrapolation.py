"""Polynomial vector extrapolation: RRE and MPE, plain and restarted (oracle).

Test infrastructure only.  Sec. 3: from iterates s_k, ..., s_{k+q+1} of a
fixed-point map (Eq. fixedpoint) the extrapolant is t_{k,q} = sum_j gamma_j
s_{k+j} (Eq. newsequence) with sum_j gamma_j = 1 and orthogonality conditions
built on the first and second differences.  Algorithms 3 (RRE) and 4 (MPE)
compute the gammas from a QR factorisation of the difference matrix
Delta S_{q+1} = [Delta s_k, ..., Delta s_{k+q}]:

* RRE: solve R^T R d = e (e = ones), lambda = sum d, gamma = d / lambda.
* MPE: solve R_q d = -r_q (r_q = first q entries of column q of R), d_q = 1,
  lambda = sum d, gamma = d / lambda.
* both: alpha_0 = 1 - gamma_0, alpha_j = alpha_{j-1} - gamma_j (j < q) and
  t = s_k + Q_q (R_q alpha).

Algorithm 5 restarts: q+1 fixed-point steps from s_0, extrapolate, test the
accuracy of t, and restart from s_0 := t.

Beyond the paper (its algorithms assume a full-rank difference matrix), one
guard is applied, identically in the GPU path.  With D_i = ||Delta s_i||, the
QR of the column-normalised difference matrix has diagonal |R_ii| / D_i.  If it
drops below BREAKDOWN_TOL at a first column i >= 1, Delta s_i lies (to that
tolerance) in the span of the earlier differences, the Krylov space is
exhausted, and the extrapolant whose generalised residual vanishes is taken:
q' = i and R_i d = -r_i, d_i = 1 (the MPE formula, which for a singular
R^T R is also the RRE minimiser).  If lambda = sum d vanishes
(|lambda| <= LAMBDA_TOL sum |d_i|) or the gammas are not finite, t is the last
iterate s_{k+q+1}; if Delta s_0 = 0, s_k is a fixed point and t = s_k.
"""
import numpy as np
import scipy.linalg as sla

BREAKDOWN_TOL = 1e-6
LAMBDA_TOL = 1e-12


def differences(S):
    """Delta S_{q+1} = [s_1 - s_0, ..., s_{q+1} - s_q] as an (N, q+1) array."""
    return np.column_stack([S[i + 1] - S[i] for i in range(len(S) - 1)])


def first_dependent_column(R, dS):
    """Smallest i >= 1 whose column-normalised R diagonal is below the
    tolerance, or q+1 when every column is independent."""
    D = np.linalg.norm(dS, axis=0)
    for i in range(1, R.shape[0]):
        if D[i] == 0.0 or abs(R[i, i]) / D[i] < BREAKDOWN_TOL:
            return i
    return R.shape[0]


def _gammas(R, method, q):
    if method == "rre":
        e = np.ones(q + 1)
        y = sla.solve_triangular(R[: q + 1, : q + 1], e, trans="T")   # R^T y = e
        d = sla.solve_triangular(R[: q + 1, : q + 1], y)              # R d = y
    elif method == "mpe":
        d = _null_vector(R, q)
    else:
        raise ValueError(method)
    return d


def _null_vector(R, q):
    """R_q d = -r_q (r_q = first q entries of column q of R), d_q = 1."""
    return np.append(sla.solve_triangular(R[:q, :q], -R[:q, q]), 1.0)


def extrapolate(S, method="rre"):
    """One RRE (Algorithm 3) or MPE (Algorithm 4) step on S = [s_k, ..., s_{k+q+1}].

    Returns (t, gamma, q_used); gamma has q_used+1 entries (empty on fallback)."""
    q = len(S) - 2
    dS = differences(S)
    if np.linalg.norm(dS[:, 0]) == 0.0:
        return S[0].copy(), np.array([1.0]), 0
    Q, R = np.linalg.qr(dS)                       # Delta S_{q+1} = Q_{q+1} R_{q+1}
    i = first_dependent_column(R, dS)
    with np.errstate(all="ignore"):
        if i <= q:                                # exhausted Krylov space: q' = i
            d, qu = _null_vector(R, i), i
        else:
            d, qu = _gammas(R, method, q), q
        lam = d.sum()                             # lambda = sum_i d_i
        gamma = d / lam
    if not (np.all(np.isfinite(gamma)) and abs(lam) > LAMBDA_TOL * np.abs(d).sum()):
        return S[-1].copy(), np.array([]), -1
    alpha = np.empty(qu)
    alpha[0] = 1.0 - gamma[0]
    for j in range(1, qu):
        alpha[j] = alpha[j - 1] - gamma[j]
    t = S[0] + Q[:, :qu] @ (R[:qu, :qu] @ alpha)   # t = s_k + Q_q (R_q alpha)
    return t, gamma, qu


def extrapolate_schur(S, method="rre"):
    """Eq. (extrapolapprox): t = s_k - Delta S (Y^T Delta^2 S)^{-1} Y^T Delta s_k with
    Y = Delta^2 S (RRE) or Delta S (MPE), both with q columns."""
    q = len(S) - 2
    dS = differences(S)                     # columns Delta s_0..Delta s_q
    d2S = dS[:, 1:] - dS[:, :-1]            # Delta^2 s_0..Delta^2 s_{q-1}
    dSq = dS[:, :q]
    Y = d2S if method == "rre" else dSq
    return S[0] - dSq @ np.linalg.solve(Y.T @ d2S, Y.T @ dS[:, 0])


def extrapolate_pinv(S):
    """Eq. (rreapproxim): t = s_k - Delta S (Delta^2 S)^+ Delta s_k (RRE)."""
    q = len(S) - 2
    dS = differences(S)
    d2S = dS[:, 1:] - dS[:, :-1]
    return S[0] - dS[:, :q] @ (np.linalg.pinv(d2S) @ dS[:, 0])


def generalized_residual(S, gamma):
    """Eq. (resgeneralized): r~(t) = t~ - t = sum_j gamma_j Delta s_{k+j}."""
    dS = differences(S)
    return dS[:, : len(gamma)] @ gamma


def restarted(G, residual, s0, q, method="rre", tol=1e-10, max_cycles=100,
              bnorm=1.0, keep_iterates=False):
    """Algorithm 5.  G is the fixed-point map, residual(x) = ||b - A x||.
    The accuracy test is residual(t) / bnorm <= tol.

    Returns dict(x, history, cycles, vcycles, converged[, iterates])."""
    s = np.asarray(s0, dtype=np.float64).copy()
    hist = [residual(s) / bnorm]
    out = {"iterates": []} if keep_iterates else {}
    vcycles = 0
    if hist[0] <= tol:
        out.update(x=s, history=hist, cycles=0, vcycles=0, converged=True)
        return out
    for cyc in range(1, max_cycles + 1):
        S = [s]
        for _ in range(q + 1):
            S.append(G(S[-1]))
            vcycles += 1
        t, gamma, _ = extrapolate(S, method)
        rel = residual(t) / bnorm
        hist.append(rel)
        if keep_iterates:
            out["iterates"].append(t.copy())
        if rel <= tol:
            out.update(x=t, history=hist, cycles=cyc, vcycles=vcycles, converged=True)
            return out
        s = t
    out.update(x=s, history=hist, cycles=max_cycles, vcycles=vcycles, converged=False)
    return out
