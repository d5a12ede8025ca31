"""Pins of the oracle's RRE / MPE (Sec. 3, Eq. newsequence-resgeneralized,
Algorithms 3-5) against closed forms and textbook Krylov methods."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import extrapolation as ex
from oracle import krylov, multigrid as mg, solver
from oracle.galerkin import load_vector


def _linear_sequence(N=40, q=5, seed=0):
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.standard_normal((N, N)))[0]
    B = Q @ np.diag(rng.uniform(-0.9, 0.9, N)) @ Q.T
    c = rng.standard_normal(N)
    S = [rng.standard_normal(N)]
    for _ in range(q + 1):
        S.append(B @ S[-1] + c)
    return B, c, S


@pytest.mark.parametrize("q", [1, 2, 5, 8])
def test_rre_alg3_equals_schur_and_pseudoinverse_forms(q):
    _, _, S = _linear_sequence(q=q, seed=q)
    t, gamma, qu = ex.extrapolate(S, "rre")
    assert qu == q and abs(gamma.sum() - 1) < 1e-13
    assert np.allclose(t, ex.extrapolate_schur(S, "rre"), atol=1e-10)
    assert np.allclose(t, ex.extrapolate_pinv(S), atol=1e-10)
    assert np.allclose(t, sum(g * s for g, s in zip(gamma, S)), atol=1e-12)


@pytest.mark.parametrize("q", [1, 3, 6])
def test_mpe_alg4_equals_schur_form(q):
    _, _, S = _linear_sequence(q=q, seed=10 + q)
    t, gamma, _ = ex.extrapolate(S, "mpe")
    assert np.allclose(t, ex.extrapolate_schur(S, "mpe"), atol=1e-9)
    # MPE: generalised residual orthogonal to Delta s_0..Delta s_{q-1}
    r = ex.generalized_residual(S, gamma)
    dS = ex.differences(S)
    assert np.allclose(dS[:, :q].T @ r, 0.0, atol=1e-10 * np.linalg.norm(r) * np.linalg.norm(dS))


def test_rre_generalized_residual_norm_identity():
    """RRE minimises ||sum gamma_j Delta s_j|| under sum gamma_j = 1, whose
    minimum is 1 / (e^T (Delta S^T Delta S)^{-1} e)."""
    _, _, S = _linear_sequence(q=4, seed=3)
    t, gamma, _ = ex.extrapolate(S, "rre")
    dS = ex.differences(S)
    d = np.linalg.solve(dS.T @ dS, np.ones(dS.shape[1]))
    r = ex.generalized_residual(S, gamma)
    assert abs(np.dot(r, r) * d.sum() - 1) < 1e-10


@pytest.mark.parametrize("q", [2, 4])
def test_rre_is_gmres_and_mpe_is_fom_on_multigrid_preconditioned_system(q):
    """With G(x) = B x + c the V-cycle map, RRE(q) = GMRES(q) and MPE(q) = FOM(q)
    on (I - B) x = c from x_0 = s_0."""
    H = mg.Hierarchy(2, 16, 3)
    b = load_vector(H.finest.breaks, 3, np.random.default_rng(4).standard_normal((3, 3)))
    N = H.finest.N
    G = lambda x: mg.cycle(H, x, b)
    c = G(np.zeros(N))
    F = lambda v: v - (G(v) - c)
    s0 = np.random.default_rng(5).standard_normal(N)
    S = [s0]
    for _ in range(q + 1):
        S.append(G(S[-1]))
    t_rre = ex.extrapolate(S, "rre")[0]
    t_mpe = ex.extrapolate(S, "mpe")[0]
    scale = np.linalg.norm(t_rre)
    assert np.linalg.norm(t_rre - krylov.gmres(F, c, s0, q)) < 1e-10 * scale
    assert np.linalg.norm(t_mpe - krylov.fom(F, c, s0, q)) < 1e-10 * scale


@pytest.mark.parametrize("method", ["rre", "mpe"])
@pytest.mark.parametrize("q", [6, 8])
def test_finite_termination_on_a_linear_map(method, q):
    """For s_{j+1} = B s_j + c in R^6, q >= 6 exhausts the Krylov space and the
    first extrapolant is the fixed point (I - B)^{-1} c."""
    B, c, S = _linear_sequence(N=6, q=q, seed=21)
    t, _, qu = ex.extrapolate(S, method)
    x = np.linalg.solve(np.eye(6) - B, c)
    assert qu == 6
    assert np.allclose(t, x, atol=1e-9 * np.abs(x).max())


@pytest.mark.parametrize("method", ["rre", "mpe"])
def test_finite_termination_on_a_tiny_multigrid_system(method):
    """2D n=4, p=2 has N=16 unknowns: with q = 16 one restart cycle of the
    V-cycle iteration reaches the discrete solution."""
    prob = solver.Problem(2, 4, 2, np.array([[1.0, 0.3], [-0.2, 0.5]]), n_levels=2)
    assert prob.H.finest.N == 16
    out = solver.solve(prob, method, k=16, tol=1e-12, max_cycles=1)
    u = spla.spsolve(prob.H.finest.A.tocsc(), prob.b)
    assert out["history"][1] < 1e-12
    assert np.allclose(out["x"], u, atol=1e-11 * np.abs(u).max())


@pytest.mark.parametrize("method", ["rre", "mpe"])
def test_restarted_solver_reaches_tolerance_and_the_discrete_solution(method):
    prob = solver.Problem(2, 32, 3, np.array([[2 * np.pi ** 2]]))
    out = solver.solve(prob, method, k=5, tol=1e-10, max_cycles=30)
    assert out["converged"] and out["history"][-1] <= 1e-10
    assert out["vcycles"] == 6 * out["cycles"]
    u = spla.spsolve(prob.H.finest.A.tocsc(), prob.b)
    assert np.linalg.norm(out["x"] - u) <= 1e-6 * np.linalg.norm(u)


@pytest.mark.parametrize("method,krylov_step", [("rre", krylov.gmres), ("mpe", krylov.fom)])
@pytest.mark.parametrize("q", [2, 4])
def test_restarted_extrapolation_is_restarted_krylov(method, krylov_step, q):
    """Algorithm 5 restarts from the extrapolant t (s_0 := t).  Each restart
    cycle from s_0 is one RRE (MPE) step, i.e. GMRES(q) (FOM(q)) from x_0 = s_0
    on the V-cycle-preconditioned system, so three restart cycles of the oracle
    equal three cycles of restarted GMRES(q) (FOM(q)), iterate by iterate.  An
    oracle that restarted from the last V-cycle iterate s_{q+1}, or ran q
    instead of q+1 V-cycles per restart, fails this."""
    H = mg.Hierarchy(2, 16, 3)
    b = load_vector(H.finest.breaks, 3, np.random.default_rng(6).standard_normal((3, 3)))
    N = H.finest.N
    G = lambda x: mg.cycle(H, x, b)
    c = G(np.zeros(N))
    F = lambda v: v - (G(v) - c)
    A = H.finest.A
    res = lambda x: float(np.linalg.norm(b - A @ x))
    out = ex.restarted(G, res, np.zeros(N), q, method, tol=0.0, max_cycles=3, keep_iterates=True)
    assert out["cycles"] == 3 and out["vcycles"] == 3 * (q + 1)
    x = np.zeros(N)
    for cyc in range(3):
        x = krylov_step(F, c, x, q)
        t = out["iterates"][cyc]
        assert np.linalg.norm(t - x) < 1e-10 * np.linalg.norm(x), cyc
        # the history holds ||b - A t|| of the same iterate (cancellation in b - A t
        # limits the agreement of two nearby iterates' residuals to about cond(A) eps)
        assert abs(out["history"][cyc + 1] - res(x)) < 1e-5 * res(x), cyc
