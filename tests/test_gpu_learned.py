"""The learned post-smoother inside the solver (2D), through the C ABI.

* igamg_vcycle_probe: the captured iterate is the oracle's V-cycle stopped
  before the finest post-smoothing (composed here from oracle steps), and the
  returned iterate is the oracle's full V-cycle; FP64, relative 1e-11.
* A network with zero weights adds nothing, so each learned cycle is the
  V-cycle without finest post-smoothing: checked against the oracle
  composition over three FP32-IR cycles (relative 1e-5: FP32 corrections).
* Solves with a network converge; a harmful network triggers the fallback to
  Gauss-Seidel post-smoothing and the solve still converges.
* Training pairs satisfy A e = r and have unit RMS error; training on them
  lowers the loss.
* The fused inference kernel matches the oracle network on a many-tile image.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import multigrid as omg  # noqa: E402
import workloads  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build_library()
    import paper_2412_20205_gb300 as p
    assert torch.cuda.is_available()
    return p


DEV = "cuda"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _oracle_mid(H, x, b):
    """Finest-level V-cycle up to the coarse correction (Algorithm 2 without
    the last post-smoothing), composed from oracle steps."""
    l = len(H.levels) - 1
    lev = H.levels[l]
    u = omg.gs_sweep(lev, x, b)
    r = b - lev.A @ u
    ec = omg.mu_cycle(H, l - 1, np.zeros(H.levels[l - 1].N), H.P[l].T @ r)
    return u + H.P[l] @ ec


@pytest.mark.parametrize("n,p", [(32, 3), (27, 2), (20, 5)])
def test_probe_matches_oracle(pkg, n, p):
    s = pkg.Solver(2, p, n, k=5)
    H = omg.Hierarchy(2, [n, n], p)
    rng = np.random.default_rng(n + p)
    b = rng.standard_normal(H.finest.N)
    x = rng.standard_normal(H.finest.N)
    dx, db = _t(x), _t(b)
    mid = torch.empty_like(dx)
    pkg.igamg_vcycle_probe(s.ctx, dx, db, mid, s.ws)
    ref_mid = _oracle_mid(H, x, b)
    ref_x = omg.cycle(H, x, b)
    assert _rel(_np(mid), ref_mid) < 1e-11
    assert _rel(_np(dx), ref_x) < 1e-11
    s.close()


def test_zero_network_is_cycle_without_post_smoothing(pkg):
    n, p = 32, 3
    s = pkg.Solver(2, p, n, k=5)
    H = omg.Hierarchy(2, [n, n], p)
    w = torch.zeros(pkg.igamg_cnn_num_weights(), dtype=torch.float32, device=DEV)
    s.set_smoother(w, stall_ratio=10.0)            # never fall back
    b = np.random.default_rng(3).standard_normal(H.finest.N)
    out = s.solve(_t(b), tol=0.0, method="none", max_cycles=3, prec="fp32_ir_learned")
    assert out["cycles"] == 3 and not out["fell_back"]
    x = np.zeros(H.finest.N)
    for _ in range(3):
        x = _oracle_mid(H, x, b)
    assert _rel(_np(out["x"]), x) < 1e-5
    s.close()


def test_learned_solve_converges(pkg):
    from paper_2412_20205_gb300 import learned
    s = pkg.Solver(2, 3, 128, k=5)
    w = learned.init_weights(seed=1)
    s.set_smoother(w, stall_ratio=0.9)
    b = s.rhs_sine(workloads.random_sine_coeffs(2, seed=5))
    out = s.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir_learned", max_cycles=100)
    assert out["converged"], out["history"]
    ref = s.solve(b, tol=1e-12, method="rre", k=5, prec="fp64", max_cycles=100)
    assert _rel(_np(out["x"]), _np(ref["x"])) < 1e-6
    s.close()


def test_harmful_network_falls_back(pkg):
    from paper_2412_20205_gb300 import learned
    s = pkg.Solver(2, 3, 64, k=5)
    w = learned.init_weights(seed=2) * 30.0
    s.set_smoother(w, stall_ratio=0.9)
    b = s.rhs_sine(workloads.random_sine_coeffs(2, seed=6))
    out = s.solve(b, tol=1e-10, method="none", prec="fp32_ir_learned", max_cycles=400)
    assert out["fell_back"]
    assert out["converged"], out["history"][-5:]
    s.close()


def test_learned_needs_network_and_2d(pkg):
    s = pkg.Solver(2, 3, 16, k=5)
    b = torch.ones(s.N, dtype=torch.float64, device=DEV)
    with pytest.raises(RuntimeError):
        s.solve(b, prec="fp32_ir_learned")
    s.close()
    s3 = pkg.Solver(3, 2, 8, k=5)
    w = torch.zeros(pkg.igamg_cnn_num_weights(), dtype=torch.float32, device=DEV)
    with pytest.raises(RuntimeError):
        s3.set_smoother(w)
    s3.close()


def test_training_pairs_and_loss(pkg):
    from paper_2412_20205_gb300 import learned
    R, E = learned.generate_pairs(n=64, p=3, problems=3, k=3, modes=8)
    assert R.shape[0] >= 8 and R.shape[0] % 4 == 0 and R.shape[1:] == (65, 65)
    assert torch.isfinite(R).all() and torch.isfinite(E).all()
    # e = u_h - x_mid and r = b - A x_mid, so A e = r up to the 1e-13 solve
    # and FP32 storage (checked on the first V-cycles, where ||r|| >> 1e-13 ||b||)
    s = pkg.Solver(2, 3, 64, k=3)
    top = len(s.levels) - 1
    for i in (0, 1, 2):
        e = E[i].reshape(-1).double()
        ae = torch.empty_like(e)
        pkg.igamg_apply(s.ctx, top, e, ae, s.ws)
        r = R[i].reshape(-1).double()
        assert float((ae - r).norm() / r.norm()) < 1e-4
        assert abs(float(E[i].norm()) / 65 - 1.0) < 1e-3          # unit RMS error
    s.close()
    w, losses = learned.train(R, E, steps=400, batch=8, lr=3e-3, log_every=50)
    first = losses[0][1]
    last = np.mean([l for _, l in losses[-3:]])
    assert last < 0.7 * first, losses


def test_fused_forward_large_image(pkg):
    """The fused inference kernel on a solver-sized image with many tiles and
    ragged edges, against the FP64 oracle network."""
    from oracle import cnn as ocnn
    from paper_2412_20205_gb300 import learned
    H, W = 261, 300
    w = learned.init_weights(seed=4) * torch.tensor([1.0], device=DEV)
    w[2448:] *= 10.0
    wn = w.double().cpu().numpy()
    Ws = (wn[:144].reshape(16, 1, 3, 3), wn[144:2448].reshape(16, 16, 3, 3), wn[2448:].reshape(1, 16, 3, 3))
    r = np.random.default_rng(9).standard_normal((1, H, W))
    tr = torch.tensor(r, dtype=torch.float32, device=DEV)
    y = torch.full_like(tr, 0.5)
    ws = torch.empty(pkg.igamg_cnn_workspace_bytes(1, H, W), dtype=torch.uint8, device=DEV)
    pkg.igamg_cnn_forward(1, H, W, tr, w, y, ws)
    ref, _ = ocnn.forward(r, Ws)
    got = _np(y)
    assert _rel(got, ref) < 2e-2
    assert np.dot(got.ravel(), ref.ravel()) / (np.linalg.norm(got) * np.linalg.norm(ref)) > 0.999


def test_stored_network_saves_restarts_at_1024_p4(pkg):
    """What the trained network gains: with the stored weights (trained on
    257^2, p = 3 pairs), 1024^2 elements at p = 4 -- where multicolour
    Gauss-Seidel smooths worse -- the learned post-smoother needs fewer RRE(5)
    restart cycles than the plain mixed form on every right-hand side, without
    falling back, and its solution passes the oracle's residual test (the
    oracle's operator and load vector, FP64)."""
    import os
    from oracle import bspline as bs, galerkin as gk
    wfile = os.path.join(os.path.dirname(pkg.__file__), "weights", "smoother_2d_n256_p3.npy")
    w = torch.tensor(np.load(wfile), dtype=torch.float32, device=DEV)
    n, p = 1024, 4
    s = pkg.Solver(2, p, n, k=5)
    s.set_smoother(w)
    br = bs.uniform_breaks(n)
    f = gk.factors_1d(br, p)
    A = gk.operator([f, f])
    total_plain = total_learned = 0
    for seed in (10000, 10001, 10002):
        coeffs = workloads.random_sine_coeffs(2, seed=seed, modes=16)
        b = s.rhs_sine(coeffs)
        plain = s.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir", max_cycles=60)
        learned = s.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir_learned", max_cycles=60)
        assert plain["converged"] and learned["converged"] and not learned["fell_back"]
        assert learned["cycles"] <= plain["cycles"], (seed, learned["cycles"], plain["cycles"])
        total_plain += plain["cycles"]
        total_learned += learned["cycles"]
        bo = gk.load_vector([br, br], p, coeffs)
        x = _np(learned["x"])
        assert np.linalg.norm(bo - A @ x) / np.linalg.norm(bo) <= 1.05e-10
    assert total_learned < total_plain, (total_learned, total_plain)
    s.close()


def test_training_pairs_match_oracle(pkg):
    """igamg_training_pairs against the oracle: the first two V-cycles of the
    restarted RRE run from s_0 = 0, probed before the finest post-smoothing
    (composed from oracle steps), give pairs (b - A x_mid, u_h - x_mid) scaled
    to unit RMS error; FP32 storage, relative 1e-5."""
    import scipy.sparse.linalg as spla
    from oracle import solver as osolver
    n, p, k = 40, 3, 3
    coeffs = workloads.random_sine_coeffs(2, seed=12, modes=6)
    prob = osolver.Problem(2, n, p, coeffs)
    H, b = prob.H, prob.b
    A = H.finest.A
    uh = spla.spsolve(A.tocsc(), b)
    s = pkg.Solver(2, p, n, k=k)
    bt = s.rhs_sine(coeffs)
    uht = s.solve(bt, tol=1e-13, method="rre", k=k, prec="fp64", max_cycles=100)["x"]
    per = (k + 1) * 4
    R = torch.empty((per, s.N), dtype=torch.float32, device=DEV)
    E = torch.empty_like(R)
    ws = torch.empty(pkg.igamg_training_workspace_bytes(s.ctx, k), dtype=torch.uint8, device=DEV)
    cnt = pkg.igamg_training_pairs(s.ctx, bt, uht, k, 1e-10, 4, R, E, ws)
    assert cnt % (k + 1) == 0 and cnt >= k + 1
    x = np.zeros(H.finest.N)
    for i in range(2):
        mid = _oracle_mid(H, x, b)
        e = uh - mid
        c = np.sqrt(H.finest.N) / np.linalg.norm(e)
        assert _rel(E[i].double().cpu().numpy(), c * e) < 1e-5, i
        assert _rel(R[i].double().cpu().numpy(), c * (b - A @ mid)) < 1e-5, i
        x = omg.cycle(H, x, b)
    s.close()
