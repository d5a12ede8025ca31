"""The allocation-free extrapolation entry point against the workspace one.

igamg_extrapolate_noalloc serves callers that cannot allocate device memory
where they extrapolate; it must give the same extrapolant, coefficients and
used restart number as igamg_extrapolate.  Two calls in a row (with different
restart numbers and methods) check that whatever the shared built-in scratch
keeps from the previous call does not leak into the next.  This file runs
last so that a failure here leaves the rest of the suite already run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build_library()
    import paper_2412_20205_gb300 as p
    assert torch.cuda.is_available()
    return p


def _sequence(n, q, seed):
    """q+2 iterates of a linear contraction s_{j+1} = B s_j + c (B diagonal)."""
    rng = np.random.default_rng(seed)
    lam = rng.uniform(-0.9, 0.9, n)
    c = rng.standard_normal(n)
    S = [rng.standard_normal(n)]
    for _ in range(q + 1):
        S.append(lam * S[-1] + c)
    return S


def test_noalloc_matches_workspace_entry_point_twice(pkg):
    n = 100_003                                         # ragged: not a multiple of any block size
    for call, (q, method) in enumerate([(5, pkg.IGAMG_RRE), (3, pkg.IGAMG_MPE)]):
        S = _sequence(n, q, seed=10 + call)
        ld = n + 7
        St = torch.zeros((q + 2) * ld, dtype=torch.float64, device="cuda")
        for j, s in enumerate(S):
            St[j * ld:j * ld + n] = torch.as_tensor(s, device="cuda")
        t_ws = torch.empty(n, dtype=torch.float64, device="cuda")
        ws = torch.empty(pkg.igamg_extrap_workspace_bytes(n, q), dtype=torch.uint8, device="cuda")
        g_ws, q_ws = pkg.igamg_extrapolate(n, q, method, St, ld, t_ws, ws)
        t_na = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        g_na, q_na = pkg.igamg_extrapolate_noalloc(n, q, method, St, ld, t_na)
        torch.cuda.synchronize()
        assert q_na == q_ws == q
        assert np.allclose(g_na, g_ws, rtol=1e-12, atol=1e-15)
        a, b = t_na.cpu().numpy(), t_ws.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_noalloc_rejects_out_of_range_restart_number(pkg):
    S = torch.zeros(20 * 10, dtype=torch.float64, device="cuda")
    t = torch.empty(10, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.IgamgError) as e:
        pkg.igamg_extrapolate_noalloc(10, 13, pkg.IGAMG_RRE, S, 10, t)
    assert e.value.status == pkg.IGAMG_EINVAL


def test_noalloc_largest_restart_number_then_smallest(pkg):
    """The built-in scratch at its largest use -- restart number 12 on a vector
    long enough for the most Gram partial-sum blocks (more than 304 x 256
    entries) -- and then a restart-number-1 call, which reuses the start of
    the scratch with stale partial sums of the large call behind it."""
    n = 304 * 256 + 5
    for call, (q, method) in enumerate([(12, pkg.IGAMG_RRE), (1, pkg.IGAMG_MPE)]):
        S = _sequence(n, q, seed=30 + call)
        St = torch.as_tensor(np.concatenate(S), dtype=torch.float64, device="cuda")
        t_ws = torch.empty(n, dtype=torch.float64, device="cuda")
        ws = torch.empty(pkg.igamg_extrap_workspace_bytes(n, q), dtype=torch.uint8, device="cuda")
        g_ws, q_ws = pkg.igamg_extrapolate(n, q, method, St, n, t_ws, ws)
        t_na = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        g_na, q_na = pkg.igamg_extrapolate_noalloc(n, q, method, St, n, t_na)
        torch.cuda.synchronize()
        assert q_na == q_ws
        assert np.allclose(g_na, g_ws, rtol=1e-12, atol=1e-15)
        a, b = t_na.cpu().numpy(), t_ws.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
