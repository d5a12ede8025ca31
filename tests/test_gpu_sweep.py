"""The single-launch Gauss-Seidel sweep (one kernel per sweep, rows waiting on
their earlier-colour neighbours through flags) against the row-phase launches
it replaces: same colours, order and per-row arithmetic, so the results must
be bitwise equal, in FP64 and FP32, 2D and 3D, sweeps and whole solves.  Also
the bounded device-side wait: a wait on a flag that nothing sets runs out,
the call reports IGAMG_ETIMEOUT, and the context stays usable."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402

DEV = "cuda"


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build_library()
    import paper_2412_20205_gb300 as p
    assert torch.cuda.is_available()
    return p


CASES = [(2, 20, 2), (2, 37, 3), (2, (21, 13), 5), (2, 1024, 3), (2, 200, 7), (3, 9, 3), (3, 24, 2), (3, 40, 3),
         (2, 3, 3), (2, 2, 1)]


def _sweeps(pkg, s, form, x0, b, level):
    pkg.igamg_set_sweep_form(s.ctx, form, form)
    out = {}
    x = torch.tensor(x0, dtype=torch.float64, device=DEV)
    pkg.igamg_smooth(s.ctx, level, x, torch.tensor(b, dtype=torch.float64, device=DEV), 0, s.ws)
    pkg.igamg_smooth(s.ctx, level, x, torch.tensor(b, dtype=torch.float64, device=DEV), 1, s.ws)
    out["fp64"] = x
    xf = torch.tensor(x0, dtype=torch.float32, device=DEV)
    bf = torch.tensor(b, dtype=torch.float32, device=DEV)
    pkg.igamg_smooth_f32(s.ctx, level, xf, bf, 0, s.ws)
    pkg.igamg_smooth_f32(s.ctx, level, xf, bf, 1, s.ws, sums_current=True)
    pkg.igamg_smooth_f32(s.ctx, level, xf, bf, 0, s.ws, sums_current=True)
    out["fp32"] = xf
    assert pkg.igamg_device_status(s.ctx, s.ws) == pkg.IGAMG_OK
    return out


@pytest.mark.parametrize("dim,n,p", CASES, ids=lambda c: str(c))
def test_single_launch_sweep_is_bitwise_equal_to_row_phases(pkg, dim, n, p):
    s = pkg.Solver(dim, p, n, k=5)
    rng = np.random.default_rng(3)
    for level in range(len(s.levels)):
        m = s.levels[level]
        N = m[0] * m[1] * m[2]
        x0, b = rng.standard_normal(N), rng.standard_normal(N)
        a = _sweeps(pkg, s, 0, x0, b, level)
        c = _sweeps(pkg, s, 1, x0, b, level)
        for key in a:
            assert torch.equal(a[key], c[key]), (level, key)
    s.close()


@pytest.mark.parametrize("dim,n,p,k", [(2, 256, 3, 5), (2, 61, 5, 8), (3, 24, 3, 10)])
def test_single_launch_solves_are_bitwise_equal(pkg, dim, n, p, k):
    s = pkg.Solver(dim, p, n, k=k)
    b = s.rhs_sine(workloads.random_sine_coeffs(dim, seed=4, modes=8))
    for prec in ("fp64", "fp32_ir"):
        res = []
        for form in (0, 1):
            pkg.igamg_set_sweep_form(s.ctx, form, form)
            out = s.solve(b, tol=1e-10, method="rre", k=k, prec=prec, max_cycles=60)
            assert out["converged"], (prec, form)
            res.append(out)
        assert res[0]["cycles"] == res[1]["cycles"]
        assert np.array_equal(res[0]["history"], res[1]["history"])
        assert torch.equal(res[0]["x"], res[1]["x"]), prec
    s.close()


def test_bounded_wait_runs_out_and_is_reported(pkg):
    s = pkg.Solver(2, 3, 64, k=5)
    pkg.igamg_set_sweep_form(s.ctx, 1, 1)           # single-launch sweeps on every level
    b = s.rhs_sine(workloads.random_sine_coeffs(2, seed=5, modes=6))
    ref = s.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir")
    assert ref["converged"]
    try:
        # every sweep CTA first waits on a word nothing sets, for 1 ms
        pkg.igamg_set_wait_limit(1e-3, True)
        with pytest.raises(pkg.IgamgError) as e:
            s.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir")
        assert e.value.status == pkg.IGAMG_ETIMEOUT
        x = torch.zeros(s.N, dtype=torch.float32, device=DEV)
        bf = torch.ones(s.N, dtype=torch.float32, device=DEV)
        pkg.igamg_smooth_f32(s.ctx, len(s.levels) - 1, x, bf, 0, s.ws)
        assert pkg.igamg_device_status(s.ctx, s.ws) == pkg.IGAMG_ETIMEOUT
        assert pkg.igamg_device_status(s.ctx, s.ws) == pkg.IGAMG_OK      # the report clears the word
    finally:
        pkg.igamg_set_wait_limit(1.0, False)
    # the context and the GPU stay usable: the same solve again, same result
    again = s.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir")
    assert again["status"] == pkg.IGAMG_OK
    assert torch.equal(again["x"], ref["x"])
    s.close()
