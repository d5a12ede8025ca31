"""Batched solve of uneven problems: every problem's result equals its own
igamg_solve (same kernels, same inputs), its cycle count matches, and one
problem is checked against the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from oracle import solver as osolver  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build_library()
    import paper_2412_20205_gb300 as p
    assert torch.cuda.is_available()
    return p


@pytest.mark.parametrize("prec", ["fp32_ir", "fp64"])
def test_batch_matches_individual_solves(pkg, prec):
    ps = [2, 3, 4, 2, 3, 4, 3]
    ns = [20, 33, 24, 17, 40, 9, 64]
    coeffs = np.stack([workloads.random_sine_coeffs(2, seed=1000 + i, modes=6) for i in range(len(ps))])
    B = pkg.Batch(2, ps, ns, k=5)
    b = B.rhs_sine(coeffs)
    out = B.solve(b, tol=1e-10, method="rre", k=5, prec=prec)
    assert out["converged"], out["statuses"]
    x = out["x"].cpu().numpy()
    for i, (p, n) in enumerate(zip(ps, ns)):
        s = pkg.Solver(2, p, n, k=5)
        bi = s.rhs_sine(coeffs[i])
        o = s.solve(bi, tol=1e-10, method="rre", k=5, prec=prec)
        xi = o["x"].cpu().numpy()
        seg = x[B.offsets[i]:B.offsets[i + 1]]
        assert o["cycles"] == out["cycles"][i]
        assert np.linalg.norm(seg - xi) <= 1e-13 * np.linalg.norm(xi)
        assert out["residuals"][i] <= 1e-10
        s.close()
    # one member against the oracle
    prob = osolver.Problem(2, 33, 3, coeffs[1])
    ref = osolver.solve(prob, "rre", k=5, tol=1e-10, max_cycles=60)
    assert abs(ref["cycles"] - out["cycles"][1]) <= 1
    seg = x[B.offsets[1]:B.offsets[2]]
    assert np.linalg.norm(seg - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])
    B.close()


def test_batch_zero_rhs_member(pkg):
    ps, ns = [2, 3], [16, 20]
    coeffs = np.stack([workloads.random_sine_coeffs(2, seed=5, modes=4), np.zeros((4, 4))])
    B = pkg.Batch(2, ps, ns, k=5)
    b = B.rhs_sine(coeffs)
    out = B.solve(b, tol=1e-10, method="mpe", k=5)
    assert out["converged"] and out["cycles"][1] == 0
    x = out["x"].cpu().numpy()
    assert np.all(x[B.offsets[1]:B.offsets[2]] == 0.0)
    B.close()


def test_bench_batch_path_runs(pkg):
    """bench.py's batched workload end to end on a 4-problem batch: one JSON
    line with every problem converged (guards the bench path itself)."""
    import io
    import json
    import sys
    import contextlib
    import bench
    old = sys.argv
    sys.argv = ["bench.py", "--workload", "batch256", "--batch-count", "4", "--steps", "1", "--warmup", "1",
                "--no-cpu-baseline"]
    try:
        a = bench.parse()
    finally:
        sys.argv = old
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_batch(a, 0, 1, 0)
    lines = [l for l in buf.getvalue().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["converged"] and line["value"] > 0 and line["config"]["problems"] == 4
    assert line["gpu_launches"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 8 * line["config"]["total_dof"]
