"""The restart loop of Algorithm 5 on the GPU (a conditional WHILE graph node
whose last kernel applies the accuracy test) against the host-driven loop
(one graph launch and one residual read per restart cycle): the same kernels
in the same order, so iterates, residual histories and cycle counts must be
bitwise equal -- single problems and batches, every stopping reason."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build_library()
    import paper_2412_20205_gb300 as p
    assert torch.cuda.is_available()
    return p


def _both(s, b, **kw):
    dev = s.solve(b, **kw)
    host = s.solve(b, host_loop=True, **kw)
    return dev, host


@pytest.mark.parametrize("dim,n,p,method,k,prec", [
    (2, 64, 2, "rre", 5, "fp64"), (2, 64, 2, "rre", 5, "fp32_ir"), (2, 100, 3, "mpe", 8, "fp64"),
    (2, 37, 4, "none", 1, "fp32_ir"), (3, 16, 3, "rre", 10, "fp32_ir"), (3, 12, 2, "mpe", 5, "fp64")])
def test_device_loop_equals_host_loop(pkg, dim, n, p, method, k, prec):
    s = pkg.Solver(dim, p, n, k=max(k, 1))
    b = s.rhs_sine(workloads.random_sine_coeffs(dim, seed=9, modes=6))
    kw = dict(tol=1e-10, method=method, k=k, prec=prec, max_cycles=300)
    dev, host = _both(s, b, **kw)
    assert dev["status"] == host["status"] == pkg.IGAMG_OK
    assert dev["cycles"] == host["cycles"] and dev["vcycles"] == host["vcycles"]
    assert np.array_equal(dev["history"], host["history"])
    assert torch.equal(dev["x"], host["x"])
    # stopping at max_cycles: ENOTCONV, same iterate and history
    dev, host = _both(s, b, **dict(kw, max_cycles=2, tol=1e-30))
    assert dev["status"] == host["status"] == pkg.IGAMG_ENOTCONV
    assert dev["cycles"] == host["cycles"] == 2
    assert np.array_equal(dev["history"], host["history"])
    assert torch.equal(dev["x"], host["x"])
    s.close()


def test_device_loop_launch_accounting_and_repeat(pkg):
    """Repeated solves reuse the captured loop; the launch count per solve is
    the restart cycle's kernels times the cycles run (plus the set-up kernels)."""
    s = pkg.Solver(2, 3, 48, k=5)
    b = s.rhs_sine(workloads.random_sine_coeffs(2, seed=1, modes=4))
    outs = []
    for _ in range(3):
        l0 = pkg.igamg_launch_count()
        outs.append(s.solve(b, tol=1e-10, method="rre", k=5, prec="fp32_ir"))
        outs[-1]["launches"] = pkg.igamg_launch_count() - l0
    assert all(o["status"] == pkg.IGAMG_OK for o in outs)
    assert all(torch.equal(o["x"], outs[0]["x"]) for o in outs)
    assert outs[1]["launches"] == outs[2]["launches"] > 10 * outs[1]["cycles"]
    s.close()


@pytest.mark.parametrize("prec", ["fp32_ir", "fp64"])
def test_batch_device_loop_equals_host_rounds(pkg, prec):
    ps = [2, 3, 4, 3, 2]
    ns = [33, 40, 24, 17, 64]
    coeffs = np.stack([workloads.random_sine_coeffs(2, seed=50 + i, modes=6) for i in range(len(ps))])
    coeffs[3] = 0.0                                  # a zero right side: converged at s_0 = 0
    B = pkg.Batch(2, ps, ns, k=5)
    b = B.rhs_sine(coeffs)
    pkg.igamg_batch_set_device_loop(B.handle, True)
    dev = B.solve(b, tol=1e-10, method="rre", k=5, prec=prec)
    xd = dev["x"].clone()
    pkg.igamg_batch_set_device_loop(B.handle, False)
    host = B.solve(b, tol=1e-10, method="rre", k=5, prec=prec)
    assert dev["converged"] and host["converged"]
    assert dev["cycles"] == host["cycles"] and dev["cycles"][3] == 0
    assert np.array_equal(dev["residuals"], host["residuals"])
    assert torch.equal(xd, host["x"])
    B.close()
