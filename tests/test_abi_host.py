"""The C-ABI library loads, exports every symbol include/igamg.h declares, and
its host-side set-up (knots, quadrature, 1D factors, knot-insertion transfer)
matches the oracle.  No GPU needed: igamg_setup and igamg_get_factor are host
only."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import bspline as bs
from oracle import galerkin as gk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def igamg():
    import __graft_entry__ as g
    g.build_library()
    import paper_2412_20205_gb300 as pkg
    return pkg


def _declared():
    text = open(os.path.join(ROOT, "include", "igamg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(igamg_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(igamg):
    names = _declared()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", igamg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = igamg.lib()
    for n in names:
        getattr(lib, n)


def _band_to_dense(band, p):
    m = band.shape[0]
    A = np.zeros((m, m))
    for i in range(m):
        for k in range(2 * p + 1):
            j = i + k - p
            if 0 <= j < m:
                A[i, j] = band[i, k]
    return A


@pytest.mark.parametrize("dim,n,p", [(2, 16, 1), (2, 24, 2), (2, 33, 3), (3, 12, 4), (2, 40, 7)])
def test_host_factors_and_transfer_match_oracle(igamg, dim, n, p):
    ctx = igamg.igamg_setup(dim, p, [n] * dim, 0)
    try:
        levels = igamg.igamg_info(ctx)
        br = bs.uniform_breaks(n)
        chain = [br]
        while len(chain[-1]) - 1 > 8:
            chain.append(bs.coarsen_breaks(chain[-1]))
        chain = chain[::-1]
        assert len(levels) == len(chain)
        for l, b in enumerate(chain):
            M, K = gk.factors_1d(b, p)
            assert levels[l][0] == M.shape[0]
            for d in range(dim):
                Mb = _band_to_dense(igamg.igamg_get_factor(ctx, l, d, 0), p)
                Kb = _band_to_dense(igamg.igamg_get_factor(ctx, l, d, 1), p)
                assert np.allclose(Mb, M, rtol=0, atol=1e-15 * np.abs(M).max() * 10)
                assert np.allclose(Kb, K, rtol=0, atol=1e-13 * np.abs(K).max())
                if l > 0:
                    P = igamg.igamg_get_factor(ctx, l, d, 2)
                    Po = gk.prolongation_1d(b, chain[l - 1], p)[1]
                    assert np.allclose(P, Po, atol=1e-13)
    finally:
        igamg.igamg_destroy(ctx)


@pytest.mark.parametrize("args", [(1, 2, 16, 0), (2, 0, 16, 0), (2, 8, 16, 0), (2, 2, 1, 0), (2, 2, 16, 9)])
def test_setup_rejects_bad_arguments(igamg, args):
    dim, p, n, nl = args
    with pytest.raises(igamg.IgamgError) as e:
        igamg.igamg_setup(dim, p, [n] * max(dim, 1), nl)
    assert e.value.status == igamg.IGAMG_EINVAL


def test_workspace_size_query_is_positive_and_grows_with_k(igamg):
    ctx = igamg.igamg_setup(2, 3, [64, 64], 0)
    try:
        a = igamg.igamg_workspace_bytes(ctx, 5, igamg.IGAMG_FP64)
        b = igamg.igamg_workspace_bytes(ctx, 10, igamg.IGAMG_FP64)
        c = igamg.igamg_workspace_bytes(ctx, 10, igamg.IGAMG_FP32_IR)
        assert 0 < a < b < c
        assert igamg.igamg_workspace_bytes(ctx, 99, igamg.IGAMG_FP64) == 0
    finally:
        igamg.igamg_destroy(ctx)
