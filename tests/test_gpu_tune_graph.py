"""Autotuned launch forms and CUDA-graph replay change nothing but speed.

spaqr_autotune picks, per unit of the application, between the one-CTA and
the cluster launch forms; the application after tuning must equal the one by
the rules to rounding (both are the same arithmetic in different launch
shapes).  GMRES with the graph-replayed application must give bit-identical
results to direct launches (the same kernels with the same arguments).
"""
import numpy as np
import pytest

import paper_2010_06807_gb300 as sq
from synth.convdiff import config_problem

pytestmark = pytest.mark.gpu


def _factor(p, precision="fp64"):
    import torch
    csr = [torch.from_numpy(x).cuda() for x in (p.rowptr, p.colind, p.val)]
    o = sq.spaqr_order(p.rowptr, p.colind, p.dims)
    return sq.spaqr_factor(o, *csr, eps=1e-2, precision=precision), csr


@pytest.mark.parametrize("kind,n,nrhs,precision", [("3d_uniform_a", 16, 4, "fp64"),
                                                   ("2d_lognormal", 128, 16, "fp64"),
                                                   ("3d_uniform_a", 20, 1, "fp32")])
def test_autotune_same_result(spaqr_lib, kind, n, nrhs, precision):
    import torch
    p = config_problem(kind, n=n, seed=99)
    F, csr = _factor(p, precision)
    rng = np.random.default_rng(5)
    B = torch.from_numpy(rng.standard_normal((nrhs, p.n))).cuda().T
    X0 = sq.spaqr_solve(F, B).clone()
    ms_rule, ms_tuned = sq.spaqr_autotune(F, nrhs)
    assert ms_rule > 0 and ms_tuned > 0
    X1 = sq.spaqr_solve(F, B)
    tol = 1e-12 if precision == "fp64" else 1e-5
    d = (torch.linalg.norm(X1 - X0) / torch.linalg.norm(X0)).item()
    assert d <= tol, d
    X, it, rr = sq.spaqr_gmres(F, *csr, B, tol=1e-12)
    assert (rr <= 1e-12).all()


def test_graph_replay_bit_identical(spaqr_lib):
    import torch
    p = config_problem("2d_lognormal", n=96, seed=3)
    F, csr = _factor(p)
    rng = np.random.default_rng(6)
    B = torch.from_numpy(rng.standard_normal((3, p.n))).cuda().T
    try:
        sq.spaqr_use_graphs(True)
        Xg, itg, rrg = sq.spaqr_gmres(F, *csr, B, tol=1e-12)
        sq.spaqr_use_graphs(False)
        Xd, itd, rrd = sq.spaqr_gmres(F, *csr, B, tol=1e-12)
    finally:
        sq.spaqr_use_graphs(True)
    assert torch.equal(Xg, Xd)
    np.testing.assert_array_equal(itg, itd)
    np.testing.assert_array_equal(rrg, rrd)


def test_graph_launches_counted(spaqr_lib):
    import torch
    p = config_problem("2d_uniform_a", n=64, seed=4)
    F, csr = _factor(p)
    B = torch.ones(2, p.n, dtype=torch.float64, device="cuda").T
    counts = {}
    for g in (True, False):
        sq.spaqr_use_graphs(g)
        sq.spaqr_stats_reset()
        sq.spaqr_gmres(F, *csr, B, tol=1e-12)
        torch.cuda.synchronize()
        counts[g], per = sq.spaqr_stats()
    sq.spaqr_use_graphs(True)
    assert counts[True] == counts[False] > 0
