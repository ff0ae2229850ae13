"""Mixed-precision form: FP32 factor and application, FP64 GMRES.

The factor and its application run in FP32.  The column scaling, the
Householder scalars, the CPQR rank decisions and GMRES stay in FP64.  The
final GMRES solution must reach ||b - A x|| / ||b|| <= 1e-12.  Its error
against the FP64 oracle's solution is stated and bounded here.  A single FP32
application is compared with the FP64 oracle at FP32 accuracy.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2010_06807_gb300 as sq
from oracle import spaqr as osq
from synth.convdiff import config_problem, rhs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev(spaqr_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _dev_csr(p, dev):
    return (torch.from_numpy(p.rowptr).to(dev), torch.from_numpy(p.colind).to(dev),
            torch.from_numpy(p.val).to(dev))


def _colmajor(b, dev):
    return torch.from_numpy(np.ascontiguousarray(b.T)).to(dev).T


@pytest.mark.parametrize("kind,n,eps", [("2d_uniform_a", 64, 1e-3), ("3d_uniform_a", 16, 1e-2),
                                        ("2d_lognormal", 96, 1e-2)])
def test_fp32_factor_fp64_gmres_against_oracle(dev, kind, n, eps):
    p = config_problem(kind, n=n)
    A = _dev_csr(p, dev)
    ordl = sq.spaqr_order(A[0], A[1], p.dims)
    F32 = sq.spaqr_factor(ordl, *A, eps=eps, precision="fp32")
    Fo = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps)
    b = rhs(p, 2)
    # one FP32 application against the FP64 oracle application: FP32 accuracy
    xo = osq.solve(Fo, b)
    x1 = sq.spaqr_solve(F32, _colmajor(b, dev)).cpu().numpy()
    e1 = np.linalg.norm(x1 - xo, axis=0) / np.linalg.norm(xo, axis=0)
    assert e1.max() < 1e-3, e1
    # FP64 GMRES around the FP32 preconditioner reaches 1e-12
    X, it, rr = sq.spaqr_gmres(F32, *A, _colmajor(b, dev), tol=1e-12)
    x = X.cpu().numpy()
    rel = np.linalg.norm(b - p.matvec(x), axis=0) / np.linalg.norm(b, axis=0)
    assert rel.max() <= 1e-12 and rr.max() <= 1e-12
    # final error against the FP64 oracle's GMRES solution
    for c in range(2):
        xg, ito, rro, _ = osq.gmres(p.n, p.rowptr, p.colind, p.val, b[:, c], lambda v: osq.solve(Fo, v))
        err = np.linalg.norm(x[:, c] - xg) / np.linalg.norm(xg)
        assert err <= 1e-9, err
        assert it[c] <= ito + 3
    # ranks: FP32 pivoting with FP64 |R_kk| reproduces almost every FP64 rank
    same = total = 0
    for lev, R in enumerate(Fo.ranks):
        pairs, _ = sq.spaqr_factor_ranks(F32, lev)
        exp = [v for _, v in sorted(R.items()) if v[0] > 0]
        got = [tuple(x) for x in pairs.tolist()]
        assert len(got) == len(exp)
        for g, e in zip(got, exp):
            total += 1
            same += (g == e)
    assert total == 0 or same >= 0.9 * total


def test_config3_32cube_fp32_vs_fp64(dev):
    """32^3, a ~ U[0.1,10], v = 20 (1,1,1), eps = 1e-2: FP32 and FP64 factors,
    both with FP64 GMRES to 1e-12; the two solutions agree."""
    p = config_problem("3d_uniform_a", n=32)
    A = _dev_csr(p, dev)
    ordl = sq.spaqr_order(A[0], A[1], p.dims)
    assert ordl.L == 9
    b = rhs(p, 2)
    out = {}
    for prec in ("fp64", "fp32"):
        F = sq.spaqr_factor(ordl, *A, eps=1e-2, precision=prec)
        X, it, rr = sq.spaqr_gmres(F, *A, _colmajor(b, dev), tol=1e-12)
        x = X.cpu().numpy()
        rel = np.linalg.norm(b - p.matvec(x), axis=0) / np.linalg.norm(b, axis=0)
        assert rel.max() <= 1e-12
        out[prec] = (x, it)
    d = np.linalg.norm(out["fp32"][0] - out["fp64"][0], axis=0) / np.linalg.norm(out["fp64"][0], axis=0)
    assert d.max() <= 1e-9, d
    assert out["fp32"][1].max() <= out["fp64"][1].max() + 3
