"""Unscaled spaQR variant on the GPU (scaling = 0) against the FP64 oracle.

Bars: interface ranks bit-exact; sigma_p = 1 / sigma_min(A_p) (Lemma 1) to
1e-10 relative; one application of the factor to 1e-10 relative; GMRES to a
relative residual of 1e-12.  The FP32 form states its distance to the FP64
oracle and must still bring GMRES to 1e-12.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2010_06807_gb300 as sq
from oracle import spaqr as osq
from synth.convdiff import batch_problems, config_problem, rhs

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def dev(spaqr_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _colmajor(b, dev):
    return torch.from_numpy(np.ascontiguousarray(b.T)).to(dev).T


def _factor(p, dev, eps, L=0, skip=2, precision="fp64"):
    rp, ci, va = (torch.from_numpy(x).to(dev) for x in (p.rowptr, p.colind, p.val))
    ordl = sq.spaqr_order(rp, ci, p.dims, L)
    F = sq.spaqr_factor(ordl, rp, ci, va, eps=eps, skip=skip, scaling=0, precision=precision)
    return ordl, F, (rp, ci, va)


def _check_ranks_and_sigma(F, Fo):
    for lev, R in enumerate(Fo.ranks):
        pairs, margins = sq.spaqr_factor_ranks(F, lev)
        items = [(c, v) for c, v in sorted(R.items()) if v[0] > 0]
        got = [tuple(x) for x in pairs.tolist()]
        exp = [tuple(v) for _, v in items]
        if got != exp:
            worst = [(g, e, m) for g, e, m in zip(got, exp, margins.tolist()) if g != e]
            raise AssertionError(f"level {lev}: ranks differ {worst[:4]}")
        sg = sq.spaqr_factor_sigmas(F, lev)
        so = np.array([Fo.lemma[lev][c]["sigma"] for c, _ in items])
        assert sg.shape == so.shape
        if so.size:
            np.testing.assert_allclose(sg, so, rtol=TOL, atol=0)


CASES = [
    ("2d_uniform_a", 16, 3, 0.0, 0),
    ("2d_uniform_a", 16, 4, 1e-3, 0),    # fine columns with a leading entry zero up to rounding
    ("2d_uniform_a", 24, 4, 1e-3, 0),
    ("2d_uniform_a", 24, 4, 1e-2, 0),
    ("2d_uniform_a", 33, 0, 1e-3, 1),
    ("2d_lognormal", 40, 5, 1e-2, 2),
    ("2d_lognormal", 64, 0, 1e-1, 2),
    ("3d_uniform_a", 8, 3, 1e-2, 0),
    ("3d_uniform_a", 10, 0, 0.0, 0),
    ("2d_uniform_a", 5, 4, 1e-1, 0),
    ("3d_uniform_a", 16, 0, 1e-2, 2),    # large interfaces: cluster CPQR, long Lanczos runs
]


@pytest.mark.parametrize("kind,n,L,eps,skip", CASES)
def test_unscaled_matches_oracle(dev, kind, n, L, eps, skip):
    p = config_problem(kind, n=n)
    ordl, F, _ = _factor(p, dev, eps, L, skip)
    Fo = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, nlevels=ordl.L, skip=skip, scaling=False)
    _check_ranks_and_sigma(F, Fo)
    b = rhs(p, 3)
    xo = osq.solve(Fo, b)
    xg = sq.spaqr_solve(F, _colmajor(b, dev)).cpu().numpy()
    rel = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert rel <= TOL, rel
    if eps == 0.0:
        res = np.linalg.norm(b - p.matvec(xg), axis=0) / np.linalg.norm(b, axis=0)
        assert res.max() <= 1e-12


@pytest.mark.parametrize("kind,n,eps", [("2d_uniform_a", 64, 1e-3), ("2d_lognormal", 96, 1e-2),
                                        ("3d_uniform_a", 16, 1e-2)])
def test_unscaled_gmres(dev, kind, n, eps):
    p = config_problem(kind, n=n)
    _, F, csr = _factor(p, dev, eps)
    b = rhs(p, 2)
    x, it, rr = sq.spaqr_gmres(F, *csr, _colmajor(b, dev), tol=1e-12)
    assert (rr <= 1e-12).all()
    x = x.cpu().numpy()
    res = np.linalg.norm(b - p.matvec(x), axis=0) / np.linalg.norm(b, axis=0)
    assert res.max() <= 2e-12
    # the oracle's GMRES with the oracle's unscaled factor: same iteration count +-1
    Fo = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, skip=2, scaling=False)
    _, ito, _, _ = osq.gmres(p.n, p.rowptr, p.colind, p.val, b[:, 0], lambda v: osq.solve(Fo, v))
    assert abs(int(it[0]) - ito) <= 1, (it, ito)


def test_unscaled_fp32(dev):
    p = config_problem("3d_uniform_a", n=16)
    eps = 1e-2
    _, F, csr = _factor(p, dev, eps, precision="fp32")
    Fo = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, skip=2, scaling=False)
    b = rhs(p, 1)
    xo = osq.solve(Fo, b)
    xg = sq.spaqr_solve(F, _colmajor(b, dev)).cpu().numpy()
    d = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    print(f"unscaled FP32 factor: one application vs the FP64 oracle {d:.2e}")
    # FP32 rounding may move a rank decision or a pivot: the FP32 factor is
    # then another approximation of A^{-1} of the same order, O(eps) from the
    # FP64 one
    assert d <= eps
    x, it, rr = sq.spaqr_gmres(F, *csr, _colmajor(b, dev), tol=1e-12)
    assert (rr <= 1e-12).all()


def test_unscaled_tuned_and_batched(dev):
    p = config_problem("2d_lognormal", n=64)
    _, F, csr = _factor(p, dev, 1e-2)
    b = _colmajor(rhs(p, 4), dev)
    x0 = sq.spaqr_solve(F, b)
    sq.spaqr_autotune(F, 4)
    x1 = sq.spaqr_solve(F, b)
    assert torch.allclose(x0, x1, rtol=1e-12, atol=1e-12 * float(x0.abs().max()))
    # a block-diagonal batch factors every matrix as it is factored alone
    probs = batch_problems(3, seed=700, sides=(32, 48))
    ob = sq.spaqr_order_batch([(q.rowptr, q.colind) for q in probs], [q.dims for q in probs])
    rp, ci, v = sq.blockdiag_csr([(q.rowptr, q.colind, q.val) for q in probs])
    csrb = [torch.from_numpy(x).to(dev) for x in (rp, ci, v)]
    Fb = sq.spaqr_factor(ob, *csrb, eps=1e-2, scaling=0)
    for k in range(ob.L):
        got = sorted(tuple(x) for x in sq.spaqr_factor_ranks(Fb, k)[0].tolist())
        ref = []
        for q in probs:
            if k < sq.num_levels(q.n):
                _, Fs, _ = _factor(q, dev, 1e-2)
                ref += [tuple(x) for x in sq.spaqr_factor_ranks(Fs, k)[0].tolist()]
        assert got == sorted(ref), k
    B = torch.from_numpy(np.random.default_rng(5).standard_normal(ob.n)).to(dev)
    X, it, rr = sq.spaqr_gmres_batch(Fb, *csrb, ob.part_ptr, B, tol=1e-12)
    assert (rr <= 1e-12).all()
