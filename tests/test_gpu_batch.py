"""Batched factorisation and GMRES on the GPU against the one-matrix path.

A batch ordering + spaqr_factor on the block-diagonal CSR runs every level's
fronts of all matrices in the same launches; each matrix's factorisation must
be the one it gets alone: the same ranks at every level (bit for bit), the
same preconditioner application (to rounding) and, through
spaqr_gmres_batch, the same solutions (1e-10 relative) with every matrix's own
residual at 1e-12.
"""
import numpy as np
import pytest

import paper_2010_06807_gb300 as sq
from synth.convdiff import batch_problems, config_problem

pytestmark = pytest.mark.gpu


def _batch(probs, precision="fp64", eps=1e-2):
    import torch
    dev = torch.device("cuda:0")
    ob = sq.spaqr_order_batch([(p.rowptr, p.colind) for p in probs], [p.dims for p in probs])
    rp, ci, v = sq.blockdiag_csr([(p.rowptr, p.colind, p.val) for p in probs])
    csr = [torch.from_numpy(x).to(dev) for x in (rp, ci, v)]
    F = sq.spaqr_factor(ob, *csr, eps=eps, precision=precision)
    return ob, F, csr


def _single(p, precision="fp64", eps=1e-2):
    import torch
    dev = torch.device("cuda:0")
    o = sq.spaqr_order(p.rowptr, p.colind, p.dims)
    csr = [torch.from_numpy(x).to(dev) for x in (p.rowptr, p.colind, p.val)]
    return o, sq.spaqr_factor(o, *csr, eps=eps, precision=precision), csr


def _probs():
    ps = batch_problems(6, seed=4000, sides=(32, 48, 64))
    ps.append(config_problem("2d_uniform_a", n=16, seed=5))
    return ps


def test_batch_ranks_equal_single(spaqr_lib):
    probs = _probs()
    ob, F, _ = _batch(probs)
    singles = [_single(p)[1] for p in probs]
    for k in range(ob.L):
        pairs_b, _ = sq.spaqr_factor_ranks(F, k)
        ref = []
        for p, Fs in zip(probs, singles):
            if k < sq.num_levels(p.n):
                ref += [tuple(x) for x in sq.spaqr_factor_ranks(Fs, k)[0]]
        assert sorted(tuple(x) for x in pairs_b) == sorted(ref), k


@pytest.mark.parametrize("nrhs", [1, 3])
def test_batch_apply_equals_single(spaqr_lib, nrhs):
    import torch
    probs = _probs()
    ob, F, _ = _batch(probs)
    rng = np.random.default_rng(11)
    Bh = np.asfortranarray(rng.standard_normal((ob.n, nrhs)))
    B = torch.from_numpy(np.ascontiguousarray(Bh.T)).cuda().T
    X = sq.spaqr_solve(F, B).T.cpu().numpy().T
    for i, p in enumerate(probs):
        a, b = ob.part_ptr[i], ob.part_ptr[i + 1]
        _, Fs, _ = _single(p)
        Bs = torch.from_numpy(np.ascontiguousarray(Bh[a:b].T)).cuda().T
        Xs = sq.spaqr_solve(Fs, Bs).T.cpu().numpy().T
        np.testing.assert_allclose(X[a:b], Xs, rtol=0, atol=1e-12 * np.abs(Xs).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_gmres_equals_single(spaqr_lib, precision):
    import torch
    probs = _probs()
    ob, F, csr = _batch(probs, precision)
    nrhs = 2
    rng = np.random.default_rng(12)
    Bh = np.asfortranarray(rng.standard_normal((ob.n, nrhs)))
    B = torch.from_numpy(np.ascontiguousarray(Bh.T)).cuda().T
    X, it, rr = sq.spaqr_gmres_batch(F, *csr, ob.part_ptr, B, tol=1e-12)
    assert it.shape == (nrhs, len(probs)) and (rr <= 1e-12).all()
    X = X.T.cpu().numpy().T
    for i, p in enumerate(probs):
        a, b = ob.part_ptr[i], ob.part_ptr[i + 1]
        # the matrix's own residual
        for c in range(nrhs):
            res = np.linalg.norm(Bh[a:b, c] - p.matvec(X[a:b, c])) / np.linalg.norm(Bh[a:b, c])
            assert res <= 2e-12, (i, c, res)
        _, Fs, cs = _single(p, "fp64")
        Bs = torch.from_numpy(np.ascontiguousarray(Bh[a:b].T)).cuda().T
        Xs, its, rrs = sq.spaqr_gmres(Fs, *cs, Bs, tol=1e-12)
        Xs = Xs.T.cpu().numpy().T
        d = np.linalg.norm(X[a:b] - Xs) / np.linalg.norm(Xs)
        assert d <= 1e-10, (i, d)
        if precision == "fp64":
            assert (np.abs(it[:, i] - its) <= 1).all()


def test_batch_gmres_bad_parts(spaqr_lib):
    import torch
    probs = _probs()[:2]
    ob, F, csr = _batch(probs)
    B = torch.ones(ob.n, dtype=torch.float64, device="cuda")
    with pytest.raises(sq.SpaqrError):
        sq.spaqr_gmres_batch(F, *csr, np.array([0, 5, 5, ob.n]), B)
    with pytest.raises(sq.SpaqrError):
        sq.spaqr_gmres_batch(F, *csr, np.array([0, ob.n - 1]), B)


def test_batch_of_one_is_the_single_factor(spaqr_lib):
    import torch
    p = config_problem("2d_lognormal", n=48, seed=21)
    ob, F, csr = _batch([p])
    _, Fs, cs = _single(p)
    B = torch.from_numpy(np.random.default_rng(3).standard_normal((2, p.n))).cuda().T
    X = sq.spaqr_solve(F, B)
    Xs = sq.spaqr_solve(Fs, B)
    assert torch.equal(X, Xs)


def test_batch_mixing_2d_and_3d(spaqr_lib):
    import torch
    probs = [config_problem("3d_uniform_a", n=10, seed=31), config_problem("2d_uniform_a", n=40, seed=32),
             config_problem("3d_uniform_a", n=6, seed=33)]
    ob, F, csr = _batch(probs)
    B = torch.from_numpy(np.random.default_rng(4).standard_normal(ob.n)).cuda()
    X, it, rr = sq.spaqr_gmres_batch(F, *csr, ob.part_ptr, B, tol=1e-12)
    assert (rr <= 1e-12).all()
    X = X.cpu().numpy()
    Bh = B.cpu().numpy()
    for i, p in enumerate(probs):
        a, b = ob.part_ptr[i], ob.part_ptr[i + 1]
        _, Fs, cs = _single(p)
        Xs, _, _ = sq.spaqr_gmres(Fs, *cs, torch.from_numpy(Bh[a:b].copy()).cuda(), tol=1e-12)
        d = np.linalg.norm(X[a:b] - Xs.cpu().numpy()) / np.linalg.norm(Xs.cpu().numpy())
        assert d <= 1e-10, (i, d)


def test_batch_at_config_scale_against_oracle(spaqr_lib):
    """The 64-matrix batch of the batched configuration (sides 32 to 128,
    a ~ U[0.1, 10], Pe ~ U[1, 100]), factored together in FP64 at eps 1e-2:
    three sampled matrices (the largest side, a middle one and the smallest)
    against the oracle on that matrix alone.  Their ranks at every level are
    among the batch's ranks of that level, and the batch factor applied to a
    right-hand side that is nonzero on one matrix only equals the oracle's
    application entry by entry to 1e-10 there and is exactly zero on every
    other matrix."""
    import torch
    from oracle import spaqr as osq
    probs = batch_problems(64)
    ob, F, _ = _batch(probs)
    sides = [p.dims[0] for p in probs]
    order = np.argsort(sides, kind="stable")
    picks = [int(order[-1]), int(order[len(order) // 2]), int(order[0])]
    batch_ranks = [[tuple(x) for x in sq.spaqr_factor_ranks(F, k)[0]] for k in range(ob.L)]
    for i in picks:
        p = probs[i]
        Fo = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 1e-2)
        for k, R in enumerate(Fo.ranks):
            pool = list(batch_ranks[k])
            for e in (v for _, v in sorted(R.items()) if v[0] > 0):
                assert e in pool, (i, k, e)
                pool.remove(e)
        a, b = int(ob.part_ptr[i]), int(ob.part_ptr[i + 1])
        Bh = np.zeros((ob.n, 2))
        Bh[a:b] = np.random.default_rng(100 + i).standard_normal((b - a, 2))
        B = torch.from_numpy(np.ascontiguousarray(Bh.T)).cuda().T
        X = sq.spaqr_solve(F, B).T.cpu().numpy().T
        xo = osq.solve(Fo, Bh[a:b])
        err = np.abs(X[a:b] - xo).max(axis=0) / np.abs(xo).max(axis=0)
        assert err.max() <= 1e-10, (i, err)
        assert np.all(X[:a] == 0.0) and np.all(X[b:] == 0.0)
