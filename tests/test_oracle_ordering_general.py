"""Pins for the oracle's ordering of general sparse matrices
(oracle/ordering_general.py): what nested dissection on G(A^T A) and the
matching must satisfy, checked by brute force on explicit A^T A.

  * every separator separates: no A^T A coupling between the column sets of
    a node's two child subtrees (Section 2.1);
  * the separator of a node is a breadth-first level: the columns of its
    node set split into levels with couplings only between neighbouring
    levels;
  * perm is a permutation, atoms partition every node, interfaces nest from
    stage to stage and a separator is one cluster when it is eliminated;
  * blocks of A only couple related nodes, once rows sit with their matched
    columns;
  * the matching is perfect, uses nonzeros, is the identity on a row
    diagonally dominant matrix and undoes a row permutation;
  * the maximum-product matching reaches the largest product of |a_ij| over
    all permutations (brute force on small matrices) and the optimum of
    scipy's minimum-weight bipartite matching on the same costs;
  * eps = 0 solves exactly; GMRES converges on the general matrices.
"""
import numpy as np
import pytest

from oracle import spaqr
from oracle.ordering_general import (column_graph, level_structure, nd_general, row_matching,
                                     row_matching_max_product)
from synth.convdiff import config_problem, permuted, random_local, rhs


def _AtA(p):
    A = p.to_dense() != 0
    return (A.T.astype(int) @ A.astype(int)) > 0


def _subtree_cols(o, nd):
    out = []
    stack = [nd]
    while stack:
        x = stack.pop()
        if x is None:
            continue
        out += list(x.pts)
        stack += [x.left, x.right]
    return out


def _problems():
    g = config_problem("2d_uniform_a", n=20)
    return [("grid", g, 4), ("permuted", permuted(g, 11), 4), ("random_local", random_local(18, seed=7001), 4),
            ("random_local_L5", random_local(24, seed=7002), 5)]


@pytest.mark.parametrize("name,p,L", _problems())
def test_separators_separate(name, p, L):
    o = nd_general(p.n, p.rowptr, p.colind, p.val, L)
    S = _AtA(p)
    assert sorted(o.perm.tolist()) == list(range(p.n))
    for nd in o.nodes:
        if nd.left is None:
            continue
        lc, rc = _subtree_cols(o, nd.left), _subtree_cols(o, nd.right)
        if lc and rc:
            assert not S[np.ix_(lc, rc)].any(), (name, nd.id)


def test_level_structure_is_layered():
    p = random_local(16, seed=7003)
    adj = column_graph(p.n, p.rowptr, p.colind)
    V = list(range(0, p.n, 2)) + [1, 3, 5]
    lv = level_structure(V, adj, p.n)
    pos = {}
    for i, level in enumerate(lv):
        for x in level:
            pos[x] = i
    assert sorted(pos) == sorted(V)
    S = _AtA(p)
    for x in V:
        for y in V:
            if x != y and S[x, y]:
                assert abs(pos[x] - pos[y]) <= 1


@pytest.mark.parametrize("name,p,L", _problems())
def test_atoms_interfaces_and_blocks(name, p, L):
    o = nd_general(p.n, p.rowptr, p.colind, p.val, L)
    # atoms of a node are contiguous and partition it
    for nd in o.nodes:
        idx = [a for a in range(o.n_atoms) if o.atom_node[a] == nd.id]
        if idx:
            assert idx == list(range(idx[0], idx[-1] + 1))
            got = np.concatenate([o.perm[o.atom_ptr[a]:o.atom_ptr[a + 1]] for a in idx])
            assert sorted(got.tolist()) == sorted(nd.pts)
    # interfaces nest: a cluster at stage s is a union of clusters at stage s + 1
    for s in range(L - 1):
        coarse = o.stage_clusters(s)
        fine = set(o.stage_clusters(s + 1))
        for a0, a1 in coarse:
            b = a0
            while b < a1:
                nxt = [f for f in fine if f[0] == b]
                assert len(nxt) == 1
                b = nxt[0][1]
            assert b == a1
    # at its elimination stage a separator is one cluster
    for nd in o.nodes:
        cl = [c for c in o.stage_clusters(nd.depth) if o.atom_node[c[0]] == nd.id]
        assert len(cl) <= 1
    # blocks couple related nodes only (rows with their matched columns)
    iperm = np.empty(p.n, dtype=np.int64)
    iperm[o.perm] = np.arange(p.n)
    atom_of = np.searchsorted(o.atom_ptr, np.arange(p.n), side="right") - 1
    for r in range(p.n):
        ar = o.atom_node[atom_of[iperm[o.rowcol[r]]]]
        for c in p.colind[p.rowptr[r]:p.rowptr[r + 1]]:
            assert o.related(ar, o.atom_node[atom_of[iperm[c]]])


def test_matching():
    g = config_problem("2d_uniform_a", n=12)
    np.testing.assert_array_equal(row_matching(g.n, g.rowptr, g.colind, g.val), np.arange(g.n))
    q = permuted(g, 3, rows=True, cols=False)
    rc = row_matching(q.n, q.rowptr, q.colind, q.val)
    # row r of q is row prow[r] of g, whose diagonal sits in column prow[r]
    np.testing.assert_array_equal(rc, q.prow)
    # perfect and on nonzeros, also with the pattern only (augmenting paths)
    p = random_local(10, seed=7004)
    rc = row_matching(p.n, p.rowptr, p.colind, None)
    assert sorted(rc.tolist()) == list(range(p.n))
    A = p.to_dense()
    assert all(A[r, rc[r]] != 0 for r in range(p.n))
    # a structurally singular pattern is rejected
    rp = np.array([0, 1, 2, 3], dtype=np.int64)
    ci = np.array([0, 0, 2], dtype=np.int64)
    with pytest.raises(ValueError):
        row_matching(3, rp, ci, None)


@pytest.mark.parametrize("name,p,L", _problems())
def test_general_factor_exact_and_gmres(name, p, L):
    o = nd_general(p.n, p.rowptr, p.colind, p.val, L)
    F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, None, 0.0, ordering=o, skip=0)
    b = np.random.default_rng(5).standard_normal((p.n, 2))
    x = spaqr.solve(F, b)
    assert np.max(np.linalg.norm(b - p.matvec(x), axis=0) / np.linalg.norm(b, axis=0)) < 1e-12
    F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, None, 1e-2, ordering=o, skip=1)
    x, it, rr, _ = spaqr.gmres(p.n, p.rowptr, p.colind, p.val, b[:, 0], lambda v: spaqr.solve(F, v))
    assert rr <= 1e-12


def test_permuted_generator_is_PAQ():
    g = config_problem("2d_uniform_a", n=9)
    q = permuted(g, 17)
    A = g.to_dense()
    B = q.to_dense()
    # row r of B is row prow[r] of A; column c of B is column pcol[c] of A
    np.testing.assert_array_equal(B, A[np.ix_(q.prow, q.pcol)])
    assert q.dims is None


def _logprod(A, rc):
    return float(np.log(np.abs(A[np.arange(A.shape[0]), rc])).sum())


def test_max_product_matching_brute_force():
    """Small random unsymmetric matrices with values spread over decades:
    the matching is the permutation with the largest product of |a_ij|
    (unique with probability one), found by trying all of them."""
    import itertools
    rng = np.random.default_rng(41)
    for t in range(12):
        n = int(rng.integers(3, 8))
        M = np.where(rng.random((n, n)) < 0.45, rng.lognormal(0.0, 2.0, (n, n)) * rng.choice([-1, 1], (n, n)), 0.0)
        M[np.arange(n), rng.permutation(n)] = rng.lognormal(0.0, 2.0, n)
        rp = np.concatenate([[0], np.cumsum((M != 0).sum(1))])
        ci = np.concatenate([np.nonzero(M[r])[0] for r in range(n)])
        va = np.concatenate([M[r][M[r] != 0] for r in range(n)])
        best = max(itertools.permutations(range(n)), key=lambda pm: np.prod(np.abs(M[np.arange(n), list(pm)])))
        rc = row_matching_max_product(n, rp, ci, va)
        assert tuple(rc.tolist()) == best, t


def test_max_product_matching_against_scipy():
    """The optimum of scipy's minimum-weight full bipartite matching on the
    costs 1 + log max_k |a_kj| - log |a_ij| (the constant keeps every
    weight positive and shifts every perfect matching alike) equals the
    oracle's matched log-product."""
    scipy_sparse = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for nside, w, seed in ((20, 0.1, 7021), (28, 0.05, 7022), (24, None, 7023)):
        p = random_local(nside, seed=seed, weak_diag=w)
        A = p.to_dense()
        C = scipy_sparse.coo_matrix(np.abs(A))
        amax = np.abs(A).max(axis=0)
        W = scipy_sparse.csr_matrix((1.0 + np.log(amax[C.col]) - np.log(C.data), (C.row, C.col)), shape=A.shape)
        r, c = csgraph.min_weight_full_bipartite_matching(W)
        rc = row_matching_max_product(p.n, p.rowptr, p.colind, p.val)
        assert sorted(rc.tolist()) == list(range(p.n))
        assert _logprod(A, rc) == pytest.approx(_logprod(A, c[np.argsort(r)]), rel=1e-12, abs=1e-9)
        # never below the greedy matching's product
        assert _logprod(A, rc) >= _logprod(A, row_matching(p.n, p.rowptr, p.colind, p.val)) - 1e-9


def test_max_product_matching_special_cases():
    g = config_problem("2d_uniform_a", n=12)
    np.testing.assert_array_equal(row_matching_max_product(g.n, g.rowptr, g.colind, g.val), np.arange(g.n))
    q = permuted(g, 5, rows=True, cols=False)
    np.testing.assert_array_equal(row_matching_max_product(q.n, q.rowptr, q.colind, q.val), q.prow)
    # pattern only: every cost is 0, any perfect matching is optimal
    p = random_local(12, seed=7024, weak_diag=0.1)
    rc = row_matching_max_product(p.n, p.rowptr, p.colind, None)
    assert sorted(rc.tolist()) == list(range(p.n))
    A = p.to_dense()
    assert all(A[r, rc[r]] != 0 for r in range(p.n))
    rp = np.array([0, 1, 2, 3], dtype=np.int64)
    with pytest.raises(ValueError):
        row_matching_max_product(3, rp, np.array([0, 0, 2], dtype=np.int64), None)


def test_max_product_ordering_factor_and_gmres():
    """On a matrix whose large entries are off the diagonal, the ordering
    with the maximum-product matching factors exactly at eps = 0 and
    preconditions GMRES in fewer iterations than the greedy matching at
    eps = 1e-2 (the paper's reason to put large entries on the diagonal:
    well-conditioned diagonal blocks)."""
    p = random_local(20, seed=7010, weak_diag=0.1)
    b = np.random.default_rng(5).standard_normal(p.n)
    its = {}
    for m in ("greedy", "max_product"):
        o = nd_general(p.n, p.rowptr, p.colind, p.val, 4, matching=m)
        F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, None, 0.0, ordering=o, skip=0)
        x = spaqr.solve(F, b)
        assert np.linalg.norm(b - p.matvec(x)) <= 1e-12 * np.linalg.norm(b)
        F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, None, 1e-2, ordering=o, skip=1)
        _, its[m], rr, _ = spaqr.gmres(p.n, p.rowptr, p.colind, p.val, b, lambda v: spaqr.solve(F, v))
        assert rr <= 1e-12
    assert its["max_product"] < its["greedy"], its


@pytest.mark.parametrize("matching", ["greedy", "max_product"])
@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-3])
def test_preconditioned_operator_O_eps_on_grid_free_orderings(matching, eps):
    """Section 3.3 on grid-free orderings: the right-preconditioned operator
    is I + O(eps), ||A M^{-1} - I||_2 < 20 eps as on grids (a permuted grid
    matrix and a diagonally dominant random local one; something dropped)."""
    for p in (permuted(config_problem("2d_uniform_a", n=24), 71), random_local(20, seed=7070)):
        o = nd_general(p.n, p.rowptr, p.colind, p.val, 4, matching=matching)
        F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, None, eps, nlevels=4, skip=0, ordering=o)
        AM = p.to_dense() @ spaqr.solve(F, np.eye(p.n))
        assert np.linalg.norm(AM - np.eye(p.n), 2) < 20 * eps
        assert any(r < nb for R in F.ranks for (nb, r) in R.values())


def _golden_path(case):
    rp = np.concatenate([[0], np.cumsum([len(r) for r in case["rows"]])]).astype(np.int64)
    ci = np.asarray([c for r in case["rows"] for c, _ in r], dtype=np.int32)
    va = np.asarray([v for r in case["rows"] for _, v in r], dtype=np.float64)
    return rp, ci, va


def test_golden_hand_derived_paths():
    """Hand-derived orderings (tests/golden/general_paths.json, derived from
    the readings G1-G5 and R6, not by code): tridiagonal matrices and a case
    where a separator column touches both child subtrees of a node but not
    its separator; separators, atoms, their order and the matched rows."""
    import json
    import os
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "general_paths.json")))
    for case in golden["cases"]:
        rp, ci, va = _golden_path(case)
        o = nd_general(case["n"], rp, ci, va, case["L"])
        assert [list(nd.pts) for nd in o.nodes] == case["node_pts"], case["name"]
        for k in ("perm", "atom_ptr", "atom_node", "rperm"):
            assert getattr(o, k).tolist() == case[k], (case["name"], k)
