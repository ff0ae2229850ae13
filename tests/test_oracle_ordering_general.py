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
  * eps = 0 solves exactly; GMRES converges on the general matrices.
"""
import numpy as np
import pytest

from oracle import spaqr
from oracle.ordering_general import column_graph, level_structure, nd_general, row_matching
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
