"""Pins for the oracle's geometric modified nested dissection (oracle/ordering.py).

Brute force on small grids: the ordering is a permutation; every separator
really separates its two subdomains in G(A^T A) (A^T A formed explicitly);
interfaces partition separators and nest across merge stages; a hand-derived
16x16 case (tests/golden/nd_16x16_L3.json).
"""
import json
import os

import numpy as np
import pytest

from oracle.ordering import nd_order, num_levels
from synth.convdiff import config_problem

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_num_levels_rule():
    # ceil(log2(N/64)) (Section 4)
    assert num_levels(4096) == 6
    assert num_levels(65536) == 10
    assert num_levels(32768) == 9
    assert num_levels(64) == 1
    assert num_levels(100) == 1


def test_golden_16x16():
    g = json.load(open(os.path.join(GOLD, "nd_16x16_L3.json")))
    o = nd_order(tuple(g["dims"]), g["L"])
    sizes = [o.atom_size(a) for a in range(o.n_atoms)]
    assert sizes == g["atom_sizes"]
    assert [int(o.node_level[o.atom_node[a]]) for a in range(o.n_atoms)] == g["atom_level"]
    root_atoms = [a for a in range(o.n_atoms) if o.atom_node[a] == 0]
    firsts = []
    for a in root_atoms:
        gi = o.perm[o.atom_ptr[a]]
        firsts.append([int(gi % 16), int(gi // 16)])
    assert firsts == g["root_atom_first_points"]
    root_cl = lambda st: [c for c in o.stage_clusters(st) if o.atom_node[c[0]] == 0]
    assert len(root_cl(0)) == g["root_stage0_clusters"]
    assert len(root_cl(1)) == g["root_stage1_clusters"]


def _ata_pattern(p):
    A = p.to_dense() != 0
    return (A.T.astype(np.int64) @ A.astype(np.int64)) != 0


@pytest.mark.parametrize("dims,L", [((16, 16), 3), ((20, 13), 4), ((24, 24), 4),
                                    ((8, 8, 8), 3), ((9, 7, 6), 3)])
def test_nd_separators_separate_in_AtA(dims, L):
    kind = "2d_uniform_a" if len(dims) == 2 else "3d_uniform_a"
    n = dims[0]
    o = nd_order(dims, L)
    N = int(np.prod(dims))
    assert sorted(o.perm.tolist()) == list(range(N))
    # build an A with the right stencil on this (possibly non-cubic) grid
    from synth.convdiff import convdiff
    rng = np.random.Generator(np.random.PCG64(1))
    rp, ci, va = _stencil(dims)
    A = np.zeros((N, N), dtype=bool)
    for r in range(N):
        A[r, ci[rp[r]:rp[r + 1]]] = True
    S = (A.T.astype(np.int64) @ A.astype(np.int64)) != 0
    # node -> set of grid points in its subtree
    node_pts = {}
    for a in range(o.n_atoms):
        node_pts.setdefault(int(o.atom_node[a]), []).extend(
            o.perm[o.atom_ptr[a]:o.atom_ptr[a + 1]].tolist())
    nodes = o.nodes

    def subtree_pts(nd):
        if nd is None:
            return []
        return node_pts.get(nd.id, []) + subtree_pts(nd.left) + subtree_pts(nd.right)

    for nd in nodes:
        if nd.left is None:
            continue
        lp = subtree_pts(nd.left)
        rpn = subtree_pts(nd.right)
        if lp and rpn:
            assert not S[np.ix_(lp, rpn)].any(), f"separator of node {nd.id} leaks"
    # every block of A couples related nodes only
    atom_of = np.searchsorted(o.atom_ptr, np.arange(N), side="right") - 1
    iperm = np.empty(N, dtype=np.int64)
    iperm[o.perm] = np.arange(N)
    rows, cols = np.nonzero(A)
    for r, c in zip(rows, cols):
        na = o.atom_node[atom_of[iperm[r]]]
        nb = o.atom_node[atom_of[iperm[c]]]
        assert o.related(int(na), int(nb))


def _stencil(dims):
    """Plain 5/7-point pattern on an arbitrary box (x fastest)."""
    d = len(dims)
    N = int(np.prod(dims))
    strides = [1]
    for k in range(1, d):
        strides.append(strides[-1] * dims[k - 1])
    rp = [0]
    ci = []
    for idx in range(N):
        co = [(idx // strides[k]) % dims[k] for k in range(d)]
        nb = [idx]
        for k in range(d):
            if co[k] > 0:
                nb.append(idx - strides[k])
            if co[k] < dims[k] - 1:
                nb.append(idx + strides[k])
        nb.sort()
        ci.extend(nb)
        rp.append(len(ci))
    return np.array(rp), np.array(ci), None


@pytest.mark.parametrize("dims,L", [((32, 32), 4), ((64, 64), 6), ((12, 12, 12), 4)])
def test_interfaces_partition_and_nest(dims, L):
    o = nd_order(dims, L)
    prev = None
    for stage in range(L - 2, -1, -1):
        cl = o.stage_clusters(stage)
        # contiguous, covering, one node each
        assert cl[0][0] == 0 and cl[-1][1] == o.n_atoms
        for (a0, a1), (b0, b1) in zip(cl, cl[1:]):
            assert a1 == b0
        for a0, a1 in cl:
            assert len(set(o.atom_node[a0:a1].tolist())) == 1
        if prev is not None:
            # finer stage clusters nest inside coarser ones
            bounds = set(a0 for a0, _ in cl)
            assert bounds <= set(a0 for a0, _ in prev)
        prev = cl
    # at stage 0 every ND node is one cluster
    cl0 = o.stage_clusters(0)
    assert len(cl0) == len(set(o.atom_node.tolist()))
    # a separator at depth d is a single cluster under cuts of depth <= d
    for (a0, a1) in o.stage_clusters(L - 2):
        pass
    for nd in o.nodes:
        d = nd.depth
        if d > L - 2:
            continue
        cls = [c for c in o.stage_clusters(d) if o.atom_node[c[0]] == nd.id]
        assert len(cls) <= 1


def test_leaf_sizes_balanced():
    o = nd_order((64, 64), 6)
    leaf_sizes = [o.atom_size(a) for a in range(o.n_atoms) if o.node_level[o.atom_node[a]] == 6]
    assert len(leaf_sizes) == 32
    assert max(leaf_sizes) <= 2 * min(leaf_sizes)
    assert abs(np.mean(leaf_sizes) - 4096 / 32) < 0.5 * 4096 / 32
