"""Batch ordering: the ordering of diag(A_0, ..., A_{k-1}) restricted to one
matrix is that matrix's own ordering, aligned at the leaves.

spaqr_order_batch is integer host work, so this runs without a GPU.  Every
matrix's permutation, nodes, clusters, fronts, colours and R(s) / C(s) lists
must equal the single-matrix ordering after mapping atom ids, with level k
of the batch (from the leaves) holding level k of each matrix.
"""
import numpy as np
import pytest

import paper_2010_06807_gb300 as sq
from synth.convdiff import config_problem

BATCHES = [
    [("2d_uniform_a", 16), ("2d_uniform_a", 32), ("2d_lognormal", 24)],
    [("2d_uniform_a", 48), ("3d_uniform_a", 8), ("2d_uniform_a", 8), ("2d_uniform_a", 40)],
]


def _single(p):
    o = sq.spaqr_order(p.rowptr, p.colind, p.dims)
    return o, o.arrays(), o.plan()


@pytest.mark.parametrize("batch", BATCHES)
def test_batch_ordering_restricts_to_each_matrix(spaqr_lib, batch):
    probs = [config_problem(kind, n=n, seed=7 + i) for i, (kind, n) in enumerate(batch)]
    ob = sq.spaqr_order_batch([(p.rowptr, p.colind) for p in probs], [p.dims for p in probs])
    ab = ob.arrays()
    plan_b = ob.plan()
    singles = [_single(p) for p in probs]
    assert ob.L == max(o.L for o, _, _ in singles)
    assert ob.n == sum(p.n for p in probs)
    np.testing.assert_array_equal(ob.part_ptr, np.cumsum([0] + [p.n for p in probs]))
    # node ranges and atom maps per matrix
    node_off = np.cumsum([0] + [o.n_nodes for o, _, _ in singles])
    atom_mat = np.searchsorted(node_off, ab["atom_node"], side="right") - 1
    for i, (p, (o, a, plan)) in enumerate(zip(probs, singles)):
        base = ob.part_ptr[i]
        # permutation restricted to the matrix
        sel = (ab["perm"] >= base) & (ab["perm"] < base + p.n)
        np.testing.assert_array_equal(ab["perm"][sel] - base, a["perm"])
        # atoms of the matrix, in order, and their sizes / nodes
        atoms_b = np.nonzero(atom_mat == i)[0]
        assert atoms_b.size == a["atom_node"].size
        np.testing.assert_array_equal(np.diff(ab["atom_ptr"])[atoms_b], np.diff(a["atom_ptr"]))
        np.testing.assert_array_equal(ab["atom_node"][atoms_b] - node_off[i], a["atom_node"])
        amap = {int(b): s for s, b in enumerate(atoms_b)}
        shift = ob.L - o.L
        lv_b = ab["node_level"][node_off[i]:node_off[i + 1]]
        np.testing.assert_array_equal(lv_b - shift, a["node_level"])
        for k, st in enumerate(plan_b):
            mine = [amap[c] for c in st["clusters"] if c in amap]
            fr = [f for f in st["fronts"] if f["id"] in amap]
            if k >= o.L:
                assert not mine and not fr
                continue
            ref = plan[k]
            assert mine == ref["clusters"]
            assert len(fr) == len(ref["fronts"])
            for fb, fs in zip(fr, ref["fronts"]):
                assert amap[fb["id"]] == fs["id"]
                assert fb["colour"] == fs["colour"]
                assert [amap[x] for x in fb["R"]] == fs["R"]
                assert [amap[x] for x in fb["C"]] == fs["C"]


def test_blockdiag_csr_layout():
    probs = [config_problem("2d_uniform_a", n=n, seed=3 + n) for n in (8, 12, 5)]
    rp, ci, v = sq.blockdiag_csr([(p.rowptr, p.colind, p.val) for p in probs])
    A = np.zeros((rp.size - 1, rp.size - 1))
    for r in range(rp.size - 1):
        A[r, ci[rp[r]:rp[r + 1]]] = v[rp[r]:rp[r + 1]]
    b = 0
    for p in probs:
        np.testing.assert_array_equal(A[b:b + p.n, b:b + p.n], p.to_dense())
        assert not A[b:b + p.n, :b].any() and not A[b:b + p.n, b + p.n:].any()
        b += p.n


def test_batch_ordering_errors(spaqr_lib):
    p = config_problem("2d_uniform_a", n=8)
    with pytest.raises(sq.SpaqrError):
        sq.spaqr_order_batch([(p.rowptr, p.colind)], [(9, 8)])
    with pytest.raises(ValueError):
        sq.spaqr_order_batch([], [])
