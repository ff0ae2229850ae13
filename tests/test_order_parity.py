"""The library's host ordering and symbolic plan match the oracle bit for bit.

spaqr_order is integer host work, so this runs without a GPU.  The oracle
(oracle/ordering.py, oracle/spaqr.py) is an independent implementation of the
same readings of Section 2.3 / Algorithm 2.
"""
import numpy as np
import pytest

import paper_2010_06807_gb300 as sq
from oracle import spaqr as osq
from oracle.ordering import nd_order
from synth.convdiff import config_problem, convdiff


CASES = [
    ("2d_uniform_a", 16, 3), ("2d_uniform_a", 24, 4), ("2d_uniform_a", 32, 0),
    ("2d_uniform_a", 64, 0), ("2d_lognormal", 40, 5), ("3d_uniform_a", 8, 3),
    ("3d_uniform_a", 12, 0), ("2d_uniform_a", 5, 4), ("2d_uniform_a", 4, 0),
]


@pytest.mark.parametrize("kind,n,L", CASES)
def test_ordering_and_plan_bit_exact(spaqr_lib, kind, n, L):
    p = config_problem(kind, n=n)
    ordl = sq.spaqr_order(p.rowptr, p.colind, p.dims, L)
    arr = ordl.arrays()
    o = nd_order(p.dims, L if L > 0 else None)
    assert ordl.L == o.L
    np.testing.assert_array_equal(arr["perm"], o.perm)
    np.testing.assert_array_equal(arr["atom_ptr"], o.atom_ptr)
    np.testing.assert_array_equal(arr["atom_node"], o.atom_node)
    np.testing.assert_array_equal(arr["node_level"], o.node_level)
    # symbolic plan against the oracle's factorisation record (eps irrelevant)
    F = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 1e-2, nlevels=o.L, skip=1, ordering=o)
    plan = ordl.plan()
    assert len(plan) == len(F.steps)
    for st_l, st_o in zip(plan, F.steps):
        assert st_l["level"] == st_o["level"]
        assert st_l["clusters"] == sorted(st_o["sizes"].keys())
        assert [f["id"] for f in st_l["fronts"]] == list(st_o["order"])
        for f in st_l["fronts"]:
            s = f["id"]
            assert f["colour"] == st_o["colour"][s]
            assert f["R"] == list(st_o["R"][s])
            assert f["C"] == list(st_o["C"][s])


def test_order_rejects_bad_input(spaqr_lib):
    p = config_problem("2d_uniform_a", n=8)
    with pytest.raises(sq.SpaqrError) as e:
        sq.spaqr_order(p.rowptr, p.colind, (8, 9))
    assert e.value.name == "INVALID_ARG"
    # a pattern that couples points two separators apart is not a stencil
    rp = p.rowptr.copy()
    ci = p.colind.copy()
    ci[1] = 63 if ci[1] != 0 else ci[1]
    with pytest.raises(sq.SpaqrError):
        sq.spaqr_order(rp, np.sort(ci.reshape(-1)), (8, 8), 3)


def _general_cases():
    from synth.convdiff import permuted, random_local
    g = config_problem("2d_uniform_a", n=20)
    return [("grid_no_dims", g, 4), ("row_col_permuted", permuted(g, 21), 4),
            ("rows_permuted_3d", permuted(config_problem("3d_uniform_a", n=7), 22, cols=False), 3),
            ("random_local", random_local(18, seed=7011), 4), ("random_local_auto_L", random_local(26, seed=7012), 0)]


@pytest.mark.parametrize("name,p,L", _general_cases())
def test_general_ordering_bit_exact(spaqr_lib, name, p, L):
    """Ordering of a general matrix (no grid): nested dissection on
    G(A^T A), interfaces, row matching and symbolic plan equal the oracle's."""
    from oracle.ordering_general import nd_general
    ordl = sq.spaqr_order(p.rowptr, p.colind, None, L, val=p.val)
    arr = ordl.arrays()
    o = nd_general(p.n, p.rowptr, p.colind, p.val, L if L > 0 else None)
    assert ordl.L == o.L
    for k in ("perm", "atom_ptr", "atom_node", "node_level", "rperm"):
        np.testing.assert_array_equal(arr[k], getattr(o, k), err_msg=k)
    F = osq.factor(p.n, p.rowptr, p.colind, p.val, None, 1e-2, nlevels=o.L, skip=1, ordering=o)
    plan = ordl.plan()
    assert len(plan) == len(F.steps)
    for st_l, st_o in zip(plan, F.steps):
        assert st_l["clusters"] == sorted(st_o["sizes"].keys())
        assert [f["id"] for f in st_l["fronts"]] == list(st_o["order"])
        for f in st_l["fronts"]:
            assert f["R"] == list(st_o["R"][f["id"]]) and f["C"] == list(st_o["C"][f["id"]])


def test_general_ordering_rejects_singular_pattern(spaqr_lib):
    rp = np.array([0, 1, 2, 3], dtype=np.int64)
    ci = np.array([0, 0, 2], dtype=np.int32)
    with pytest.raises(sq.SpaqrError) as e:
        sq.spaqr_order(rp, ci, None, 1)
    assert e.value.name == "SINGULAR"


def test_general_ordering_rejects_dense_rows(spaqr_lib):
    """Squared row lengths above 2^31: G(A^T A) is not formed (UNSUPPORTED)."""
    n = 47000
    rp = np.concatenate([[0, n], n + np.arange(1, n)]).astype(np.int64)
    ci = np.concatenate([np.arange(n), np.arange(1, n)]).astype(np.int32)
    with pytest.raises(sq.SpaqrError) as e:
        sq.spaqr_order(rp, ci, None, 2)
    assert e.value.name == "UNSUPPORTED"


def _disconnected():
    from synth.convdiff import permuted, random_local
    a, b = permuted(config_problem("2d_uniform_a", n=7), 51), random_local(6, seed=7031)
    rp, ci, v = sq.blockdiag_csr([(a.rowptr, a.colind, a.val), (b.rowptr, b.colind, b.val)])
    from synth.convdiff import Problem
    return Problem(None, rp, ci.astype(np.int32), v, name="disconnected")


@pytest.mark.parametrize("case", ["disconnected", "many_levels", "tiny"])
def test_general_ordering_edge_cases(spaqr_lib, case):
    """Disconnected patterns (components in order of their smallest column),
    more levels than the columns can fill (empty subtrees) and a 1 x 1 matrix:
    the host ordering still equals the oracle's, and the oracle's factor with
    eps = 0 solves exactly."""
    from oracle.ordering_general import nd_general
    from synth.convdiff import Problem, permuted
    if case == "disconnected":
        p, L = _disconnected(), 4
    elif case == "many_levels":
        p, L = permuted(config_problem("2d_uniform_a", n=5), 52), 6
    else:
        p, L = Problem(None, np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32),
                       np.array([2.0])), 1
    ordl = sq.spaqr_order(p.rowptr, p.colind, None, L, val=p.val)
    arr = ordl.arrays()
    o = nd_general(p.n, p.rowptr, p.colind, p.val, L)
    for k in ("perm", "atom_ptr", "atom_node", "node_level", "rperm"):
        np.testing.assert_array_equal(arr[k], getattr(o, k), err_msg=k)
    F = osq.factor(p.n, p.rowptr, p.colind, p.val, None, 0.0, nlevels=o.L, skip=0, ordering=o)
    b = np.random.default_rng(2).standard_normal(p.n)
    x = osq.solve(F, b)
    assert np.linalg.norm(b - p.matvec(x)) <= 1e-12 * np.linalg.norm(b)


def _with_duplicates_and_zeros(p, seed):
    """p with some entries split into two stored parts (same sum up to one
    rounding), explicit zeros at new positions of existing rows, and every
    row's entries in a shuffled storage order."""
    from synth.convdiff import Problem
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for r in range(p.n):
        ent = [(int(c), float(x)) for c, x in zip(p.colind[p.rowptr[r]:p.rowptr[r + 1]],
                                                  p.val[p.rowptr[r]:p.rowptr[r + 1]])]
        out = []
        for c, x in ent:
            if rng.random() < 0.3:
                t = rng.uniform(0.2, 0.8)
                out += [(c, t * x), (c, x - t * x)]
            else:
                out.append((c, x))
        if rng.random() < 0.3:
            out.append((int(rng.integers(p.n)), 0.0))
        rng.shuffle(out)
        for c, x in out:
            rows.append(r)
            cols.append(c)
            vals.append(x)
    counts = np.bincount(np.asarray(rows), minlength=p.n)
    rp = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return Problem(None, rp, np.asarray(cols, dtype=np.int32), np.asarray(vals), name=p.name + "_dup")


def _max_product_cases():
    from synth.convdiff import permuted, random_local
    g = config_problem("2d_uniform_a", n=20)
    w = random_local(16, seed=7016, weak_diag=0.1)
    return [("weak_18", random_local(18, seed=7013, weak_diag=0.1), 4, True),
            ("weak_30_auto_L", random_local(30, seed=7014, weak_diag=0.05), 0, True),
            ("row_col_permuted", permuted(g, 23), 4, True),
            ("pattern_only", random_local(16, seed=7015, weak_diag=0.1), 4, False),
            ("duplicates_zeros", _with_duplicates_and_zeros(w, 3), 4, True)]


@pytest.mark.parametrize("name,p,L,values", _max_product_cases())
def test_general_ordering_max_product_bit_exact(spaqr_lib, name, p, L, values):
    """The maximum-product row matching (and the ordering and plan built on
    it) equals the oracle's, ties included (pattern only: every cost is 0)."""
    from oracle.ordering_general import nd_general
    val = p.val if values else None
    ordl = sq.spaqr_order(p.rowptr, p.colind, None, L, val=val, matching="max_product")
    arr = ordl.arrays()
    o = nd_general(p.n, p.rowptr, p.colind, val, L if L > 0 else None, matching="max_product")
    assert ordl.L == o.L
    for k in ("perm", "atom_ptr", "atom_node", "node_level", "rperm"):
        np.testing.assert_array_equal(arr[k], getattr(o, k), err_msg=k)
    F = osq.factor(p.n, p.rowptr, p.colind, p.val, None, 1e-2, nlevels=o.L, skip=1, ordering=o)
    plan = ordl.plan()
    assert len(plan) == len(F.steps)
    for st_l, st_o in zip(plan, F.steps):
        assert st_l["clusters"] == sorted(st_o["sizes"].keys())
        assert [f["id"] for f in st_l["fronts"]] == list(st_o["order"])


def test_general_ordering_matching_errors(spaqr_lib):
    import ctypes
    g = config_problem("2d_uniform_a", n=6)
    with pytest.raises(ValueError):
        sq.spaqr_order(g.rowptr, g.colind, None, 2, val=g.val, matching="mc64")
    with pytest.raises(ValueError):   # grids keep every row with its column
        sq.spaqr_order(g.rowptr, g.colind, g.dims, 2, matching="max_product")
    # an unknown matching code at the C ABI
    csr, keep = sq._make_csr(g.rowptr, g.colind, g.val)
    h = ctypes.c_void_p(1)
    assert sq._lib.spaqr_order_general(ctypes.byref(csr), 2, 7, ctypes.byref(h)) == -1
    assert not h.value
    # column 0 holds only explicit zeros: a perfect matching on the pattern,
    # none on the values
    rp = np.array([0, 2, 4, 5], dtype=np.int64)
    ci = np.array([0, 1, 0, 2, 1], dtype=np.int32)
    v = np.array([0.0, 1.0, 0.0, 3.0, 2.0])
    sq.spaqr_order(rp, ci, None, 1, val=v, matching="greedy")   # greedy: uses the pattern
    with pytest.raises(sq.SpaqrError) as e:
        sq.spaqr_order(rp, ci, None, 1, val=v)   # the default, maximum product
    assert e.value.name == "SINGULAR"
    from oracle.ordering_general import row_matching_max_product
    with pytest.raises(ValueError):
        row_matching_max_product(3, rp, ci, v)


def test_orderings_reject_decreasing_rowptr(spaqr_lib):
    """A rowptr that starts at 0 and ends at nnz but decreases in between
    would send the host loops outside colind: all three ordering paths
    refuse it (INVALID_ARG) before reading the rows."""
    p = config_problem("2d_uniform_a", n=8)
    rp = p.rowptr.copy()
    rp[3] = rp[5] + 1          # rows 2 and 3 now run backwards
    for call in (lambda: sq.spaqr_order(rp, p.colind, p.dims, 2),
                 lambda: sq.spaqr_order(rp, p.colind, None, 2, val=p.val),
                 lambda: sq.spaqr_order(rp, p.colind, None, 2, val=p.val, matching="max_product"),
                 lambda: sq.spaqr_order_batch([(p.rowptr, p.colind), (rp, p.colind)], [p.dims, p.dims])):
        with pytest.raises(sq.SpaqrError) as e:
            call()
        assert e.value.name == "INVALID_ARG"
        assert "rowptr" in str(e.value)


@pytest.mark.parametrize("matching", ["greedy", "max_product"])
def test_matchings_random_small_matrices(spaqr_lib, matching):
    """Many small random patterns with heavy ties (values from a six-value
    set, zeros included), duplicate entries, shuffled rows and pattern-only
    runs: the host matching equals the oracle's, and both refuse the same
    structurally singular cases."""
    from oracle.ordering_general import row_matching, row_matching_max_product
    ref_fn = row_matching if matching == "greedy" else row_matching_max_product
    rng = np.random.default_rng(321 if matching == "greedy" else 123)
    tested = 0
    for t in range(150):
        n = int(rng.integers(2, 40))
        M = rng.random((n, n)) < rng.uniform(0.05, 0.4)
        M[np.arange(n), rng.permutation(n)] = True
        rows, cols, vals = [], [], []
        for r in range(n):
            cs = list(np.nonzero(M[r])[0])
            rng.shuffle(cs)
            for c in cs:
                for _ in range(2 if rng.random() < 0.15 else 1):
                    rows.append(r)
                    cols.append(int(c))
                    vals.append(float(rng.choice([1.0, -1.0, 2.0, 0.5, -3.0, 0.0])) if t % 2
                                else float(rng.lognormal()))
        rp = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]).astype(np.int64)
        ci = np.asarray(cols, dtype=np.int32)
        va = None if t % 7 == 0 else np.asarray(vals)
        try:
            ref = ref_fn(n, rp, ci, va)
        except ValueError:
            ref = None
        try:
            arr = sq.spaqr_order(rp, ci, None, 2 if n > 8 else 1, val=va, matching=matching).arrays()
        except sq.SpaqrError as e:
            assert e.name == "SINGULAR", e
            arr = None
        assert (ref is None) == (arr is None), t
        if ref is None:
            continue
        colrow = np.empty(n, dtype=np.int64)
        colrow[ref] = np.arange(n)
        np.testing.assert_array_equal(arr["rperm"], colrow[arr["perm"]], err_msg=str(t))
        tested += 1
    assert tested >= 100


def test_general_ordering_random_patterns(spaqr_lib):
    """Random sparse patterns of 1-60 columns (some split into two
    disconnected blocks, some with shuffled rows and columns) at 1-5 levels:
    the host ordering equals the oracle's, and every fifth plan too."""
    from oracle.ordering_general import nd_general
    rng = np.random.default_rng(77)
    for t in range(120):
        n = int(rng.integers(1, 60))
        M = rng.random((n, n)) < rng.uniform(0.02, 0.2)
        M[np.arange(n), np.arange(n)] = True
        if t % 3 == 0 and n > 4:
            h = n // 2
            M[:h, h:] = False
            M[h:, :h] = False
        if t % 2:
            M = M[rng.permutation(n)][:, rng.permutation(n)]
        rp = np.concatenate([[0], np.cumsum(M.sum(1))]).astype(np.int64)
        ci = np.concatenate([np.nonzero(M[r])[0] for r in range(n)]).astype(np.int32)
        va = rng.standard_normal(ci.shape[0])
        L = int(rng.integers(1, 6))
        o = nd_general(n, rp, ci, va, L)
        ol = sq.spaqr_order(rp, ci, None, L, val=va)
        arr = ol.arrays()
        for k in ("perm", "atom_ptr", "atom_node", "node_level", "rperm"):
            np.testing.assert_array_equal(arr[k], getattr(o, k), err_msg=f"{t} {k}")
        if t % 5 == 0:
            F = osq.factor(n, rp, ci, va, None, 1e-2, nlevels=L, skip=1, ordering=o)
            plan = ol.plan()
            assert len(plan) == len(F.steps)
            for st_l, st_o in zip(plan, F.steps):
                assert st_l["clusters"] == sorted(st_o["sizes"].keys())
                assert [f["id"] for f in st_l["fronts"]] == list(st_o["order"])
                for f in st_l["fronts"]:
                    assert f["R"] == list(st_o["R"][f["id"]]) and f["C"] == list(st_o["C"][f["id"]])


def test_grid_ordering_random_shapes(spaqr_lib):
    """Random 2D (1-23 per side) and 3D (1-8 per side) grids, degenerate
    sides of 1 included, at 0 (automatic) to 5 levels: the geometric
    ordering equals the oracle's, and every third plan too."""
    rng = np.random.default_rng(5)
    for t in range(100):
        if t % 2:
            dims = (int(rng.integers(1, 24)), int(rng.integers(1, 24)))
        else:
            dims = (int(rng.integers(1, 9)), int(rng.integers(1, 9)), int(rng.integers(1, 9)))
        L = int(rng.integers(0, 6))
        N = int(np.prod(dims))
        rp, ci, va = convdiff(dims, np.ones(N), np.ones((N, len(dims))))[:3]
        ol = sq.spaqr_order(rp, ci, dims, L)
        arr = ol.arrays()
        o = nd_order(dims, L if L > 0 else None)
        for k in ("perm", "atom_ptr", "atom_node", "node_level"):
            np.testing.assert_array_equal(arr[k], getattr(o, k), err_msg=f"{dims} L={L} {k}")
        if t % 3 == 0:
            F = osq.factor(N, rp, ci, va, dims, 1e-2, nlevels=o.L, skip=1, ordering=o)
            plan = ol.plan()
            assert len(plan) == len(F.steps)
            for st_l, st_o in zip(plan, F.steps):
                assert st_l["clusters"] == sorted(st_o["sizes"].keys())
                assert [f["id"] for f in st_l["fronts"]] == list(st_o["order"])


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_general_ordering_rejects_non_finite_values(spaqr_lib, bad):
    """The matchings order entries by |a_ij|; a NaN or infinite value is
    refused (INVALID_ARG) by the host and the oracle alike."""
    from oracle.ordering_general import nd_general
    g = config_problem("2d_uniform_a", n=6)
    v = g.val.copy()
    v[7] = bad
    for m in ("greedy", "max_product"):
        with pytest.raises(sq.SpaqrError) as e:
            sq.spaqr_order(g.rowptr, g.colind, None, 2, val=v, matching=m)
        assert e.value.name == "INVALID_ARG"
        with pytest.raises(ValueError):
            nd_general(g.n, g.rowptr, g.colind, v, 2, matching=m)
    sq.spaqr_order(g.rowptr, g.colind, None, 2, val=None)   # pattern only: no values to check


def test_general_ordering_hand_derived_golden(spaqr_lib):
    """The host library's grid-free ordering reproduces the hand-derived
    cases of tests/golden/general_paths.json directly."""
    import json
    import os
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "general_paths.json")))
    for case in golden["cases"]:
        rp = np.concatenate([[0], np.cumsum([len(r) for r in case["rows"]])]).astype(np.int64)
        ci = np.asarray([c for r in case["rows"] for c, _ in r], dtype=np.int32)
        va = np.asarray([v for r in case["rows"] for _, v in r], dtype=np.float64)
        arr = sq.spaqr_order(rp, ci, None, case["L"], val=va).arrays()
        for k in ("perm", "atom_ptr", "atom_node", "rperm"):
            assert arr[k].tolist() == case[k], (case["name"], k)
