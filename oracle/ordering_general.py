"""Oracle: modified nested dissection of a general sparse square matrix on
G(A^T A), and the row assignment by a bipartite matching.

TEST INFRASTRUCTURE ONLY (see package docstring).

The paper (Section 2.3) orders general matrices with a hypergraph partitioner
(PaToH, HUND) and assigns rows with MC64; neither is available here.  This is
our own restatement of the same steps, in the paper's terms:
  * nested dissection on the graph of A^T A gives the column partition
    (Section 2.1: a vertex separator of G(A^T A) leaves no fill between the
    two sides);
  * modified nested dissection splits every separator into interfaces by the
    descendant subdomains its columns connect to, and the cluster hierarchy
    says which interfaces merge after each level (Sections 2.3, 2.6);
  * rows are assigned through a matching that puts large entries on the
    diagonal (Section 2.3, second heuristic), row i then sitting with its
    matched column.

Readings (also in the design notes):
  G1  G(A^T A): columns i != j are adjacent when a row holds nonzeros in
      both.  It is walked through A's rows and columns, never formed.
  G2  Separator of a vertex set V (the columns of a node): a level set of a
      breadth-first search.  Components of G restricted to V are taken in
      the order of their smallest column; in each, the search starts from a
      pseudo-peripheral column (start at the component's smallest column;
      repeat: search, take the column of the last level with the fewest
      neighbours in V, ties to the smallest index, and move there while the
      number of levels grows).  The levels of all components are
      concatenated; the separator is the first level l whose cumulative size
      reaches half of |V|; the left child gets the levels before l, the right
      child those after it.  The separator then keeps only its columns that
      are adjacent to the right side; the others join the left side (they
      touch no right column, so the sides stay uncoupled).  Nodes at depth L-1
      are leaves; empty sets still get their subtree (no columns).
  G3  Interfaces: a column x of the separator of node B gets, for every
      non-leaf strict descendant D of B, a key (depth D, D, k) when x is
      adjacent in G(A^T A) to some column of D's subtree: k = 1 if x touches
      D's own separator or both of D's child subtrees, 0 if only the left
      one, 2 if only the right one.  Keys are sorted by (depth, id); classes
      of equal keys restricted to depths <= s are the interfaces at stage s
      (as reading R5 of the grid ordering), atoms are the finest classes.
  G4  Column order as reading R6 of the grid ordering, with the column index
      in place of the grid index.
  G5  Row matching: entries by decreasing |a_ij| (ties: row, then column)
      are matched greedily; every row left unmatched (ascending) is then
      matched by an augmenting path (columns of a row tried in ascending
      order, depth first).  A structurally singular pattern is rejected.
  G6  Maximum-product row matching (the option closest to the MC64 matching
      Section 2.3 uses): the perfect matching maximising prod |a_{i,m(i)}|,
      i.e. minimising sum c_ij with c_ij = log max_k |a_kj| - log |a_ij| over
      the nonzero entries (duplicates summed in storage order, explicit
      zeros dropped).  Found by shortest augmenting paths with dual
      potentials u (rows), v (columns), reduced costs (c_ij - u_i) - v_j:
      start v = 0, u_i = min_j c_ij, and match every row (ascending) to its
      first free zero-reduced-cost column (ascending); then every row left
      free (ascending) starts a Dijkstra search over columns (ties: the
      smaller column), crossing matched edges at no cost, up to the first
      free column at distance D; every column k settled meanwhile gets
      v_k -= D - d_k, its matched row u += D - d_k, the start row u += D; the
      path is then flipped.  No path: structurally singular.
  Both matchings order entries by |a_ij|: a NaN or infinite value is refused.
"""
import heapq
import math
import sys

import numpy as np

from .ordering import NDOrdering, hierarchical_atoms, num_levels

__all__ = ["nd_general", "row_matching", "row_matching_max_product", "column_graph"]


class _GNode:
    __slots__ = ("id", "depth", "parent", "left", "right", "size", "pts")

    def __init__(self, nid, depth, parent):
        self.id = nid
        self.depth = depth
        self.parent = parent
        self.left = None
        self.right = None
        self.size = 1
        self.pts = []


def column_graph(n, rowptr, colind):
    """Adjacency of G(A^T A) (reading G1): sorted neighbour lists, no self."""
    rows = [set(int(c) for c in colind[rowptr[r]:rowptr[r + 1]]) for r in range(n)]
    adj = [set() for _ in range(n)]
    for cols in rows:
        for c in cols:
            adj[c] |= cols
    return [sorted(a - {j}) for j, a in enumerate(adj)]


def _bfs_levels(root, inV, adj):
    levels = [[root]]
    seen = {root}
    while True:
        nxt = sorted({y for x in levels[-1] for y in adj[x] if inV[y] and y not in seen})
        if not nxt:
            return levels
        seen.update(nxt)
        levels.append(nxt)


def _pseudo_peripheral(start, inV, adj):
    root = start
    lv = _bfs_levels(root, inV, adj)
    while True:
        cand = min(lv[-1], key=lambda v: (sum(1 for y in adj[v] if inV[y]), v))
        lv2 = _bfs_levels(cand, inV, adj)
        if len(lv2) <= len(lv):
            return root, lv
        root, lv = cand, lv2


def level_structure(V, adj, n):
    """Breadth-first levels of G restricted to V, component by component (G2)."""
    inV = np.zeros(n, dtype=bool)
    inV[list(V)] = True
    done = set()
    levels = []
    for s in sorted(V):
        if s in done:
            continue
        _, lv = _pseudo_peripheral(s, inV, adj)
        for level in lv:
            done.update(level)
        levels += lv
    return levels


def row_matching(n, rowptr, colind, val=None):
    """rowcol[r] = the column row r is matched to (reading G5)."""
    rowptr = np.asarray(rowptr)
    colind = np.asarray(colind)
    mag = np.ones(colind.shape[0]) if val is None else np.abs(np.asarray(val, dtype=np.float64))
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    order = np.lexsort((colind, rows, -mag))
    rowcol = -np.ones(n, dtype=np.int64)
    colrow = -np.ones(n, dtype=np.int64)
    for e in order:
        r, c = int(rows[e]), int(colind[e])
        if rowcol[r] < 0 and colrow[c] < 0:
            rowcol[r] = c
            colrow[c] = r
    sys.setrecursionlimit(max(10000, 4 * n))

    def augment(r, seen):
        for c in sorted(set(int(x) for x in colind[rowptr[r]:rowptr[r + 1]])):
            if c in seen:
                continue
            seen.add(c)
            if colrow[c] < 0 or augment(int(colrow[c]), seen):
                rowcol[r] = c
                colrow[c] = r
                return True
        return False

    for r in range(n):
        if rowcol[r] < 0 and not augment(r, set()):
            raise ValueError("structurally singular matrix: no perfect matching")
    return rowcol


def _row_entries(n, rowptr, colind, val):
    """Per row the distinct columns (ascending) with their values, duplicates
    summed in storage order; explicit zeros dropped (reading G6)."""
    out = []
    for r in range(n):
        acc = {}
        for e in range(int(rowptr[r]), int(rowptr[r + 1])):
            c = int(colind[e])
            x = 1.0 if val is None else float(val[e])
            acc[c] = acc[c] + x if c in acc else x
        out.append([(c, acc[c]) for c in sorted(acc) if acc[c] != 0.0])
    return out


def row_matching_max_product(n, rowptr, colind, val=None):
    """rowcol[r] = the column row r is matched to, maximising the product of
    the matched |a_ij| (reading G6)."""
    rows = _row_entries(n, rowptr, colind, val)
    amax = [0.0] * n
    for ent in rows:
        for c, x in ent:
            amax[c] = max(amax[c], abs(x))
    if any(a == 0.0 for a in amax):
        raise ValueError("structurally singular matrix: an empty column")
    cost = [[(c, math.log(amax[c]) - math.log(abs(x))) for c, x in ent] for ent in rows]
    v = [0.0] * n
    u = [min((w for _, w in ent), default=0.0) for ent in cost]
    rowcol = [-1] * n
    colrow = [-1] * n
    for r in range(n):
        for c, w in cost[r]:
            if colrow[c] < 0 and (w - u[r]) - v[c] == 0.0:
                rowcol[r] = c
                colrow[c] = r
                break
    for r in range(n):
        if rowcol[r] >= 0:
            continue
        d = {}
        pred = {}
        heap = []
        for c, w in cost[r]:
            nd = (w - u[r]) - v[c]
            if c not in d or nd < d[c]:
                d[c] = nd
                pred[c] = r
                heapq.heappush(heap, (nd, c))
        settled = []
        done = set()
        end = -1
        while heap:
            dj, j = heapq.heappop(heap)
            if j in done:
                continue
            done.add(j)
            settled.append(j)
            if colrow[j] < 0:
                end = j
                break
            i = colrow[j]
            for c, w in cost[i]:
                if c in done:
                    continue
                nd = dj + ((w - u[i]) - v[c])
                if c not in d or nd < d[c]:
                    d[c] = nd
                    pred[c] = i
                    heapq.heappush(heap, (nd, c))
        if end < 0:
            raise ValueError("structurally singular matrix: no perfect matching")
        D = d[end]
        u[r] = u[r] + D
        for k in settled:
            delta = D - d[k]
            v[k] = v[k] - delta
            if k != end:
                u[colrow[k]] = u[colrow[k]] + delta
        j = end
        while True:
            i = pred[j]
            prev = rowcol[i]
            rowcol[i] = j
            colrow[j] = i
            if i == r:
                break
            j = prev
    return np.array(rowcol, dtype=np.int64)


def nd_general(n, rowptr, colind, val=None, L=None, matching="max_product"):
    """Modified nested dissection of a general matrix (readings G1-G5).

    Returns an NDOrdering (as the grid ordering) with two more fields:
    rowcol[r] (the column row r is matched to) and rperm[new] (old row of the
    new position: the row matched to column perm[new]).  matching:
    "max_product" (reading G6, the default) or "greedy" (reading G5).
    """
    if matching not in ("greedy", "max_product"):
        raise ValueError("matching must be 'greedy' or 'max_product'")
    if val is not None and not np.all(np.isfinite(np.asarray(val, dtype=np.float64))):
        raise ValueError("non-finite matrix value: the matchings order entries by |a_ij|")
    rowptr = np.asarray(rowptr, dtype=np.int64)
    colind = np.asarray(colind, dtype=np.int64)
    if L is None or L <= 0:
        L = num_levels(n)
    adj = column_graph(n, rowptr, colind)
    nodes = []

    def build(V, depth, parent):
        nd = _GNode(len(nodes), depth, parent)
        nodes.append(nd)
        if depth == L - 1:
            nd.pts = list(V)
            return nd
        if V:
            levels = level_structure(V, adj, n)
            cum = 0
            for l, level in enumerate(levels):
                cum += len(level)
                if 2 * cum >= len(V):
                    break
            left = [x for lv in levels[:l] for x in lv]
            right = sorted(x for lv in levels[l + 1:] for x in lv)
            rset = set(right)
            sep = sorted(levels[l])
            nd.pts = [x for x in sep if any(y in rset for y in adj[x])]
            left = sorted(left + [x for x in sep if not any(y in rset for y in adj[x])])
        else:
            left, right = [], []
        nd.left = build(left, depth + 1, nd)
        nd.right = build(right, depth + 1, nd)
        nd.size = 1 + nd.left.size + nd.right.size
        return nd

    build(list(range(n)), 0, None)
    owner = np.zeros(n, dtype=np.int64)
    for nd in nodes:
        owner[nd.pts] = nd.id

    node_atoms = {}
    for nd in nodes:
        if not nd.pts:
            node_atoms[nd.id] = []
            continue
        if nd.depth == L - 1:
            node_atoms[nd.id] = [(np.array(nd.pts, dtype=np.int64), [])]
            continue
        keys = []
        for x in nd.pts:
            marks = {}
            for y in adj[x]:
                o = int(owner[y])
                if not (nd.id < o < nd.id + nd.size):
                    continue
                # every non-leaf node D on the path from owner(y) up to (not incl.) nd
                child = None
                D = nodes[o]
                while D is not nd:
                    if D.depth < L - 1:
                        m = marks.setdefault(D.id, [False, False, False])
                        if child is None:
                            m[1] = True
                        elif child is D.left:
                            m[0] = True
                        else:
                            m[2] = True
                    child = D
                    D = D.parent
            kk = []
            for did in sorted(marks, key=lambda i: (nodes[i].depth, i)):
                a, b, c = marks[did]
                kk.append((nodes[did].depth, did, 1 if (b or (a and c)) else (0 if a else 2)))
            keys.append(kk)
        node_atoms[nd.id] = hierarchical_atoms(nd.pts, keys)

    order_nodes = sorted(nodes, key=lambda nd: (-nd.depth, nd.id))
    perm, atom_ptr, atom_node, atom_keys = [], [0], [], []
    for nd in order_nodes:
        for gi, kk in node_atoms[nd.id]:
            perm.append(gi)
            atom_ptr.append(atom_ptr[-1] + gi.shape[0])
            atom_node.append(nd.id)
            atom_keys.append(kk)
    perm = np.concatenate(perm) if perm else np.zeros(0, dtype=np.int64)
    assert perm.shape[0] == n
    o = NDOrdering((n,), L, nodes, perm.astype(np.int64), np.array(atom_ptr, dtype=np.int64),
                   np.array(atom_node, dtype=np.int32), atom_keys)
    if matching == "greedy":
        o.rowcol = row_matching(n, rowptr, colind, val)
    else:
        o.rowcol = row_matching_max_product(n, rowptr, colind, val)
    colrow = np.empty(n, dtype=np.int64)
    colrow[o.rowcol] = np.arange(n)
    o.rperm = colrow[o.perm]
    return o
