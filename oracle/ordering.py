"""Oracle: geometric modified nested dissection on G(A^T A) for regular grids.

TEST INFRASTRUCTURE ONLY (see package docstring).

Follows the paper's ordering step (Section 2.3 and Algorithm 2 step 1):
  * nested dissection on the graph of A^T A gives the column partition
    (Section 2.1); on a regular grid the separators are geometric;
  * the number of levels is ceil(log2(N/64)) (Section 4);
  * modified nested dissection (Section 2.3, figure "mnd_multilvl") splits each
    separator into interfaces by the cuts of descendant subdomains, and the
    cluster hierarchy says which interfaces merge after each level
    (Section 2.6);
  * rows are ordered like columns for diagonally dominant matrices
    (Section 2.3).

Readings where the paper is silent (each also listed in the design notes):
  R1  A vertex separator of G(A^T A) for a 5/7-point stencil must be two grid
      planes thick (A^T A couples nodes up to stencil distance 2).
  R2  Cut the longest box extent (ties: x, then y, then z) at
      m = lo + max(0, (ext - 2) // 2); the separator is planes [m, m+2)
      clipped to the box; the children are [lo, m) and [m+2, hi).
  R3  Nodes at depth L-1 are leaves (interiors); a node at depth d is at level
      d+1, the root at level 1.
  R4  The cut of a non-leaf descendant box D of box B splits B's separator S
      when D touches S (D ends where B's left child ends or starts where B's
      right child starts along B's cut dimension) and D's cut dimension is
      tangent to S.  It applies to a node v of S when, in every tangent
      dimension other than D's cut dimension, v lies within D's extent widened
      by two planes on each side.  It puts v below, inside or above D's
      two-plane slab.
  R5  Interfaces after eliminating level l are the classes of S under the cuts
      of depth <= l-1; the merge after level l removes the cuts of depth l-1.
      The finest classes are the atoms.
  R6  Column order: nodes by level (leaves first, root last), then by
      depth-first preorder; inside a separator, atoms in hierarchical order
      (classes of shallower cuts first, each class ordered by its smallest
      grid index); inside an atom, by grid index (x fastest).
"""
import math
import numpy as np

__all__ = ["NDOrdering", "nd_order", "num_levels", "hierarchical_atoms"]


def num_levels(N):
    """L = ceil(log2(N / 64)), at least 1 (Section 4)."""
    if N <= 64:
        return 1
    return max(1, int(math.ceil(math.log2(N / 64.0) - 1e-12)))


class _Node:
    __slots__ = ("id", "depth", "lo", "hi", "parent", "left", "right",
                 "cut_dim", "cut_m", "size")

    def __init__(self, nid, depth, lo, hi, parent):
        self.id = nid
        self.depth = depth
        self.lo = list(lo)
        self.hi = list(hi)
        self.parent = parent
        self.left = None
        self.right = None
        self.cut_dim = -1
        self.cut_m = -1
        self.size = 1  # subtree size in preorder ids

    def empty(self):
        return any(h <= l for l, h in zip(self.lo, self.hi))


class NDOrdering:
    """Result of the oracle's ordering.

    perm[new] = old grid index; atom_ptr[a]..atom_ptr[a+1] are the new
    indices of atom a; atom_node[a] = preorder id of its ND node;
    node_level[id], node_parent[id], node_size[id] (subtree size);
    stage_clusters(s) lists clusters (atom ranges) under cuts of depth <= s.
    """

    def __init__(self, dims, L, nodes, perm, atom_ptr, atom_node, atom_keys):
        self.dims = dims
        self.L = L
        self.nodes = nodes
        self.perm = perm
        self.atom_ptr = atom_ptr
        self.atom_node = atom_node
        self._atom_keys = atom_keys  # per atom: list of (depth, cut node id, key)
        self.node_level = np.array([nd.depth + 1 for nd in nodes], dtype=np.int32)
        self.node_parent = np.array([(-1 if nd.parent is None else nd.parent.id) for nd in nodes],
                                    dtype=np.int32)
        self.node_size = np.array([nd.size for nd in nodes], dtype=np.int32)

    @property
    def n_atoms(self):
        return len(self.atom_node)

    def atom_size(self, a):
        return int(self.atom_ptr[a + 1] - self.atom_ptr[a])

    def related(self, na, nb):
        """True when ND nodes na and nb are equal or one is an ancestor of the other."""
        if na > nb:
            na, nb = nb, na
        return nb < na + self.node_size[na]

    def stage_clusters(self, stage):
        """Clusters under the cuts of depth <= stage, as [first_atom, end_atom) ranges."""
        out = []
        a = 0
        n = self.n_atoms
        while a < n:
            b = a + 1
            key_a = [k for k in self._atom_keys[a] if k[0] <= stage]
            while (b < n and self.atom_node[b] == self.atom_node[a]
                   and [k for k in self._atom_keys[b] if k[0] <= stage] == key_a):
                b += 1
            out.append((a, b))
            a = b
        return out


def hierarchical_atoms(gidx, keys):
    """Atoms of one separator (reading R6): the finest classes of equal keys,
    ordered hierarchically (for each stage depth, coarser classes first, each
    class by the smallest index in it), points by index.  Returns a list of
    (index array, key list)."""
    gidx = np.asarray(gidx, dtype=np.int64)
    depths = sorted(set(k[0] for kk in keys for k in kk))
    sort_cols = []
    for s in depths:
        cls = [tuple(k for k in kk if k[0] <= s) for kk in keys]
        minidx = {}
        for i, cl in enumerate(cls):
            if cl not in minidx or gidx[i] < minidx[cl]:
                minidx[cl] = gidx[i]
        sort_cols.append(np.array([minidx[cl] for cl in cls], dtype=np.int64))
    order = np.lexsort(tuple([gidx] + sort_cols[::-1]))
    atoms = []
    cur = None
    for i in order:
        kk = tuple(keys[i])
        if cur is None or kk != cur[1]:
            cur = ([], kk)
            atoms.append(cur)
        cur[0].append(int(gidx[i]))
    return [(np.array(a, dtype=np.int64), list(k)) for a, k in atoms]


def nd_order(dims, L=None):
    dims = tuple(int(d) for d in dims)
    dim = len(dims)
    N = int(np.prod(dims))
    if L is None:
        L = num_levels(N)
    nodes = []

    def build(lo, hi, depth, parent):
        nd = _Node(len(nodes), depth, lo, hi, parent)
        nodes.append(nd)
        if depth < L - 1:
            ext = [h - l for l, h in zip(lo, hi)]
            c = 0
            for k in range(1, dim):
                if ext[k] > ext[c]:
                    c = k
            m = lo[c] + max(0, (ext[c] - 2) // 2)
            nd.cut_dim = c
            nd.cut_m = m
            llo, lhi = list(lo), list(hi)
            lhi[c] = m
            rlo, rhi = list(lo), list(hi)
            rlo[c] = min(m + 2, hi[c])
            nd.left = build(llo, lhi, depth + 1, nd)
            nd.right = build(rlo, rhi, depth + 1, nd)
            nd.size = 1 + nd.left.size + nd.right.size
        return nd

    build([0] * dim, list(dims), 0, None)

    def node_points(nd):
        """Grid points owned by the node (separator slab or leaf box), sorted by index."""
        lo, hi = list(nd.lo), list(nd.hi)
        if nd.cut_dim >= 0:
            c = nd.cut_dim
            lo[c] = nd.cut_m
            hi[c] = min(nd.cut_m + 2, nd.hi[c])
        if any(h <= l for l, h in zip(lo, hi)):
            return np.zeros((0, dim), dtype=np.int64)
        axes = [np.arange(l, h) for l, h in zip(lo, hi)]
        mesh = np.meshgrid(*axes[::-1], indexing="ij")  # z, y, x with x fastest
        pts = np.stack([m.reshape(-1) for m in mesh[::-1]], axis=1)
        return pts

    strides = [1]
    for k in range(1, dim):
        strides.append(strides[-1] * dims[k - 1])
    strides = np.array(strides, dtype=np.int64)

    def descendants(nd):
        out = []
        stack = [nd.left, nd.right]
        while stack:
            x = stack.pop()
            if x is None:
                continue
            out.append(x)
            stack.append(x.left)
            stack.append(x.right)
        return out

    # per node: list of atoms (each an array of grid indices) and their keys
    node_atoms = {}
    for nd in nodes:
        pts = node_points(nd)
        if pts.shape[0] == 0:
            node_atoms[nd.id] = []
            continue
        gidx = pts @ strides
        if nd.cut_dim < 0:
            node_atoms[nd.id] = [(gidx, [])]
            continue
        c = nd.cut_dim
        left_hi = nd.left.hi[c]
        right_lo = nd.right.lo[c]
        cuts = []
        for D in descendants(nd):
            if D.cut_dim < 0 or D.cut_dim == c or D.empty():
                continue
            if not (D.hi[c] == left_hi or D.lo[c] == right_lo):
                continue
            cuts.append(D)
        cuts.sort(key=lambda D: (D.depth, D.id))
        keys = [[] for _ in range(pts.shape[0])]
        for D in cuts:
            cd = D.cut_dim
            ok = np.ones(pts.shape[0], dtype=bool)
            for e in range(dim):
                if e == c or e == cd:
                    continue
                ok &= (pts[:, e] >= D.lo[e] - 2) & (pts[:, e] < D.hi[e] + 2)
            kv = np.where(pts[:, cd] < D.cut_m, 0, np.where(pts[:, cd] < D.cut_m + 2, 1, 2))
            for i in np.nonzero(ok)[0]:
                keys[i].append((D.depth, D.id, int(kv[i])))
        node_atoms[nd.id] = hierarchical_atoms(gidx, keys)

    order_nodes = sorted(nodes, key=lambda nd: (-nd.depth, nd.id))
    perm = []
    atom_ptr = [0]
    atom_node = []
    atom_keys = []
    for nd in order_nodes:
        for gi, kk in node_atoms[nd.id]:
            perm.append(gi)
            atom_ptr.append(atom_ptr[-1] + gi.shape[0])
            atom_node.append(nd.id)
            atom_keys.append(kk)
    perm = np.concatenate(perm) if perm else np.zeros(0, dtype=np.int64)
    assert perm.shape[0] == N
    return NDOrdering(dims, L, nodes, perm.astype(np.int64), np.array(atom_ptr, dtype=np.int64),
                      np.array(atom_node, dtype=np.int32), atom_keys)
