"""Oracle: the spaQR factorisation, its application and GMRES, in plain FP64.

TEST INFRASTRUCTURE ONLY.  Slow and direct; written from the paper
(Gnanasekaran & Darve, "Hierarchical Orthogonal Factorization: Sparse Square
Matrices", arXiv 2010.06807):

  column pre-normalisation ........ Section 2.7 (columns scaled to unit 2-norm)
  ordering ........................ Section 2.3 (oracle.ordering)
  level loop ...................... Algorithm 2 (Section 2.7)
  factor separator s .............. Section 2.4 (block Householder on the
                                    stacked column block, fill among neighbours)
  block-diagonal scaling .......... Section 2.5 ("Scaling of Interfaces")
  sparsification (scaled form) .... Sections 2.2/2.5, rank rule of Section 4
  sparsification (unscaled form) .. Sections 2.2/3.2 with sigma of Lemma 1
  merge ........................... Section 2.6
  factor application .............. Section 2.7 (Q^T A W^{-1} ~ I)
  GMRES to ||Ax-b||/||b|| <= 1e-12  Section 4

Readings where the paper is silent (also in the design notes):
  F1  Blocks only ever exist between clusters whose ND nodes are equal or in an
      ancestor/descendant relation (Section 2.1: no fill between separated
      subtrees; Theorem 2.1).  A front of separator s has rows
      R(s) = {i : block (i, s) exists} and columns C(s) = {j related to s :
      block (i, j) exists for some i in R(s)}; H_s^T is applied to those
      columns only.  R(s) and C(s) of every front of a level are taken from
      the block pattern at the start of that level.
  F2  Fronts of one level that share a row cluster are ordered: colour the
      fronts greedily in ascending id (two fronts conflict when they share a
      row cluster), then process them by (colour, id).
  F3  Scaling and sparsification start after `skip` levels (default 2: the
      paper "skips two levels" / starts "on levels 3 or 4").
  F4  Sparsification is two-phase: every interface's Q_p is computed from the
      matrix after scaling, then all are applied (A_ij <- Q_i^T A_ij Q_j,
      keeping coarse rows/columns).  The paper's loop is sequential and does
      not fix an order.
  F5  M_p = [A_{k1 p}^T ... | A_{p j1} ...], row-neighbours first, then
      column-neighbours, each in ascending cluster id.
  F6  Q_p keeps only the r reflectors of the truncated CPQR; the first r
      columns of Q_p are the coarse basis, and the fine space is its
      complement (the solve only depends on that subspace).
  F7  Unscaled variant (scaling=False; Sections 2.2 and 3.2, Lemma 1): no
      scaling step; every interface p of a sparsified level gets
      sigma_p = 1 / sigma_min(A_p), A_p = [A_pp; A_np] stacked over all rows
      of column p, and M_p = [A_{k1 p}^T ... | sigma_p A_pp^T A_{p j1} ...]
      (row-neighbours first, then column-neighbours, ascending ids).  After the
      CPQR, T_p = A_pp Q_p; the fine columns f = T_p[:, r:] get a Householder
      QR H_p (R_ff), H_p^T is applied to the coarse columns (top |f| rows:
      R_fc, bottom rows: the new coarse diagonal block) and to every block
      A_pj (top |f| rows: R_fn, dropped).  A_np Q_pf and R_fn are dropped.
      Two-phase like F4: every sigma_p, Q_p and H_p comes from the matrix at
      the start of the step, then all blocks are transformed,
      A_ij <- (H_i^T A_ij)[f_i:, :] Q_j[:, :r_j].
  F8  The fine columns A_pp Q_pf often have a leading entry that is zero in
      exact arithmetic, and either reflector sign is valid there.  In the QR
      of those columns a leading entry within 1e-12 |column| of zero takes
      beta = -|column| (sign +1), so that rounding cannot choose the
      reflection and with it the basis of the coarse rows.
"""
from collections import defaultdict

import numpy as np

from . import dense
from .ordering import nd_order, num_levels

__all__ = ["Factor", "factor", "solve", "gmres", "column_norms"]


def column_norms(n, rowptr, colind, val):
    """2-norm of every column of the CSR matrix."""
    s = np.zeros(n)
    np.add.at(s, colind, val * val)
    return np.sqrt(s)


class Factor:
    pass


def _greedy_colours(fronts, rows_of):
    colour = {}
    for s in fronts:  # ascending id
        used = set()
        rs = set(rows_of[s])
        for t in fronts:
            if t >= s:
                break
            if rs & set(rows_of[t]):
                used.add(colour[t])
        c = 0
        while c in used:
            c += 1
        colour[s] = c
    return colour


def factor(n, rowptr, colind, val, dims, eps, nlevels=0, skip=2, ordering=None,
           col_normalize=True, scaling=True, sequential=False):
    """Compute the spaQR factorisation (Algorithm 2) of the CSR matrix A.

    scaling=False gives the unscaled variant of Sections 2.2 / 3.2 (reading
    F7).  sequential=True (scaled variant) sparsifies the interfaces of a
    level one after the other, as the loop of Algorithm 2 is written: each
    CPQR sees the matrix already transformed by the interfaces before it
    (ascending id), instead of the two-phase reading F4.  Returns a Factor with the op sequence and diagnostics (ranks per
    level, CPQR pivot norms, algorithmic flop counts; for the unscaled
    variant also sigma_p and the Lemma 1 quantities per interface).
    """
    rowptr = np.asarray(rowptr, dtype=np.int64)
    colind = np.asarray(colind, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    if ordering is None:
        L = nlevels if nlevels > 0 else num_levels(n)
        ordering = nd_order(dims, L)
    o = ordering
    L = o.L
    F = Factor()
    F.n = n
    F.ordering = o
    F.eps = eps
    F.skip = skip
    # column pre-normalisation (Section 2.7)
    if col_normalize:
        d = 1.0 / column_norms(n, rowptr, colind, val)
    else:
        d = np.ones(n)
    F.d = d
    iperm = np.empty(n, dtype=np.int64)
    iperm[o.perm] = np.arange(n)
    # a row sits with its matched column (general orderings); else rows = columns
    rowcol = getattr(o, "rowcol", None)
    rowpos = iperm[rowcol] if rowcol is not None else iperm
    atom_of = np.searchsorted(o.atom_ptr, np.arange(n), side="right") - 1
    natom = o.n_atoms
    size = {a: o.atom_size(a) for a in range(natom)}
    node = {a: int(o.atom_node[a]) for a in range(natom)}
    span = {a: (a, a + 1) for a in range(natom)}  # atom range of a cluster
    blocks = {}
    for r in range(n):
        nr = rowpos[r]
        ar = atom_of[nr]
        for e in range(rowptr[r], rowptr[r + 1]):
            c = colind[e]
            nc = iperm[c]
            ac = atom_of[nc]
            key = (ar, ac)
            if key not in blocks:
                blocks[key] = np.zeros((size[ar], size[ac]))
            blocks[key][nr - o.atom_ptr[ar], nc - o.atom_ptr[ac]] += val[e] * d[c]
    for (i, j) in blocks:
        assert o.related(node[i], node[j]), "pattern couples separated subtrees"
    active = set(range(natom))
    ops = []
    F.ranks = []       # per level: {cluster: (n_before, r)}
    F.rdiag = []       # per level: {cluster: pivot norms}
    F.dropped = []     # per level: {cluster: (||dropped||_F, #cols of M_p, |R_11|)}
    F.steps = []       # per level: dict(fronts, colours, R, C)
    F.scaling = bool(scaling)
    F.lemma = []       # per level (unscaled): {cluster: dict(sigma, smin, Rff, Wfn2, Rfn)}
    flops = defaultdict(float)

    for k in range(1, L + 1):
        lev = L - k + 1
        col_rows = defaultdict(list)
        row_cols = defaultdict(list)
        for (i, j) in blocks:
            col_rows[j].append(i)
            row_cols[i].append(j)
        fronts = sorted(c for c in active if o.node_level[node[c]] == lev)
        nodes_seen = [node[c] for c in fronts]
        assert len(set(nodes_seen)) == len(nodes_seen), "separator not merged"
        Rof = {}
        Cof = {}
        for s in fronts:
            Rof[s] = sorted(col_rows[s])
            assert Rof[s][0] == s
            cs = set()
            for i in Rof[s]:
                for j in row_cols[i]:
                    if o.related(node[j], node[s]):
                        cs.add(j)
            Cof[s] = sorted(cs)
            assert Cof[s][0] == s
        colour = _greedy_colours(fronts, Rof)
        seq = sorted(fronts, key=lambda s: (colour[s], s))
        F.steps.append(dict(level=lev, fronts=fronts, colour=colour, R=Rof, C=Cof, order=seq,
                            sizes={c: size[c] for c in active}))
        # (i) factor every separator of this level (Section 2.4)
        for s in seq:
            rows = Rof[s]
            rsz = [size[i] for i in rows]
            ns = size[s]
            Fr = np.vstack([blocks[(i, s)] for i in rows])
            m = Fr.shape[0]
            V, tau, R = dense.qr(Fr)
            flops["factor"] += 2.0 * m * ns * ns - 2.0 / 3.0 * ns ** 3
            Rsj = {}
            for j in Cof[s][1:]:
                B = np.vstack([blocks.get((i, j), np.zeros((size[i], size[j]))) for i in rows])
                B = dense.apply_qt(V, tau, B)
                flops["factor"] += (4.0 * m * ns - 2.0 * ns * ns) * size[j]
                Rsj[j] = B[:ns].copy()
                off = ns
                for i, sz in zip(rows[1:], rsz[1:]):
                    blocks[(i, j)] = B[off:off + sz].copy()
                    off += sz
            ops.append(("house", k, s, list(zip(rows, rsz)), V, tau, R[:ns, :ns].copy(), Rsj))
            for key in [key for key in blocks if key[0] == s or key[1] == s]:
                del blocks[key]
            active.discard(s)
        F.ranks.append({})
        F.rdiag.append({})
        F.dropped.append({})
        F.lemma.append({})
        if k > skip and active and not scaling:
            blocks = _sparsify_unscaled(F, k, eps, blocks, active, size, ops, flops)
        # (ii) block-diagonal scaling, (iii) sparsification
        if k > skip and active and scaling:
            act = sorted(active)
            U = {}
            for p in act:
                if size[p] == 0:
                    continue
                Vp, tp, Rp = dense.qr(blocks[(p, p)])
                flops["scale"] += 4.0 / 3.0 * size[p] ** 3
                U[p] = (Vp, tp, Rp)
                ops.append(("scale", k, p, Vp, tp, Rp))
            for key in list(blocks):
                i, j = key
                if i == j:
                    blocks[key] = np.eye(size[i])
                    continue
                B = blocks[key]
                if size[i] > 0 and size[j] > 0:
                    B = dense.apply_qt(U[i][0], U[i][1], B)
                    B = dense.solve_upper_right(B, U[j][2])
                    flops["scale"] += 2.0 * size[i] ** 2 * size[j] + size[j] ** 2 * size[i]
                blocks[key] = B
            col_rows = defaultdict(list)
            row_cols = defaultdict(list)
            for (i, j) in blocks:
                col_rows[j].append(i)
                row_cols[i].append(j)
            Qs = {}
            if sequential:
                blocks = _sparsify_sequential(F, k, eps, blocks, act, size, ops, flops)
                act = []
            for p in act:
                if size[p] == 0:
                    continue
                parts = [blocks[(i, p)].T for i in sorted(col_rows[p]) if i != p]
                parts += [blocks[(p, j)] for j in sorted(row_cols[p]) if j != p]
                Mp = np.hstack(parts) if parts else np.zeros((size[p], 0))
                Vq, tq, r, rd, _ = dense.cpqr_truncated(Mp, eps)
                flops["sparsify"] += 4.0 * size[p] * Mp.shape[1] * r
                Qs[p] = (Vq, tq, r)
                F.ranks[-1][p] = (size[p], r)
                F.rdiag[-1][p] = rd
                # what this interface drops: the fine rows of Q_p^T M_p
                QtM = dense.apply_qt(Vq, tq, Mp) if r > 0 else Mp
                F.dropped[-1][p] = (float(np.linalg.norm(QtM[r:])), Mp.shape[1],
                                    float(rd[0]) if len(rd) else 0.0)
                ops.append(("sparsify", k, p, Vq, tq, r, size[p]))
            newb = {} if not sequential else dict(blocks)
            for (i, j), B in (blocks.items() if not sequential else []):
                if i == j:
                    ri = Qs[i][2] if i in Qs else 0
                    newb[(i, j)] = np.eye(ri)
                    continue
                if i in Qs and Qs[i][2] > 0 and size[j] > 0:
                    B = dense.apply_qt(Qs[i][0], Qs[i][1], B)
                if j in Qs and Qs[j][2] > 0 and size[i] > 0:
                    B = dense.apply_qt(Qs[j][0], Qs[j][1], B.T).T
                ri = Qs[i][2] if i in Qs else 0
                rj = Qs[j][2] if j in Qs else 0
                newb[(i, j)] = B[:ri, :rj].copy()
            blocks = newb
            for p in act:
                size[p] = Qs[p][2] if p in Qs else 0
        # (iv) merge (Section 2.6): classes under cuts of depth <= L-k-1
        if k < L and active:
            stage = L - k - 1
            groups = defaultdict(list)
            for (a0, a1) in o.stage_clusters(stage):
                for c in active:
                    if a0 <= span[c][0] and span[c][1] <= a1:
                        groups[a0].append(c)
            mapping = {}
            for g, members in groups.items():
                members.sort()
                mapping[g] = [(c, size[c]) for c in members]
            child_off = {}
            for g, members in mapping.items():
                off = 0
                for c, sz in members:
                    child_off[c] = (g, off)
                    off += sz
            newb = {}
            newsize = {g: sum(sz for _, sz in mem) for g, mem in mapping.items()}
            for (i, j), B in blocks.items():
                gi, oi = child_off[i]
                gj, oj = child_off[j]
                if (gi, gj) not in newb:
                    newb[(gi, gj)] = np.zeros((newsize[gi], newsize[gj]))
                newb[(gi, gj)][oi:oi + B.shape[0], oj:oj + B.shape[1]] = B
            blocks = newb
            new_active = set()
            for g, mem in mapping.items():
                size[g] = newsize[g]
                node[g] = node[mem[0][0]]
                span[g] = (span[mem[0][0]][0], span[mem[-1][0]][1])
                new_active.add(g)
            active = new_active
            ops.append(("merge", k, mapping))
    assert not active and not blocks
    F.ops = ops
    F.flops = dict(flops)
    return F


def _sparsify_sequential(F, k, eps, blocks, act, size, ops, flops):
    """Scaled sparsification of one level, interface after interface in
    ascending id (Algorithm 2's loop taken literally): M_p is built from the
    current blocks, and Q_p is applied at once -- rows p <- Q_p^T, columns
    p <- Q_p, fine rows / columns dropped, A_pp <- I_r."""
    for p in act:
        if size[p] == 0:
            continue
        rows_of_p = sorted(i for (i, j) in blocks if j == p and i != p)
        cols_of_p = sorted(j for (i, j) in blocks if i == p and j != p)
        parts = [blocks[(i, p)].T for i in rows_of_p] + [blocks[(p, j)] for j in cols_of_p]
        Mp = np.hstack(parts) if parts else np.zeros((size[p], 0))
        Vq, tq, r, rd, _ = dense.cpqr_truncated(Mp, eps)
        flops["sparsify"] += 4.0 * size[p] * Mp.shape[1] * r
        F.ranks[-1][p] = (size[p], r)
        F.rdiag[-1][p] = rd
        QtM = dense.apply_qt(Vq, tq, Mp) if r > 0 else Mp
        F.dropped[-1][p] = (float(np.linalg.norm(QtM[r:])), Mp.shape[1], float(rd[0]) if len(rd) else 0.0)
        ops.append(("sparsify", k, p, Vq, tq, r, size[p]))
        for j in cols_of_p:
            B = dense.apply_qt(Vq, tq, blocks[(p, j)]) if r > 0 and blocks[(p, j)].shape[1] > 0 else blocks[(p, j)]
            blocks[(p, j)] = B[:r].copy()
        for i in rows_of_p:
            B = blocks[(i, p)]
            if r > 0 and B.shape[0] > 0:
                B = dense.apply_qt(Vq, tq, B.T).T
            blocks[(i, p)] = B[:, :r].copy()
        blocks[(p, p)] = np.eye(r)
        size[p] = r
    return blocks


def _sparsify_unscaled(F, k, eps, blocks, active, size, ops, flops):
    """One sparsified level of the unscaled variant (reading F7).

    Returns the new block dictionary (coarse blocks only) and updates size.
    """
    act = sorted(active)
    col_rows = defaultdict(list)
    row_cols = defaultdict(list)
    for (i, j) in blocks:
        col_rows[j].append(i)
        row_cols[i].append(j)
    info = {}
    for p in act:
        np_ = size[p]
        if np_ == 0:
            continue
        rows = sorted(col_rows[p])
        Ap = np.vstack([blocks[(i, p)] for i in rows])
        smin = float(np.linalg.svd(Ap, compute_uv=False)[-1])
        if smin == 0.0:
            raise ZeroDivisionError("interface column block A_p is rank deficient")
        sigma = 1.0 / smin
        App = blocks[(p, p)]
        rparts = [blocks[(i, p)].T for i in rows if i != p]
        cparts = [sigma * (App.T @ blocks[(p, j)]) for j in sorted(row_cols[p]) if j != p]
        nrow = sum(b.shape[1] for b in rparts)
        Mp = np.hstack(rparts + cparts) if rparts or cparts else np.zeros((np_, 0))
        Vq, tq, r, rd, _ = dense.cpqr_truncated(Mp, eps)
        flops["sparsify"] += 4.0 * np_ * Mp.shape[1] * r
        QtM = dense.apply_qt(Vq, tq, Mp) if r > 0 else Mp
        # T_p = A_pp Q_p, Householder QR of its fine columns, H^T on the coarse ones
        Tp = dense.apply_qt(Vq, tq, App.T).T if r > 0 else App.copy()
        f = np_ - r
        if f > 0:
            Vh, th, Rff = dense.qr(Tp[:, r:], sign_tol=1e-12)
            if np.any(np.diag(Rff) == 0.0):
                raise ZeroDivisionError("zero diagonal in R_ff")
            Cc = dense.apply_qt(Vh, th, Tp[:, :r])
        else:
            Vh, th, Rff = np.zeros((np_, 0)), np.zeros(0), np.zeros((0, 0))
            Cc = Tp[:, :r]
        info[p] = dict(Vq=Vq, tq=tq, r=r, Vh=Vh, th=th, f=f, Acc=Cc[f:].copy())
        F.ranks[-1][p] = (np_, r)
        F.rdiag[-1][p] = rd
        F.dropped[-1][p] = (float(np.linalg.norm(QtM[r:])), Mp.shape[1], float(rd[0]) if len(rd) else 0.0)
        F.lemma[-1][p] = dict(sigma=sigma, smin=smin, Rff=Rff, Wfn2=QtM[r:, nrow:].copy(),
                              Wfn1=QtM[r:, :nrow].copy(), Ap=Ap, App=App.copy(),
                              Apn=np.hstack([blocks[(p, j)] for j in sorted(row_cols[p]) if j != p] or
                                            [np.zeros((np_, 0))]), Rfn=[])
        ops.append(("usparsify", k, p, Vq, tq, r, Vh, th, Rff, Cc[:f].copy(), np_))
    newb = {}
    for (i, j), B in blocks.items():
        ri = info[i]["r"] if i in info else 0
        rj = info[j]["r"] if j in info else 0
        if i == j:
            newb[(i, i)] = info[i]["Acc"] if i in info else np.zeros((0, 0))
            continue
        fi = info[i]["f"] if i in info else 0
        if fi > 0 and size[j] > 0:
            B = dense.apply_qt(info[i]["Vh"], info[i]["th"], B)
            F.lemma[-1][i]["Rfn"].append((j, B[:fi].copy()))
        B = B[fi:]
        if rj > 0 and B.shape[0] > 0:
            B = dense.apply_qt(info[j]["Vq"], info[j]["tq"], B.T).T
        newb[(i, j)] = B[:, :rj].copy()
    for p in act:
        size[p] = info[p]["r"] if p in info else 0
    return newb


def _apply_inverse_permuted(F, y):
    """Apply C_1 ... C_K L_K ... L_1 to y (rows in the new ordering)."""
    o = F.ordering
    nrhs = y.shape[1]
    cur = {}
    for a in range(o.n_atoms):
        cur[a] = y[o.atom_ptr[a]:o.atom_ptr[a + 1]].copy()
    saved = {}
    # forward pass: left ops in factor order
    for op in F.ops:
        kind = op[0]
        if kind == "house":
            _, k, s, rows, V, tau, Rss, Rsj = op
            stack = np.vstack([cur[i] for i, _ in rows])
            stack = dense.apply_qt(V, tau, stack)
            off = 0
            for i, sz in rows:
                cur[i] = stack[off:off + sz]
                off += sz
            saved[("z", k, s)] = cur.pop(s)
        elif kind == "scale":
            _, k, p, V, tau, R = op
            cur[p] = dense.apply_qt(V, tau, cur[p])
        elif kind == "sparsify":
            _, k, p, V, tau, r, nb = op
            if r > 0:
                cur[p] = dense.apply_qt(V, tau, cur[p])
            saved[("f", k, p)] = cur[p][r:].copy()
            cur[p] = cur[p][:r].copy()
        elif kind == "usparsify":
            _, k, p, Vq, tq, r, Vh, th, Rff, Rfc, nb = op
            f = nb - r
            yp = dense.apply_qt(Vh, th, cur[p]) if f > 0 else cur[p]
            saved[("f", k, p)] = yp[:f].copy()
            cur[p] = yp[f:].copy()
        elif kind == "merge":
            _, k, mapping = op
            new = {}
            for g, mem in mapping.items():
                new[g] = np.vstack([cur[c] for c, _ in mem]) if mem else np.zeros((0, nrhs))
            cur = new
    assert not cur
    # backward pass: right ops in reverse order
    x = {}
    for op in reversed(F.ops):
        kind = op[0]
        if kind == "merge":
            _, k, mapping = op
            for g, mem in mapping.items():
                xg = x.pop(g)
                off = 0
                for c, sz in mem:
                    x[c] = xg[off:off + sz]
                    off += sz
        elif kind == "sparsify":
            _, k, p, V, tau, r, nb = op
            xp = np.vstack([x[p], saved[("f", k, p)]])
            if r > 0:
                xp = dense.apply_q(V, tau, xp)
            x[p] = xp
        elif kind == "usparsify":
            _, k, p, Vq, tq, r, Vh, th, Rff, Rfc, nb = op
            xc = x[p]
            yf = saved[("f", k, p)]
            xf = dense.solve_upper(Rff, yf - Rfc @ xc) if nb > r else yf
            xp = np.vstack([xc, xf])
            if r > 0:
                xp = dense.apply_q(Vq, tq, xp)
            x[p] = xp
        elif kind == "scale":
            _, k, p, V, tau, R = op
            x[p] = dense.solve_upper(R, x[p])
        elif kind == "house":
            _, k, s, rows, V, tau, Rss, Rsj = op
            rhs = saved[("z", k, s)].copy()
            for j, B in Rsj.items():
                rhs -= B @ x[j]
            x[s] = dense.solve_upper(Rss, rhs)
    out = np.zeros_like(y)
    for a in range(o.n_atoms):
        out[o.atom_ptr[a]:o.atom_ptr[a + 1]] = x[a]
    return out


def solve(F, b):
    """x = M^{-1} b for the spaQR factor F (one application, Section 2.7)."""
    b = np.asarray(b, dtype=np.float64)
    vec = b.ndim == 1
    B = b.reshape(F.n, -1)
    rperm = getattr(F.ordering, "rperm", None)
    yp = _apply_inverse_permuted(F, B[rperm if rperm is not None else F.ordering.perm])
    y = np.empty_like(yp)
    y[F.ordering.perm] = yp
    x = F.d[:, None] * y
    return x.reshape(b.shape) if not vec else x[:, 0]


def _matvec(n, rowptr, colind, val, x):
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    y = np.zeros(n)
    np.add.at(y, rows, val * x[colind])
    return y


def gmres(n, rowptr, colind, val, b, precond, tol=1e-12, maxit=300):
    """Right-preconditioned GMRES (modified Gram-Schmidt Arnoldi, Givens).

    x0 = 0; no restart within maxit.  Convergence: the recomputed true
    residual ||b - A x|| / ||b|| <= tol (Section 4).  x and the true residual
    are formed only at an iteration whose Arnoldi residual estimate
    |g_{j+1}| / ||b|| is <= tol, at a breakdown (zero subdiagonal entry before
    its rotation: the Krylov space is invariant) and at maxit.  Returns (x,
    iters, relres, history of the Arnoldi residual estimates).
    """
    rowptr = np.asarray(rowptr, dtype=np.int64)
    colind = np.asarray(colind, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    x = np.zeros(n)
    if bnorm == 0.0:
        return x, 0, 0.0, [0.0]
    Vb = np.zeros((maxit + 1, n))
    H = np.zeros((maxit + 1, maxit))
    cs = np.zeros(maxit)
    sn = np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = bnorm
    Vb[0] = b / bnorm
    hist = [1.0]
    relres = 1.0
    Z = []
    for j in range(maxit):
        z = precond(Vb[j])
        Z.append(z)
        w = _matvec(n, rowptr, colind, val, z)
        for i in range(j + 1):
            H[i, j] = Vb[i] @ w
            w = w - H[i, j] * Vb[i]
        H[j + 1, j] = float(np.linalg.norm(w))
        # breakdown: the Krylov space is invariant, and the Arnoldi step has
        # no next basis vector (tested here, before the rotation below
        # zeroes this entry)
        breakdown = H[j + 1, j] == 0.0
        if not breakdown:
            Vb[j + 1] = w / H[j + 1, j]
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        den = np.hypot(H[j, j], H[j + 1, j])
        cs[j] = H[j, j] / den
        sn[j] = H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        est = abs(g[j + 1]) / bnorm
        hist.append(est)
        if est <= tol or breakdown or j == maxit - 1:
            yk = dense.solve_upper(H[:j + 1, :j + 1], g[:j + 1])
            xt = np.zeros(n)
            for i in range(j + 1):
                xt += yk[i] * Z[i]
            res = float(np.linalg.norm(b - _matvec(n, rowptr, colind, val, xt))) / bnorm
            x, relres = xt, res
            if res <= tol or breakdown:
                return x, j + 1, relres, hist
    return x, maxit, relres, hist
