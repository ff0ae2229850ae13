"""Expected factor blocks from the oracle, keyed like the GPU's stored blocks
(spaqr_factor_block): (level, kind, cluster, other).

The oracle's op sequence (oracle/spaqr.py) holds every factor the GPU keeps:
  house     -> front panel (reflectors below the diagonal, R_ss on and above),
               its Householder scalars, and R_sj per column cluster j
  scale     -> U_pp reflectors below the diagonal with R_pp on and above, tau
  sparsify  -> the CPQR reflectors Q_pp (explicit, |p| x r) and their tau
  usparsify -> the same CPQR factors, plus the unscaled form's fine QR: R_fc
               (top |f| rows of columns :r) and the QR of the fine columns
               (columns r:), and the scalars of H_p
Levels: the oracle counts steps k = 1..L from the leaves, the GPU levels
0..L-1.
"""
import numpy as np


def _panel(V, R, ns):
    """Reflectors strictly below the diagonal, R (first ns rows) on and above."""
    P = np.tril(V, -1).astype(np.float64)
    P[:ns, :] += np.triu(R[:ns, :V.shape[1]])
    return P


def expected_blocks(Fo):
    """dict key -> (array, mask): mask selects the entries the GPU block is
    compared on (None: all of them)."""
    out = {}
    for op in Fo.ops:
        kind = op[0]
        if kind == "house":
            _, k, s, rows, V, tau, Rss, Rsj = op
            ns = Rss.shape[0]
            if ns == 0:
                continue
            lev = k - 1
            out[(lev, "front", s, -1)] = (_panel(V, Rss, ns), None)
            out[(lev, "front_tau", s, -1)] = (np.asarray(tau, dtype=np.float64).reshape(-1, 1), None)
            for j, B in Rsj.items():
                if B.shape[1] > 0:
                    out[(lev, "rsj", s, j)] = (B, None)
        elif kind == "scale":
            _, k, p, Vp, tp, Rp = op
            out[(k - 1, "scale", p, -1)] = (_panel(Vp, Rp, Rp.shape[0]), None)
            out[(k - 1, "scale_tau", p, -1)] = (np.asarray(tp).reshape(-1, 1), None)
        elif kind == "sparsify":
            _, k, p, Vq, tq, r, nb = op
            if r > 0:
                out[(k - 1, "cpqr", p, -1)] = (Vq, None)
                out[(k - 1, "cpqr_tau", p, -1)] = (np.asarray(tq).reshape(-1, 1), None)
        elif kind == "usparsify":
            _, k, p, Vq, tq, r, Vh, th, Rff, Rfc, nb = op
            if r > 0:
                out[(k - 1, "cpqr", p, -1)] = (Vq, None)
                out[(k - 1, "cpqr_tau", p, -1)] = (np.asarray(tq).reshape(-1, 1), None)
            f = nb - r
            E = np.zeros((nb, nb))
            M = np.zeros((nb, nb), dtype=bool)
            E[:f, :r] = Rfc
            M[:f, :r] = True
            if f > 0:
                E[:, r:] = _panel(Vh, Rff, f)
                M[:, r:] = True
                out[(k - 1, "fine_tau", p, -1)] = (np.asarray(th).reshape(-1, 1), None)
            out[(k - 1, "fine", p, -1)] = (E, M)
    return out


def compare_blocks(blocks, Fo, tol):
    """Every GPU block against the oracle's, entry by entry: the largest
    entry difference of a block, over its largest entry (its Frobenius norm
    for the relative Frobenius error), at most tol.  An R_sj block is a piece
    of the row s of the triangular factor, and some are zero in exact
    arithmetic (rounding residue of order 1e-18 against entries of order 1 in
    R_ss): its scale is the larger of its own and that of R_ss of the same
    front, so that it is compared relative to the factor row it belongs to.
    The two sets of keys must be equal.  Returns (number of blocks, worst
    max-entry error, worst Frobenius error)."""
    exp = expected_blocks(Fo)
    got = {}
    for b in blocks:
        key = (b["level"], b["kind"], b["cluster"], b["other"])
        assert key not in got, f"block {key} stored twice"
        got[key] = b["data"]
    missing = sorted(set(exp) - set(got))
    extra = sorted(set(got) - set(exp))
    assert not missing and not extra, f"blocks missing on the GPU: {missing[:5]}; not in the oracle: {extra[:5]}"
    worst_max = worst_fro = 0.0
    for key, (E, mask) in exp.items():
        G = got[key]
        assert G.shape == E.shape, f"{key}: shape {G.shape} vs {E.shape}"
        if mask is not None:
            G = np.where(mask, G, 0.0)
            E = np.where(mask, E, 0.0)
        d = np.abs(G - E)
        scale = np.abs(E).max() if E.size else 0.0
        fscale = float(np.linalg.norm(E))
        if key[1] == "rsj":
            P = exp[(key[0], "front", key[2], -1)][0]
            Rss = np.triu(P[:P.shape[1], :])
            scale = max(scale, float(np.abs(Rss).max()))
            fscale = max(fscale, float(np.linalg.norm(Rss)))
        if scale == 0.0:
            assert d.max(initial=0.0) <= 1e-14, f"{key}: nonzero entries where the oracle has none"
            continue
        em = float(d.max()) / scale
        ef = float(np.linalg.norm(G - E)) / fscale
        assert em <= tol and ef <= tol, f"{key}: max-entry error {em:.3e}, Frobenius {ef:.3e}"
        worst_max = max(worst_max, em)
        worst_fro = max(worst_fro, ef)
    return len(exp), worst_max, worst_fro
