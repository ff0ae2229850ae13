"""Oracle: textbook dense Householder kernels in FP64 (numpy).

TEST INFRASTRUCTURE ONLY.

Householder convention (LAPACK dlarfg reading; the paper only says
"Householder"): for a column (alpha, x), if x = 0 then tau = 0 and the
reflector is the identity; otherwise beta = -sign(alpha) * sqrt(alpha^2 + x.x)
with sign(0) = +1, tau = (beta - alpha) / beta, v = (1, x / (alpha - beta)).
H = I - tau v v^T.  A QR factor stores the reflectors in the strictly lower
part of the factored matrix (unit diagonal implied) and R in the upper part.
"""
import numpy as np

__all__ = ["house", "qr", "apply_qt", "apply_q", "cpqr_truncated", "solve_upper",
           "solve_upper_right"]


def house(col, sign_tol=0.0):
    """Return (v, tau, beta) for the column vector col (length >= 1).

    sign_tol > 0: alpha counts as negative only below -sign_tol * |col|, so a
    leading entry that is zero up to rounding always gives beta = -|col|
    (both signs give a valid reflector; the tolerance keeps rounding from
    choosing between them).
    """
    alpha = float(col[0])
    x = col[1:]
    xnorm2 = float(np.dot(x, x)) if x.shape[0] else 0.0
    v = np.zeros_like(col)
    v[0] = 1.0
    if xnorm2 == 0.0:
        return v, 0.0, alpha
    s = np.sqrt(alpha * alpha + xnorm2)
    beta = -s if alpha >= -sign_tol * s else s
    tau = (beta - alpha) / beta
    v[1:] = x / (alpha - beta)
    return v, tau, beta


def qr(A, sign_tol=0.0):
    """Unblocked Householder QR of an m x n matrix (m >= n not required).

    Returns (V, tau, R): V is m x t unit lower trapezoidal, tau has t entries,
    R is t x n upper trapezoidal, t = min(m, n).  A = Q R with
    Q = H_0 H_1 ... H_{t-1} (first t columns).  sign_tol: see house().
    """
    A = np.array(A, dtype=np.float64, copy=True)
    m, n = A.shape
    t = min(m, n)
    V = np.zeros((m, t))
    tau = np.zeros(t)
    for k in range(t):
        v, tk, beta = house(A[k:, k], sign_tol)
        V[k:, k] = v
        tau[k] = tk
        A[k, k] = beta
        A[k + 1:, k] = 0.0
        if tk != 0.0 and k + 1 < n:
            w = v @ A[k:, k + 1:]
            A[k:, k + 1:] -= tk * np.outer(v, w)
    return V, tau, np.triu(A[:t, :])


def apply_qt(V, tau, B):
    """Q^T B with Q = H_0 ... H_{t-1}; B has V.shape[0] rows."""
    B = np.array(B, dtype=np.float64, copy=True)
    for k in range(V.shape[1]):
        if tau[k] == 0.0:
            continue
        v = V[k:, k]
        w = v @ B[k:]
        B[k:] -= tau[k] * np.outer(v, w)
    return B


def apply_q(V, tau, B):
    """Q B with Q = H_0 ... H_{t-1}."""
    B = np.array(B, dtype=np.float64, copy=True)
    for k in range(V.shape[1] - 1, -1, -1):
        if tau[k] == 0.0:
            continue
        v = V[k:, k]
        w = v @ B[k:]
        B[k:] -= tau[k] * np.outer(v, w)
    return B


def solve_upper(R, B):
    """R^{-1} B by back substitution (R upper triangular, non-singular)."""
    R = np.asarray(R, dtype=np.float64)
    X = np.array(B, dtype=np.float64, copy=True)
    n = R.shape[0]
    for i in range(n - 1, -1, -1):
        if i + 1 < n:
            X[i] -= R[i, i + 1:] @ X[i + 1:]
        X[i] /= R[i, i]
    return X


def solve_upper_right(B, R):
    """B R^{-1} (column-wise forward substitution)."""
    R = np.asarray(R, dtype=np.float64)
    X = np.array(B, dtype=np.float64, copy=True)
    n = R.shape[0]
    for j in range(n):
        if j > 0:
            X[:, j] -= X[:, :j] @ R[:j, j]
        X[:, j] /= R[j, j]
    return X


# Leading entries within this fraction of the column norm count as zero in
# the CPQR's reflectors (beta = -|column|).
CPQR_SIGN_TOL = 1e-12


def cpqr_truncated(M, eps):
    """Column-pivoted Householder QR of M (m x c), truncated at tolerance eps.

    Rank rule (Section 4): keep step k while |R_kk| >= eps |R_11|.  At step k
    every remaining column's norm over rows k..m-1 is recomputed from scratch
    (no downdating); the pivot is the largest, ties to the lowest column index.
    |R_kk| is taken as that recomputed pivot norm.  Stops at the first step that
    fails the rule.  If M has no rows/columns or R_11 = 0, the rank is 0.
    The reflector of each step takes the sign tolerance CPQR_SIGN_TOL (see
    house()): M_p is assembled from sparse blocks, so the pivot column's
    leading entry is often zero in exact arithmetic, and only a tolerance
    keeps rounding from choosing the reflection (and with it the coarse basis
    vectors' signs and every later reflector).

    Returns (V, tau, r, rdiag, perm): V is m x r, tau r entries, rdiag the
    pivot norms |R_kk| of the r kept steps plus the first rejected one (if any),
    perm the column permutation applied.
    """
    M = np.array(M, dtype=np.float64, copy=True)
    m, c = M.shape
    perm = np.arange(c)
    t = min(m, c)
    V = np.zeros((m, t))
    tau = np.zeros(t)
    rdiag = []
    r = 0
    R11 = 0.0
    for k in range(t):
        norms2 = np.sum(M[k:, k:] * M[k:, k:], axis=0)
        j = k + int(np.argmax(norms2))
        pn = float(np.sqrt(norms2[j - k]))
        rdiag.append(pn)
        if k == 0:
            R11 = pn
            if R11 == 0.0:
                break
        if pn < eps * R11:
            break
        if j != k:
            M[:, [k, j]] = M[:, [j, k]]
            perm[[k, j]] = perm[[j, k]]
        v, tk, beta = house(M[k:, k], CPQR_SIGN_TOL)
        V[k:, k] = v
        tau[k] = tk
        M[k, k] = beta
        M[k + 1:, k] = 0.0
        if tk != 0.0 and k + 1 < c:
            w = v @ M[k:, k + 1:]
            M[k:, k + 1:] -= tk * np.outer(v, w)
        r = k + 1
    return V[:, :r].copy(), tau[:r].copy(), r, np.array(rdiag), perm
