"""Pins for the oracle's spaQR factorisation, solve and GMRES (oracle/spaqr.py).

What fixes the answer here is mathematics the paper states, not the oracle:
  * without scaling/sparsification the block factorisation is plain
    Householder QR of A D P in nested-dissection order, so its R must equal
    LAPACK's R of the dense permuted matrix (Section 2.1/2.4; R is unique for
    a fixed reflector sign convention);
  * eps = 0 drops nothing: one application solves A x = b to rounding
    (rank rule of Section 4, drop step of Section 2.5);
  * eps > 0: ||A M^{-1} - I|| = O(eps) and kappa <= (1+|E|)/(1-|E|) (Section 3.3) and each interface drops
    at most sqrt(#cols) * eps * |R_11| (rank rule);
  * GMRES reaches ||b - A x|| / ||b|| <= 1e-12 and needs fewer iterations for
    smaller eps (Section 4, Figure "ad_eps").
"""
import numpy as np
import pytest

from oracle import spaqr, dense
from oracle.ordering import nd_order
from synth.convdiff import config_problem, rhs


def _prob(kind, n, seed=None):
    return config_problem(kind, n=n, seed=seed)


def _assembled_R(F):
    o = F.ordering
    N = F.n
    R = np.zeros((N, N))
    for op in F.ops:
        if op[0] != "house":
            continue
        _, k, s, rows, V, tau, Rss, Rsj = op
        r0 = o.atom_ptr[s]
        ns = Rss.shape[0]
        R[r0:r0 + ns, r0:r0 + ns] = Rss
        for j, B in Rsj.items():
            c0 = o.atom_ptr[j]
            R[r0:r0 + ns, c0:c0 + B.shape[1]] = B
    return R


@pytest.mark.parametrize("kind,n,L", [("2d_uniform_a", 16, 3), ("2d_uniform_a", 24, 4),
                                      ("2d_lognormal", 16, 3), ("3d_uniform_a", 6, 3)])
def test_direct_mode_equals_dense_householder_R(kind, n, L):
    p = _prob(kind, n)
    F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 0.0, nlevels=L, skip=L + 1)
    A = p.to_dense() * F.d[None, :]
    Ap = A[np.ix_(F.ordering.perm, F.ordering.perm)]
    Rref = np.linalg.qr(Ap, mode="r")
    R = _assembled_R(F)
    scale = np.abs(Rref).max()
    assert np.abs(R - Rref).max() <= 1e-12 * scale
    # column pre-normalisation: every column of A D has unit norm
    np.testing.assert_allclose(np.linalg.norm(A, axis=0), 1.0, rtol=1e-14)


@pytest.mark.parametrize("kind,n,L,skip", [("2d_uniform_a", 16, 3, 0), ("2d_uniform_a", 32, 4, 0),
                                           ("2d_uniform_a", 32, 4, 1), ("2d_lognormal", 32, 4, 0),
                                           ("3d_uniform_a", 8, 3, 0)])
def test_eps0_is_exact(kind, n, L, skip):
    p = _prob(kind, n)
    F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 0.0, nlevels=L, skip=skip)
    b = rhs(p, 3)
    x = spaqr.solve(F, b)
    rel = np.linalg.norm(b - p.matvec(x), axis=0) / np.linalg.norm(b, axis=0)
    assert rel.max() < 1e-12
    # with eps = 0 the rank is min(|p|, #cols) for every interface
    for lev, R in enumerate(F.ranks):
        for c, (nb, r) in R.items():
            assert r == min(nb, F.dropped[lev][c][1])


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-4])
def test_preconditioned_operator_is_identity_plus_O_eps(eps):
    p = _prob("2d_uniform_a", 24)
    F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, nlevels=4, skip=0)
    A = p.to_dense()
    AM = A @ spaqr.solve(F, np.eye(p.n))   # right-preconditioned operator = Q S Q^T
    E = np.linalg.norm(AM - np.eye(p.n), 2)
    assert E < 20 * eps
    if E < 1:
        sv = np.linalg.svd(AM, compute_uv=False)
        assert sv[0] / sv[-1] <= (1 + E) / (1 - E) * (1 + 1e-10)
    assert any(r < nb for R in F.ranks for (nb, r) in R.values())  # something was dropped


def test_dropped_blocks_bounded_by_rank_rule():
    p = _prob("2d_uniform_a", 32)
    eps = 1e-2
    F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, nlevels=4, skip=0)
    n_checked = 0
    for lev in F.dropped:
        for c, (fro, ncols, R11) in lev.items():
            assert fro <= np.sqrt(max(ncols, 1)) * eps * R11 * (1 + 1e-12)
            n_checked += 1
    assert n_checked > 10


def test_stored_orthogonal_factors():
    p = _prob("2d_uniform_a", 32)
    F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 1e-3, nlevels=4, skip=0)
    for op in F.ops:
        if op[0] in ("house", "scale", "sparsify"):
            V, tau = op[4], op[5]
            if op[0] in ("scale",):
                V, tau = op[3], op[4]
            if op[0] == "sparsify":
                V, tau = op[3], op[4]
            m = V.shape[0]
            Q = dense.apply_q(V, tau, np.eye(m))
            np.testing.assert_allclose(Q.T @ Q, np.eye(m), atol=1e-13)


def test_gmres_converges_and_iterations_fall_with_eps():
    p = _prob("2d_uniform_a", 32)
    b = rhs(p, 1)[:, 0]
    its = []
    for eps in (1e-1, 1e-3, 1e-6):
        F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, nlevels=4, skip=0)
        x, it, rel, hist = spaqr.gmres(p.n, p.rowptr, p.colind, p.val, b, lambda v: spaqr.solve(F, v))
        assert rel <= 1e-12
        assert np.linalg.norm(b - p.matvec(x)) / np.linalg.norm(b) <= 1e-12
        its.append(it)
    assert its[0] > its[1] >= its[2]


def test_singleton_and_tiny_grids():
    # L = 1: the whole matrix is one leaf; one dense QR
    p = _prob("2d_uniform_a", 4)
    F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 1e-2)
    assert F.ordering.L == 1
    b = rhs(p, 1)
    x = spaqr.solve(F, b)
    assert np.linalg.norm(b - p.matvec(x)) / np.linalg.norm(b) < 1e-13
    # degenerate boxes (extent < 3) still factor exactly
    p = _prob("2d_uniform_a", 5)
    F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 0.0, nlevels=4, skip=0)
    b = rhs(p, 2)
    x = spaqr.solve(F, b)
    assert np.linalg.norm(b - p.matvec(x)) / np.linalg.norm(b) < 1e-12


@pytest.mark.parametrize("kind,n,eps", [("2d_uniform_a", 32, 1e-2), ("2d_lognormal", 48, 1e-1), ("3d_uniform_a", 10, 1e-2)])
def test_sequential_sparsification_close_to_two_phase(kind, n, eps):
    """Algorithm 2's loop taken literally (each interface's CPQR sees the
    earlier interfaces' transformations) against the two-phase reading F4:
    eps = 0 stays exact, and the GMRES iterations and total ranks are close."""
    p = _prob(kind, n)
    b = rhs(p, 1)[:, 0]
    F0 = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 0.0, skip=0, sequential=True)
    x = spaqr.solve(F0, b)
    assert np.linalg.norm(b - p.matvec(x)) / np.linalg.norm(b) < 1e-12
    out = []
    for seq in (False, True):
        F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, skip=1, sequential=seq)
        _, it, rr, _ = spaqr.gmres(p.n, p.rowptr, p.colind, p.val, b, lambda v: spaqr.solve(F, v))
        assert rr <= 1e-12
        out.append((it, sum(r for lev in F.ranks for (_, r) in lev.values())))
    assert abs(out[0][0] - out[1][0]) <= 3
    assert abs(out[0][1] - out[1][1]) <= 0.05 * out[0][1]


def _krylov_min_residuals(Aop, b, jmax):
    """min over y in K_j(A, b) of ||b - A y|| / ||b||, j = 1..jmax, by brute
    force: an orthonormal basis of the Krylov space from numpy's QR of
    [b, Ab, ..., A^{j-1} b] (columns normalised first) and a least-squares
    solve over it (the definition of the GMRES iterate, Section 4)."""
    n = b.shape[0]
    K = np.zeros((n, jmax))
    v = b / np.linalg.norm(b)
    for j in range(jmax):
        K[:, j] = v
        v = Aop(v)
        v = v / np.linalg.norm(v)
    out = []
    for j in range(1, jmax + 1):
        Qk, _ = np.linalg.qr(K[:, :j])
        AQ = np.column_stack([Aop(Qk[:, i]) for i in range(j)])
        y, *_ = np.linalg.lstsq(AQ, b, rcond=None)
        out.append(np.linalg.norm(b - AQ @ y) / np.linalg.norm(b))
    return np.array(out)


def test_gmres_estimates_equal_krylov_minimum():
    """The Arnoldi residual estimates are the minimum residuals over the
    Krylov spaces of A M^{-1} (right preconditioning), computed here by
    brute force; a dropped Givens rotation, a wrong sign in it or a
    left-preconditioned residual fails this."""
    p = _prob("2d_uniform_a", 12)
    b = rhs(p, 1)[:, 0]
    F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 1e-1, nlevels=3, skip=0)
    _, it, rr, hist = spaqr.gmres(p.n, p.rowptr, p.colind, p.val, b, lambda v: spaqr.solve(F, v))
    jm = min(it, 6)
    ref = _krylov_min_residuals(lambda v: p.matvec(spaqr.solve(F, v)), b, jm)
    np.testing.assert_allclose(hist[1:jm + 1], ref, rtol=1e-6, atol=1e-14)


def test_gmres_stops_at_first_estimate_below_tol():
    """The true residual is recomputed only once the Arnoldi estimate passes
    tol, so the iteration count is the first j with estimate <= tol (when the
    recomputed residual passes there too), and a looser tol stops earlier."""
    p = _prob("2d_uniform_a", 16)
    b = rhs(p, 1)[:, 0]
    F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 1e-1, nlevels=3, skip=0)
    for tol in (1e-6, 1e-12):
        x, it, rr, hist = spaqr.gmres(p.n, p.rowptr, p.colind, p.val, b, lambda v: spaqr.solve(F, v), tol=tol)
        first = next(j for j in range(1, len(hist)) if hist[j] <= tol)
        assert it == first and rr <= tol
        assert np.linalg.norm(b - p.matvec(x)) / np.linalg.norm(b) == pytest.approx(rr, rel=1e-12)
        assert all(h > tol for h in hist[1:it])


def test_gmres_exact_breakdown():
    """A M^{-1} = I (the exact inverse as preconditioner): the first Arnoldi
    vector spans an invariant space, the next basis vector is exactly zero,
    and GMRES stops after one iteration with the exact solution."""
    p = _prob("2d_uniform_a", 6)
    b = rhs(p, 1)[:, 0]
    Ad = np.zeros((p.n, p.n))
    for r in range(p.n):
        for e in range(p.rowptr[r], p.rowptr[r + 1]):
            Ad[r, p.colind[e]] += p.val[e]
    Ainv = np.linalg.inv(Ad)

    def exact(v):
        return Ainv @ v

    def ident_matvec_solver(v):
        return v

    # identity matrix and identity preconditioner: w = v_0 exactly
    n = 8
    rp = np.arange(n + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int64)
    va = np.ones(n)
    bb = np.linspace(1.0, 2.0, n)
    x, it, rr, hist = spaqr.gmres(n, rp, ci, va, bb, ident_matvec_solver, tol=0.0, maxit=5)
    assert it == 1 and rr == 0.0 and np.array_equal(x, bb)
    # the exact inverse on a grid matrix: converged after one iteration
    x, it, rr, _ = spaqr.gmres(p.n, p.rowptr, p.colind, p.val, b, exact)
    assert it == 1 and rr <= 1e-13
