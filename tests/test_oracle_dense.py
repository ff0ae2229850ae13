"""Pins for the oracle's dense Householder kernels (oracle/dense.py).

Each kernel is checked against something other than itself: LAPACK through
numpy/scipy (same dlarfg sign convention), orthogonality and reconstruction
identities, and matrices with a constructed singular-value gap.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import dense


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (12, 12), (40, 17), (7, 9)])
def test_qr_matches_lapack_geqrf(m, n):
    A = _rng(m * 100 + n).standard_normal((m, n))
    V, tau, R = dense.qr(A)
    # LAPACK dgeqrf (numpy 'raw' mode) uses the same reflector convention
    h, tau_ref = np.linalg.qr(A, mode="raw")
    h = h.T
    t = min(m, n)
    np.testing.assert_allclose(tau, tau_ref[:t], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(R, np.triu(h[:t, :]), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(np.tril(V, -1), np.tril(h[:, :t], -1), rtol=1e-11, atol=1e-12)
    # Q R = A and Q^T Q = I
    Q = dense.apply_q(V, tau, np.eye(m)[:, :t])
    np.testing.assert_allclose(Q @ R, A, atol=1e-12)
    np.testing.assert_allclose(Q.T @ Q, np.eye(t), atol=1e-13)


def test_qr_zero_column_gives_identity_reflector():
    A = np.zeros((4, 2))
    A[0, 1] = 3.0
    V, tau, R = dense.qr(A)
    assert tau[0] == 0.0
    # second column: alpha = 0 (sign(0) = +1), x = 0 -> tau 0 too
    assert R[0, 1] == 3.0


def test_house_sign_convention():
    v, tau, beta = dense.house(np.array([3.0, 4.0]))
    assert beta == -5.0 and abs(tau - 1.6) < 1e-15
    v, tau, beta = dense.house(np.array([-3.0, 4.0]))
    assert beta == 5.0
    v, tau, beta = dense.house(np.array([0.0, 2.0]))
    assert beta == -2.0  # sign(0) = +1


def test_house_sign_tolerance():
    """A leading entry within sign_tol |col| of zero takes beta = -|col| on
    either side of zero; both reflections map col to beta e_1 exactly."""
    for alpha in (-1e-18, 1e-18, -3e-13):
        col = np.array([alpha, 3.0, 4.0])
        v, tau, beta = dense.house(col, sign_tol=1e-12)
        assert beta == -np.sqrt(alpha * alpha + 25.0)
        h = col - tau * v * (v @ col)
        assert abs(h[0] - beta) <= 1e-15 * 5 and np.abs(h[1:]).max() <= 1e-15 * 5
    # outside the tolerance the LAPACK sign stands
    v, tau, beta = dense.house(np.array([-1e-11, 3.0, 4.0]), sign_tol=1e-12)
    assert beta > 0
    v, tau, beta = dense.house(np.array([-1e-18, 3.0, 4.0]))
    assert beta > 0


def test_apply_qt_and_q_are_inverse():
    A = _rng(3).standard_normal((20, 8))
    V, tau, R = dense.qr(A)
    B = _rng(4).standard_normal((20, 5))
    np.testing.assert_allclose(dense.apply_q(V, tau, dense.apply_qt(V, tau, B)), B, atol=1e-13)
    Q = dense.apply_q(V, tau, np.eye(20))
    np.testing.assert_allclose(dense.apply_qt(V, tau, B), Q.T @ B, atol=1e-13)


def test_triangular_solves():
    R = np.triu(_rng(5).standard_normal((9, 9))) + 5 * np.eye(9)
    B = _rng(6).standard_normal((9, 4))
    np.testing.assert_allclose(dense.solve_upper(R, B), np.linalg.solve(R, B), rtol=1e-12)
    C = _rng(7).standard_normal((4, 9))
    np.testing.assert_allclose(dense.solve_upper_right(C, R), C @ np.linalg.inv(R), rtol=1e-11)


@pytest.mark.parametrize("m,c", [(10, 30), (25, 12), (16, 16)])
def test_cpqr_full_matches_lapack_geqp3(m, c):
    """eps = 0: full CPQR; pivots and |R_kk| agree with LAPACK dgeqp3 on generic data."""
    M = _rng(m + 7 * c).standard_normal((m, c)) * np.logspace(0, -3, c)[None, :]
    V, tau, r, rdiag, perm = dense.cpqr_truncated(M, 0.0)
    t = min(m, c)
    assert r == t
    Rref, piv = sla.qr(M, mode="r", pivoting=True)
    np.testing.assert_array_equal(perm[:t], piv[:t])
    np.testing.assert_allclose(rdiag[:t], np.abs(np.diag(Rref))[:t], rtol=1e-10)
    # Q^T M P = R with R upper trapezoidal
    QtM = dense.apply_qt(V, tau, M[:, perm])
    np.testing.assert_allclose(np.tril(QtM, -1)[:, :t], 0.0, atol=1e-12)


def test_cpqr_rank_on_constructed_gap():
    """A matrix with 6 singular values O(1) and the rest 1e-9: rank 6 at eps = 1e-5."""
    rng = _rng(11)
    U, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    W, _ = np.linalg.qr(rng.standard_normal((80, 80)))
    s = np.r_[np.linspace(3, 1, 6), 1e-9 * np.ones(24)]
    M = U @ np.diag(s) @ W[:30]
    V, tau, r, rdiag, perm = dense.cpqr_truncated(M, 1e-5)
    assert r == 6
    assert rdiag[-1] < 1e-5 * rdiag[0] <= rdiag[-2]
    # what is dropped is bounded by sqrt(#cols) * eps * |R_11|
    QtM = dense.apply_qt(V, tau, M)
    assert np.linalg.norm(QtM[r:]) <= np.sqrt(M.shape[1]) * 1e-5 * rdiag[0]
    # numerical rank by SVD at the same relative tolerance agrees here
    assert np.sum(np.linalg.svd(M, compute_uv=False) >= 1e-5 * s[0]) == 6


def test_cpqr_degenerate():
    V, tau, r, rd, perm = dense.cpqr_truncated(np.zeros((5, 0)), 1e-3)
    assert r == 0
    V, tau, r, rd, perm = dense.cpqr_truncated(np.zeros((5, 4)), 1e-3)
    assert r == 0
    V, tau, r, rd, perm = dense.cpqr_truncated(np.zeros((0, 4)), 1e-3)
    assert r == 0
    # ties go to the lowest column index
    M = np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 0.0]])
    V, tau, r, rd, perm = dense.cpqr_truncated(M, 0.0)
    assert perm[0] == 0


def test_cpqr_zero_leading_entry_takes_negative_beta():
    """A pivot column whose leading entry is zero in exact arithmetic: exact
    zero and rounding residue of either sign give the same reflectors and
    the same R (beta = -|column|), so rounding cannot choose the coarse
    basis; a leading entry well outside the tolerance keeps LAPACK's sign."""
    base = np.array([[0.0, 1.0, 0.5],
                     [3.0, 0.2, 0.1],
                     [4.0, 0.3, 0.7],
                     [0.0, 0.4, 0.2]])
    outs = []
    for a in (0.0, 1e-17, -1e-17):
        M = base.copy()
        M[0, 0] = a
        V, tau, r, rd, perm = dense.cpqr_truncated(M, 0.0)
        assert perm[0] == 0 and r == 3
        R = dense.apply_qt(V, tau, M[:, perm])
        assert R[0, 0] < 0
        outs.append((V, tau, R))
    for V, tau, R in outs[1:]:
        np.testing.assert_allclose(V, outs[0][0], atol=1e-15)
        np.testing.assert_allclose(R, outs[0][2], atol=1e-14)
    M = base.copy()
    M[0, 0] = -1e-6
    V, tau, r, rd, perm = dense.cpqr_truncated(M, 0.0)
    assert dense.apply_qt(V, tau, M[:, perm])[0, 0] > 0
