"""Pins for the oracle's unscaled spaQR variant (oracle/spaqr.py, scaling=False).

What fixes the answer here is mathematics the paper states, not the oracle:
  * eps = 0 drops nothing, so one application solves A x = b to rounding;
  * the proof of Lemma 1 (Section 3.2 / appendix) rests on the identity
    sigma R_ff^T R_fn = W_fn^(2): the dropped R_fn is tied to the dropped rows
    of the CPQR of M_p by R_ff.  Both sides are computed independently (R_fn
    from the Householder QR of the fine columns applied to the rows of p,
    W_fn from the CPQR of M_p), so a wrong sigma, a transposed A_pp, H taken on
    the wrong columns or a swapped fine/coarse split breaks it;
  * from that identity and sigma = 1 / sigma_min(A_p):
    ||R_fn|| <= ||W_fn^(2)|| / sqrt(1 - (sigma ||W_fn^(1)||)^2), the exact form
    of the bound of Lemma 1;
  * sigma_p sigma_min(A_p) = 1 with sigma_min from the eigenvalues of
    A_p^T A_p (another route than the SVD the oracle calls);
  * with no sparsified level the variant is the plain block QR, equal to the
    scaled variant;
  * GMRES reaches 1e-12 and needs fewer iterations for smaller eps.
"""
import numpy as np
import pytest

from oracle import spaqr
from synth.convdiff import config_problem, rhs


def _fac(kind, n, eps, L, skip, scaling=False, seed=None):
    p = config_problem(kind, n=n, seed=seed)
    return p, spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, nlevels=L, skip=skip, scaling=scaling)


def _interfaces(F):
    for lev in F.lemma:
        for c, d in lev.items():
            yield c, d


@pytest.mark.parametrize("kind,n,L,skip", [("2d_uniform_a", 16, 3, 0), ("2d_uniform_a", 32, 4, 0),
                                           ("2d_lognormal", 32, 4, 1), ("3d_uniform_a", 8, 3, 0)])
def test_unscaled_eps0_is_exact(kind, n, L, skip):
    p, F = _fac(kind, n, 0.0, L, skip)
    assert any(F.lemma), "no sparsified level"
    b = rhs(p, 2)
    x = spaqr.solve(F, b)
    rel = np.linalg.norm(b - p.matvec(x), axis=0) / np.linalg.norm(b, axis=0)
    assert rel.max() < 1e-12
    for lev, R in enumerate(F.ranks):
        for c, (nb, r) in R.items():
            assert r == min(nb, F.dropped[lev][c][1])


@pytest.mark.parametrize("kind,n,L,eps", [("2d_uniform_a", 32, 4, 1e-2), ("2d_lognormal", 32, 4, 1e-1),
                                          ("2d_uniform_a", 48, 5, 1e-3), ("3d_uniform_a", 10, 4, 1e-2)])
def test_lemma1_identity_and_bound(kind, n, L, eps):
    _, F = _fac(kind, n, eps, L, 0)
    checked = 0
    for c, d in _interfaces(F):
        f = d["Rff"].shape[0]
        if f == 0 or not d["Rfn"]:
            continue
        Rfn = np.hstack([B for _, B in sorted(d["Rfn"], key=lambda t: t[0])])
        W2 = d["Wfn2"]
        W1 = d["Wfn1"]
        assert Rfn.shape == W2.shape
        sigma = d["sigma"]
        lhs = sigma * d["Rff"].T @ Rfn
        # rounding scale of W2 = sigma Q_f^T A_pp^T A_pn (cancellation to O(eps))
        scale = sigma * np.linalg.norm(d["App"], 2) * np.linalg.norm(d["Apn"], 2)
        assert np.linalg.norm(lhs - W2) <= 1e-12 * scale * np.sqrt(W2.size) + 1e-12 * np.linalg.norm(W2)
        # Lemma 1, exact form
        w1 = sigma * np.linalg.norm(W1, 2) if W1.size else 0.0
        if w1 < 0.5:
            bound = np.linalg.norm(W2, 2) / np.sqrt(1.0 - w1 * w1)
            assert np.linalg.norm(Rfn, 2) <= bound * (1 + 1e-9) + 1e-13 * scale
        if np.linalg.norm(W2) > 1e3 * 1e-12 * scale:
            checked += 1
    assert checked >= 3


def test_sigma_is_inverse_smallest_singular_value():
    _, F = _fac("2d_lognormal", 32, 1e-2, 4, 0)
    n = 0
    for c, d in _interfaces(F):
        Ap = d["Ap"]
        lam = np.linalg.eigvalsh(Ap.T @ Ap)
        smin = np.sqrt(lam[0])
        assert abs(d["sigma"] * smin - 1.0) <= 1e-8
        # A_p stacks the diagonal block and every row-neighbour block of column p
        assert Ap.shape[0] >= Ap.shape[1]
        n += 1
    assert n > 5


def test_dropped_parts_follow_rank_rule():
    """What the variant drops of Q^T M_p obeys the rank rule: below
    sqrt(#cols) eps |R_11| whenever the CPQR stopped early."""
    _, F = _fac("2d_uniform_a", 32, 1e-2, 4, 0)
    for lev, drops in enumerate(F.dropped):
        for c, (dnorm, ncols, r11) in drops.items():
            nb, r = F.ranks[lev][c]
            if r < min(nb, ncols):
                assert dnorm <= np.sqrt(ncols) * 1e-2 * r11 * (1 + 1e-12)


@pytest.mark.parametrize("kind,n,L", [("2d_uniform_a", 24, 3), ("3d_uniform_a", 8, 3)])
def test_no_sparsified_level_equals_scaled(kind, n, L):
    p = config_problem(kind, n=n)
    a = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 1e-2, nlevels=L, skip=L + 1, scaling=False)
    b = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 1e-2, nlevels=L, skip=L + 1, scaling=True)
    assert not any(a.lemma)
    x = rhs(p, 1)
    np.testing.assert_array_equal(spaqr.solve(a, x), spaqr.solve(b, x))


def test_unscaled_operator_error_falls_with_eps():
    p = config_problem("2d_uniform_a", n=24)
    A = p.to_dense()
    errs = []
    for eps in (1e-1, 1e-2, 1e-3, 1e-5):
        F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, nlevels=4, skip=0, scaling=False)
        E = A @ spaqr.solve(F, np.eye(p.n)) - np.eye(p.n)
        errs.append(np.linalg.norm(E, 2))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-2


def test_unscaled_gmres_converges_and_iterations_fall():
    p = config_problem("2d_uniform_a", n=48)
    b = rhs(p, 1)[:, 0]
    its = []
    for eps in (1e-1, 1e-3):
        F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, nlevels=5, skip=1, scaling=False)
        x, it, rr, _ = spaqr.gmres(p.n, p.rowptr, p.colind, p.val, b, lambda v: spaqr.solve(F, v))
        assert rr <= 1e-12
        assert np.linalg.norm(b - p.matvec(x)) / np.linalg.norm(b) <= 1e-12
        its.append(it)
    assert its[1] < its[0]


def test_fine_column_sign_rule_is_benign(monkeypatch):
    """Reading F8 only fixes which of two valid reflectors the fine-column QR
    takes when its leading entry is zero up to rounding.  With the plain
    LAPACK sign instead the factor is another valid one: GMRES converges with
    the same iteration count within one, and eps = 0 stays exact."""
    from oracle import dense
    p = config_problem("2d_uniform_a", n=16)
    b = rhs(p, 1)[:, 0]
    its = []
    orig = dense.qr
    for strict in (False, True):
        if strict:
            monkeypatch.setattr(dense, "qr", lambda A, sign_tol=0.0: orig(A, 0.0))
        F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 1e-3, nlevels=4, skip=0, scaling=False)
        _, it, rr, _ = spaqr.gmres(p.n, p.rowptr, p.colind, p.val, b, lambda v: spaqr.solve(F, v))
        assert rr <= 1e-12
        its.append(it)
        F0 = spaqr.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 0.0, nlevels=4, skip=0, scaling=False)
        x = spaqr.solve(F0, b)
        assert np.linalg.norm(b - p.matvec(x)) / np.linalg.norm(b) < 1e-12
    assert abs(its[0] - its[1]) <= 1, its


def _general_cases():
    from oracle.ordering_general import nd_general
    from synth.convdiff import permuted, random_local
    q = permuted(config_problem("2d_uniform_a", n=24), 61)
    r = random_local(20, seed=7060)
    w = random_local(20, seed=7061, weak_diag=0.1)
    return [("permuted_grid", q, nd_general(q.n, q.rowptr, q.colind, q.val, 4)),
            ("random_local", r, nd_general(r.n, r.rowptr, r.colind, r.val, 4)),
            ("weak_diag_max_product", w, nd_general(w.n, w.rowptr, w.colind, w.val, 4, matching="max_product"))]


@pytest.mark.parametrize("name,p,o", _general_cases())
def test_unscaled_on_grid_free_orderings(name, p, o):
    """The unscaled variant on matrices without a grid (rows matched to
    columns): eps = 0 solves exactly, and Lemma 1's identity
    sigma R_ff^T R_fn = W_fn^(2) holds at eps = 1e-2 on every interface
    that drops something."""
    b = np.random.default_rng(9).standard_normal((p.n, 2))
    F0 = spaqr.factor(p.n, p.rowptr, p.colind, p.val, None, 0.0, nlevels=o.L, skip=0, ordering=o, scaling=False)
    x = spaqr.solve(F0, b)
    assert np.max(np.linalg.norm(b - p.matvec(x), axis=0) / np.linalg.norm(b, axis=0)) < 1e-11
    F = spaqr.factor(p.n, p.rowptr, p.colind, p.val, None, 1e-2, nlevels=o.L, skip=0, ordering=o, scaling=False)
    checked = 0
    for c, d in _interfaces(F):
        if d["Rff"].shape[0] == 0 or not d["Rfn"]:
            continue
        Rfn = np.hstack([B for _, B in sorted(d["Rfn"], key=lambda t: t[0])])
        W2 = d["Wfn2"]
        scale = d["sigma"] * np.linalg.norm(d["App"], 2) * np.linalg.norm(d["Apn"], 2)
        lhs = d["sigma"] * d["Rff"].T @ Rfn
        assert np.linalg.norm(lhs - W2) <= 1e-12 * scale * np.sqrt(W2.size) + 1e-12 * np.linalg.norm(W2)
        checked += 1
    assert checked >= 1
