"""GPU spaQR (through the C ABI) against the FP64 CPU oracle.

Bars (FP64): ordering/plan and interface ranks bit-exact; one application of
the factor and GMRES solutions agree with the oracle to 1e-10 relative;
GMRES reaches ||b - A x|| / ||b|| <= 1e-12.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2010_06807_gb300 as sq
from oracle import spaqr as osq
from synth.convdiff import Problem, config_problem, convdiff, rhs

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def dev(spaqr_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _to_dev(p, dev):
    return (torch.from_numpy(p.rowptr).to(dev), torch.from_numpy(p.colind).to(dev),
            torch.from_numpy(p.val).to(dev))


def _colmajor(b, dev):
    t = torch.from_numpy(np.ascontiguousarray(b.T)).to(dev)  # (nrhs, n) rows = columns of b
    return t.T


def _gpu_factor(p, dev, eps, L=0, skip=2):
    rp, ci, va = _to_dev(p, dev)
    ordl = sq.spaqr_order(rp, ci, p.dims, L)
    F = sq.spaqr_factor(ordl, rp, ci, va, eps=eps, skip=skip)
    return ordl, F, (rp, ci, va)


def _oracle_ranks(Fo):
    return [sorted(R.items()) for R in Fo.ranks]


def _check_ranks(F, Fo):
    for lev, R in enumerate(Fo.ranks):
        pairs, margins = sq.spaqr_factor_ranks(F, lev)
        exp = [v for _, v in sorted(R.items()) if v[0] > 0]
        got = [tuple(x) for x in pairs.tolist()]
        assert got == [tuple(e) for e in exp], f"level {lev}: ranks differ"


CASES = [
    ("2d_uniform_a", 16, 3, 0.0, 0),
    ("2d_uniform_a", 16, 3, 1e-2, 0),
    ("2d_uniform_a", 24, 4, 1e-3, 1),
    ("2d_uniform_a", 33, 0, 1e-2, 2),
    ("2d_lognormal", 40, 5, 1e-4, 2),
    ("3d_uniform_a", 8, 3, 1e-2, 0),
    ("3d_uniform_a", 10, 0, 0.0, 0),
    ("2d_uniform_a", 5, 4, 1e-1, 0),
    ("2d_uniform_a", 4, 0, 1e-2, 2),
    ("3d_uniform_a", 16, 0, 1e-2, 2),    # large interfaces: cluster CPQR
    ("2d_lognormal", 128, 0, 1e-4, 2),
]


@pytest.mark.parametrize("kind,n,L,eps,skip", CASES)
def test_solve_matches_oracle(dev, kind, n, L, eps, skip):
    p = config_problem(kind, n=n)
    ordl, F, _ = _gpu_factor(p, dev, eps, L, skip)
    Fo = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, nlevels=ordl.L, skip=skip)
    _check_ranks(F, Fo)
    b = rhs(p, 3)
    xo = osq.solve(Fo, b)
    xg = sq.spaqr_solve(F, _colmajor(b, dev)).cpu().numpy()
    err = np.linalg.norm(xg - xo, axis=0) / np.linalg.norm(xo, axis=0)
    assert err.max() <= TOL, err
    if eps == 0.0:
        rel = np.linalg.norm(b - p.matvec(xg), axis=0) / np.linalg.norm(b, axis=0)
        assert rel.max() < 1e-12


@pytest.mark.parametrize("dims,eps,skip", [((20, 36), 1e-2, 2), ((37, 12), 1e-3, 1), ((6, 8, 11), 1e-2, 2),
                                            ((3, 70), 1e-2, 0)])
def test_nonsquare_grids_match_oracle(dev, dims, eps, skip):
    """Boxes whose cuts change dimension between levels, a mixed-sign
    velocity, and a strip two cells short of a single cut."""
    rng = np.random.Generator(np.random.PCG64(77 + len(dims)))
    N = int(np.prod(dims))
    a = rng.uniform(0.1, 10.0, N)
    v = np.tile(rng.uniform(-20.0, 20.0, len(dims)), (N, 1))
    p = Problem(dims, *convdiff(dims, a, v))
    ordl, F, _ = _gpu_factor(p, dev, eps, 0, skip)
    Fo = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, nlevels=ordl.L, skip=skip)
    _check_ranks(F, Fo)
    b = rhs(p, 2, seed=5)
    xo = osq.solve(Fo, b)
    xg = sq.spaqr_solve(F, _colmajor(b, dev)).cpu().numpy()
    err = np.linalg.norm(xg - xo, axis=0) / np.linalg.norm(xo, axis=0)
    assert err.max() <= TOL, err


def test_host_buffers_match_device_buffers(dev):
    p = config_problem("2d_uniform_a", n=32)
    ordl, F, _ = _gpu_factor(p, dev, 1e-3)
    b = rhs(p, 2)
    xh = sq.spaqr_solve(F, np.asfortranarray(b))
    xd = sq.spaqr_solve(F, _colmajor(b, dev)).cpu().numpy()
    assert np.array_equal(xh, xd)


def test_config1_64x64_parity_and_gmres(dev):
    """64x64, a ~ U[0.1,10], v = (10,10), L = 6, eps = 1e-3, one RHS."""
    p = config_problem("2d_uniform_a", n=64)
    ordl, F, A = _gpu_factor(p, dev, 1e-3)
    assert ordl.L == 6
    Fo = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 1e-3)
    _check_ranks(F, Fo)
    b = rhs(p, 1)
    xo = osq.solve(Fo, b)
    xg = sq.spaqr_solve(F, _colmajor(b, dev)).cpu().numpy()
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= TOL
    X, it, rr = sq.spaqr_gmres(F, *A, _colmajor(b, dev), tol=1e-12, maxit=300)
    x = X.cpu().numpy()
    assert rr[0] <= 1e-12
    assert np.linalg.norm(b - p.matvec(x)) / np.linalg.norm(b) <= 1e-12
    xo2, ito, rro, _ = osq.gmres(p.n, p.rowptr, p.colind, p.val, b[:, 0], lambda v: osq.solve(Fo, v))
    assert abs(int(it[0]) - ito) <= 1
    assert np.linalg.norm(x[:, 0] - xo2) / np.linalg.norm(xo2) <= 1e-9


def test_gmres_multi_rhs_host_and_initial_guess(dev):
    p = config_problem("2d_uniform_a", n=32)
    ordl, F, A = _gpu_factor(p, dev, 1e-2)
    b = rhs(p, 5)
    X, it, rr = sq.spaqr_gmres(F, p.rowptr, p.colind, p.val, np.asfortranarray(b), tol=1e-12)
    assert rr.max() <= 1e-12
    rel = np.linalg.norm(b - p.matvec(X), axis=0) / np.linalg.norm(b, axis=0)
    assert rel.max() <= 1e-12
    # a converged initial guess needs no iterations
    X2, it2, rr2 = sq.spaqr_gmres(F, p.rowptr, p.colind, p.val, np.asfortranarray(b),
                                   X=np.asfortranarray(X.copy()), tol=1e-10)
    assert (it2 == 0).all()
    # zero right-hand side gives x = 0
    z = np.zeros((p.n, 1), order="F")
    X3, it3, rr3 = sq.spaqr_gmres(F, p.rowptr, p.colind, p.val, z, tol=1e-12)
    assert np.all(X3 == 0)


def test_deterministic(dev):
    p = config_problem("2d_uniform_a", n=48)
    b = _colmajor(rhs(p, 2), dev)
    _, F1, _ = _gpu_factor(p, dev, 1e-3)
    _, F2, _ = _gpu_factor(p, dev, 1e-3)
    x1 = sq.spaqr_solve(F1, b).cpu().numpy()
    x2 = sq.spaqr_solve(F2, b).cpu().numpy()
    assert np.array_equal(x1, x2)


def test_errors(dev):
    p = config_problem("2d_uniform_a", n=16)
    rp, ci, va = _to_dev(p, dev)
    ordl = sq.spaqr_order(rp, ci, p.dims)
    with pytest.raises(sq.SpaqrError) as e:
        sq.spaqr_factor(ordl, rp, ci, va, eps=1e-2, scaling=2)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(sq.SpaqrError) as e:
        sq.spaqr_factor(ordl, rp, ci, va, eps=-1.0)
    assert e.value.name == "INVALID_ARG"
    # a loose factor (sparsified from the leaves up) cannot reach 1e-14 in one step
    ordl3 = sq.spaqr_order(rp, ci, p.dims, 3)
    F = sq.spaqr_factor(ordl3, rp, ci, va, eps=0.9, skip=0)
    b = rhs(p, 1)
    with pytest.raises(sq.SpaqrError) as e:
        sq.spaqr_gmres(F, p.rowptr, p.colind, p.val, np.asfortranarray(b), tol=1e-15, maxit=1)
    assert e.value.name == "NOT_CONVERGED"
    # the error carries the best iterate and the per-column counts
    assert e.value.iters.tolist() == [1] and e.value.relres[0] > 1e-15 and e.value.X.shape == (p.n, 1)


def test_gmres_rejects_mismatched_or_bad_host_csr(dev):
    """GMRES reads A's CSR in its SpMV kernels: a host CSR with another entry
    count than the factored pattern, a decreasing rowptr or a column index
    out of range is refused on the host (INVALID_ARG) before any kernel."""
    p = config_problem("2d_uniform_a", n=16)
    rp, ci, va = _to_dev(p, dev)
    F = sq.spaqr_factor(sq.spaqr_order(rp, ci, p.dims), rp, ci, va, eps=1e-2)
    b = np.asfortranarray(rhs(p, 1))
    short = p.rowptr.copy()
    short[-1] -= 1
    bad_rp = p.rowptr.copy()
    bad_rp[3] = bad_rp[5] + 1
    bad_ci = p.colind.copy()
    bad_ci[5] = p.n
    for A in ((short, p.colind[:-1], p.val[:-1]), (bad_rp, p.colind, p.val), (p.rowptr, bad_ci, p.val)):
        with pytest.raises(sq.SpaqrError) as e:
            sq.spaqr_gmres(F, *A, b, tol=1e-12)
        assert e.value.name == "INVALID_ARG"
    # the factor is untouched: the right matrix still converges
    _, it, rr = sq.spaqr_gmres(F, p.rowptr, p.colind, p.val, b, tol=1e-12)
    assert rr[0] <= 1e-12


def test_csr_location_flag_checked_on_device(dev):
    """Device arrays flagged as host memory are refused by the ordering, the
    factorisation and GMRES before the host or a kernel reads them."""
    import ctypes
    p = config_problem("2d_uniform_a", n=16)
    rp, ci, va = _to_dev(p, dev)
    ordl = sq.spaqr_order(rp, ci, p.dims)
    F = sq.spaqr_factor(ordl, rp, ci, va, eps=1e-2)
    csr, keep = sq._make_csr(rp, ci, va)
    assert csr.on_device == 1
    csr.on_device = 0
    h = ctypes.c_void_p()
    g = sq._Grid(2, 16, 16, 1)
    assert sq._lib.spaqr_order(ctypes.byref(csr), ctypes.byref(g), 0, ctypes.byref(h)) == -1
    assert b"device memory" in sq._lib.spaqr_last_error()
    o = sq._Opts()
    sq._lib.spaqr_opts_default(ctypes.byref(o))
    assert sq._lib.spaqr_factor(ordl._h, ctypes.byref(csr), ctypes.byref(o), ctypes.byref(h)) == -1
    b = torch.zeros(p.n, dtype=torch.float64, device=dev)
    x = torch.zeros(p.n, dtype=torch.float64, device=dev)
    it = np.zeros(1, dtype=np.int32)
    rr = np.zeros(1)
    assert sq._lib.spaqr_gmres(F._h, ctypes.byref(csr), 1, b.data_ptr(), p.n, x.data_ptr(), p.n, 1e-12, 10,
                               it.ctypes.data, rr.ctypes.data, None) == -1
    del keep


def test_gmres_residual_history(dev):
    """spaqr_gmres_history: per column the Arnoldi estimate of the relative
    residual after every iteration -- non-increasing, at most tol when it
    stopped the column -- equal to the oracle's estimates (MGS there, CGS2
    here) over the first iterations; NaN after the column stopped."""
    import ctypes
    p = config_problem("2d_uniform_a", n=32)
    rp, ci, va = _to_dev(p, dev)
    F = sq.spaqr_factor(sq.spaqr_order(rp, ci, p.dims), rp, ci, va, eps=1e-2)
    b = rhs(p, 2)
    X, it, rr, hist = sq.spaqr_gmres(F, p.rowptr, p.colind, p.val, np.asfortranarray(b), tol=1e-12, history=True)
    assert (rr <= 1e-12).all()
    Fo = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, 1e-2)
    for c in range(2):
        h = hist[c]
        assert len(h) == it[c] and np.all(np.isfinite(h)) and h[-1] <= 1e-12
        assert np.all(h[1:] <= h[:-1] * (1 + 1e-12))
        _, ito, _, ho = osq.gmres(p.n, p.rowptr, p.colind, p.val, b[:, c], lambda v: osq.solve(Fo, v))
        k = min(3, len(h), len(ho) - 1)
        np.testing.assert_allclose(h[:k], np.asarray(ho[1:k + 1]), rtol=1e-6)
    # the raw array: NaN after each column's last iteration
    csr, keep = sq._make_csr(p.rowptr, p.colind, p.val)
    maxit = 40
    raw = np.zeros((2, maxit))
    its = np.zeros(2, dtype=np.int32)
    res = np.zeros(2)
    Xh = np.zeros((p.n, 2), order="F")
    bf = np.asfortranarray(b)
    assert sq._lib.spaqr_gmres_history(F._h, ctypes.byref(csr), 2, bf.ctypes.data, p.n, Xh.ctypes.data, p.n,
                                       1e-12, maxit, its.ctypes.data, res.ctypes.data, raw.ctypes.data, None) == 0
    for c in range(2):
        assert np.all(np.isfinite(raw[c, :its[c]])) and np.all(np.isnan(raw[c, its[c]:]))
    assert sq._lib.spaqr_gmres_history(F._h, ctypes.byref(csr), 2, bf.ctypes.data, p.n, Xh.ctypes.data, p.n,
                                       1e-12, maxit, its.ctypes.data, res.ctypes.data, None, None) == -1
    del keep
