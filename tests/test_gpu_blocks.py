"""Every stored factor block of the GPU factorisation against the oracle's,
entry by entry, and the application of the factor element by element.

The GPU exports its blocks through the C ABI (spaqr_factor_nblocks /
spaqr_factor_block): per level the front panels (reflectors and R_ss), the
Householder scalars, every R_sj, the scaling factors U_pp / R_pp, the CPQR
reflectors Q_pp and, in the unscaled form, the QR of the fine columns with
R_fc.  Both sides use the same Householder sign rule (Section 2.4's QR in the
LAPACK convention), so the blocks are compared as they are, no sign fix-up.
Bar (FP64): per block, the largest entry difference and the Frobenius norm of
the difference are at most 1e-10 of the oracle block's largest entry and
Frobenius norm; the set of blocks is the same on both sides; one application
agrees entry by entry to 1e-10 of each column's largest entry.  (An R_sj
block is measured against the scale of R_ss of its front: some are zero in
exact arithmetic, rounding residue against entries of order one.)  The coarse
blocks a level's sparsification writes are the next level's fronts, so they
are compared as those fronts' panels and R_sj.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2010_06807_gb300 as sq
from oracle import spaqr as osq
from synth.convdiff import config_problem, rhs

from blockparity import compare_blocks
from test_gpu_parity import CASES

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def dev(spaqr_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _colmajor(b, dev):
    return torch.from_numpy(np.ascontiguousarray(b.T)).to(dev).T


def _elementwise(xg, xo):
    """Largest entry difference of each column over the column's largest entry."""
    return np.abs(xg - xo).max(axis=0) / np.abs(xo).max(axis=0)


def _run(p, dev, eps, L, skip, scaling=1, nrhs=3):
    A = [torch.from_numpy(x).to(dev) for x in (p.rowptr, p.colind, p.val)]
    ordl = sq.spaqr_order(A[0], A[1], p.dims, L)
    F = sq.spaqr_factor(ordl, *A, eps=eps, skip=skip, scaling=scaling)
    Fo = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, nlevels=ordl.L, skip=skip,
                    scaling=bool(scaling))
    nb, em, ef = compare_blocks(sq.spaqr_factor_blocks(F), Fo, TOL)
    b = rhs(p, nrhs)
    xg = sq.spaqr_solve(F, _colmajor(b, dev)).cpu().numpy()
    xo = osq.solve(Fo, b)
    e = _elementwise(xg, xo)
    assert e.max() <= TOL, e
    return F, Fo, A, b, nb


@pytest.mark.parametrize("kind,n,L,eps,skip", CASES)
def test_blocks_match_oracle(dev, kind, n, L, eps, skip):
    _run(config_problem(kind, n=n), dev, eps, L, skip)


@pytest.mark.parametrize("kind,n,eps,skip", [("2d_uniform_a", 24, 1e-3, 1), ("3d_uniform_a", 8, 1e-2, 0),
                                             ("2d_lognormal", 40, 1e-3, 2)])
def test_unscaled_blocks_match_oracle(dev, kind, n, eps, skip):
    _run(config_problem(kind, n=n), dev, eps, 0, skip, scaling=0)


def test_config1_gmres_iterations_match_oracle(dev):
    """64 x 64, eps 1e-3, L = 6: the GMRES iteration count equals the
    oracle's, and so do the Arnoldi residual estimates of every iteration
    (the two differ only in the rounding of the factor and of the
    orthogonalisation: classical Gram-Schmidt twice on the GPU, modified
    Gram-Schmidt in the oracle)."""
    p = config_problem("2d_uniform_a", n=64)
    F, Fo, A, _, _ = _run(p, dev, 1e-3, 0, 2)
    b = rhs(p, 1)
    X, it, rr, hist = sq.spaqr_gmres(F, *A, _colmajor(b, dev), tol=1e-12, history=True)
    xo, ito, rro, histo = osq.gmres(p.n, p.rowptr, p.colind, p.val, b[:, 0], lambda v: osq.solve(Fo, v))
    assert int(it[0]) == ito, (int(it[0]), ito, hist[0][-3:], histo[-3:])
    np.testing.assert_allclose(hist[0][:ito], histo[1:ito + 1], rtol=1e-6, atol=1e-14)
    assert _elementwise(X.cpu().numpy(), xo[:, None]).max() <= 1e-9


@pytest.mark.parametrize("eps", [1e-2, 1e-4])
def test_256x256_blocks_and_16_columns(dev, eps):
    """The bench workload (256 x 256, a = exp(g), Pe = 50 with random angles)
    at both tolerances of its configuration: every block against the oracle,
    one application of all 16 right-hand sides element by element, GMRES to
    1e-12 on all 16, and the iteration counts of two columns against the
    oracle's GMRES."""
    p = config_problem("2d_lognormal", n=256)
    F, Fo, A, b, nb = _run(p, dev, eps, 0, 2, nrhs=16)
    assert nb > 1000
    X, it, rr = sq.spaqr_gmres(F, *A, _colmajor(b, dev), tol=1e-12, maxit=300)
    x = X.cpu().numpy()
    rel = np.linalg.norm(b - p.matvec(x), axis=0) / np.linalg.norm(b, axis=0)
    assert rel.max() <= 1e-12 and rr.max() <= 1e-12
    for c in (0, 9):
        xo, ito, rro, _ = osq.gmres(p.n, p.rowptr, p.colind, p.val, b[:, c], lambda v: osq.solve(Fo, v))
        assert int(it[c]) == ito, (c, int(it[c]), ito)
        assert _elementwise(x[:, [c]], xo[:, None]).max() <= 1e-9
