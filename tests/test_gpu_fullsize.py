"""Full-size workload (256x256, a = exp(g), Pe = 50 with random angles, 16 RHS)
in the launch configuration the benchmark times: ranks bit-exact against the
oracle, one application and GMRES checked against the oracle on the same
inputs, GMRES to 1e-12 on every right-hand side.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2010_06807_gb300 as sq
from oracle import spaqr as osq
from synth.convdiff import config_problem, rhs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eps", [1e-2])
def test_256x256_16rhs(spaqr_lib, eps):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    p = config_problem("2d_lognormal", n=256)
    b = rhs(p, 16)
    rp, ci, va = (torch.from_numpy(p.rowptr).to(dev), torch.from_numpy(p.colind).to(dev),
                  torch.from_numpy(p.val).to(dev))
    ordl = sq.spaqr_order(rp, ci, p.dims)
    F = sq.spaqr_factor(ordl, rp, ci, va, eps=eps)
    Fo = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps)
    for lev, R in enumerate(Fo.ranks):
        pairs, _ = sq.spaqr_factor_ranks(F, lev)
        assert [tuple(x) for x in pairs.tolist()] == [v for _, v in sorted(R.items()) if v[0] > 0]
    bd = torch.from_numpy(np.ascontiguousarray(b.T)).to(dev).T
    xg = sq.spaqr_solve(F, bd).cpu().numpy()
    # sampled columns against the oracle (each oracle application is ~0.1 s)
    for c in (0, 7, 15):
        xo = osq.solve(Fo, b[:, c])
        assert np.linalg.norm(xg[:, c] - xo) / np.linalg.norm(xo) <= 1e-10
    X, it, rr = sq.spaqr_gmres(F, rp, ci, va, bd, tol=1e-12, maxit=300)
    x = X.cpu().numpy()
    rel = np.linalg.norm(b - p.matvec(x), axis=0) / np.linalg.norm(b, axis=0)
    assert rel.max() <= 1e-12 and rr.max() <= 1e-12
