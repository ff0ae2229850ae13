"""spaqr_solve_noalloc, the allocation-free variant of spaqr_solve.

It is for callers that cannot allocate device memory while they run (their
device memory is reserved by another allocator, or their loop must not enter
the CUDA allocator).  The test calls it through the C ABI twice in a row, with
different right-hand sides, and checks each result against spaqr_solve within
the parity tolerance of the GPU tests.  It also checks the two rejections: a
call that needs more scratch than the fixed array, and host buffers.

This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2010_06807_gb300 as sq
from synth.convdiff import config_problem, rhs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _colmajor(b, dev):
    return torch.from_numpy(np.ascontiguousarray(b.T)).to(dev).T


def test_noalloc_solve_matches_solve_on_two_calls(spaqr_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    p = config_problem("2d_uniform_a", n=64)
    rp, ci, va = (torch.from_numpy(p.rowptr).to(dev), torch.from_numpy(p.colind).to(dev),
                  torch.from_numpy(p.val).to(dev))
    ordl = sq.spaqr_order(rp, ci, p.dims)
    F = sq.spaqr_factor(ordl, rp, ci, va, eps=1e-3)
    for seed in (11, 12):
        b = rhs(p, 4, seed=seed)
        B = _colmajor(b, dev)
        ref = sq.spaqr_solve(F, B).cpu().numpy()
        X = torch.full((4, p.n), float("nan"), dtype=torch.float64, device=dev).T
        sq.spaqr_solve_noalloc(F, B, X)
        got = X.cpu().numpy()
        err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert np.all(np.isfinite(got))
        assert err.max() <= TOL, err


def test_noalloc_solve_rejections(spaqr_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    p = config_problem("2d_uniform_a", n=32)
    rp, ci, va = (torch.from_numpy(p.rowptr).to(dev), torch.from_numpy(p.colind).to(dev),
                  torch.from_numpy(p.val).to(dev))
    ordl = sq.spaqr_order(rp, ci, p.dims)
    F = sq.spaqr_factor(ordl, rp, ci, va, eps=1e-2)
    # more right-hand sides than the fixed scratch array holds
    big = torch.zeros(2048, p.n, dtype=torch.float64, device=dev).T
    with pytest.raises(sq.SpaqrError) as e:
        sq.spaqr_solve_noalloc(F, big, torch.zeros_like(big.T).T)
    assert e.value.name == "INVALID_ARG"
    # host buffers are refused (copying them would need device staging memory)
    bh = np.asfortranarray(rhs(p, 1))
    with pytest.raises(sq.SpaqrError) as e:
        sq.spaqr_solve_noalloc(F, bh, np.zeros_like(bh, order="F"))
    assert e.value.name == "INVALID_ARG"
