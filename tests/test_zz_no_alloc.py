"""spaqr_solve_noalloc, the allocation-free variant of spaqr_solve.

It is for callers that cannot allocate device memory while they run (their
device memory is reserved by another allocator, or their loop must not enter
the CUDA allocator).  The test calls it through the C ABI twice in a row, with
different right-hand sides, and checks each result against spaqr_solve on the
same factor within the parity tolerance of the GPU tests: for an FP64 and an
FP32 factor, on the default stream and on a stream of the caller's.  It also
checks the two rejections: a call that needs more scratch than the fixed
array (the size taken from the factor's reported workspace), and host
buffers.

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


def _need_doubles(F, nrhs):
    """Scratch doubles of one call: the factor's workspace rows x nrhs in its
    precision, rounded up to whole doubles."""
    info = sq.spaqr_factor_info(F)
    esz = 8 if info["precision"] == sq.SPAQR_FP64 else 4
    return (info["workspace_rows"] * nrhs * esz + 7) // 8


@pytest.mark.parametrize("precision,own_stream", [("fp64", False), ("fp32", True)])
def test_noalloc_solve_matches_solve_on_two_calls(spaqr_lib, precision, own_stream):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    p = config_problem("2d_uniform_a", n=64)
    rp, ci, va = (torch.from_numpy(p.rowptr).to(dev), torch.from_numpy(p.colind).to(dev),
                  torch.from_numpy(p.val).to(dev))
    ordl = sq.spaqr_order(rp, ci, p.dims)
    st = torch.cuda.Stream(device=dev) if own_stream else None
    F = sq.spaqr_factor(ordl, rp, ci, va, eps=1e-3, precision=precision, stream=st)
    assert _need_doubles(F, 4) <= sq.SPAQR_NOALLOC_SCRATCH_DOUBLES
    for seed in (11, 12):
        b = rhs(p, 4, seed=seed)
        B = _colmajor(b, dev)
        ref = sq.spaqr_solve(F, B, stream=st).cpu().numpy()
        X = torch.full((4, p.n), float("nan"), dtype=torch.float64, device=dev).T
        sq.spaqr_solve_noalloc(F, B, X, stream=st)
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
    # the fewest right-hand sides whose scratch exceeds the fixed array
    rows = sq.spaqr_factor_info(F)["workspace_rows"]
    nbig = sq.SPAQR_NOALLOC_SCRATCH_DOUBLES // rows + 1
    assert _need_doubles(F, nbig) > sq.SPAQR_NOALLOC_SCRATCH_DOUBLES >= _need_doubles(F, nbig - 1)
    big = torch.zeros(nbig, p.n, dtype=torch.float64, device=dev).T
    with pytest.raises(sq.SpaqrError) as e:
        sq.spaqr_solve_noalloc(F, big, torch.zeros_like(big.T).T)
    assert e.value.name == "INVALID_ARG"
    # host buffers are refused (copying them would need device staging memory)
    bh = np.asfortranarray(rhs(p, 1))
    with pytest.raises(sq.SpaqrError) as e:
        sq.spaqr_solve_noalloc(F, bh, np.zeros_like(bh, order="F"))
    assert e.value.name == "INVALID_ARG"
