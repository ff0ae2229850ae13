"""Failure handling without a GPU fault: device allocations are made to fail
on the host (spaqr_test_fail_alloc, a fake of the failing cudaMallocAsync)
at every point of a factorisation and of a GMRES call.  Every such call must
return OOM (no other error, no crash), leave nothing behind that breaks the
next call, and the next factorisation / solve must give the same result as
before bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2010_06807_gb300 as sq
from synth.convdiff import config_problem, rhs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(spaqr_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    p = config_problem("2d_uniform_a", n=40)
    A = [torch.from_numpy(x).to(dev) for x in (p.rowptr, p.colind, p.val)]
    o = sq.spaqr_order(p.rowptr, p.colind, p.dims)
    b = torch.from_numpy(np.ascontiguousarray(rhs(p, 2).T)).to(dev).T
    F = sq.spaqr_factor(o, *A, eps=1e-3, skip=1)
    x_ref = sq.spaqr_solve(F, b).clone()
    g_ref, _, _ = sq.spaqr_gmres(F, *A, b, tol=1e-12)
    yield dev, o, A, b, x_ref, g_ref.clone()
    sq.spaqr_test_fail_alloc(-1)


@pytest.mark.parametrize("scaling", [1, 0])
def test_factor_allocation_failures(setup, scaling):
    dev, o, A, b, x_ref, _ = setup
    failed = 0
    for after in range(0, 400, 7):
        sq.spaqr_test_fail_alloc(after)
        try:
            F = sq.spaqr_factor(o, *A, eps=1e-3, skip=1, scaling=scaling)
        except sq.SpaqrError as e:
            assert e.name == "OOM", e
            failed += 1
            continue
        finally:
            sq.spaqr_test_fail_alloc(-1)
        del F
        break          # `after` is past the factorisation's last allocation
    assert failed >= 5
    if scaling:
        F = sq.spaqr_factor(o, *A, eps=1e-3, skip=1)
        assert torch.equal(sq.spaqr_solve(F, b), x_ref)


def test_gmres_allocation_failures(setup):
    dev, o, A, b, _, g_ref = setup
    F = sq.spaqr_factor(o, *A, eps=1e-3, skip=1)
    failed = 0
    for after in range(0, 60):
        sq.spaqr_test_fail_alloc(after)
        try:
            X, it, rr = sq.spaqr_gmres(F, *A, b, tol=1e-12)
        except sq.SpaqrError as e:
            assert e.name == "OOM", e
            failed += 1
            continue
        finally:
            sq.spaqr_test_fail_alloc(-1)
        break
    assert failed >= 1
    X, it, rr = sq.spaqr_gmres(F, *A, b, tol=1e-12)
    assert torch.equal(X, g_ref)


def test_buffers_of_another_gpu_are_refused(setup):
    """B or X in device memory of a GPU other than the factor's is refused
    on the host (INVALID_ARG) before any kernel is launched: kernels on the
    factor's GPU would otherwise reach the other GPU's memory through
    unified addressing.  Needs two visible GPUs."""
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU visible")
    dev, o, A, b, x_ref, _ = setup
    F = sq.spaqr_factor(o, *A, eps=1e-3, skip=1)
    other = torch.device("cuda:1")
    b1 = b.T.contiguous().to(other).T
    sq.spaqr_stats_reset()
    for fn in (lambda: sq.spaqr_solve(F, b1), lambda: sq.spaqr_solve_noalloc(F, b1, torch.zeros_like(b1.T).T),
               lambda: sq.spaqr_gmres(F, *A, b1)):
        with pytest.raises(sq.SpaqrError) as e:
            fn()
        assert e.value.name == "INVALID_ARG"
    launches, _ = sq.spaqr_stats()
    assert launches == 0
