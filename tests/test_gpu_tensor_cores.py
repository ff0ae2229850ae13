"""The mixed-precision factorisation with its large fronts applied on the
tensor cores (tcgen05, compact-WY form of Section 2.4's block Householder
step) against the same factorisation with every front on the CUDA cores, and
against the FP64 factor through GMRES: the application agrees with the
CUDA-core FP32 form to FP32-level rounding (three TF32 passes) or TF32-level
rounding (one pass), ranks agree within 1%, and FP64 GMRES still reaches
1e-12 with at most one iteration more than the FP64 factor needs (three
passes)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2010_06807_gb300 as sq
from synth.convdiff import config_problem, rhs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev(spaqr_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _factor(o, A, eps, precision, tc):
    sq.spaqr_use_tensor_cores(tc)
    try:
        return sq.spaqr_factor(o, *A, eps=eps, precision=precision)
    finally:
        sq.spaqr_use_tensor_cores(True)


def _rank_sum(F):
    return sq.spaqr_factor_info(F)["rank_sum"]


@pytest.mark.parametrize("kind,n,eps", [("3d_uniform_a", 16, 1e-2), ("3d_uniform_a", 20, 1e-3)])
def test_tensor_core_apply_matches_cuda_core_apply(dev, kind, n, eps):
    """The application of each FP32-storage factor is compared with the FP64
    factor's: FP32 storage alone moves it by the conditioning of the blocks
    times FP32 rounding, so the bar is relative to the CUDA-core FP32 form's
    own distance from FP64.  Three TF32 passes represent each operand to
    2^-22 (x = hi + lo + O(2^-22 x)) against FP32's 2^-24, and the tensor
    core's FP32 accumulation adds its own rounding: the bar is 50x the
    CUDA-core form's distance plus 1e-5 (measured: 19x on 3D 20^3, 31x on
    2D 128^2 once the CUDA-core form's Householder norms were accumulated in
    FP64)."""
    p = config_problem(kind, n=n)
    A = [torch.from_numpy(x).to(dev) for x in (p.rowptr, p.colind, p.val)]
    o = sq.spaqr_order(p.rowptr, p.colind, p.dims)
    b = rhs(p, 4)
    B = torch.from_numpy(np.ascontiguousarray(b.T)).to(dev).T
    F64 = sq.spaqr_factor(o, *A, eps=eps)
    x64 = sq.spaqr_solve(F64, B).cpu().numpy()
    Fcc = _factor(o, A, eps, "fp32", False)
    assert sq.spaqr_factor_info(Fcc)["tc_levels"] == 0
    xcc = sq.spaqr_solve(Fcc, B).cpu().numpy()
    e_cc = (np.linalg.norm(xcc - x64, axis=0) / np.linalg.norm(x64, axis=0)).max()
    _, it64, _ = sq.spaqr_gmres(F64, *A, B, tol=1e-12)
    for prec in ("fp32", "tf32"):
        sq.spaqr_stats_reset()
        F = _factor(o, A, eps, prec, True)
        assert sq.spaqr_factor_info(F)["tc_levels"] > 0
        # the scaling and sparsification products of the large interfaces
        # ran on the tensor cores too
        assert sq.spaqr_stats()[1]["interface_tc"]["launches"] > 0
        # rank decisions are FP64 on FP32 data: rounding may move a pivot
        # that sits at the threshold
        assert abs(_rank_sum(F) - _rank_sum(Fcc)) <= 0.01 * _rank_sum(Fcc)
        x = sq.spaqr_solve(F, B).cpu().numpy()
        e = (np.linalg.norm(x - x64, axis=0) / np.linalg.norm(x64, axis=0)).max()
        if prec == "fp32":
            assert e <= 50 * e_cc + 1e-5, (e, e_cc)
        X, it, rr = sq.spaqr_gmres(F, *A, B, tol=1e-12)
        res = np.linalg.norm(b - p.matvec(X.cpu().numpy()), axis=0) / np.linalg.norm(b, axis=0)
        assert res.max() <= 1e-12 and rr.max() <= 1e-12
        assert int(it.max()) <= int(it64.max()) + (1 if prec == "fp32" else 3)


def test_small_fronts_stay_on_cuda_cores(dev):
    """2D fronts (at most 193 rows here) are too small to be tensor-core
    products: the FP32 factorisation keeps every level on the CUDA cores,
    bit for bit the factor the CUDA-core form gives."""
    p = config_problem("2d_lognormal", n=128)
    A = [torch.from_numpy(x).to(dev) for x in (p.rowptr, p.colind, p.val)]
    o = sq.spaqr_order(p.rowptr, p.colind, p.dims)
    B = torch.from_numpy(np.ascontiguousarray(rhs(p, 2).T)).to(dev).T
    F = _factor(o, A, 1e-2, "fp32", True)
    Fcc = _factor(o, A, 1e-2, "fp32", False)
    assert sq.spaqr_factor_info(F)["tc_levels"] == 0
    assert np.array_equal(sq.spaqr_solve(F, B).cpu().numpy(), sq.spaqr_solve(Fcc, B).cpu().numpy())
