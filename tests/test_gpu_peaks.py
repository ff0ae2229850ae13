"""The tcgen05 TF32 tile (the tensor-core building block of the
mixed-precision factorisation) against a plain FP64 product of the same
TF32-rounded inputs, and the arithmetic peak microbenchmarks (positive,
plausible rates)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2010_06807_gb300 as sq

pytestmark = pytest.mark.gpu


def tf32_round(x):
    """FP32 -> TF32 (10 explicit mantissa bits), round to nearest with ties
    away from zero, as cvt.rna.tf32.f32 does for finite values."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000) & 0xFFFFFFFF
    return b.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def dev(spaqr_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("N,K", [(16, 8), (64, 32), (256, 128), (128, 24), (240, 72)])
def test_tc_tile_matches_fp64_product(dev, N, K):
    rng = np.random.default_rng(N * 1000 + K)
    A = rng.standard_normal((128, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    D = sq.spaqr_tc_tile_check(torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)).cpu().numpy()
    ref = tf32_round(A).astype(np.float64) @ tf32_round(B).astype(np.float64).T
    # FP32 accumulation of K products of TF32 values
    bound = 2 * K * np.finfo(np.float32).eps * (np.abs(tf32_round(A)).astype(np.float64) @
                                                 np.abs(tf32_round(B)).astype(np.float64).T)
    assert np.all(np.abs(D - ref) <= bound + 1e-30)
    # and the rounding of the inputs matters: the FP64 product of the
    # unrounded inputs differs by far more than that
    raw = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.abs(raw - ref).max() > 10 * bound.max() / K


def test_tc_tile_rejects_bad_shapes(dev):
    A = torch.zeros(128, 12, device=dev)
    with pytest.raises(sq.SpaqrError):
        sq.spaqr_tc_tile_check(A, torch.zeros(16, 12, device=dev))


def test_peaks_plausible(dev):
    rates = {}
    for w in ("dfma", "dmma", "ffma", "tf32"):
        f, ms = sq.spaqr_peak(w, reps=3)
        assert f > 0 and ms > 0
        rates[w] = f / ms / 1e9
    assert 0.2 < rates["dfma"] < 10 and 0.1 < rates["dmma"] < 10
    assert 10 < rates["ffma"] < 200
    assert rates["tf32"] > rates["ffma"]


def test_op_cycles_fp64_cost_model(dev):
    """The FP64 cost model the kernels are designed around: a dependent FP64
    operation takes several times an FP32 one, its cost does not depend on
    how many lanes are active, and division and square root take several
    FMAs' time."""
    dfma1 = sq.spaqr_op_cycles("dfma", 1, 1)
    dfma32 = sq.spaqr_op_cycles("dfma", 1, 32)
    ffma = sq.spaqr_op_cycles("ffma", 1, 32)
    assert 0 < ffma < dfma32 / 4
    assert abs(dfma1 - dfma32) <= 0.1 * dfma32
    assert sq.spaqr_op_cycles("ddiv", 1, 32) > 4 * dfma32
    assert sq.spaqr_op_cycles("dsqrt", 1, 32) > 4 * dfma32
    # eight warps share the SM's FP64 pipe: each waits longer per operation
    assert sq.spaqr_op_cycles("dfma", 8, 32) > 1.5 * dfma32
    with pytest.raises(sq.SpaqrError):
        sq._check(sq._lib.spaqr_op_cycles(7, 1, 1, None))


def _refl(P):
    """Unit lower trapezoidal reflector matrix of a stored panel."""
    V = np.tril(P, -1)
    k = min(P.shape)
    V[np.arange(k), np.arange(k)] = 1.0
    return V


@pytest.mark.parametrize("M,N,K,layout,refl,alpha,beta", [
    (200, 70, 45, "cc", False, 1.5, -0.5),
    (128, 128, 32, "rr", False, 1.0, 0.0),
    (1, 1, 1, "cc", False, 2.0, 1.0),
    (300, 257, 129, "rc", True, -1.0, 1.0),
    (1300, 600, 370, "cr", True, -1.0, 1.0),
    (90, 33, 0, "cc", False, 1.0, 0.25),
])
@pytest.mark.parametrize("split3", [False, True])
def test_tc_gemm_matches_fp64(dev, M, N, K, layout, refl, alpha, beta, split3):
    """C = alpha A B + beta C on the tensor cores against an FP64 product:
    ragged tiles on every edge, both memory orders of A and B, the reflector
    view of A, K = 0.  One TF32 pass is within the FP32-accumulation bound of
    the TF32-rounded operands; three passes within a few FP32 roundings of
    the exact product."""
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    C0 = rng.standard_normal((M, N)).astype(np.float32)

    def place(x, order):
        t = torch.from_numpy(np.ascontiguousarray(x if order == "r" else x.T)).to(dev)
        return t if order == "r" else t.T

    Ad, Bd = place(A, layout[0]), place(B, layout[1])
    Cd = place(C0, "c")
    sq.spaqr_tc_gemm(Ad, Bd, Cd, alpha=alpha, beta=beta, reflectors=refl, split3=split3)
    got = Cd.cpu().numpy().astype(np.float64)
    Ae = _refl(A) if refl else A
    if split3:
        ref = alpha * (Ae.astype(np.float64) @ B.astype(np.float64)) + beta * C0
        mag = np.abs(alpha) * (np.abs(Ae) @ np.abs(B)) + np.abs(beta * C0)
        assert np.all(np.abs(got - ref) <= (3 * K + 8) * np.finfo(np.float32).eps * mag + 1e-30)
    else:
        At, Bt = tf32_round(Ae), tf32_round(B)
        ref = alpha * (At.astype(np.float64) @ Bt.astype(np.float64)) + beta * C0
        mag = np.abs(alpha) * (np.abs(At).astype(np.float64) @ np.abs(Bt).astype(np.float64)) + np.abs(beta * C0)
        assert np.all(np.abs(got - ref) <= (2 * K + 4) * np.finfo(np.float32).eps * mag + 1e-30)
