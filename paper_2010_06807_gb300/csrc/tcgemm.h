// Batched FP32 matrix products on the fifth-generation tensor cores
// (tcgen05.mma kind::tf32, FP32 accumulation in tensor memory), used by the
// mixed-precision factorisation for its dense contractions: the compact-WY
// application of a front's reflectors, Q^T B = B - V T^T (V^T B)
// (Section 2.4's block Householder step).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace spaqr {

// One operand of a product: element (i, k) of an rows x cols matrix is
// p[i * rs + k * cs].  unit_lower: the operand is the unit lower trapezoidal
// reflector matrix stored with R above it (a factored panel): entry (i, k) is
// read only below the diagonal of the stored panel, 1 on it and 0 above it,
// where the stored panel's row is i and column k (trans = 0) or row k and
// column i (trans = 1).
struct GemmOperand {
    const float* p;
    int64_t rs, cs;
    int unit_lower;
    int trans;
};

// C (M x N) = alpha A (M x K) B (K x N) + beta C.  B is given as its
// transpose's operand: element (j, k) of B^T, so that both operands are read
// along K.
struct GemmTask {
    GemmOperand a;    // M x K
    GemmOperand bt;   // N x K
    float* c;
    int64_t c_rs, c_cs;
    int M, N, K;
    float alpha, beta;
    int tile_begin;   // first output tile of this task in the launch (128 x 128 tiles, row-major over the task's tiles)
    int ntn;          // tiles along N
};

constexpr int kGemmBM = 128, kGemmBN = 128, kGemmBK = 32;

// Launch the products of `tasks` (device array `dtasks`, host copy `tasks`
// for the grid size) on `st`.  split3: three-pass TF32 (hi*hi + hi*lo +
// lo*hi), about FP32 accuracy; else one TF32 pass.  err: device flag set if a
// bounded tensor-core wait ran out.  Returns the number of CTAs launched.
int launch_tc_gemm(const GemmTask* dtasks, const std::vector<GemmTask>& tasks, bool split3, int* err,
                   cudaStream_t st);

// Fill tile_begin / ntn of every task; returns the total tile count.
int gemm_tiles(std::vector<GemmTask>& tasks);

}  // namespace spaqr
