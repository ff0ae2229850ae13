// Batched FP32 matrix products on the tcgen05 tensor cores (see tcgemm.h).
//
// One CTA of 128 threads computes one 128 x 128 output tile: the tile's
// accumulator lives in tensor memory (128 lanes x 128 FP32 columns); the K
// dimension is walked in chunks of BK elements, each chunk of A and B^T
// loaded from global memory with plain loads (any strides, reflector views,
// zero fill past the edges), rounded to TF32 and written to shared memory in
// the K-major core-matrix layout of tcgen05.cuh.  Two shared-memory stages:
// while the tensor core works on chunk k, the threads load chunk k + 1; a
// stage is refilled only after the MMAs that read it have signalled their
// mbarrier.  Thread 0 issues the MMAs (BK / 8 per chunk, three per step in
// the three-pass form: hi*hi + hi*lo + lo*hi, with x = hi + lo, hi and lo
// TF32).  The epilogue reads the accumulator back with tcgen05.ld (warp w
// owns rows 32 w .. 32 w + 31) and writes C = alpha acc + beta C.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "spaqr_internal.h"
#include "tcgemm.h"
#include "tcgen05.cuh"

namespace spaqr {

namespace {

// Stage one BM x BK (or BN x BK) chunk of an operand at K offset k0 into
// shared memory (TF32 hi, and lo for the three-pass form).
template <int BK, bool SPLIT3>
__device__ __forceinline__ void stage_operand(const GemmOperand& o, int rows, int K, int i0, int k0, float* hi,
                                              float* lo) {
    // thread t reads element (ib + di u, kb + dk u) at its u-th load: along K
    // when the operand is contiguous along K (a warp reads a row), else along
    // the rows (a warp reads a column)
    const bool kfast = o.cs == 1 || (o.rs != 1 && o.cs < o.rs);
    const int t = threadIdx.x;
    const int ib = kfast ? t / BK : t, kb = kfast ? t % BK : 0;
    const int di = kfast ? 128 / BK : 0, dk = kfast ? 0 : 1;
    const int64_t step = (int64_t)di * o.rs + (int64_t)dk * o.cs;
    const float* p0 = o.p + (int64_t)(i0 + ib) * o.rs + (int64_t)(k0 + kb) * o.cs;
    // every load of the chunk is issued before the first is used (BK values
    // per thread in flight), then converted and stored
    float x[BK];
#pragma unroll
    for (int u = 0; u < BK; u++) {
        const int i = i0 + ib + di * u, k = k0 + kb + dk * u;
        float v = 0.0f;
        if (i < rows && k < K) {
            if (o.unit_lower) {
                const int r = o.trans ? k : i, c = o.trans ? i : k;
                v = r > c ? p0[step * u] : (r == c ? 1.0f : 0.0f);
            } else {
                v = p0[step * u];
            }
        }
        x[u] = v;
    }
#pragma unroll
    for (int u = 0; u < BK; u++) {
        const float h = tc::to_tf32(x[u]);
        const uint32_t off = tc::kmajor_off(ib + di * u, kb + dk * u, BK) >> 2;
        hi[off] = h;
        if constexpr (SPLIT3) lo[off] = tc::to_tf32(x[u] - h);
    }
}

template <bool SPLIT3>
__global__ void __launch_bounds__(128) k_tc_gemm(const GemmTask* __restrict__ tasks, int ntask, int* err) {
    constexpr int BM = kGemmBM, BN = kGemmBN;
    constexpr int BK = SPLIT3 ? 16 : kGemmBK;
    constexpr int TILE = 128 * BK;                   // floats per operand tile
    constexpr int PER_STAGE = (SPLIT3 ? 4 : 2) * TILE;
    extern __shared__ __align__(1024) float sm[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;

    // the task of this tile: the last one whose first tile is <= blockIdx.x
    int lo = 0, hi = ntask - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile_begin <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const GemmTask t = tasks[lo];
    const int lt = (int)blockIdx.x - t.tile_begin;
    const int m0 = (lt / t.ntn) * BM, n0 = (lt % t.ntn) * BN;

    if (threadIdx.x < 32) {
        __syncwarp();
        tc::tmem_alloc(&tslot, BN);
    }
    if (threadIdx.x == 0) {
        tc::bar_init(&bar[0], 1);
        tc::bar_init(&bar[1], 1);
        abort_flag = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t idesc = tc::idesc_tf32(BM, BN);
    const uint32_t sbo = (uint32_t)(BK / 4) * 128;
    const int nk = (t.K + BK - 1) / BK;
    for (int kc = 0; kc < nk; kc++) {
        const int s = kc & 1;
        float* st = sm + s * PER_STAGE;
        if (kc >= 2) {
            // the MMAs of chunk kc - 2 read this stage: wait until they are done
            if (!tc::bar_wait(&bar[s], (uint32_t)((kc - 2) >> 1) & 1u, err)) abort_flag = 1;
            tc::fence_after_sync();
        }
        __syncthreads();
        if (abort_flag) break;
        float* aH = st;
        float* bH = st + TILE;
        float* aL = SPLIT3 ? st + 2 * TILE : nullptr;
        float* bL = SPLIT3 ? st + 3 * TILE : nullptr;
        stage_operand<BK, SPLIT3>(t.a, t.M, t.K, m0, kc * BK, aH, aL);
        stage_operand<BK, SPLIT3>(t.bt, t.N, t.K, n0, kc * BK, bH, bL);
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_u32(aH), b0 = tc::smem_u32(bH);
#pragma unroll
            for (int j = 0; j < BK / 8; j++) {
                const uint32_t acc = (kc | j) != 0;
                tc::mma_tf32(tmem, tc::smem_desc(a0 + 256u * j, 128, sbo), tc::smem_desc(b0 + 256u * j, 128, sbo),
                             idesc, acc);
                if constexpr (SPLIT3) {
                    const uint32_t a1 = tc::smem_u32(aL), b1 = tc::smem_u32(bL);
                    tc::mma_tf32(tmem, tc::smem_desc(a0 + 256u * j, 128, sbo), tc::smem_desc(b1 + 256u * j, 128, sbo),
                                 idesc, 1);
                    tc::mma_tf32(tmem, tc::smem_desc(a1 + 256u * j, 128, sbo), tc::smem_desc(b0 + 256u * j, 128, sbo),
                                 idesc, 1);
                }
            }
            tc::mma_commit(&bar[s]);
        }
    }
    // the last commit covers every MMA issued before it
    bool ok = !abort_flag;
    if (ok && nk > 0) ok = tc::bar_wait(&bar[(nk - 1) & 1], (uint32_t)((nk - 1) >> 1) & 1u, err);
    ok = __all_sync(0xffffffffu, ok);
    tc::fence_after_sync();
    if (ok) {
        const int w = threadIdx.x >> 5;
        const int row = m0 + 32 * w + (threadIdx.x & 31);
        for (int c0 = 0; c0 < BN && n0 + c0 < t.N; c0 += 8) {
            float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (nk > 0) tc::tmem_ld8(tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c0, v);
            if (row < t.M) {
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int col = n0 + c0 + j;
                    if (col < t.N) {
                        float* cp = t.c + (int64_t)row * t.c_rs + (int64_t)col * t.c_cs;
                        *cp = t.beta != 0.0f ? t.alpha * v[j] + t.beta * *cp : t.alpha * v[j];
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_free(tmem, BN);
}

}  // namespace

int gemm_tiles(std::vector<GemmTask>& tasks) {
    int tot = 0;
    for (GemmTask& t : tasks) {
        t.ntn = std::max(1, (t.N + kGemmBN - 1) / kGemmBN);
        const int ntm = std::max(1, (t.M + kGemmBM - 1) / kGemmBM);
        t.tile_begin = tot;
        tot += ntm * t.ntn;
    }
    return tot;
}

int launch_tc_gemm(const GemmTask* dtasks, const std::vector<GemmTask>& tasks, bool split3, int* err,
                   cudaStream_t st) {
    if (tasks.empty()) return 0;
    const GemmTask& last = tasks.back();
    const int tiles = last.tile_begin + std::max(1, (last.M + kGemmBM - 1) / kGemmBM) * last.ntn;
    // (the attribute is per device; setting it is cheap next to a launch)
    if (split3) {
        const int smem = 2 * 4 * 128 * 16 * 4;
        cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_tc_gemm<true><<<tiles, 128, smem, st>>>(dtasks, (int)tasks.size(), err);
    } else {
        const int smem = 2 * 2 * 128 * kGemmBK * 4;
        cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_tc_gemm<false><<<tiles, 128, smem, st>>>(dtasks, (int)tasks.size(), err);
    }
    return tiles;
}

}  // namespace spaqr

using namespace spaqr;

extern "C" int spaqr_tc_gemm(int M, int N, int K, float alpha, const float* A, int64_t a_rs, int64_t a_cs,
                             int a_reflectors, const float* B, int64_t b_rs, int64_t b_cs, float beta, float* C,
                             int64_t c_rs, int64_t c_cs, int split3, void* stream) {
    if (M < 0 || N < 0 || K < 0 || (M > 0 && N > 0 && (!C || (K > 0 && (!A || !B))))) {
        set_error("bad size or NULL pointer");
        return SPAQR_ERR_INVALID_ARG;
    }
    if (M == 0 || N == 0) return SPAQR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<GemmTask> tv(1);
    GemmTask& t = tv[0];
    t.a = GemmOperand{A, a_rs, a_cs, a_reflectors != 0, 0};
    t.bt = GemmOperand{B, b_cs, b_rs, 0, 0};   // B^T(j, k) = B(k, j)
    t.c = C;
    t.c_rs = c_rs;
    t.c_cs = c_cs;
    t.M = M;
    t.N = N;
    t.K = K;
    t.alpha = alpha;
    t.beta = beta;
    gemm_tiles(tv);
    GemmTask* d = nullptr;
    int* err = nullptr;
    if (cudaMallocAsync(&d, sizeof(GemmTask), st) != cudaSuccess || cudaMallocAsync(&err, sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        if (d) cudaFreeAsync(d, st);
        set_error("device allocation failed");
        return SPAQR_ERR_OOM;
    }
    cudaMemcpyAsync(d, tv.data(), sizeof(GemmTask), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(err, 0, sizeof(int), st);
    launch_tc_gemm(d, tv, split3 != 0, err, st);
    int herr = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d, st);
    cudaFreeAsync(err, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("CUDA: ") + cudaGetErrorString(e));
        return SPAQR_ERR_CUDA;
    }
    if (herr) { set_error("tensor-core wait ran out"); return SPAQR_ERR_TIMEOUT; }
    return SPAQR_OK;
}
