// Arithmetic peaks of the GPU, measured by microbenchmarks (the paper has no
// counterpart: these are the denominators of the roofline fractions the
// benchmark reports), and a self-check of the tcgen05 TF32 tile used by the
// mixed-precision factorisation.
//
//   DFMA   FP64 fused multiply-add on the CUDA cores
//   DMMA   FP64 mma.sync m8n8k4 (the FP64 tensor path of earlier chips)
//   FFMA   FP32 fused multiply-add on the CUDA cores
//   TF32   tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, FP32 accumulate
//          in tensor memory, operands in shared memory
//
// Each kernel keeps independent dependency chains in flight so that the
// pipe, not latency, bounds it; results are stored so that nothing is
// eliminated.
#include <cuda_runtime.h>

#include <string>

#include "spaqr_internal.h"
#include "tcgen05.cuh"

namespace spaqr {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_peak_dfma(const double* __restrict__ in, double* __restrict__ out, int iters) {
    double a[kChains];
    const double x = in[0], y = in[1];
#pragma unroll
    for (int c = 0; c < kChains; c++) a[c] = in[2] + c * threadIdx.x;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) a[c] = fma(a[c], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += a[c];
    if (s == 12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true for the inputs given
}

__global__ void __launch_bounds__(256) k_peak_ffma(const float* __restrict__ in, float* __restrict__ out, int iters) {
    float a[2 * kChains];
    const float x = in[0], y = in[1];
#pragma unroll
    for (int c = 0; c < 2 * kChains; c++) a[c] = in[2] + c * threadIdx.x;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < 2 * kChains; c++) a[c] = fmaf(a[c], x, y);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 2 * kChains; c++) s += a[c];
    if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One warp: D(8x8) += A(8x4) B(4x8) per instruction, four independent accumulators.
__global__ void __launch_bounds__(256) k_peak_dmma(const double* __restrict__ in, double* __restrict__ out, int iters) {
    double c[4][2];
    const double a = in[0] + threadIdx.x, b = in[1];
#pragma unroll
    for (int j = 0; j < 4; j++) c[j][0] = c[j][1] = in[2];
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 4; j++)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                         : "+d"(c[j][0]), "+d"(c[j][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 4; j++) s += c[j][0] + c[j][1];
    if (s == 12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

constexpr int kTcM = 128, kTcN = 256, kTcK = 16;

// Two CTAs per SM: A (128 x 16) and B (256 x 16) TF32 tiles in shared memory,
// thread 0 issues `iters` rounds of two K-steps into one TMEM accumulator,
// then the CTA waits for them (bounded) and reads one value back.
__global__ void __launch_bounds__(128) k_peak_tf32(const float* __restrict__ in, float* __restrict__ out, int iters,
                                                  int* err) {
    __shared__ __align__(128) float sA[kTcM * kTcK];
    __shared__ __align__(128) float sB[kTcN * kTcK];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    for (int o = threadIdx.x; o < kTcM * kTcK; o += blockDim.x) sA[o] = tc::to_tf32(in[o & 7] * 0.5f);
    for (int o = threadIdx.x; o < kTcN * kTcK; o += blockDim.x) sB[o] = tc::to_tf32(in[o & 7] * 0.25f);
    __syncwarp();
    if (threadIdx.x < 32) tc::tmem_alloc(&tslot, kTcN);
    if (threadIdx.x == 0) tc::bar_init(&bar, 1);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    if (threadIdx.x == 0) {
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
        const uint32_t sbo = (kTcK / 4) * 128;
        const uint32_t idesc = tc::idesc_tf32(kTcM, kTcN);
        for (int i = 0; i < iters; i++) {
#pragma unroll
            for (int k = 0; k < kTcK / 8; k++)
                tc::mma_tf32(tmem, tc::smem_desc(a0 + 256u * k, 128, sbo), tc::smem_desc(b0 + 256u * k, 128, sbo), idesc,
                             (i | k) != 0);
        }
        tc::mma_commit(&bar);
    }
    // warp-uniform (the TMEM loads below are warp-collective)
    const bool ok = __all_sync(0xffffffffu, tc::bar_wait(&bar, 0, err));
    tc::fence_after_sync();
    if (ok) {
        const int w = threadIdx.x >> 5;
        float v[8];
        tc::tmem_ld8(tmem + ((uint32_t)(32 * w) << 16), v);
        if (v[0] == 12345.678f) out[blockIdx.x] = v[0];
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_free(tmem, kTcN);
}

// D (128 x N, row-major) = A (128 x K, row-major) B^T (B N x K, row-major)
// with TF32 inputs (rounded to nearest) and FP32 accumulation: one CTA, the
// tile staged in the K-major layout, K / 8 MMAs, the result read from TMEM.
__global__ void __launch_bounds__(128) k_tc_tile(const float* __restrict__ A, const float* __restrict__ B,
                                                float* __restrict__ D, int N, int K, int* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    float* sA = reinterpret_cast<float*>(smem);
    float* sB = reinterpret_cast<float*>(smem + (size_t)kTcM * K * 4);
    for (int o = threadIdx.x; o < kTcM * K; o += blockDim.x) {
        const int r = o / K, k = o % K;
        sA[tc::kmajor_off(r, k, K) / 4] = tc::to_tf32(A[o]);
    }
    for (int o = threadIdx.x; o < N * K; o += blockDim.x) {
        const int r = o / K, k = o % K;
        sB[tc::kmajor_off(r, k, K) / 4] = tc::to_tf32(B[o]);
    }
    __syncwarp();
    if (threadIdx.x < 32) tc::tmem_alloc(&tslot, 256);
    if (threadIdx.x == 0) tc::bar_init(&bar, 1);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    if (threadIdx.x == 0) {
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
        const uint32_t sbo = (uint32_t)(K / 4) * 128;
        const uint32_t idesc = tc::idesc_tf32(kTcM, N);
        for (int k = 0; k < K / 8; k++)
            tc::mma_tf32(tmem, tc::smem_desc(a0 + 256u * k, 128, sbo), tc::smem_desc(b0 + 256u * k, 128, sbo), idesc,
                         k != 0);
        tc::mma_commit(&bar);
    }
    // warp-uniform (the TMEM loads below are warp-collective)
    const bool ok = __all_sync(0xffffffffu, tc::bar_wait(&bar, 0, err));
    tc::fence_after_sync();
    if (ok) {
        const int w = threadIdx.x >> 5, row = 32 * w + (threadIdx.x & 31);
        for (int c0 = 0; c0 < N; c0 += 8) {
            float v[8];
            tc::tmem_ld8(tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 8; i++) D[(size_t)row * N + c0 + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_free(tmem, 256);
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// Latency of one kind of operation in a dependent chain, per warp: each
// of the CTA's warps runs `iters` dependent operations in its lanes below
// `lanes` and records its clock cycles.  The FP64 rows show what the FP64
// kernels are designed around (an FP64 instruction costs the same pipe time
// whatever its active lanes, and its latency is tens of cycles).
__global__ void k_op_chain(int op, int iters, int lanes, double a, double b, double* out, long long* cyc) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double x = 1.0 + threadIdx.x * 1e-3;
    float xf = (float)x;
    __syncwarp();
    const long long t0 = clock64();
    if (lane < lanes) {
        switch (op) {
            case 0: for (int i = 0; i < iters; i++) x = fma(x, a, b); break;
            case 1: for (int i = 0; i < iters; i++) x = x + b; break;
            case 2: for (int i = 0; i < iters; i++) x = a / x; break;
            case 3: for (int i = 0; i < iters; i++) x = sqrt(x + a); break;
            case 4: for (int i = 0; i < iters; i++) xf = fmaf(xf, (float)a, (float)b); break;
            case 5: for (int i = 0; i < iters; i++) x = (double)(float)x + b; break;
            default: for (int i = 0; i < iters; i++) x = x > b ? x * a : x + a; break;
        }
    }
    __syncwarp();
    const long long t1 = clock64();
    if (lane == 0) cyc[w] = t1 - t0;
    out[threadIdx.x] = x + xf;
}

}  // namespace
}  // namespace spaqr

using namespace spaqr;

extern "C" int spaqr_op_cycles(int op, int warps, int lanes, double* cycles) {
    if (op < 0 || op > 6 || warps < 1 || warps > 32 || lanes < 1 || lanes > 32 || !cycles) {
        set_error("need 0 <= op <= 6, 1 <= warps <= 32, 1 <= lanes <= 32 and an output");
        return SPAQR_ERR_INVALID_ARG;
    }
    double* out = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&out, 1024 * sizeof(double)) != cudaSuccess || cudaMalloc(&cyc, 32 * sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
        if (out) cudaFree(out);
        set_error("device allocation failed");
        return SPAQR_ERR_OOM;
    }
    const int iters = 2048;
    long long h[32] = {0};
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {   // the first run warms up
        k_op_chain<<<1, 32 * warps>>>(op, iters, lanes, 0.999999, 1e-7, out, cyc);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, cyc, warps * sizeof(long long), cudaMemcpyDeviceToHost);
    cudaFree(out);
    cudaFree(cyc);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("CUDA: ") + cudaGetErrorString(e));
        return SPAQR_ERR_CUDA;
    }
    long long mx = 0;
    for (int i = 0; i < warps; i++) mx = h[i] > mx ? h[i] : mx;
    *cycles = (double)mx / iters;
    return SPAQR_OK;
}

extern "C" int spaqr_peak(int which, int reps, double* flops, double* ms) {
    if (which < 0 || which > 3 || reps < 1 || !flops || !ms) { set_error("bad argument"); return SPAQR_ERR_INVALID_ARG; }
    const int sms = sm_count();
    void* buf = nullptr;
    int* err = nullptr;
    if (cudaMalloc(&buf, 1 << 20) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (buf) cudaFree(buf);
        set_error("device allocation failed");
        return SPAQR_ERR_OOM;
    }
    const double hin[3] = {0.999999, 1e-7, 0.5};
    const float fin[8] = {0.999f, 1e-6f, 0.5f, 0.25f, 0.75f, 1.5f, 0.125f, 2.0f};
    double* din = static_cast<double*>(buf);
    float* fbuf = reinterpret_cast<float*>(static_cast<char*>(buf) + 4096);
    cudaMemcpy(din, hin, sizeof(hin), cudaMemcpyHostToDevice);
    cudaMemcpy(fbuf, fin, sizeof(fin), cudaMemcpyHostToDevice);
    cudaMemset(err, 0, sizeof(int));
    double* dout = reinterpret_cast<double*>(static_cast<char*>(buf) + 8192);
    float* fout = reinterpret_cast<float*>(static_cast<char*>(buf) + 8192);
    const int blocks = sms * 8, threads = 256;
    int iters = 0;
    double per = 0.0;
    auto launch = [&]() {
        switch (which) {
            case 0: k_peak_dfma<<<blocks, threads>>>(din, dout, iters); break;
            case 1: k_peak_dmma<<<blocks, threads>>>(din, dout, iters); break;
            case 2: k_peak_ffma<<<blocks, threads>>>(fbuf, fout, iters); break;
            default: k_peak_tf32<<<2 * sms, 128>>>(fbuf, fout, iters, err); break;
        }
    };
    switch (which) {
        case 0: iters = 4096; per = 2.0 * kChains * iters * (double)blocks * threads; break;
        case 1: iters = 2048; per = 512.0 * 4 * iters * (double)blocks * (threads / 32); break;
        case 2: iters = 4096; per = 2.0 * 2 * kChains * iters * (double)blocks * threads; break;
        default: iters = 4096; per = 2.0 * kTcM * kTcN * kTcK * (double)iters * 2 * sms; break;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();   // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < reps; r++) launch();
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(err);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("CUDA: ") + cudaGetErrorString(e));
        return SPAQR_ERR_CUDA;
    }
    if (herr) { set_error("tensor-core wait ran out"); return SPAQR_ERR_TIMEOUT; }
    *flops = per;
    *ms = t / reps;
    return SPAQR_OK;
}

extern "C" int spaqr_tc_tile_check(const float* A, const float* B, float* D, int N, int K, void* stream) {
    if (!A || !B || !D || N < 16 || N > 256 || N % 16 != 0 || K < 8 || K % 8 != 0 || K > 128) {
        set_error("need device A (128 x K), B (N x K), D (128 x N); 16 <= N <= 256, N % 16 == 0, 8 <= K <= 128, K % 8 == 0");
        return SPAQR_ERR_INVALID_ARG;
    }
    int* err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) { cudaGetLastError(); set_error("device allocation failed"); return SPAQR_ERR_OOM; }
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemsetAsync(err, 0, sizeof(int), st);
    const size_t smem = (size_t)(128 + N) * K * 4;
    cudaFuncSetAttribute(k_tc_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_tc_tile<<<1, 128, smem, st>>>(A, B, D, N, K, err);
    int herr = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(err);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("CUDA: ") + cudaGetErrorString(e));
        return SPAQR_ERR_CUDA;
    }
    if (herr) { set_error("tensor-core wait ran out"); return SPAQR_ERR_TIMEOUT; }
    return SPAQR_OK;
}
