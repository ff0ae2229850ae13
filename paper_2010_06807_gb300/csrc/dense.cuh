// CTA-level dense FP64 routines used by the factor and solve kernels.
//
// Householder convention (LAPACK dlarfg reading; the paper only says
// "Householder", Section 2.4): for a column (alpha, x) with x = 0 the
// reflector is the identity (tau = 0); otherwise
// beta = -sign(alpha) sqrt(alpha^2 + x.x) with sign(0) = +1,
// tau = (beta - alpha) / beta, v = (1, x / (alpha - beta)).  A factored
// matrix keeps v below the diagonal (unit diagonal implied) and R on and
// above it.  Block reflector (compact WY): H_0 ... H_{t-1} = I - V T V^T with
// T upper triangular.
//
// Every routine is called by all NT threads of a CTA and synchronises
// internally; operands may be in global or shared memory.
#pragma once

#include <cstdint>

namespace spaqr {

constexpr int NT = 256;          // threads per CTA of every kernel
constexpr int NWARP = NT / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA, result returned to every thread.  `red` holds NWARP
// doubles of shared memory.  Fixed reduction order (deterministic).
__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < NWARP; i++) s += red[i];
    return s;
}

// Largest value over the CTA, ties to the smallest index; every thread gets it.
__device__ __forceinline__ void block_argmax(double v, int idx, double* redv, int* redi, double& bv,
                                             int& bi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) { redv[w] = v; redi[w] = idx; }
    __syncthreads();
    bv = redv[0];
    bi = redi[0];
    for (int i = 1; i < NWARP; i++) {
        if (redv[i] > bv || (redv[i] == bv && redi[i] < bi)) { bv = redv[i]; bi = redi[i]; }
    }
}

// Householder vector of column `col` (rows k..m-1) in place: col[k] <- beta,
// col[k+1..] <- v (below the unit).  Returns tau.  All threads get tau.
__device__ __forceinline__ double cta_house(double* col, int k, int m, double* red) {
    double part = 0.0;
    for (int r = k + 1 + threadIdx.x; r < m; r += NT) {
        double x = col[r];
        part += x * x;
    }
    const double xn2 = block_sum(part, red);
    const double alpha = col[k];
    double tk = 0.0, beta = alpha, denom = 1.0;
    if (xn2 != 0.0) {
        const double s = sqrt(alpha * alpha + xn2);
        beta = alpha >= 0.0 ? -s : s;
        tk = (beta - alpha) / beta;
        denom = alpha - beta;
    }
    __syncthreads();
    if (threadIdx.x == 0) col[k] = beta;
    if (tk != 0.0)
        for (int r = k + 1 + threadIdx.x; r < m; r += NT) col[r] = col[r] / denom;
    __syncthreads();
    return tk;
}

// Apply H_k = I - tau v v^T (v = e_k + col[k+1..m-1]) to columns j0..j1-1 of A.
// One warp per column.
__device__ __forceinline__ void cta_reflect_cols(const double* col, double tk, int k, int m, double* A,
                                                 int64_t lda, int j0, int j1) {
    if (tk == 0.0) return;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int j = j0 + w; j < j1; j += NWARP) {
        double* cj = A + (int64_t)j * lda;
        const double ck = cj[k];
        double d = 0.0;
        for (int r = k + 1 + l; r < m; r += 32) d += col[r] * cj[r];
        d = warp_sum(d) + ck;
        const double f = tk * d;
        if (l == 0) cj[k] = ck - f;
        for (int r = k + 1 + l; r < m; r += 32) cj[r] -= f * col[r];
    }
}

// T factor (forward, columnwise) of the t reflectors stored in A (m rows).
// T is t x t upper triangular, leading dimension ldt.  `z` holds t doubles of
// shared memory.
static __device__ void cta_form_t(const double* A, int64_t lda, int m, int t, const double* tau, double* T,
                           int ldt, double* z) {
    for (int k = 0; k < t; k++) {
        const double tk = tau[k];
        // z_i = V(:,i)^T v_k for i < k
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        for (int i = w; i < k; i += NWARP) {
            const double* vi = A + (int64_t)i * lda;
            const double* vk = A + (int64_t)k * lda;
            double d = 0.0;
            for (int r = k + 1 + l; r < m; r += 32) d += vi[r] * vk[r];
            d = warp_sum(d) + vi[k];
            if (l == 0) z[i] = d;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < k; i += NT) {
            double s = 0.0;
            for (int p = i; p < k; p++) s += T[i + (int64_t)p * ldt] * z[p];
            T[i + (int64_t)k * ldt] = -tk * s;
        }
        if (threadIdx.x == 0) T[k + (int64_t)k * ldt] = tk;
        // zero the strictly lower part of column k for clean storage
        for (int i = k + 1 + threadIdx.x; i < t; i += NT) T[i + (int64_t)k * ldt] = 0.0;
        __syncthreads();
    }
}

// In-place Householder QR of A (m x n, lda); tau gets min(m, n) entries; if T
// is non-null the compact-WY T (t x t, ldt) is formed.  `smem` holds
// NWARP + t doubles.
static __device__ void cta_qr(double* A, int64_t lda, int m, int n, double* tau, double* T, int ldt,
                       double* smem) {
    double* red = smem;
    const int t = m < n ? m : n;
    for (int k = 0; k < t; k++) {
        double* col = A + (int64_t)k * lda;
        const double tk = cta_house(col, k, m, red);
        if (threadIdx.x == 0) tau[k] = tk;
        cta_reflect_cols(col, tk, k, m, A, lda, k + 1, n);
        __syncthreads();
    }
    if (T != nullptr) cta_form_t(A, lda, m, t, tau, T, ldt, smem + NWARP);
}

// Element (r, c) of an m x q operand addressed through an optional row map:
// row r lives at base[(rmap ? rmap[r] : r) + c * ld].
struct RowMapped {
    double* base;
    int64_t ld;
    const int* rmap;
    __device__ __forceinline__ double& at(int r, int c) const {
        return base[(rmap ? (int64_t)rmap[r] : (int64_t)r) + (int64_t)c * ld];
    }
};

// B <- (I - V T V^T)^T B  (trans = true, i.e. Q^T B)  or  (I - V T V^T) B.
// V: m x n unit lower trapezoidal stored in place (v below the diagonal,
// diagonal/upper part ignored) unless `explicit_v` (then read as is).
// B: m x q through a row map.  W: 2 * n * q doubles of shared memory.
static __device__ void cta_apply_wy(const double* V, int64_t ldv, int m, int n, const double* T, int ldt,
                             bool explicit_v, RowMapped B, int q, bool trans, double* W) {
    if (n == 0 || q == 0) return;
    double* W1 = W;
    double* W2 = W + (int64_t)n * q;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    // W1 = V^T B (n x q)
    for (int o = w; o < n * q; o += NWARP) {
        const int i = o % n, c = o / n;
        const double* vi = V + (int64_t)i * ldv;
        double d = 0.0;
        for (int r = i + 1 + l; r < m; r += 32) d += vi[r] * B.at(r, c);
        d = warp_sum(d);
        if (l == 0) W1[o] = d + (explicit_v ? vi[i] : 1.0) * B.at(i, c);
    }
    __syncthreads();
    // W2 = T^T W1 (trans) or T W1
    for (int o = threadIdx.x; o < n * q; o += NT) {
        const int i = o % n, c = o / n;
        double s = 0.0;
        if (trans) {
            for (int p = 0; p <= i; p++) s += T[p + (int64_t)i * ldt] * W1[p + c * n];
        } else {
            for (int p = i; p < n; p++) s += T[i + (int64_t)p * ldt] * W1[p + c * n];
        }
        W2[o] = s;
    }
    __syncthreads();
    // B -= V W2
    for (int o = threadIdx.x; o < m * q; o += NT) {
        const int r = o % m, c = o / m;
        const int top = r < n ? r : n;  // strictly-lower part: columns i < min(r, n)
        double s = 0.0;
        for (int i = 0; i < top; i++) s += V[r + (int64_t)i * ldv] * W2[i + c * n];
        if (r < n) s += (explicit_v ? V[r + (int64_t)r * ldv] : 1.0) * W2[r + c * n];
        B.at(r, c) -= s;
    }
    __syncthreads();
}

// B <- B R^{-1}: B is mi x nj (ldb), R upper triangular nj x nj (ldr).
// Thread-per-row forward substitution; returns false (via flag) on a zero
// diagonal.
static __device__ void cta_trsm_right_upper(double* B, int64_t ldb, int mi, int nj, const double* R,
                                     int64_t ldr, int* singular) {
    for (int r = threadIdx.x; r < mi; r += NT) {
        for (int c = 0; c < nj; c++) {
            double s = B[r + (int64_t)c * ldb];
            for (int p = 0; p < c; p++) s -= B[r + (int64_t)p * ldb] * R[p + (int64_t)c * ldr];
            const double d = R[c + (int64_t)c * ldr];
            if (d == 0.0) { *singular = 1; s = 0.0; }
            else s = s / d;
            B[r + (int64_t)c * ldb] = s;
        }
    }
    __syncthreads();
}

// X <- R^{-1} X for X n x q through a row map, R upper n x n (ldr).
// Column-oriented back substitution.
static __device__ void cta_trsv_upper(const double* R, int64_t ldr, int n, RowMapped X, int q, int* singular) {
    for (int i = n - 1; i >= 0; i--) {
        const double d = R[i + (int64_t)i * ldr];
        for (int c = threadIdx.x; c < q; c += NT) {
            if (d == 0.0) { *singular = 1; X.at(i, c) = 0.0; }
            else X.at(i, c) = X.at(i, c) / d;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < i * q; o += NT) {
            const int r = o % i, c = o / i;
            X.at(r, c) -= R[r + (int64_t)i * ldr] * X.at(i, c);
        }
        __syncthreads();
    }
}

}  // namespace spaqr
