// CTA-level dense FP64 routines used by the factor and solve kernels.
//
// Householder convention (LAPACK dlarfg reading; the paper only says
// "Householder", Section 2.4): for a column (alpha, x) with x = 0 the
// reflector is the identity (tau = 0); otherwise
// beta = -sign(alpha) sqrt(alpha^2 + x.x) with sign(0) = +1,
// tau = (beta - alpha) / beta, v = (1, x / (alpha - beta)).  A factored
// matrix keeps v below the diagonal (unit diagonal implied) and R on and
// above it.
//
// Blocked reflectors: reflectors are grouped in panels of NB consecutive
// ones; panel b (reflectors p0 .. p0+pb-1) is I - V_b T_b V_b^T with T_b upper
// triangular, stored as the diagonal block T[p0:p0+pb, p0:p0+pb] of an array
// with leading dimension ldt (the off-diagonal blocks are unused).
// Q = H_0 H_1 ... = Q_0 Q_1 ... so Q^T B applies panels 0, 1, ... with T_b^T
// and Q B applies them in reverse order with T_b.
//
// GB300 executes FP64 at ~2 DFMA per clock per SM, and a warp shuffle
// reduction costs one DADD per step on that same pipe.  The routines therefore
// compute every dot product as one thread's sequential DFMA chain (thread per
// output) and only reduce across threads where a result is needed once per
// column (norms, Householder scalars).
//
// Every routine is templated on the storage/arithmetic type `real` (double
// for the FP64 form, float for the mixed-precision form; Householder scalars
// and pivot decisions stay FP64 in both), is called by all NT threads of a
// CTA and synchronises internally; operands may be in global or shared
// memory.
#pragma once

#include <cstdint>

namespace spaqr {

constexpr int NT = 256;          // threads per CTA of every kernel
constexpr int NWARP = NT / 32;
constexpr int NB = 16;           // reflectors per panel

// Asynchronous element copies global -> shared (cp.async, 4 or 8 bytes):
// a thread issues many without waiting, so a staged block has all its loads
// in flight at once.  cp_async_wait<N> waits until at most N of this thread's
// committed groups are pending; a __syncthreads must follow before other
// threads read the data.
template <class real>
__device__ __forceinline__ void cp_async_elem(real* dst, const real* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(real) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Doubles of shared memory that block_sum and cta_house work in.
constexpr int RED = NT + 8;

// Sum over the CTA, result returned to every thread.  `red` holds RED doubles
// of shared memory.  Fixed reduction order (deterministic): the NT partials go
// to shared memory and warp 0 alone adds them (eight per lane, then across the
// warp).  On GB300 an FP64 instruction occupies the SM's FP64 pipe for the
// same time whatever its active lanes, so an FP64 reduction run by one warp
// instead of all of them costs a fraction of the pipe time and less latency.
__device__ __forceinline__ double block_sum(double v, double* red) {
    red[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        const double* p = red + threadIdx.x;
        double s = ((p[0] + p[32]) + (p[64] + p[96])) + ((p[128] + p[160]) + (p[192] + p[224]));
        s = warp_sum(s);
        if (threadIdx.x == 0) red[NT] = s;
    }
    __syncthreads();
    return red[NT];
}

// Order key of a non-negative value: its IEEE bit pattern, which orders like
// the value, so that comparisons run on the integer pipe (an FP64 compare
// occupies the slow FP64 pipe on GB300).
__device__ __forceinline__ long long nonneg_key(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ long long nonneg_key(float v) { return (long long)__float_as_int(v); }

// Largest key over the CTA, ties to the smallest index; every thread gets it.
__device__ __forceinline__ void block_argmax_key(long long key, int idx, long long* redv, int* redi, long long& bk,
                                                 int& bi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long ok = __shfl_xor_sync(0xffffffffu, key, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ok > key || (ok == key && oi < idx)) { key = ok; idx = oi; }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) { redv[w] = key; redi[w] = idx; }
    __syncthreads();
    bk = redv[0];
    bi = redi[0];
    for (int i = 1; i < NWARP; i++) {
        if (redv[i] > bk || (redv[i] == bk && redi[i] < bi)) { bk = redv[i]; bi = redi[i]; }
    }
}

// Strided view of a matrix: element (r, c) is base[row(r) * rs + c * cs] with
// row(r) = rmap ? rmap[r] : r.
template <class real>
struct Mat {
    real* base;
    int64_t rs, cs;
    const int* rmap;
    __device__ __forceinline__ real& at(int r, int c) const {
        const int64_t rr = rmap ? (int64_t)rmap[r] : (int64_t)r;
        return base[rr * rs + (int64_t)c * cs];
    }
    __device__ __forceinline__ Mat cols(int c0) const { return Mat{base + (int64_t)c0 * cs, rs, cs, rmap}; }
};

// Householder vector of column `col` (rows k..m-1, element stride `stride`)
// in place: col[k] <- beta, col[k+1..] <- v.  Returns tau to every thread.
// The squared norm (every partial sum), beta, tau and alpha - beta are FP64
// whatever the storage type; v = x / (alpha - beta) is divided in FP64 in the
// FP64 form and by alpha - beta rounded to FP32 in the FP32 form.
// sign_tol > 0: alpha counts as negative only below
// -sign_tol sqrt(alpha^2 + x.x), so that a leading entry that is zero up to
// rounding always gives beta = -norm.  `red`: RED doubles of shared memory.
template <class real>
__device__ __forceinline__ double cta_house(real* col, int64_t stride, int k, int m, double* red,
                                            double sign_tol = 0.0) {
    static_assert(NT == 256, "the reduction below adds eight partials per lane");
    double part = 0.0;
    for (int r = k + 1 + threadIdx.x; r < m; r += NT) {
        const double x = (double)col[(int64_t)r * stride];
        part += x * x;
    }
    // squared norm by warp 0; the scalars by its lane 0 (FP64 work of one
    // warp, not of every warp), shared through red[NT..]
    red[threadIdx.x] = part;
    __syncthreads();
    if (threadIdx.x < 32) {
        const double* p = red + threadIdx.x;
        double xn2 = ((p[0] + p[32]) + (p[64] + p[96])) + ((p[128] + p[160]) + (p[192] + p[224]));
        xn2 = warp_sum(xn2);
        if (threadIdx.x == 0) {
            const double alpha = (double)col[(int64_t)k * stride];
            double beta = alpha, denom = 1.0;
            if (xn2 != 0.0) {
                const double s = sqrt(alpha * alpha + xn2);
                beta = alpha >= -sign_tol * s ? -s : s;
                denom = alpha - beta;
            }
            red[NT] = denom;
            red[NT + 1] = beta;
            red[NT + 2] = alpha;
            reinterpret_cast<float*>(red + NT + 3)[0] = (float)denom;
            reinterpret_cast<int*>(red + NT + 4)[0] = xn2 != 0.0;
        }
    }
    __syncthreads();
    const bool reflect = reinterpret_cast<const int*>(red + NT + 4)[0] != 0;
    if (reflect) {
        if constexpr (sizeof(real) == 8) {
            const double denom = red[NT];
            for (int r = k + 1 + threadIdx.x; r < m; r += NT) col[(int64_t)r * stride] = col[(int64_t)r * stride] / denom;
        } else {
            const float denom = reinterpret_cast<const float*>(red + NT + 3)[0];
            for (int r = k + 1 + threadIdx.x; r < m; r += NT) col[(int64_t)r * stride] /= denom;
        }
    }
    if (threadIdx.x == 0) {
        // tau off the critical path: thread 0 forms it while the others divide
        const double beta = red[NT + 1], alpha = red[NT + 2];
        red[NT + 5] = reflect ? (beta - alpha) / beta : 0.0;
        col[(int64_t)k * stride] = (real)beta;
    }
    __syncthreads();
    return red[NT + 5];
}

// Diagonal T blocks of the t reflectors in V (m rows, column-major, ldv); the
// diagonal/upper part of V is not read (unit diagonal implied).  `G` holds
// NB * NB and `X` NB * NB / 2 elements of shared memory.  cta_t_from_g forms
// one block (pb <= NB reflectors) from G (strict upper part, ld ldg) and tau.
//
// A block's T is built by doubling (the compact-WY identity for a product of
// two block reflectors): with T11, T22 the factors of reflectors [a, b) and
// [b, c), the factor of [a, c) is [[T11, -T11 G12 T22], [0, T22]],
// G12 = V(:, a:b)^T V(:, b:c).  Merging pairs of blocks of 1, 2, 4 and 8
// reflectors gives the same T as the column recurrence
// T(0:k, k) = -tau_k T(0:k, 0:k) G(0:k, k), in four steps instead of sixteen
// sequential ones (every FP64 operation costs ~64 cycles of latency on GB300).
template <class real>
static __device__ void cta_t_from_g(const real* G, int ldg, const real* tau, real* Tb, int ldt, int pb, real* X) {
    // the diagonal of T and zeros elsewhere
    for (int o = threadIdx.x; o < pb * pb; o += NT) {
        const int i = o % pb, k = o / pb;
        Tb[i + (int64_t)k * ldt] = i == k ? tau[i] : (real)0;
    }
    __syncthreads();
    for (int h = 1; h < pb; h *= 2) {
        // merges of [b0, b0 + h) and [b0 + h, b0 + h + h2), b0 = 2 h g
        const int nm = (pb + 2 * h - 1) / (2 * h);
        // X_g = G12 T22 (h x h2; T22 upper triangular)
        for (int o = threadIdx.x; o < nm * h * h; o += NT) {
            const int g = o / (h * h), i = o % h, j = (o / h) % h;
            const int b0 = 2 * h * g, h2 = min(h, pb - b0 - h);
            if (j >= h2) continue;
            real s = 0;
            for (int u = 0; u <= j; u++)
                s += G[(b0 + i) + (b0 + h + u) * ldg] * Tb[(b0 + h + u) + (int64_t)(b0 + h + j) * ldt];
            X[g * h * h + i + j * h] = s;
        }
        __syncthreads();
        // T12 = -T11 X_g (T11 upper triangular)
        for (int o = threadIdx.x; o < nm * h * h; o += NT) {
            const int g = o / (h * h), i = o % h, j = (o / h) % h;
            const int b0 = 2 * h * g, h2 = min(h, pb - b0 - h);
            if (j >= h2) continue;
            real s = 0;
            for (int u = i; u < h; u++) s += Tb[(b0 + i) + (int64_t)(b0 + u) * ldt] * X[g * h * h + u + j * h];
            Tb[(b0 + i) + (int64_t)(b0 + h + j) * ldt] = -s;
        }
        __syncthreads();
    }
}

template <class real>
static __device__ void cta_form_tblocks(const real* V, int64_t ldv, int m, int t, const real* tau, real* T, int ldt,
                                        real* G, real* X) {
    for (int p0 = 0; p0 < t; p0 += NB) {
        const int pb = t - p0 < NB ? t - p0 : NB;
        // G(i, k) = V(:, p0+i)^T V(:, p0+k), i < k
        for (int o = threadIdx.x; o < pb * pb; o += NT) {
            const int i = o % pb, k = o / pb;
            if (i >= k) continue;
            const real* vi = V + (int64_t)(p0 + i) * ldv;
            const real* vk = V + (int64_t)(p0 + k) * ldv;
            real s = vi[p0 + k];
            for (int r = p0 + k + 1; r < m; r++) s += vi[r] * vk[r];
            G[i + k * NB] = s;
        }
        __syncthreads();
        cta_t_from_g(G, NB, tau + p0, T + p0 + (int64_t)p0 * ldt, ldt, pb, X);
    }
}

// Number of row groups that split each dot product so that nout outputs keep
// all NT threads busy (a power of two, 1 when nout >= NT / 2).
__device__ __forceinline__ int row_groups(int nout) {
    int g = 1;
    while (g < 16 && nout * g * 2 <= NT) g *= 2;
    return g;
}

// W1(i, c) = sum over the rows of Vcol_i(r) * Bv(r, c) for the pb x q outputs;
// `dot(i, c, r0, step)` returns a partial sum over rows r0, r0 + step, ...
// P holds NT doubles.
template <class real, class Dot>
__device__ __forceinline__ void cta_small_gemv(int pb, int q, real* W1, real* P, Dot dot) {
    const int nout = pb * q;
    const int G = row_groups(nout);
    if (G == 1) {
        for (int o = threadIdx.x; o < nout; o += NT) W1[o] = dot(o % pb, o / pb, 0, 1);
        __syncthreads();
        return;
    }
    if (threadIdx.x < nout * G) {
        const int o = threadIdx.x % nout, g = threadIdx.x / nout;
        P[threadIdx.x] = dot(o % pb, o / pb, g, G);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += NT) {
        // the G row-group partials added as a tree (G a power of two <= 16)
        real v[16];
#pragma unroll
        for (int g = 0; g < 16; g++) v[g] = g < G ? P[o + g * nout] : (real)0;
#pragma unroll
        for (int h = 8; h > 0; h >>= 1)
            if (h < G)
#pragma unroll
                for (int g = 0; g < h; g++) v[g] += v[g + h];
        W1[o] = v[0];
    }
    __syncthreads();
}

// W2 = T_b^T W1 (trans) or T_b W1 for the diagonal T block at p0.
template <class real>
__device__ __forceinline__ void cta_tblock_mul(const real* T, int ldt, int p0, int pb, int q, bool trans,
                                               const real* W1, real* W2) {
    for (int o = threadIdx.x; o < pb * q; o += NT) {
        const int i = o % pb, c = o / pb;
        real s = 0;
        if (trans) {
            for (int u = 0; u <= i; u++) s += T[(p0 + u) + (int64_t)(p0 + i) * ldt] * W1[u + c * pb];
        } else {
            for (int u = i; u < pb; u++) s += T[(p0 + i) + (int64_t)(p0 + u) * ldt] * W1[u + c * pb];
        }
        W2[o] = s;
    }
    __syncthreads();
}

// B <- Q^T B (trans) or Q B for the t reflectors in V (m rows) with diagonal T
// blocks; B is m x q, read and written in place (global or shared memory).
// explicit_v: V holds its unit diagonal (and zeros above it) explicitly;
// otherwise the diagonal is taken as 1 and the upper part is ignored.
// W holds 2 * NB * q + NT doubles of shared memory.
template <class real>
static __device__ void cta_apply_q(const real* V, int64_t ldv, int m, int t, const real* T, int ldt,
                                   bool explicit_v, Mat<real> B, int q, bool trans, real* W) {
    if (t <= 0 || q <= 0) return;
    real* W1 = W;
    real* W2 = W + NB * q;
    real* P = W + 2 * NB * q;
    const int nbk = (t + NB - 1) / NB;
    for (int bb = 0; bb < nbk; bb++) {
        const int b = trans ? bb : nbk - 1 - bb;
        const int p0 = b * NB;
        const int pb = t - p0 < NB ? t - p0 : NB;
        cta_small_gemv(pb, q, W1, P, [&](int i, int c, int g, int G) {
            const int col = p0 + i;
            const real* v = V + (int64_t)col * ldv;
            real s = 0;
            if (g == 0) s = (explicit_v ? v[col] : (real)1) * B.at(col, c);
            // rows col+1+.. with stride G, loaded four at a time before use
            // (the additions keep the row order)
            constexpr int U = 4;
            int r = col + 1 + (g == 0 ? G - 1 : g - 1);
            for (; r + (U - 1) * G < m; r += U * G) {
                real a[U], b[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    a[u] = v[r + u * G];
                    b[u] = B.at(r + u * G, c);
                }
#pragma unroll
                for (int u = 0; u < U; u++) s += a[u] * b[u];
            }
            for (; r < m; r += G) s += v[r] * B.at(r, c);
            return s;
        });
        cta_tblock_mul(T, ldt, p0, pb, q, trans, W1, W2);
        // B(r, c) -= sum_{i <= r - p0} V(r, p0+i) W2(i, c), r >= p0
        const int rows = m - p0;
        for (int o = threadIdx.x; o < rows * q; o += NT) {
            const int rr = o % rows, c = o / rows, r = p0 + rr;
            const int top = rr < pb - 1 ? rr : pb - 1;   // last i with p0 + i <= r
            real s = 0;
            for (int i = 0; i < top; i++) s += V[r + (int64_t)(p0 + i) * ldv] * W2[i + c * pb];
            const real vd = (rr == top) ? (explicit_v ? V[r + (int64_t)r * ldv] : (real)1)
                                        : V[r + (int64_t)(p0 + top) * ldv];
            s += vd * W2[top + c * pb];
            B.at(r, c) -= s;
        }
        __syncthreads();
    }
}

// Shared memory (elements) of cta_apply_q_staged for m rows and q columns.
__host__ __device__ constexpr int64_t staged_smem_elems(int m, int q) {
    return (int64_t)(m | 1) * (q + NB) + 2 * NB * q + NT;
}

// Same as cta_apply_q, with B (m x q) staged into shared memory once and each
// panel of V staged before use, so the inner loops read shared memory only.
// smem: staged_smem_elems(m, q) elements.
template <class real>
static __device__ void cta_apply_q_staged(const real* V, int64_t ldv, int m, int t, const real* T, int ldt,
                                          bool explicit_v, Mat<real> B, int q, bool trans, real* sm) {
    if (t <= 0 || q <= 0) return;
    const int ld = m | 1;
    real* Bs = sm;
    real* Vs = Bs + (int64_t)ld * q;
    real* W1 = Vs + (int64_t)ld * NB;
    real* W2 = W1 + NB * q;
    real* P = W2 + NB * q;
    for (int o = threadIdx.x; o < m * q; o += NT) {
        const int r = o % m, c = o / m;
        Bs[r + c * ld] = B.at(r, c);
    }
    const int nbk = (t + NB - 1) / NB;
    for (int bb = 0; bb < nbk; bb++) {
        const int b = trans ? bb : nbk - 1 - bb;
        const int p0 = b * NB;
        const int pb = t - p0 < NB ? t - p0 : NB;
        const int rows = m - p0;
        // Vs(rr, i) = V(p0 + rr, p0 + i) with the unit diagonal and zeros above
        for (int o = threadIdx.x; o < rows * pb; o += NT) {
            const int rr = o % rows, i = o / rows;
            const int r = p0 + rr, col = p0 + i;
            real v = 0;
            if (r > col) v = V[r + (int64_t)col * ldv];
            else if (r == col) v = explicit_v ? V[r + (int64_t)col * ldv] : (real)1;
            Vs[rr + i * ld] = v;
        }
        __syncthreads();
        cta_small_gemv(pb, q, W1, P, [&](int i, int c, int g, int G) {
            const real* vi = Vs + i * ld;
            const real* bc = Bs + p0 + c * ld;
            real s = 0;
            for (int rr = i + g; rr < rows; rr += G) s += vi[rr] * bc[rr];
            return s;
        });
        cta_tblock_mul(T, ldt, p0, pb, q, trans, W1, W2);
        for (int o = threadIdx.x; o < rows * q; o += NT) {
            const int rr = o % rows, c = o / rows;
            const int top = rr < pb - 1 ? rr : pb - 1;
            real s = 0;
            for (int i = 0; i <= top; i++) s += Vs[rr + i * ld] * W2[i + c * pb];
            Bs[p0 + rr + c * ld] -= s;
        }
        __syncthreads();
    }
    for (int o = threadIdx.x; o < m * q; o += NT) {
        const int r = o % m, c = o / m;
        B.at(r, c) = Bs[r + c * ld];
    }
    __syncthreads();
}

// cta_apply_q over q columns in chunks of qc (W: 2 * NB * qc + NT elements).
template <class real>
static __device__ void cta_apply_q_chunked(const real* V, int64_t ldv, int m, int t, const real* T, int ldt,
                                           bool explicit_v, Mat<real> B, int q, int qc, bool trans, real* W) {
    for (int c0 = 0; c0 < q; c0 += qc) {
        const int w = q - c0 < qc ? q - c0 : qc;
        cta_apply_q(V, ldv, m, t, T, ldt, explicit_v, B.cols(c0), w, trans, W);
    }
}

// Shared memory (bytes) needed by cta_qr with column chunk qc and a staged
// panel of up to prow rows (prow = 0: panels stay in global memory).
__host__ __device__ constexpr int64_t qr_smem_bytes(int esz, int qc, int prow = 0) {
    return 8 * RED + (int64_t)esz * (NT + NB + NB * NB + 2 * NB * qc + NT + (int64_t)prow * NB);
}

// Factor the panel columns [p0, pe) of A (rows p0..m-1) in place, column by
// column, and form its T block (T + p0 + p0 ldt).  With staged (m <= prow) the
// panel is worked on in shared memory Ps and written back at the end.  Returns
// the panel view (reflectors) for the trailing update: Vp with leading
// dimension *ldv (shared memory when staged, otherwise A itself).
template <class real>
static __device__ const real* cta_qr_panel(real* A, int64_t lda, int m, int p0, int pe, real* tau, real* T, int ldt,
                                           bool staged, double* red, real* P, real* Wk, real* G, real* Ps,
                                           int64_t* ldv, double sign_tol = 0.0) {
    // panel view: column k, row r -> Pb[r + (k - p0) * ldp]
    real* Pb;
    int64_t ldp;
    if (staged) {
        ldp = m - p0;
        Pb = Ps - p0;
        for (int o = threadIdx.x; o < (m - p0) * (pe - p0); o += NT) {
            const int rr = o % (m - p0), j = o / (m - p0);
            Ps[rr + (int64_t)j * ldp] = A[(p0 + rr) + (int64_t)(p0 + j) * lda];
        }
        __syncthreads();
    } else {
        ldp = lda;
        Pb = A + (int64_t)p0 * lda;
    }
    for (int k = p0; k < pe; k++) {
        real* col = Pb + (int64_t)(k - p0) * ldp;
        const double tkd = cta_house(col, 1, k, m, red, sign_tol);
        const real tk = (real)tkd;
        if (threadIdx.x == 0) tau[k] = tk;
        const int ncol = pe - k - 1;
        if (ncol > 0 && tkd != 0.0) {
            // partial dots: NB column slots x (NT / NB) row groups
            const int js = threadIdx.x % NB, g = threadIdx.x / NB;
            real part = 0;
            if (js < ncol) {
                const real* cj = Pb + (int64_t)(k + 1 + js - p0) * ldp;
                constexpr int S = NT / NB, U = 8;
                int r = k + 1 + g;
                for (; r + (U - 1) * S < m; r += U * S) {   // eight loads in flight, order kept
                    real a[U], b[U];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        a[u] = col[r + u * S];
                        b[u] = cj[r + u * S];
                    }
#pragma unroll
                    for (int u = 0; u < U; u++) part += a[u] * b[u];
                }
                for (; r < m; r += S) part += col[r] * cj[r];
            }
            P[threadIdx.x] = part;
            __syncthreads();
            if (threadIdx.x < ncol) {
                // row k's entry plus the 16 row-group partials (added as a tree)
                static_assert(NT / NB == 16, "sixteen row groups");
                const real* pp = P + threadIdx.x;
                const real s = (((pp[0] + pp[NB]) + (pp[2 * NB] + pp[3 * NB])) +
                                ((pp[4 * NB] + pp[5 * NB]) + (pp[6 * NB] + pp[7 * NB]))) +
                               (((pp[8 * NB] + pp[9 * NB]) + (pp[10 * NB] + pp[11 * NB])) +
                                ((pp[12 * NB] + pp[13 * NB]) + (pp[14 * NB] + pp[15 * NB])));
                Wk[threadIdx.x] = tk * (Pb[k + (int64_t)(k + 1 + threadIdx.x - p0) * ldp] + s);
            }
            __syncthreads();
            const int rows = m - k;
            for (int o = threadIdx.x; o < rows * ncol; o += NT) {
                const int rr = o % rows, jj = o / rows, r = k + rr;
                const real v = rr == 0 ? (real)1 : col[r];
                Pb[r + (int64_t)(k + 1 + jj - p0) * ldp] -= Wk[jj] * v;
            }
        }
        __syncthreads();
    }
    if (staged) {
        for (int o = threadIdx.x; o < (m - p0) * (pe - p0); o += NT) {
            const int rr = o % (m - p0), j = o / (m - p0);
            A[(p0 + rr) + (int64_t)(p0 + j) * lda] = Ps[rr + (int64_t)j * ldp];
        }
    }
    // T block of the panel (reflectors = panel rows p0.. of the panel view)
    const real* Vp = Pb + p0;
    cta_form_tblocks(Vp, ldp, m - p0, pe - p0, tau + p0, T + p0 + (int64_t)p0 * ldt, ldt, G, P);
    *ldv = ldp;
    return Vp;
}

// In-place blocked Householder QR of A (m x n, lda).  tau gets min(m, n)
// entries and T the diagonal NB blocks (ldt).  A panel of NB columns is
// factored column by column (in shared memory when m <= prow), then applied
// to the columns right of it as a block reflector.
// smem: qr_smem_bytes(sizeof(real), qc, prow).
template <class real>
static __device__ void cta_qr(real* A, int64_t lda, int m, int n, real* tau, real* T, int ldt, int qc, int prow,
                              double* smem, double sign_tol = 0.0) {
    double* red = smem;                               // RED
    real* P = reinterpret_cast<real*>(red + RED);     // NT partial dots
    real* Wk = P + NT;         // NB
    real* G = Wk + NB;         // NB * NB
    real* W = G + NB * NB;     // 2 * NB * qc + NT
    real* Ps = W + 2 * NB * qc + NT;   // prow * NB
    const int t = m < n ? m : n;
    const bool staged = m <= prow;
    for (int p0 = 0; p0 < t; p0 += NB) {
        const int pe = (t - p0 < NB ? t : p0 + NB);   // panel columns [p0, pe)
        int64_t ldp;
        const real* Vp = cta_qr_panel(A, lda, m, p0, pe, tau, T, ldt, staged, red, P, Wk, G, Ps, &ldp, sign_tol);
        // trailing update of the columns right of the panel
        if (pe < n) {
            Mat<real> B{A + p0 + (int64_t)pe * lda, 1, lda, nullptr};
            cta_apply_q_chunked(Vp, ldp, m - p0, pe - p0, T + p0 + (int64_t)p0 * ldt, ldt, false, B, n - pe, qc,
                                true, W);
        }
        __syncthreads();
    }
}

// Inverses of the diagonal NB x NB blocks of the upper triangular R (n x n,
// ldr): block b (rows/columns [b NB, b NB + bs)) goes to Dinv rows
// [b NB, b NB + bs), columns [0, bs) (ld n), upper triangular, zeros below.
// One thread per column of a block (back substitution).  Sets *singular on a
// zero diagonal entry (and writes zeros for it).
template <class real>
static __device__ void cta_tri_inv_blocks(const real* R, int64_t ldr, int n, real* Dinv, int* singular) {
    const int nbk = (n + NB - 1) / NB;
    for (int o = threadIdx.x; o < nbk * NB; o += NT) {
        const int b = o / NB, j = o % NB, b0 = b * NB;
        const int bs = n - b0 < NB ? n - b0 : NB;
        if (j >= bs) continue;
        real* dj = Dinv + b0 + (int64_t)j * n;
        for (int i = bs - 1; i > j; i--) dj[i] = 0;
        for (int i = j; i >= 0; i--) {
            double s = i == j ? 1.0 : 0.0;
            for (int u = i + 1; u <= j; u++) s -= (double)R[(b0 + i) + (int64_t)(b0 + u) * ldr] * (double)dj[u];
            const double d = (double)R[(b0 + i) + (int64_t)(b0 + i) * ldr];
            if (d == 0.0) {
                if (singular) *singular = 1;
                dj[i] = 0;
            } else {
                dj[i] = (real)(s / d);
            }
        }
    }
    __syncthreads();
}

// B <- B R^{-1}: B is mi x nj (ldb), R upper triangular nj x nj (ldr) with
// inverted diagonal blocks Dinv (ld nj).  Per block of NB columns (left to
// right): the update by the solved columns runs one thread per entry, then
// the block is multiplied by Dinv_b one thread per row.
template <class real>
static __device__ void cta_trsm_right_upper(real* B, int64_t ldb, int mi, int nj, const real* R, int64_t ldr,
                                            const real* Dinv) {
    for (int b0 = 0; b0 < nj; b0 += NB) {
        const int bs = nj - b0 < NB ? nj - b0 : NB;
        if (b0 > 0) {
            for (int o = threadIdx.x; o < mi * bs; o += NT) {
                const int r = o % mi, j = o / mi;
                const real* rc = R + (int64_t)(b0 + j) * ldr;
                real s = B[r + (int64_t)(b0 + j) * ldb];
                // solved columns u < b0, loaded four at a time (order kept)
                constexpr int U = 4;
                int u = 0;
                for (; u + U <= b0; u += U) {
                    real x[U], y[U];
#pragma unroll
                    for (int w = 0; w < U; w++) {
                        x[w] = B[r + (int64_t)(u + w) * ldb];
                        y[w] = rc[u + w];
                    }
#pragma unroll
                    for (int w = 0; w < U; w++) s -= x[w] * y[w];
                }
                for (; u < b0; u++) s -= B[r + (int64_t)u * ldb] * rc[u];
                B[r + (int64_t)(b0 + j) * ldb] = s;
            }
            __syncthreads();
        }
        const real* D = Dinv + b0;
        for (int r = threadIdx.x; r < mi; r += NT) {
            real* br = B + r + (int64_t)b0 * ldb;
            real t[NB];
#pragma unroll
            for (int j = 0; j < NB; j++) t[j] = j < bs ? br[(int64_t)j * ldb] : (real)0;
#pragma unroll
            for (int j = NB - 1; j >= 0; j--) {
                if (j < bs) {
                    real x = 0;
#pragma unroll
                    for (int l = 0; l <= j; l++) x += t[l] * D[l + (int64_t)j * nj];
                    br[(int64_t)j * ldb] = x;
                }
            }
        }
        __syncthreads();
    }
}

// X <- R^{-1} X for X n x q, R upper n x n (ldr) with inverted diagonal
// blocks Dinv (ld n).  Block back substitution: per block (bottom up)
// x_b = Dinv_b y_b, then the rows above are updated.  tmp: NB * q doubles of
// shared memory.
template <class real>
static __device__ void cta_trsv_upper(const real* R, int64_t ldr, int n, const real* Dinv, Mat<real> X, int q,
                                      real* tmp) {
    const int nbk = (n + NB - 1) / NB;
    for (int b = nbk - 1; b >= 0; b--) {
        const int b0 = b * NB;
        const int bs = n - b0 < NB ? n - b0 : NB;
        for (int o = threadIdx.x; o < bs * q; o += NT) {
            const int i = o % bs, c = o / bs;
            real s = 0;
            for (int u = i; u < bs; u++) s += Dinv[(b0 + i) + (int64_t)u * n] * X.at(b0 + u, c);
            tmp[o] = s;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < bs * q; o += NT) X.at(b0 + o % bs, o / bs) = tmp[o];
        __syncthreads();
        for (int o = threadIdx.x; o < b0 * q; o += NT) {
            const int r = o % b0, c = o / b0;
            real s = 0;
            for (int u = 0; u < bs; u++) s += R[r + (int64_t)(b0 + u) * ldr] * X.at(b0 + u, c);
            X.at(r, c) -= s;
        }
        __syncthreads();
    }
}

}  // namespace spaqr
