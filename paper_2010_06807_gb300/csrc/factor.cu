// Numeric spaQR factorisation on the GPU (Algorithm 2 of the paper).
//
// Per level (leaves first):
//   (i)   every separator s of the level: Householder QR of its front (the
//         column panel of s: rows R(s) stacked), then H_s^T applied to the
//         columns C(s) of the front rows (Section 2.4);
//   (ii)  block-diagonal scaling of every remaining interface p: A_pp = U R,
//         rows p <- U^T, columns p <- R^{-1} (Section 2.5);
//   (iii) sparsification: truncated column-pivoted QR of
//         M_p = [A_np^T | A_pn] (rank rule of Section 4), then
//         A_ij <- Q_i^T A_ij Q_j keeping the coarse rows/columns (Sections
//         2.2, 2.5); all Q_p of a level are computed before any is applied;
//   (iv)  merge of interfaces along the cluster hierarchy (Section 2.6),
//         fused into (iii): every coarse block is written at its place in the
//         merged blocks of the next level.
// Storage: per level one arena of column panels (panel j = all blocks of
// column j stacked, rows ascending), column-major.  The arena of a level is
// kept: it holds the front reflectors, R_ss, the R_sj rows and the scaled
// diagonal blocks the solve needs.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdio>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dense.cuh"
#include "spaqr_internal.h"
#include "tasks.h"
#include "tcgemm.h"

#define SPAQR_LAUNCH(kind, flops, bytes, stream, ...)                            \
    do {                                                                         \
        const int rec_ = prof_begin((void*)(stream), (kind), (flops), (bytes)); \
        __VA_ARGS__;                                                             \
        prof_end((void*)(stream), rec_);                                         \
    } while (0)

namespace spaqr {

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// d_j = 1 / ||A(:, j)||_2 (Section 2.7); sums in ascending row order.
__global__ void k_colscale(int64_t n, const int64_t* __restrict__ csc_ptr,
                           const int64_t* __restrict__ csc_entry, const double* __restrict__ val,
                           int normalize, double* __restrict__ d, int* __restrict__ bad) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (!normalize) { d[j] = 1.0; return; }
    double s = 0.0;
    for (int64_t e = csc_ptr[j]; e < csc_ptr[j + 1]; e++) {
        const double v = val[csc_entry[e]];
        s += v * v;
    }
    if (s == 0.0) { *bad = 1; d[j] = 0.0; return; }
    d[j] = 1.0 / sqrt(s);
}

// Level-1 arena <- A D scattered into column panels (rounded to the storage type).
template <class real>
__global__ void k_gather(int64_t nnz, const int64_t* __restrict__ off, const int32_t* __restrict__ colind,
                         const double* __restrict__ val, const double* __restrict__ d, real* __restrict__ arena) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    arena[off[e]] = (real)(val[e] * d[colind[e]]);
}

constexpr int QC = 32;       // column chunk of the blocked updates
// CTAs per cluster of the large-front QR: 16, the largest (non-portable)
// cluster, so that the few large fronts of the upper levels keep more SMs
// busy.  The large-interface CPQR takes 16 in FP64, whose steps are bound by
// the FP64 pipe of the cluster's SMs, and 8 in FP32, where the per-step
// cluster barriers dominate (measured on 3D 32^3: FP64 151 -> 139 ms, FP32
// 64 -> 82 ms with 16).
template <class real>
constexpr int cpqr_cs() { return sizeof(real) == 8 ? 16 : 8; }
constexpr int64_t kBigCPQR = 1 << 17;   // n_p x ncols from which an interface uses a cluster
constexpr int QR_CS = 16;
constexpr int64_t kBigQR = 1 << 16;     // m x n from which a front uses a cluster
constexpr int kNumSM = 152;             // SMs of a GB300
constexpr int QAPPLY = 32;   // column chunk of one front-apply task
// CPQR reflectors: a pivot column's leading entry within this fraction of
// the column's norm counts as zero (beta = -norm).  M_p is assembled from
// sparse blocks, so that entry is often zero in exact arithmetic, and the
// tolerance keeps rounding from choosing the reflection.
constexpr double kCpqrSignTol = 1e-12;

template <class real>
__global__ void __launch_bounds__(NT) k_qr(const QRTask<real>* __restrict__ tasks, int prow) {
    extern __shared__ double sm[];
    const QRTask<real> t = tasks[blockIdx.x];
    const int tt = t.m < t.n ? t.m : t.n;
    cta_qr(t.A, t.lda, t.m, t.n, t.tau, t.T, tt, QC, prow, sm, t.sign_tol);
    if (t.Dinv) cta_tri_inv_blocks(t.A, t.lda, tt, t.Dinv, t.singular);
}

// Shared memory (bytes) of k_qr_cluster for panel slabs of `slab` rows.
__host__ __device__ constexpr size_t qrcl_smem_bytes(int esz, int slab) {
    return (size_t)8 * (NWARP + 2 * (2 + 2 * NB) + NB * NB + NT) +
           (size_t)esz * (NB + 2 * NB * QC + NT + (size_t)slab * NB);
}

// Cluster form of k_qr for large fronts.  Each panel of NB columns is
// factored by all CS CTAs together, the panel's rows p0..m-1 split into one
// slab per CTA (staged in its shared memory).  For column k every CTA sums,
// over its own rows below k, the squares of column k and its products with
// the panel's later columns; the owner of row k adds that row.  One cluster
// barrier later warp 0 of every CTA adds the CTAs' sums (a fixed tree over
// the ranks, read through distributed shared memory) and forms the same
// Householder scalars and the same
// w_j = tau (A(k, j) + sum_r A(r, k) A(r, j) / (alpha - beta)), the dot
// product of the reflector with column j; then every CTA updates its rows.
// The T block comes from the slabs' partial V^T V the same way.  The CS CTAs
// then apply the panel to their slices of the trailing columns (reflectors
// read from global memory).  Distributed-shared-memory slots alternate
// between two buffers by the parity of the cluster barrier count, so a slot
// is rewritten only two barriers after it was read.
template <class real, int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(NT)
    k_qr_cluster(const QRTask<real>* __restrict__ tasks, int prow) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double sm[];
    constexpr int SL = 2 + 2 * NB;                 // slot: norm, alpha, NB sums, NB entries of row k
    double* red = sm;                              // NWARP
    double* slot = red + NWARP;                    // 2 x SL
    double* Gp = slot + 2 * SL;                    // NB x NB partial V^T V
    double* Pd = Gp + NB * NB;                     // NT partial sums
    real* Wk = reinterpret_cast<real*>(Pd + NT);   // NB
    real* W = Wk + NB;                             // 2 NB QC + NT (trailing update)
    real* Ps = W + 2 * NB * QC + NT;               // slab x NB panel rows of this CTA
    (void)prow;
    const int q = (int)cl.block_rank();
    const QRTask<real> t = tasks[blockIdx.x / CS];
    const int m = t.m, n = t.n, tt = m < n ? m : n;
    real* A = t.A;
    const int64_t lda = t.lda;
    int ph = 0;
    for (int p0 = 0; p0 < tt; p0 += NB) {
        const int pe = (tt - p0 < NB ? tt : p0 + NB), pb = pe - p0;
        const int mr = m - p0, slab = (mr + CS - 1) / CS;
        const int lo = p0 + min(mr, q * slab), hi = p0 + min(mr, (q + 1) * slab), rows = hi - lo;
        for (int o = threadIdx.x; o < rows * pb; o += NT) {
            const int r = o % rows, jj = o / rows;
            Ps[r + jj * slab] = A[(lo + r) + (int64_t)(p0 + jj) * lda];
        }
        __syncthreads();
        for (int k = p0; k < pe; k++) {
            const int jk = k - p0, ncol = pe - k - 1;
            real* col = Ps + jk * slab - lo;   // col[r], r in [lo, hi)
            const bool own_k = k >= lo && k < hi;
            // thread (js, g): js = 0 the squared norm, js = 1 + jj the sum for column k + 1 + jj
            {
                const int js = threadIdx.x % NB, g = threadIdx.x / NB;
                double pd = 0.0;
                if (js <= ncol) {
                    const real* cj = Ps + (jk + js) * slab - lo;
                    for (int r = max(lo, k + 1) + g; r < hi; r += NT / NB) pd += (double)col[r] * (double)cj[r];
                }
                Pd[threadIdx.x] = pd;
            }
            __syncthreads();
            double* sl = slot + (ph & 1) * SL;
            if (threadIdx.x <= ncol) {
                // the NT / NB = 16 row-group partials of this column, added as a tree
                const double* pp = Pd + threadIdx.x;
                const double sacc = (((pp[0] + pp[NB]) + (pp[2 * NB] + pp[3 * NB])) +
                                     ((pp[4 * NB] + pp[5 * NB]) + (pp[6 * NB] + pp[7 * NB]))) +
                                    (((pp[8 * NB] + pp[9 * NB]) + (pp[10 * NB] + pp[11 * NB])) +
                                     ((pp[12 * NB] + pp[13 * NB]) + (pp[14 * NB] + pp[15 * NB])));
                sl[threadIdx.x == 0 ? 0 : 1 + threadIdx.x] = sacc;
            }
            if (threadIdx.x < NB) {
                // alpha = A(k, k) and row k's entries A(k, k + 1 + jj) from the owner of row k
                const int jj = threadIdx.x;
                sl[2 + NB + jj] = (own_k && jj < ncol) ? (double)Ps[(k - lo) + (jk + 1 + jj) * slab] : 0.0;
                if (jj == 0) sl[1] = own_k ? (double)col[k] : 0.0;
            }
            cl.sync();
            ph++;
            // the CTAs' sums added by warp 0 (a tree over the ranks, the same
            // in every CTA), the scalars by its lane 0, the w_j by lane j: FP64
            // work of one warp instead of every thread
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                double x2 = 0.0, alpha = 0.0;
                if (lane < CS) {
                    const double* o = cl.map_shared_rank(sl, lane);
                    x2 = o[0];
                    alpha = o[1];
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    x2 += __shfl_xor_sync(0xffffffffu, x2, off);
                    alpha += __shfl_xor_sync(0xffffffffu, alpha, off);
                }
                x2 = __shfl_sync(0xffffffffu, x2, 0);
                alpha = __shfl_sync(0xffffffffu, alpha, 0);
                double beta = alpha, denom = 1.0;
                if (x2 != 0.0) {
                    const double sq = sqrt(alpha * alpha + x2);
                    beta = alpha >= -t.sign_tol * sq ? -sq : sq;
                    denom = alpha - beta;
                }
                double u = 0.0;
                if (lane < ncol && x2 != 0.0) {
                    double sa[CS], ak[CS];
#pragma unroll
                    for (int rr = 0; rr < CS; rr++) {
                        const double* o = cl.map_shared_rank(sl, rr);
                        sa[rr] = o[2 + lane];
                        ak[rr] = o[2 + NB + lane];
                    }
#pragma unroll
                    for (int h = CS / 2; h > 0; h >>= 1)
#pragma unroll
                        for (int rr = 0; rr < h; rr++) {
                            sa[rr] += sa[rr + h];
                            ak[rr] += ak[rr + h];
                        }
                    u = ak[0] + sa[0] / denom;
                }
                const double tk = x2 != 0.0 ? (beta - alpha) / beta : 0.0;
                if (lane < ncol && tk != 0.0) Wk[lane] = (real)(tk * u);
                if (lane == 0) {
                    Pd[0] = tk;
                    Pd[1] = beta;
                    Pd[2] = denom;
                }
            }
            __syncthreads();
            const double tk = Pd[0], beta = Pd[1], denom = Pd[2];
            if (tk != 0.0) {
                if constexpr (sizeof(real) == 8) {
                    for (int r = max(lo, k + 1) + (int)threadIdx.x; r < hi; r += NT) col[r] = col[r] / denom;
                } else {
                    const real dn = (real)denom;
                    for (int r = max(lo, k + 1) + (int)threadIdx.x; r < hi; r += NT) col[r] /= dn;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0 && own_k) col[k] = (real)beta;
            if (threadIdx.x == 0 && q == 0) t.tau[k] = (real)tk;
            if (ncol > 0 && tk != 0.0) {
                const int r0 = max(lo, k), nr = hi - r0;
                for (int o = threadIdx.x; o < nr * ncol; o += NT) {
                    const int r = r0 + o % nr, jj = o / nr;
                    const real v = r == k ? (real)1 : col[r];
                    Ps[(r - lo) + (jk + 1 + jj) * slab] -= Wk[jj] * v;
                }
            }
            __syncthreads();
        }
        // the factored panel back to global memory, and the partial
        // G(i, j) = V(:, p0+i)^T V(:, p0+j), i < j, over own rows
        for (int o = threadIdx.x; o < rows * pb; o += NT) {
            const int r = o % rows, jj = o / rows;
            A[(lo + r) + (int64_t)(p0 + jj) * lda] = Ps[r + jj * slab];
        }
        for (int o = threadIdx.x; o < pb * pb; o += NT) {
            const int i = o % pb, jj = o / pb;
            double acc = 0.0;
            if (i < jj) {
                for (int r = max(lo, p0 + jj); r < hi; r++) {
                    const double vi = r == p0 + i ? 1.0 : (double)Ps[(r - lo) + i * slab];
                    const double vj = r == p0 + jj ? 1.0 : (double)Ps[(r - lo) + jj * slab];
                    acc += vi * vj;
                }
            }
            Gp[o] = acc;
        }
        cl.sync();
        ph++;
        if (q == 0) {
            // G summed over the ranks (a tree), then the T block
            real* Gs = reinterpret_cast<real*>(Pd);
            for (int o = threadIdx.x; o < pb * pb; o += NT) {
                if (o % pb >= o / pb) continue;   // strict upper part only
                double a[CS];
#pragma unroll
                for (int rr = 0; rr < CS; rr++) a[rr] = cl.map_shared_rank(Gp, rr)[o];
#pragma unroll
                for (int h = CS / 2; h > 0; h >>= 1)
#pragma unroll
                    for (int rr = 0; rr < h; rr++) a[rr] += a[rr + h];
                Gs[o] = (real)a[0];   // pb * pb <= NT
            }
            __syncthreads();
            cta_t_from_g(Gs, pb, t.tau + p0, t.T + p0 + (int64_t)p0 * tt, tt, pb, W);
        }
        cl.sync();   // panel, tau and T visible to the cluster; Gp read before it is rewritten
        ph++;
        if (pe < n) {
            const int w = (n - pe + CS - 1) / CS;
            const int c0 = pe + q * w, c1 = min(n, c0 + w);
            if (c1 > c0) {
                Mat<real> B{A + p0 + (int64_t)c0 * lda, 1, lda, nullptr};
                cta_apply_q_chunked(A + p0 + (int64_t)p0 * lda, lda, m - p0, pb, t.T + p0 + (int64_t)p0 * tt, tt,
                                    false, B, c1 - c0, QC, true, W);
            }
        }
        cl.sync();
        ph++;
    }
    if (q == 0 && t.Dinv) cta_tri_inv_blocks(A, lda, tt, t.Dinv, t.singular);
}

// smem layout: rmap (rmap_doubles doubles) then the work area of the apply
// (staged: staged_smem_elems(m, q); otherwise 2 * NB * q + NT elements).
template <class real>
__global__ void __launch_bounds__(NT) k_front_apply(const ApplyTask<real>* __restrict__ tasks,
                                                    const ApplyFront<real>* __restrict__ fronts,
                                                    const Seg* __restrict__ segs, int rmap_doubles, int staged) {
    extern __shared__ double sm[];
    int* rmap = reinterpret_cast<int*>(sm);
    real* W = reinterpret_cast<real*>(sm + rmap_doubles);
    const ApplyTask<real> t = tasks[blockIdx.x];
    for (int f = 0; f < t.nfr; f++) {
        const ApplyFront<real> F = fronts[t.fr_begin + f];
        // a segment per thread: its descriptor is one load, not one of a
        // chain of loads every thread would wait for in turn
        for (int s = threadIdx.x; s < F.nseg; s += NT) {
            const Seg g = segs[F.seg_begin + s];
            for (int r = 0; r < g.len; r++) rmap[g.pos + r] = (int)(g.off + r);
        }
        __syncthreads();
        const Mat<real> B{t.B, 1, t.ldb, rmap};
        if (staged) cta_apply_q_staged(F.V, F.ldv, F.m, F.n, F.T, F.n, false, B, t.q, true, W);
        else cta_apply_q(F.V, F.ldv, F.m, F.n, F.T, F.n, false, B, t.q, true, W);
    }
}

// ---------------------------------------------------------------------------
// Tensor-core application of a level's fronts (FP32 storage).  A front's
// rows R(s) of its columns C(s) \ {s} are copied into one dense m x w matrix
// B, and Q_s^T B = B - V T^T (V^T B) is formed by products on the tensor
// cores (tcgemm.h) with the full n x n compact-WY factor T of the front's n
// reflectors (Section 2.4's block Householder step); T comes from
// G = V^T V and tau.  Fronts of one colour share no row cluster, so their
// copies are disjoint; the colours run in order.
// ---------------------------------------------------------------------------

// One column panel j of a front: rows R(s) of the panel <-> the panel's
// columns in the front's dense copy.
struct FrontCopy {
    float* panel;     // first column of panel j (column-major, ld)
    int64_t ld;
    float* dense;     // first of its columns in the dense copy (ld m)
    int m, ncol;
    int seg_begin, nseg;   // row segments R(s) in panel j, in front row order
};

constexpr int kCopyCols = 8;   // columns of one k_front_copy CTA

// to_dense = 1: panel -> dense copy; 0: dense copy -> panel.  CTA
// (x, y) copies columns [8 y, 8 y + 8) of (front, panel) pair x; smem: the
// front's row map (m ints).
__global__ void __launch_bounds__(NT) k_front_copy(const FrontCopy* __restrict__ tasks, const Seg* __restrict__ segs,
                                                   int to_dense) {
    extern __shared__ int rmap_sm[];
    const FrontCopy c = tasks[blockIdx.x];
    const int c0 = (int)blockIdx.y * kCopyCols;
    if (c0 >= c.ncol) return;
    const int c1 = min(c.ncol, c0 + kCopyCols);
    for (int s = threadIdx.x; s < c.nseg; s += NT) {   // a segment per thread
        const Seg g = segs[c.seg_begin + s];
        for (int r = 0; r < g.len; r++) rmap_sm[g.pos + r] = (int)(g.off + r);
    }
    __syncthreads();
    for (int col = c0; col < c1; col++) {
        float* p = c.panel + (int64_t)col * c.ld;
        float* d = c.dense + (int64_t)col * c.m;
        if (to_dense)
            for (int r = threadIdx.x; r < c.m; r += NT) d[r] = p[rmap_sm[r]];
        else
            for (int r = threadIdx.x; r < c.m; r += NT) p[rmap_sm[r]] = d[r];
    }
}

struct TfullTask {
    const float* G;     // n x n, G = V^T V (ld n)
    const float* tau;   // n
    float* T;           // out: n x n upper triangular (ld n), zeros below
    float* X;           // scratch n x 16
    int n;
};

// Full compact-WY factor of a front's reflectors, Q = I - V T V^T, by blocks
// of 16 columns: the diagonal block by the column recurrence
// T(0:k, k) = -tau_k T(0:k, 0:k) G(0:k, k), the rows above it by
// T_12 = -T_11 G_12 T_22 (the product of two block reflectors).  One CTA per
// front, FP32.
__global__ void __launch_bounds__(NT) k_tfull(const TfullTask* __restrict__ tasks) {
    const TfullTask t = tasks[blockIdx.x];
    const int n = t.n;
    const float* G = t.G;
    float* T = t.T;
    for (int64_t o = threadIdx.x; o < (int64_t)n * n; o += NT) {
        const int r = (int)(o % n), c = (int)(o / n);
        if (r > c) T[o] = 0.0f;
    }
    for (int c0 = 0; c0 < n; c0 += NB) {
        const int cb = n - c0 < NB ? n - c0 : NB;
        for (int k = 0; k < cb; k++) {
            const float tk = t.tau[c0 + k];
            for (int i = threadIdx.x; i < k; i += NT) {
                float s = 0.0f;
                for (int u = i; u < k; u++) s += T[(c0 + i) + (int64_t)(c0 + u) * n] * G[(c0 + u) + (int64_t)(c0 + k) * n];
                T[(c0 + i) + (int64_t)(c0 + k) * n] = -tk * s;
            }
            if (threadIdx.x == 0) T[(c0 + k) + (int64_t)(c0 + k) * n] = tk;
            __syncthreads();
        }
        if (c0 == 0) continue;
        for (int o = threadIdx.x; o < c0 * cb; o += NT) {
            const int i = o % c0, j = o / c0;
            float s = 0.0f;
            for (int u = i; u < c0; u++) s += T[i + (int64_t)u * n] * G[u + (int64_t)(c0 + j) * n];
            t.X[i + (int64_t)j * c0] = s;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < c0 * cb; o += NT) {
            const int i = o % c0, j = o / c0;
            float s = 0.0f;
            for (int l = 0; l <= j; l++) s += t.X[i + (int64_t)l * c0] * T[(c0 + l) + (int64_t)(c0 + j) * n];
            T[i + (int64_t)(c0 + j) * n] = -s;
        }
        __syncthreads();
    }
}

template <class real>
__global__ void __launch_bounds__(NT) k_scale_apply(const ScaleTask<real>* __restrict__ tasks,
                                                    const ScalePiece* __restrict__ pieces, int right) {
    extern __shared__ double sm[];
    real* W = reinterpret_cast<real*>(sm);
    const ScalePiece pc = pieces[blockIdx.x];
    const ScaleTask<real> t = tasks[pc.task];
    if (!right) {
        // rows i <- U_i^T (rows i): columns [off, off + len) of the block
        cta_apply_q_chunked(t.Vi, t.ldvi, t.mi, t.mi, t.Ti, t.mi, false,
                            Mat<real>{t.A + (int64_t)pc.off * t.lda, 1, t.lda, nullptr}, pc.len, QC, true, W);
    } else {
        // columns j <- (columns j) R_j^{-1}: rows [off, off + len) of the block
        cta_trsm_right_upper(t.A + pc.off, t.lda, pc.len, t.nj, t.Rj, t.ldrj, t.Dj);
    }
}

// One column of the CPQR trailing update: a_j <- (I - tau v v^T) a_j over
// rows k.. (v_k = 1, v_r = vs[r] below), returning the new squared norm of
// rows k+1.. (the next step's pivot norm).  Column entries are row-major
// with stride ld.  Rows are loaded sixteen at a time before they are used,
// so a thread keeps sixteen loads in flight; the additions keep the row order.
template <class real>
__device__ __forceinline__ real cpqr_reflect_column(real* a, int ld, int k, int m, const real* vs, real tk) {
    constexpr int U = 16;
    real d = a[(int64_t)k * ld];
    int r = k + 1;
    for (; r + U <= m; r += U) {
        real x[U];
#pragma unroll
        for (int u = 0; u < U; u++) x[u] = a[(int64_t)(r + u) * ld];
#pragma unroll
        for (int u = 0; u < U; u++) d += vs[r + u] * x[u];
    }
    for (; r < m; r++) d += vs[r] * a[(int64_t)r * ld];
    const real f = tk * d;
    a[(int64_t)k * ld] -= f;
    real nrm = 0;
    r = k + 1;
    for (; r + U <= m; r += U) {
        real x[U];
#pragma unroll
        for (int u = 0; u < U; u++) x[u] = a[(int64_t)(r + u) * ld];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const real y = x[u] - f * vs[r + u];
            a[(int64_t)(r + u) * ld] = y;
            nrm += y * y;
        }
    }
    for (; r < m; r++) {
        const real y = a[(int64_t)r * ld] - f * vs[r];
        a[(int64_t)r * ld] = y;
        nrm += y * y;
    }
    return nrm;
}

// Truncated CPQR of M_p (stored row-major) with column norms recomputed from
// scratch at every step (fused into the reflector update, one thread per
// column), pivot = largest norm, ties to the lowest column index; stops at the
// first |R_kk| < eps |R_11|.  The rank decision is taken in FP64: in the FP64
// form |R_kk| is the pivot's recomputed norm; in the mixed form the norms that
// choose the pivot are FP32 and |R_kk| is recomputed in FP64 from the pivot
// column.
template <class real>
__global__ void __launch_bounds__(NT) k_cpqr(const CPQRTask<real>* __restrict__ tasks,
                                             const GatherSeg<real>* __restrict__ gsegs, double eps) {
    extern __shared__ double sm[];
    double* red = sm;                                                // RED
    long long* redv = reinterpret_cast<long long*>(sm + RED);        // NWARP
    int* redi = reinterpret_cast<int*>(sm + RED + NWARP);            // NWARP ints
    real* G = reinterpret_cast<real*>(sm + RED + 2 * NWARP);         // NB * NB
    real* X = G + NB * NB;                                           // NB * NB / 2
    real* vs = X + NB * NB / 2;                                      // n_p
    const CPQRTask<real> t = tasks[blockIdx.x];
    const int m = t.np, c = t.ncols;
    real* M = t.M;  // M(r, j) = M[r * c + j]
    for (int s = 0; s < t.nseg; s++) {
        const GatherSeg<real> g = gsegs[t.seg_begin + s];
        const int64_t tot = (int64_t)g.rows * g.cols;
        if (g.transpose) {
            // M(r, col_off + cc) = src[cc + r * ld], r < n_p (= cols), cc < rows
            for (int64_t o = threadIdx.x; o < tot; o += NT) {
                const int cc = (int)(o % g.rows), r = (int)(o / g.rows);
                M[(int64_t)r * c + g.col_off + cc] = g.src[cc + (int64_t)r * g.ld];
            }
        } else {
            for (int64_t o = threadIdx.x; o < tot; o += NT) {
                const int r = (int)(o % g.rows), cc = (int)(o / g.rows);
                M[(int64_t)r * c + g.col_off + cc] = g.src[r + (int64_t)cc * g.ld];
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < c; j += NT) {
        real s = 0;
        for (int r = 0; r < m; r++) {
            const real x = M[(int64_t)r * c + j];
            s += x * x;
        }
        t.norms[j] = s;
    }
    __syncthreads();
    const int tmax = m < c ? m : c;
    int rank = 0;
    double R11 = 0.0;
    __shared__ int s_stop;
    for (int k = 0; k < tmax; k++) {
        // pivot: largest norm, ties to the lowest column (integer keys)
        long long bk = -1;
        int bi = 0x7fffffff;
        for (int j = k + threadIdx.x; j < c; j += NT) {
            const long long key = nonneg_key(t.norms[j]);
            if (key > bk || (key == bk && j < bi)) { bk = key; bi = j; }
        }
        long long gk;
        int gi;
        block_argmax_key(bk, bi, redv, redi, gk, gi);
        double gv = 0.0;
        if constexpr (sizeof(real) == 8) {
            gv = __longlong_as_double(gk);
        } else {
            // |R_kk| in FP64 from the pivot column (rows k..m-1)
            double part = 0.0;
            for (int r = k + threadIdx.x; r < m; r += NT) {
                const double x = (double)M[(int64_t)r * c + gi];
                part += x * x;
            }
            gv = block_sum(part, red);
        }
        // the rank decision by one thread (FP64), shared with the CTA
        if (threadIdx.x == 0) {
            const double pn = sqrt(gv);
            t.rdiag[k] = pn;
            if (k == 0) R11 = pn;
            s_stop = (R11 == 0.0) || (pn < eps * R11);
        }
        __syncthreads();
        if (s_stop) break;
        if (gi != k) {
            for (int r = threadIdx.x; r < m; r += NT) {
                real* row = M + (int64_t)r * c;
                const real x = row[k];
                row[k] = row[gi];
                row[gi] = x;
            }
            __syncthreads();
            if (threadIdx.x == 0) t.norms[gi] = t.norms[k];
        }
        __syncthreads();
        const double tkd = cta_house(M + k, c, k, m, red, kCpqrSignTol);
        const real tk = (real)tkd;
        if (threadIdx.x == 0) t.tau[k] = tk;
        for (int r = k + 1 + threadIdx.x; r < m; r += NT) vs[r] = M[(int64_t)r * c + k];
        __syncthreads();
        for (int j = k + 1 + threadIdx.x; j < c; j += NT) {
            t.norms[j] = cpqr_reflect_column(M + j, c, k, m, vs, tk);
        }
        __syncthreads();
        rank = k + 1;
    }
    // explicit reflectors V (n_p x rank, column-major), unit diagonal, zeros above
    for (int64_t o = threadIdx.x; o < (int64_t)m * rank; o += NT) {
        const int r = (int)(o % m), i = (int)(o / m);
        t.V[r + (int64_t)i * m] = r < i ? (real)0 : (r == i ? (real)1 : M[(int64_t)r * c + i]);
    }
    if (threadIdx.x == 0) *t.rank = rank;
    __syncthreads();
    cta_form_tblocks(t.V, m, m, rank, t.tau, t.T, t.kmax, G, X);
}

// Cluster form of k_cpqr for large interfaces: the CS CTAs of a thread-block
// cluster share one M_p.  CTA q owns the columns [q cw, (q+1) cw); each step
// combines the CTAs' pivot candidates through distributed shared memory, the
// owner of column k swaps, forms the reflector and publishes it through
// global memory, and every CTA reflects its own columns.  Per column the
// arithmetic is that of k_cpqr, so ranks and reflectors are identical.
template <class real, int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(NT)
    k_cpqr_cluster(const CPQRTask<real>* __restrict__ tasks, const GatherSeg<real>* __restrict__ gsegs, double eps) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double sm[];
    double* red = sm;                                                // RED
    long long* redv = reinterpret_cast<long long*>(sm + RED);        // NWARP
    int* redi = reinterpret_cast<int*>(sm + RED + NWARP);            // NWARP ints
    real* G = reinterpret_cast<real*>(sm + RED + 2 * NWARP);         // NB * NB
    real* X = G + NB * NB;                                           // NB * NB / 2
    real* vs = X + NB * NB / 2;                                      // n_p
    __shared__ long long slot_k;
    __shared__ double slot_n;
    __shared__ int slot_i, s_gi, s_stop;
    const int q = (int)cl.block_rank();
    const CPQRTask<real> t = tasks[blockIdx.x / CS];
    const int m = t.np, c = t.ncols;
    const int cw = (c + CS - 1) / CS;
    const int j0 = q * cw, j1 = min(c, j0 + cw);
    real* M = t.M;  // M(r, j) = M[r * c + j]
    // gather, elements split over the cluster's CTAs
    const int gt = q * NT + threadIdx.x, gstride = CS * NT;
    for (int s = 0; s < t.nseg; s++) {
        const GatherSeg<real> g = gsegs[t.seg_begin + s];
        const int64_t tot = (int64_t)g.rows * g.cols;
        if (g.transpose) {
            for (int64_t o = gt; o < tot; o += gstride) {
                const int cc = (int)(o % g.rows), r = (int)(o / g.rows);
                M[(int64_t)r * c + g.col_off + cc] = g.src[cc + (int64_t)r * g.ld];
            }
        } else {
            for (int64_t o = gt; o < tot; o += gstride) {
                const int r = (int)(o % g.rows), cc = (int)(o / g.rows);
                M[(int64_t)r * c + g.col_off + cc] = g.src[r + (int64_t)cc * g.ld];
            }
        }
    }
    cl.sync();
    for (int j = j0 + threadIdx.x; j < j1; j += NT) {
        real s = 0;
        for (int r = 0; r < m; r++) {
            const real x = M[(int64_t)r * c + j];
            s += x * x;
        }
        t.norms[j] = s;
    }
    __syncthreads();
    const int tmax = m < c ? m : c;
    int rank = 0;
    double R11 = 0.0;
    for (int k = 0; k < tmax; k++) {
        // pivot candidate of this CTA, then of the cluster (integer keys)
        long long bk = -1;
        int bi = 0x7fffffff;
        for (int j = max(k, j0) + threadIdx.x; j < j1; j += NT) {
            const long long key = nonneg_key(t.norms[j]);
            if (key > bk || (key == bk && j < bi)) { bk = key; bi = j; }
        }
        long long lk;
        int li;
        block_argmax_key(bk, bi, redv, redi, lk, li);
        // FP64 |R_kk|^2 of this CTA's candidate, published with it (computed
        // before any CTA may swap columns)
        double ln2 = 0.0;
        if constexpr (sizeof(real) == 8) {
            if (lk >= 0) ln2 = __longlong_as_double(lk);
        } else {
            double part = 0.0;
            if (li < c)
                for (int r = k + threadIdx.x; r < m; r += NT) {
                    const double x = (double)M[(int64_t)r * c + li];
                    part += x * x;
                }
            ln2 = block_sum(part, red);
        }
        if (threadIdx.x == 0) { slot_k = lk; slot_i = li; slot_n = ln2; }
        cl.sync();
        // the cluster's pivot and the rank decision by one thread per CTA
        // (every CTA reaches the same result)
        if (threadIdx.x == 0) {
            long long ks[CS];
            int is[CS];
#pragma unroll
            for (int r = 0; r < CS; r++) {   // all loads in flight, then the compares
                ks[r] = *cl.map_shared_rank(&slot_k, r);
                is[r] = *cl.map_shared_rank(&slot_i, r);
            }
            long long gk = -1;
            int gi = 0x7fffffff, gr = 0;
#pragma unroll
            for (int r = 0; r < CS; r++)
                if (ks[r] > gk || (ks[r] == gk && is[r] < gi)) { gk = ks[r]; gi = is[r]; gr = r; }
            const double gn = *cl.map_shared_rank(&slot_n, gr);
            const double pn = sqrt(gn);
            if (q == 0) t.rdiag[k] = pn;
            if (k == 0) R11 = pn;
            s_gi = gi;
            s_stop = (R11 == 0.0) || (pn < eps * R11);
        }
        __syncthreads();
        const int gi = s_gi;
        const bool stop = s_stop != 0;
        const int owner = k / cw;
        if (!stop && q == owner && gi != k) {
            for (int r = threadIdx.x; r < m; r += NT) {
                real* row = M + (int64_t)r * c;
                const real x = row[k];
                row[k] = row[gi];
                row[gi] = x;
            }
            __syncthreads();
            if (threadIdx.x == 0) t.norms[gi] = t.norms[k];
        }
        // every CTA has read the slots and sees the swap before they change
        cl.sync();
        if (stop) break;
        if (q == owner) {
            const double tkd = cta_house(M + k, c, k, m, red, kCpqrSignTol);
            if (threadIdx.x == 0) t.tau[k] = (real)tkd;
        }
        cl.sync();
        const real tk = t.tau[k];
        for (int r = k + 1 + threadIdx.x; r < m; r += NT) vs[r] = M[(int64_t)r * c + k];
        __syncthreads();
        for (int j = max(k + 1, j0) + threadIdx.x; j < j1; j += NT) {
            t.norms[j] = cpqr_reflect_column(M + j, c, k, m, vs, tk);
        }
        __syncthreads();
        rank = k + 1;
    }
    // explicit reflectors V (n_p x rank), split over the cluster
    for (int64_t o = gt; o < (int64_t)m * rank; o += gstride) {
        const int r = (int)(o % m), i = (int)(o / m);
        t.V[r + (int64_t)i * m] = r < i ? (real)0 : (r == i ? (real)1 : M[(int64_t)r * c + i]);
    }
    cl.sync();
    if (q == 0) {
        if (threadIdx.x == 0) *t.rank = rank;
        cta_form_tblocks(t.V, m, m, rank, t.tau, t.T, t.kmax, G, X);
    }
}

// Coarse block [Q_i^T A Q_j](0:r_i, 0:r_j) into the merged block of the next
// level; identity for diagonal blocks; plain copy when not sparsified.
template <class real>
__global__ void __launch_bounds__(NT) k_sparsify(const SparsifyTask<real>* __restrict__ tasks,
                                                 const ScalePiece* __restrict__ pieces, int right) {
    extern __shared__ double sm[];
    real* W = reinterpret_cast<real*>(sm);
    const ScalePiece pc = pieces[blockIdx.x];
    const SparsifyTask<real> t = tasks[pc.task];
    if (t.mode == 2) {
        const int64_t tot = (int64_t)t.mi * t.nj;
        for (int64_t o = threadIdx.x; o < tot; o += NT) {
            const int r = (int)(o % t.mi), c = (int)(o / t.mi);
            t.D[r + (int64_t)c * t.ldd] = t.A[r + (int64_t)c * t.lda];
        }
        return;
    }
    if (t.mode == 1) {
        for (int i = threadIdx.x; i < t.ri; i += NT) t.D[i + (int64_t)i * t.ldd] = (real)1;
        return;
    }
    const int mi = t.mi, nj = t.nj;
    real* X = t.scratch;  // mi x nj, ld mi
    if (!right) {
        // columns [off, off + len): X <- Q_i^T A
        const int c0 = pc.off, qn = pc.len;
        for (int64_t o = threadIdx.x; o < (int64_t)mi * qn; o += NT) {
            const int r = (int)(o % mi), c = c0 + (int)(o / mi);
            X[r + (int64_t)c * mi] = t.A[r + (int64_t)c * t.lda];
        }
        __syncthreads();
        if (t.li > 0)
            cta_apply_q_chunked(t.Vi, mi, mi, t.li, t.Ti, t.ldti, t.lexp != 0,
                                Mat<real>{X + (int64_t)c0 * mi, 1, mi, nullptr}, qn, QC, true, W);
        return;
    }
    // kept rows lkeep + [off, off + len): X <- X Q_j, i.e. X^T <- Q_j^T X^T
    // with X^T(r, c) = X[c + r * mi]; then the r_i x r_j coarse block
    const int r0 = pc.off, rn = pc.len;
    real* Xk = X + t.lkeep;
    cta_apply_q_chunked(t.Vj, nj, nj, t.rj, t.Tj, t.ldtj, true, Mat<real>{Xk + r0, mi, 1, nullptr}, rn, QC, true, W);
    for (int64_t o = threadIdx.x; o < (int64_t)rn * t.rj; o += NT) {
        const int p = r0 + (int)(o % rn), q = (int)(o / rn);
        t.D[p + (int64_t)q * t.ldd] = Xk[p + (int64_t)q * mi];
    }
}

// Merge of a level below the sparsified ones: one CTA per column chunk
// copies its row segments into the merged panel (one task per chunk instead
// of one per block keeps the host's planning of the many small blocks of the
// lower levels short).
template <class real>
__global__ void __launch_bounds__(NT) k_merge_copy(const CopyCol<real>* __restrict__ cols,
                                                   const RowSeg* __restrict__ segs) {
    const CopyCol<real> t = cols[blockIdx.x];
    for (int s = 0; s < t.nseg; s++) {
        const RowSeg g = segs[t.seg_begin + s];
        const int64_t tot = (int64_t)g.len * t.ncols;
        for (int64_t o = threadIdx.x; o < tot; o += NT) {
            const int r = (int)(o % g.len), c = (int)(o / g.len);
            t.D[(g.dst + r) + (int64_t)c * t.ldd] = t.A[(g.src + r) + (int64_t)c * t.lda];
        }
    }
}

// B <- Q^T B over a column chunk, or B <- B Q over a row chunk (Q^T applied
// to the transposed view).
template <class real>
__global__ void __launch_bounds__(NT) k_refl_apply(const ReflTask<real>* __restrict__ tasks,
                                                   const ScalePiece* __restrict__ pieces) {
    extern __shared__ double sm[];
    real* W = reinterpret_cast<real*>(sm);
    const ScalePiece pc = pieces[blockIdx.x];
    const ReflTask<real> t = tasks[pc.task];
    const Mat<real> B = t.right ? Mat<real>{t.B + pc.off, t.ldb, 1, nullptr}
                                : Mat<real>{t.B + (int64_t)pc.off * t.ldb, 1, t.ldb, nullptr};
    cta_apply_q_chunked(t.V, t.ldv, t.m, t.t, t.T, t.ldt, t.vexp != 0, B, pc.len, QC, true, W);
}

// C = sigma_p (A_pp^T A_pj) over a column chunk of A_pj (the second part of
// the unscaled M_p, Section 3.2): one output per thread, its dot product one
// sequential chain.
template <class real>
__global__ void __launch_bounds__(NT) k_atb_sigma(const AtbTask<real>* __restrict__ tasks,
                                                  const ScalePiece* __restrict__ pieces) {
    const ScalePiece pc = pieces[blockIdx.x];
    const AtbTask<real> t = tasks[pc.task];
    const double sg = *t.sigma;
    const int n = t.n;
    for (int o = threadIdx.x; o < n * pc.len; o += NT) {
        const int r = o % n, c = pc.off + o / n;
        const real* a = t.A + (int64_t)r * t.lda;
        const real* b = t.B + (int64_t)c * t.ldb;
        real acc = 0;
        for (int u = 0; u < n; u++) acc += a[u] * b[u];
        t.C[r + (int64_t)c * n] = (real)(sg * (double)acc);
    }
}

// ---------------------------------------------------------------------------
// sigma_p = 1 / sigma_min(A_p) (Lemma 1) from the triangular factor R of A_p:
// sigma_p^2 is the largest eigenvalue of (R^T R)^{-1}.  Lanczos on that
// operator (two triangular solves per step) with full reorthogonalisation
// (classical Gram-Schmidt, two passes), from a fixed hashed start vector.
// Every fourth step the largest eigenvalue of the Lanczos tridiagonal is
// found by multisection (32 points per round on one warp, Sturm counts) to
// the last bits, and the iteration stops once it grew by at most 1e-15
// relative over those four steps, at an invariant subspace, or after kmax
// steps.  All of it in FP64; one CTA per interface.
// ---------------------------------------------------------------------------
constexpr int kLanczosMax = 160;

// Eigenvalues of the k x k symmetric tridiagonal (diagonal a, squared
// off-diagonal b2) below x: negative pivots of the LDL^T of T - x I.
__device__ __forceinline__ int sturm_below(const double* a, const double* b2, int k, double x) {
    int c = 0;
    double q = a[0] - x;
    c += q < 0.0;
    for (int i = 1; i < k; i++) {
        const double qq = q != 0.0 ? q : 1e-300;
        q = a[i] - x - b2[i - 1] / qq;
        c += q < 0.0;
    }
    return c;
}

__device__ __forceinline__ double warp_max_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Largest eigenvalue in [lo, hi] (lo below it, hi above it); warp 0 only.
__device__ double warp_top_eig(const double* a, const double* b2, int k, double lo, double hi) {
    const int lane = threadIdx.x & 31;
    for (int it = 0; it < 20 && hi - lo > 2.3e-16 * hi; it++) {
        const double x = lo + (hi - lo) * (double)(lane + 1) * (1.0 / 33.0);
        const unsigned m = __ballot_sync(0xffffffffu, sturm_below(a, b2, k, x) == k);
        const double xf = __shfl_sync(0xffffffffu, x, m ? __ffs(m) - 1 : 31);
        const double xp = __shfl_sync(0xffffffffu, x, m ? (__ffs(m) > 1 ? __ffs(m) - 2 : 0) : 31);
        if (!m) lo = xf;
        else {
            hi = xf;
            if (__ffs(m) > 1) lo = xp;
        }
    }
    return 0.5 * (lo + hi);
}

// w <- R^{-T} w (R upper n x n, ld; idg = 1 / diag R), blocks of 32: warp 0
// solves the diagonal block, every thread updates the rows below it.
template <class real>
__device__ void lanczos_solve_rt(const real* R, int64_t ld, int n, const double* idg, double* w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b0 = 0; b0 < n; b0 += 32) {
        const int bs = n - b0 < 32 ? n - b0 : 32;
        if (warp == 0) {
            double x = lane < bs ? w[b0 + lane] : 0.0;
            for (int k = 0; k < bs; k++) {
                const double xk = __shfl_sync(0xffffffffu, x, k) * idg[b0 + k];
                if (lane == k) x = xk;
                else if (lane > k && lane < bs) x -= (double)R[(b0 + k) + (int64_t)(b0 + lane) * ld] * xk;
            }
            if (lane < bs) w[b0 + lane] = x;
        }
        __syncthreads();
        for (int i = b0 + bs + threadIdx.x; i < n; i += NT) {
            const real* col = R + b0 + (int64_t)i * ld;
            double s = 0.0;
            for (int k = 0; k < bs; k++) s += (double)col[k] * w[b0 + k];
            w[i] -= s;
        }
        __syncthreads();
    }
}

// w <- R^{-1} w, same blocking from the bottom block up.
template <class real>
__device__ void lanczos_solve_r(const real* R, int64_t ld, int n, const double* idg, double* w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b0 = ((n - 1) / 32) * 32; b0 >= 0; b0 -= 32) {
        const int bs = n - b0 < 32 ? n - b0 : 32;
        if (warp == 0) {
            double x = lane < bs ? w[b0 + lane] : 0.0;
            for (int k = bs - 1; k >= 0; k--) {
                const double xk = __shfl_sync(0xffffffffu, x, k) * idg[b0 + k];
                if (lane == k) x = xk;
                else if (lane < k) x -= (double)R[(b0 + lane) + (int64_t)(b0 + k) * ld] * xk;
            }
            if (lane < bs) w[b0 + lane] = x;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < b0; i += NT) {
            double s = 0.0;
            for (int k = 0; k < bs; k++) s += (double)R[i + (int64_t)(b0 + k) * ld] * w[b0 + k];
            w[i] -= s;
        }
        __syncthreads();
    }
}

template <class real>
__global__ void __launch_bounds__(NT) k_sigma_min(const SigmaTask<real>* __restrict__ tasks) {
    __shared__ double alpha[kLanczosMax], beta2[kLanczosMax], hc[kLanczosMax];
    __shared__ double red[RED];
    __shared__ double theta_sh;
    __shared__ int bad;
    const SigmaTask<real> t = tasks[blockIdx.x];
    const int n = t.n, kmax = t.kmax;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* Vl = t.work;                         // Lanczos vectors, vector j at Vl + j n
    double* w = t.work + (int64_t)(kmax + 1) * n;
    double* idg = w + n;
    const real* R = t.R;
    const int64_t ld = t.ldr;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += NT) {
        const double d = (double)R[i + (int64_t)i * ld];
        if (d == 0.0) bad = 1;
        idg[i] = d != 0.0 ? 1.0 / d : 0.0;
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) {
            *t.singular = 1;
            *t.sigma = 0.0;
        }
        return;
    }
    // start vector: hashed entries in [0.5, 1.5), normalised
    double part = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) {
        const unsigned h = (unsigned)(i + 1) * 2654435761u;
        const double v = 0.5 + (double)(h >> 8) * (1.0 / 16777216.0);
        Vl[i] = v;
        part += v * v;
    }
    const double nrm = sqrt(block_sum(part, red));
    for (int i = threadIdx.x; i < n; i += NT) Vl[i] /= nrm;
    __syncthreads();
    double theta = 0.0;
    for (int j = 0; j < kmax; j++) {
        const double* v = Vl + (int64_t)j * n;
        for (int i = threadIdx.x; i < n; i += NT) w[i] = v[i];
        __syncthreads();
        lanczos_solve_rt(R, ld, n, idg, w);
        lanczos_solve_r(R, ld, n, idg, w);
        part = 0.0;
        for (int i = threadIdx.x; i < n; i += NT) part += w[i] * v[i];
        const double a = block_sum(part, red);
        const double bp = j > 0 ? sqrt(beta2[j - 1]) : 0.0;
        for (int i = threadIdx.x; i < n; i += NT) {
            double x = w[i] - a * v[i];
            if (j > 0) x -= bp * Vl[(int64_t)(j - 1) * n + i];
            w[i] = x;
        }
        if (threadIdx.x == 0) alpha[j] = a;
        __syncthreads();
        for (int pass = 0; pass < 2; pass++) {
            for (int q = warp; q <= j; q += NWARP) {
                const double* vq = Vl + (int64_t)q * n;
                double s = 0.0;
                for (int i = lane; i < n; i += 32) s += vq[i] * w[i];
                s = warp_sum(s);
                if (lane == 0) hc[q] = s;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += NT) {
                double x = w[i];
                for (int q = 0; q <= j; q++) x -= hc[q] * Vl[(int64_t)q * n + i];
                w[i] = x;
            }
            __syncthreads();
        }
        part = 0.0;
        for (int i = threadIdx.x; i < n; i += NT) part += w[i] * w[i];
        const double b2 = block_sum(part, red);
        if (threadIdx.x == 0) beta2[j] = b2;
        const int k = j + 1;
        const bool last = k == kmax || !(sqrt(b2) > 1e-15 * fmax(fabs(a), theta));
        if (last || (k & 3) == 0) {
            __syncthreads();
            if (warp == 0) {
                double lo = theta, hi = 0.0;
                for (int i = lane; i < k; i += 32) {
                    const double bl = i > 0 ? sqrt(beta2[i - 1]) : 0.0, br = i + 1 < k ? sqrt(beta2[i]) : 0.0;
                    lo = fmax(lo, alpha[i]);
                    hi = fmax(hi, alpha[i] + bl + br);
                }
                lo = warp_max_d(lo);
                hi = warp_max_d(hi) * (1.0 + 1e-13);
                if (lo > hi) lo = hi;
                const double th = warp_top_eig(alpha, beta2, k, lo, hi);
                if (lane == 0) theta_sh = th;
            }
            __syncthreads();
            const double th_old = theta;
            theta = theta_sh;
            if (last || (k >= 8 && theta - th_old <= 1e-15 * theta)) break;
        }
        const double b = sqrt(b2);
        double* vn = Vl + (int64_t)(j + 1) * n;
        for (int i = threadIdx.x; i < n; i += NT) vn[i] = w[i] / b;
        __syncthreads();
    }
    if (threadIdx.x == 0) *t.sigma = sqrt(theta);
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------

namespace {

// Pinned host staging for the task arrays a factorisation uploads (copies
// from pageable memory are synchronous staging copies).  One buffer per host
// thread, reused by the thread's next factorisation, which starts after this
// one has synchronised its stream; it grows between calls to the largest
// total seen.
struct PinnedStage {
    char* p = nullptr;
    size_t cap = 0, want = 0;
    void grow() {
        if (want <= cap) return;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        const size_t bytes = want + want / 4;
        if (cudaHostAlloc(reinterpret_cast<void**>(&p), bytes, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return;
        }
        cap = bytes;
    }
    ~PinnedStage() {
        if (p) cudaFreeHost(p);
    }
};
thread_local PinnedStage tl_stage;

struct Ctx {
    spaqr_factor_s* F;
    cudaStream_t st;
    std::vector<std::pair<void*, size_t>> temps;
    std::vector<std::pair<void*, size_t>> kept_bytes;
    int64_t live = 0;   // bytes allocated by this factorisation and not yet given back
    int rc = SPAQR_OK;
    size_t stage_off = 0, stage_total = 0;

    template <class T>
    T* alloc(int64_t count, bool keep) {
        if (rc != SPAQR_OK) return nullptr;
        void* p = nullptr;
        size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
        bytes = (bytes + 255) & ~(size_t)255;
        if (fail_this_alloc() || cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            set_error("device allocation of " + std::to_string(bytes) + " bytes failed");
            rc = SPAQR_ERR_OOM;
            return nullptr;
        }
        if (keep) {
            F->allocs.push_back(p);
            F->bytes += (int64_t)bytes;
            kept_bytes.push_back({p, bytes});
        } else {
            temps.push_back({p, bytes});
        }
        live += (int64_t)bytes;
        F->peak_bytes = std::max(F->peak_bytes, live);
        return (T*)p;
    }
    template <class T>
    T* upload(const std::vector<T>& h, bool keep) {
        T* d = alloc<T>((int64_t)h.size(), keep);
        if (!d || h.empty()) return d;
        const size_t bytes = sizeof(T) * h.size(), rounded = (bytes + 255) & ~(size_t)255;
        stage_total += rounded;
        tl_stage.want = std::max(tl_stage.want, stage_total);
        if (stage_off + rounded <= tl_stage.cap) {
            std::memcpy(tl_stage.p + stage_off, h.data(), bytes);
            cuda(cudaMemcpyAsync(d, tl_stage.p + stage_off, bytes, cudaMemcpyHostToDevice, st));
            stage_off += rounded;
        } else {
            cuda(cudaMemcpyAsync(d, h.data(), bytes, cudaMemcpyHostToDevice, st));
        }
        return d;
    }
    void cuda(cudaError_t e) {
        if (e != cudaSuccess && rc == SPAQR_OK) {
            set_error(std::string("CUDA: ") + cudaGetErrorString(e));
            rc = SPAQR_ERR_CUDA;
        }
    }
    void launched() { cuda(cudaGetLastError()); }
    // Give back a kept allocation before the factor is complete (stream
    // ordered: work already queued on st still sees it).
    void release(void* p) {
        for (size_t i = 0; i < kept_bytes.size(); i++)
            if (kept_bytes[i].first == p) {
                F->bytes -= (int64_t)kept_bytes[i].second;
                live -= (int64_t)kept_bytes[i].second;
                kept_bytes.erase(kept_bytes.begin() + (int64_t)i);
                break;
            }
        for (size_t i = 0; i < F->allocs.size(); i++)
            if (F->allocs[i] == p) {
                F->allocs.erase(F->allocs.begin() + (int64_t)i);
                break;
            }
        cuda(cudaFreeAsync(p, st));
    }
    ~Ctx() { free_temps(); }   // temporaries of a factorisation that stopped on an error
    void free_temps() {
        for (auto& t : temps) {
            cudaFreeAsync(t.first, st);
            live -= (int64_t)t.second;
        }
        temps.clear();
    }
};

struct LevelLayout {
    std::vector<int64_t> H, poff, rowoff, voff;
    int64_t total = 0, rows = 0;
};

void layout_of(const StepPlan& sp, const std::vector<int64_t>& sz, LevelLayout& L) {
    const int ncl = (int)sp.cl.size();
    L.H.assign(ncl, 0);
    L.poff.assign(ncl + 1, 0);
    L.rowoff.assign(sp.rowidx.size(), 0);
    L.voff.assign(ncl + 1, 0);
    for (int j = 0; j < ncl; j++) {
        int64_t h = 0;
        for (int e = sp.colptr[j]; e < sp.colptr[j + 1]; e++) {
            L.rowoff[e] = h;
            h += sz[sp.rowidx[e]];
        }
        L.H[j] = h;
        L.poff[j + 1] = L.poff[j] + h * sz[j];
        L.voff[j + 1] = L.voff[j] + sz[j];
    }
    L.total = L.poff[ncl];
    L.rows = L.voff[ncl];
}

const int kSmemMax = 200 * 1024;
const int kTcMinN = 48;    // reflectors of a front from which its application is a tensor-core product
const int kTcMinM = 256;   // and rows
const int kPanelSmem = 112 * 1024;   // QR with a staged panel: two CTAs per SM

// Heaviest first: independent tasks (or pieces) reordered by their work in
// power-of-two classes, largest class first.  The block scheduler issues a
// launch's CTAs roughly in index order, so the long ones start first and the
// launch ends with short ones (the longest-processing-time rule); ncu showed
// the SMs of a 2D application launch busy only 57% of its time, the rest a
// tail of long CTAs.  Linear time, order kept within a class.
template <class T, class W>
void heaviest_first(std::vector<T>& v, W work) {
    if (v.size() < 2) return;
    constexpr int kClasses = 64;
    std::vector<unsigned char> cls(v.size());
    int cnt[kClasses + 1] = {0};
    for (size_t i = 0; i < v.size(); i++) {
        const double w = work(v[i]);
        int e = 0;
        if (w >= 1.0) std::frexp(w, &e);
        e = std::min(std::max(e, 0), kClasses - 1);
        cls[i] = (unsigned char)(kClasses - 1 - e);   // heavier -> smaller class index
        cnt[cls[i] + 1]++;
    }
    for (int c = 0; c < kClasses; c++) cnt[c + 1] += cnt[c];
    std::vector<T> out(v.size());
    for (size_t i = 0; i < v.size(); i++) out[cnt[cls[i]]++] = v[i];
    v.swap(out);
}

}  // namespace

// Launch the QR tasks: small ones on one CTA each (k_qr), large ones on a
// cluster of QR_CS CTAs (k_qr_cluster).
template <class real>
void launch_qr(Ctx& C, const std::vector<QRTask<real>>& all, size_t esz, int kind, double fl, double by) {
    std::vector<QRTask<real>> small, big;
    int pr_s = 0, pr_b = 0;
    for (const QRTask<real>& q1 : all) {
        const int tt = q1.m < q1.n ? q1.m : q1.n;
        if ((int64_t)q1.m * q1.n >= kBigQR && tt >= 4 * NB) {
            big.push_back(q1);
            pr_b = std::max(pr_b, q1.m);
        } else {
            small.push_back(q1);
            pr_s = std::max(pr_s, q1.m);
        }
    }
    auto qr_work = [](const QRTask<real>& q1) {
        const double t = q1.m < q1.n ? q1.m : q1.n;
        return (double)q1.m * q1.n * t;
    };
    heaviest_first(small, qr_work);
    heaviest_first(big, qr_work);
    if (qr_smem_bytes((int)esz, QC, pr_s) > kPanelSmem) pr_s = 0;
    if (qr_smem_bytes((int)esz, QC, pr_b) > kPanelSmem) pr_b = 0;
    cudaStream_t st = C.st;
    if (!big.empty()) {
        QRTask<real>* d = C.upload(big, false);
        if (C.rc) return;
        int mmax = 1;
        for (const QRTask<real>& q1 : big) mmax = std::max(mmax, q1.m);
        SPAQR_LAUNCH(kind, fl, by, st,
                     k_qr_cluster<real, QR_CS><<<(unsigned)(big.size() * QR_CS), NT,
                                                 qrcl_smem_bytes((int)esz, (mmax + QR_CS - 1) / QR_CS), st>>>(d, 0));
        C.launched();
        fl = 0.0;
        by = 0.0;
    }
    if (!small.empty()) {
        QRTask<real>* d = C.upload(small, false);
        if (C.rc) return;
        SPAQR_LAUNCH(kind, fl, by, st,
                     k_qr<real><<<(unsigned)small.size(), NT, (size_t)qr_smem_bytes((int)esz, QC, pr_s), st>>>(d,
                                                                                                            pr_s));
        C.launched();
    }
}

// Whether a level's fronts go to the tensor cores: the level's apply work is
// dominated by fronts wide (n reflectors) and tall (m rows, the products'
// K) enough to be dense contractions.  The 2D leaves (193 x 105) are not:
// there the tensor-core form measured 3.3 ms against 2.9 on the CUDA cores.
bool tc_level(const StepPlan& sp, const LevelLayout& lay, const std::vector<int64_t>& sz) {
    double big = 0.0, all = 0.0;
    for (size_t f = 0; f < sp.fronts.size(); f++) {
        const int s = sp.fronts[f];
        double w = 0.0;
        for (size_t t = 1; t < sp.C[f].size(); t++) w += (double)sz[sp.C[f][t]];
        const double fl = (4.0 * lay.H[s] * sz[s] - 2.0 * sz[s] * sz[s]) * w;
        all += fl;
        if (sz[s] >= kTcMinN && lay.H[s] >= kTcMinM) big += fl;
    }
    return all > 0.0 && big >= 0.8 * all;
}

// Tensor-core application of the fronts of a level (FP32 storage; see
// k_front_copy / k_tfull): per front, G = V^T V and T (once), then per
// colour the dense copies B of the fronts' columns, W = V^T B, W <- T^T W,
// B <- B - V W, and the copies written back.  split3: three TF32 passes for
// the application products (G always takes three).
int tc_front_apply(Ctx& C, const StepPlan& sp, const LevelLayout& lay, const std::vector<int64_t>& sz, float* arena,
                   const std::vector<float*>& ftau, bool split3, int* d_err) {
    cudaStream_t st = C.st;
    struct FI {
        int f, s, m, n, w;
        int64_t oB, oG, oT, oW, oW2, oX;
    };
    std::vector<FI> fi;
    int64_t tot = 0;
    for (size_t f = 0; f < sp.fronts.size(); f++) {
        const int s = sp.fronts[f];
        if (sz[s] == 0) continue;
        int64_t w = 0;
        for (size_t t = 1; t < sp.C[f].size(); t++) w += sz[sp.C[f][t]];
        if (w == 0) continue;
        FI x;
        x.f = (int)f;
        x.s = s;
        x.m = (int)lay.H[s];
        x.n = (int)sz[s];
        x.w = (int)w;
        x.oB = tot;
        tot += (int64_t)x.m * w;
        x.oG = tot;
        tot += (int64_t)x.n * x.n;
        x.oT = tot;
        tot += (int64_t)x.n * x.n;
        x.oW = tot;
        tot += (int64_t)x.n * w;
        x.oW2 = tot;
        tot += (int64_t)x.n * w;
        x.oX = tot;
        tot += (int64_t)x.n * NB;
        tot = (tot + 31) & ~(int64_t)31;
        fi.push_back(x);
    }
    if (fi.empty()) return SPAQR_OK;
    float* S = C.alloc<float>(tot, false);
    if (C.rc) return C.rc;
    auto vt = [&](const FI& x) {   // V^T as a product operand: (i, k) = V(k, i)
        return GemmOperand{arena + lay.poff[x.s], lay.H[x.s], 1, 1, 1};
    };
    {
        std::vector<GemmTask> g;
        std::vector<TfullTask> tf;
        for (const FI& x : fi) {
            GemmTask t{};
            t.a = vt(x);
            t.bt = vt(x);
            t.c = S + x.oG;
            t.c_rs = 1;
            t.c_cs = x.n;
            t.M = x.n;
            t.N = x.n;
            t.K = x.m;
            t.alpha = 1.0f;
            t.beta = 0.0f;
            g.push_back(t);
            tf.push_back(TfullTask{S + x.oG, ftau[x.f], S + x.oT, S + x.oX, x.n});
        }
        gemm_tiles(g);
        GemmTask* dg = C.upload(g, false);
        TfullTask* dtf = C.upload(tf, false);
        if (C.rc) return C.rc;
        SPAQR_LAUNCH(KK_FRONT_APPLY_TC, 0.0, 0.0, st, launch_tc_gemm(dg, g, true, d_err, st));
        C.launched();
        SPAQR_LAUNCH(KK_FRONT_APPLY_TC, 0.0, 0.0, st, k_tfull<<<(unsigned)tf.size(), NT, 0, st>>>(dtf));
        C.launched();
    }
    size_t a = 0;
    while (a < fi.size()) {
        const int colour = sp.colour[fi[a].f];
        size_t b = a;
        while (b < fi.size() && sp.colour[fi[b].f] == colour) b++;
        std::vector<FrontCopy> cp;
        std::vector<Seg> segs;
        std::vector<GemmTask> gw, gw2, gu;
        double fl = 0.0, by = 0.0;
        int mmax = 1;
        for (size_t q = a; q < b; q++) {
            const FI& x = fi[q];
            mmax = std::max(mmax, x.m);
            int64_t coff = 0;
            for (size_t t = 1; t < sp.C[x.f].size(); t++) {
                const int j = sp.C[x.f][t];
                if (sz[j] == 0) continue;
                FrontCopy c;
                c.panel = arena + lay.poff[j];
                c.ld = lay.H[j];
                c.dense = S + x.oB + coff * x.m;
                c.m = x.m;
                c.ncol = (int)sz[j];
                c.seg_begin = (int)segs.size();
                const int* ep = sp.apply_e.data() + sp.fcol_ebase[sp.fcol_ptr[x.f] + t - 1];
                int spos = 0;
                for (size_t u = 0; u < sp.R[x.f].size(); u++) {
                    const int i = sp.R[x.f][u], e = ep[u];
                    if (e < 0) { set_error("missing fill block"); return SPAQR_ERR_INVALID_ARG; }
                    if (sz[i] > 0) {
                        segs.push_back(Seg{lay.rowoff[e], (int)sz[i], spos});
                        spos += (int)sz[i];
                    }
                }
                c.nseg = (int)segs.size() - c.seg_begin;
                cp.push_back(c);
                coff += sz[j];
                by += 16.0 * x.m * sz[j] + 8.0 * x.m * x.n;
            }
            fl += (4.0 * x.m * x.n - 2.0 * x.n * x.n) * x.w;
            GemmTask t{};
            t.a = vt(x);
            t.bt = GemmOperand{S + x.oB, x.m, 1, 0, 0};
            t.c = S + x.oW;
            t.c_rs = 1;
            t.c_cs = x.n;
            t.M = x.n;
            t.N = x.w;
            t.K = x.m;
            t.alpha = 1.0f;
            t.beta = 0.0f;
            gw.push_back(t);
            t.a = GemmOperand{S + x.oT, x.n, 1, 0, 0};   // T^T: (i, k) = T(k, i)
            t.bt = GemmOperand{S + x.oW, x.n, 1, 0, 0};
            t.c = S + x.oW2;
            t.K = x.n;
            gw2.push_back(t);
            t.a = GemmOperand{arena + lay.poff[x.s], 1, lay.H[x.s], 1, 0};   // V: (i, k) = V(i, k)
            t.bt = GemmOperand{S + x.oW2, x.n, 1, 0, 0};
            t.c = S + x.oB;
            t.c_rs = 1;
            t.c_cs = x.m;
            t.M = x.m;
            t.N = x.w;
            t.K = x.n;
            t.alpha = -1.0f;
            t.beta = 1.0f;
            gu.push_back(t);
        }
        gemm_tiles(gw);
        gemm_tiles(gw2);
        gemm_tiles(gu);
        FrontCopy* dcp = C.upload(cp, false);
        Seg* dsg = C.upload(segs, false);
        GemmTask* dw = C.upload(gw, false);
        GemmTask* dw2 = C.upload(gw2, false);
        GemmTask* du = C.upload(gu, false);
        if (C.rc) return C.rc;
        const size_t smem = (size_t)mmax * sizeof(int);
        int ccmax = 1;
        for (const FrontCopy& c : cp) ccmax = std::max(ccmax, (c.ncol + kCopyCols - 1) / kCopyCols);
        const dim3 cgrid((unsigned)cp.size(), (unsigned)ccmax);
        SPAQR_LAUNCH(KK_FRONT_APPLY_TC, 0.0, 0.0, st,
                     k_front_copy<<<cgrid, NT, smem, st>>>(dcp, dsg, 1));
        C.launched();
        SPAQR_LAUNCH(KK_FRONT_APPLY_TC, 0.0, 0.0, st, launch_tc_gemm(dw, gw, split3, d_err, st));
        C.launched();
        SPAQR_LAUNCH(KK_FRONT_APPLY_TC, 0.0, 0.0, st, launch_tc_gemm(dw2, gw2, split3, d_err, st));
        C.launched();
        SPAQR_LAUNCH(KK_FRONT_APPLY_TC, fl, by, st, launch_tc_gemm(du, gu, split3, d_err, st));
        C.launched();
        SPAQR_LAUNCH(KK_FRONT_APPLY_TC, 0.0, 0.0, st,
                     k_front_copy<<<cgrid, NT, smem, st>>>(dcp, dsg, 0));
        C.launched();
        a = b;
    }
    return SPAQR_OK;
}

// Full compact-WY factors T (Q = I - V T V^T) of a set of reflector blocks
// on the tensor cores: G = V^T V (three TF32 passes), then k_tfull.  vt: V^T
// as a product operand (r x n), tau: r scalars, T: r x r output, scratch:
// r x r (G) + r x NB (k_tfull).
struct WySpec {
    GemmOperand vt;
    int n, r;
    const float* tau;
    float* T;
    float* scratch;
};

int tc_full_t(Ctx& C, const std::vector<WySpec>& ws, int kind, int* d_err) {
    if (ws.empty()) return SPAQR_OK;
    cudaStream_t st = C.st;
    std::vector<GemmTask> g;
    std::vector<TfullTask> tf;
    for (const WySpec& w : ws) {
        GemmTask t{};
        t.a = w.vt;
        t.bt = w.vt;
        t.c = w.scratch;
        t.c_rs = 1;
        t.c_cs = w.r;
        t.M = w.r;
        t.N = w.r;
        t.K = w.n;
        t.alpha = 1.0f;
        t.beta = 0.0f;
        g.push_back(t);
        tf.push_back(TfullTask{w.scratch, w.tau, w.T, w.scratch + (int64_t)w.r * w.r, w.r});
    }
    gemm_tiles(g);
    GemmTask* dg = C.upload(g, false);
    TfullTask* dtf = C.upload(tf, false);
    if (C.rc) return C.rc;
    SPAQR_LAUNCH(kind, 0.0, 0.0, st, launch_tc_gemm(dg, g, true, d_err, st));
    C.launched();
    SPAQR_LAUNCH(kind, 0.0, 0.0, st, k_tfull<<<(unsigned)tf.size(), NT, 0, st>>>(dtf));
    C.launched();
    return SPAQR_OK;
}

// One batch of products on the tensor cores (tiles filled in here).
int tc_batch(Ctx& C, std::vector<GemmTask>& g, bool split3, int kind, double fl, double by, int* d_err) {
    if (g.empty()) return SPAQR_OK;
    gemm_tiles(g);
    GemmTask* d = C.upload(g, false);
    if (C.rc) return C.rc;
    cudaStream_t st = C.st;
    SPAQR_LAUNCH(kind, fl, by, st, launch_tc_gemm(d, g, split3, d_err, st));
    C.launched();
    return SPAQR_OK;
}

// Whether the interfaces of a level are large enough for their scaling and
// sparsification products to go to the tensor cores: interfaces of at least
// kTcMinN unknowns carry 80% of the level's n_p^3.
bool tc_iface_level(const std::vector<int>& rest, const std::vector<int64_t>& sz) {
    double big = 0.0, all = 0.0;
    for (int p : rest) {
        const double w = (double)sz[p] * sz[p] * sz[p];
        all += w;
        if (sz[p] >= kTcMinN) big += w;
    }
    return all > 0.0 && big >= 0.8 * all;
}

template <class real>
int run_factor(const Ordering& o, const spaqr_csr* A, const spaqr_opts* opt, spaqr_factor_s* F) {
    Ctx C;
    C.F = F;
    C.st = (cudaStream_t)opt->stream;
    cudaStream_t st = C.st;
    const int64_t n = o.n, nnz = o.nnz;
    const int L = o.L;
    F->n = n;
    F->nnz = nnz;
    F->L = L;
    F->skip = opt->skip;
    F->eps = opt->eps;
    F->precision = sizeof(real) == 8 ? SPAQR_FP64 : SPAQR_FP32;
    F->unscaled = opt->scaling == 0;
    F->esz = (int)sizeof(real);
    // tensor-core products of the FP32 storage forms: 1 = three TF32 passes, 2 = one
    const int tcmode = (sizeof(real) == 4 && tensor_cores_on()) ? (opt->precision == SPAQR_TF32 ? 2 : 1) : 0;
    static std::once_flag attr_once;
    std::call_once(attr_once, [&] {
        C.cuda(cudaFuncSetAttribute(k_front_apply<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax));
        C.cuda(cudaFuncSetAttribute(k_scale_apply<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax));
        C.cuda(cudaFuncSetAttribute(k_qr<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax));
        C.cuda(cudaFuncSetAttribute(k_qr_cluster<real, QR_CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax));
        C.cuda(cudaFuncSetAttribute(k_qr_cluster<real, QR_CS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        C.cuda(cudaFuncSetAttribute(k_cpqr_cluster<real, cpqr_cs<real>()>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        C.cuda(cudaFuncSetAttribute(k_cpqr<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax));
        C.cuda(cudaFuncSetAttribute(k_cpqr_cluster<real, cpqr_cs<real>()>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kSmemMax));
    });
    if (C.rc != SPAQR_OK) return C.rc;
    const size_t esz = sizeof(real);
    // phase timers: (start, end, phase) event triples
    struct Timer { cudaEvent_t a, b; int ph, lev; };
    std::vector<Timer> timers;
    int cur_level = -1;
    // every timed phase is also an NVTX range "L<level> <phase>" (level -1:
    // the initial gather), so profilers can select a level's or a phase's
    // kernels; without a profiler attached the ranges cost nothing
    static const char* const kPhaseName[4] = {"factorize", "scale", "sparsify", "merge"};
    auto tstart = [&](int ph) {
        Timer t;
        t.ph = -1;
        t.lev = cur_level;
        C.cuda(cudaEventCreate(&t.a));
        C.cuda(cudaEventCreate(&t.b));
        C.cuda(cudaEventRecord(t.a, st));
        timers.push_back(t);
        char name[48];
        std::snprintf(name, sizeof(name), "L%d %s", cur_level, kPhaseName[ph]);
        nvtxRangePushA(name);
    };
    auto tstop = [&](int ph) {
        timers.back().ph = ph;
        C.cuda(cudaEventRecord(timers.back().b, st));
        nvtxRangePop();
    };

    // ---- inputs on the device ----
    const double* dval = A->val;
    const int32_t* dcol = A->colind;
    if (!A->on_device) {
        double* v = C.alloc<double>(nnz, false);
        int32_t* ci = C.alloc<int32_t>(nnz, false);
        if (C.rc) return C.rc;
        C.cuda(cudaMemcpyAsync(v, A->val, sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
        C.cuda(cudaMemcpyAsync(ci, A->colind, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
        dval = v;
        dcol = ci;
    }
    int64_t* d_cscp = C.upload(o.csc_ptr, false);
    int64_t* d_csce = C.upload(o.csc_entry, false);
    int64_t* d_goff = C.upload(o.gather_off, false);
    F->d_perm = C.upload(o.perm, true);
    F->d_rperm = o.rperm.empty() ? F->d_perm : C.upload(o.rperm, true);
    F->d_scale = C.alloc<double>(n, true);
    int* d_flags = C.alloc<int>(4, true);
    if (C.rc) return C.rc;
    C.cuda(cudaMemsetAsync(d_flags, 0, 4 * sizeof(int), st));
    tstart(3);
    SPAQR_LAUNCH(KK_COLSCALE, 2.0 * nnz, 24.0 * nnz + 16.0 * n, st,
                 k_colscale<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, d_cscp, d_csce, dval,
                                                                          opt->col_normalize, F->d_scale, d_flags));
    C.launched();

    std::vector<int64_t> sz(o.steps[0].cl.size());
    for (size_t a = 0; a < sz.size(); a++) sz[a] = o.atom_ptr[a + 1] - o.atom_ptr[a];
    LevelLayout lay;
    layout_of(o.steps[0], sz, lay);
    if (lay.total != o.arena1_size) { set_error("arena layout mismatch"); return SPAQR_ERR_INVALID_ARG; }
    real* arena = C.alloc<real>(lay.total, true);
    if (C.rc) return C.rc;
    C.cuda(cudaMemsetAsync(arena, 0, sizeof(real) * lay.total, st));
    SPAQR_LAUNCH(KK_GATHER, 1.0 * nnz, 36.0 * nnz, st,
                 k_gather<real><<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(nnz, d_goff, dcol, dval, F->d_scale, arena));
    C.launched();
    tstop(3);

    // solve-plan host arrays
    std::vector<SolveFront<real>> sfronts;
    std::vector<Seg> ssegs;
    std::vector<SolveRsj<real>> srsj;
    std::vector<SolveSS<real>> sss;
    std::vector<RsjTile> tiles;
    std::vector<SolveRsj<real>> pieces;
    std::vector<std::pair<int, int>> piece_src;   // (R_sj record, first column) of every piece
    std::vector<WideFront> wfr;
    std::vector<int> front_cl, rsj_cl, ss_cl;   // first atom of the cluster of every solve record
    int64_t zp_max = 0;
    F->lv.assign(L, SolveLevelHost());
    int64_t ws = 0;
    double flops = 0.0, sflops = 0.0;
    int64_t sbytes = 0;
    F->ranks.assign(L, {});
    F->margins.assign(L, {});
    F->sigmas.assign(L, {});
    F->pivots.assign(L, {});
    F->pivot_off.assign(L, std::vector<int32_t>(1, 0));
    F->ldiag.assign(L, LevelDiag());

    // Keep only what the solve reads of a finished level -- front panels
    // (reflectors and R_ss), the R_sj rows and the scaled diagonal blocks --
    // packed in one allocation, and give the level's block arena back: the
    // blocks between interfaces have been carried into the next level's arena
    // by the merge, and nothing else reads them.
    auto compact_level = [&](int k, real* old_arena, int piece_begin) {
        SolveLevelHost& LVk = F->lv[k];
        int64_t tot = 0;
        for (int f = LVk.front_begin; f < LVk.front_begin + LVk.nfront; f++) {
            const SolveFront<real>& sf = sfronts[f];
            tot += (int64_t)sf.m * sf.n;
            for (int b = sf.rsj_begin; b < sf.rsj_begin + sf.nrsj; b++) tot += (int64_t)sf.n * srsj[b].nj;
        }
        for (int q = LVk.ss_begin; q < LVk.ss_begin + LVk.nss; q++)
            if (sss[q].UV) tot += (int64_t)sss[q].np * sss[q].np;
        if (tot > 0) {
            real* cb = C.alloc<real>(tot, true);
            if (C.rc) return;
            std::vector<SparsifyTask<real>> cp;
            int64_t o = 0;
            auto add = [&](const real* A, int64_t lda, int m, int n) {
                SparsifyTask<real> t;
                std::memset(&t, 0, sizeof(t));
                t.A = A;
                t.lda = lda;
                t.mi = m;
                t.nj = n;
                t.D = cb + o;
                t.ldd = m;
                t.mode = 2;
                cp.push_back(t);
                o += (int64_t)m * n;
                return t.D;
            };
            for (int f = LVk.front_begin; f < LVk.front_begin + LVk.nfront; f++) {
                SolveFront<real>& sf = sfronts[f];
                sf.V = add(sf.V, sf.ldv, sf.m, sf.n);
                sf.ldv = sf.m;
                for (int b = sf.rsj_begin; b < sf.rsj_begin + sf.nrsj; b++) {
                    srsj[b].R = add(srsj[b].R, srsj[b].ldr, sf.n, srsj[b].nj);
                    srsj[b].ldr = sf.n;
                }
            }
            for (int q = LVk.ss_begin; q < LVk.ss_begin + LVk.nss; q++)
                if (sss[q].UV) {
                    sss[q].UV = add(sss[q].UV, sss[q].lduv, sss[q].np, sss[q].np);
                    sss[q].lduv = sss[q].np;
                }
            for (int pc = piece_begin; pc < (int)pieces.size(); pc++) {
                const SolveRsj<real>& R = srsj[piece_src[pc].first];
                pieces[pc].R = R.R + (int64_t)piece_src[pc].second * R.ldr;
                pieces[pc].ldr = R.ldr;
            }
            std::vector<ScalePiece> pc;
            for (int t = 0; t < (int)cp.size(); t++) pc.push_back({t, 0, 0});
            SparsifyTask<real>* d = C.upload(cp, false);
            ScalePiece* dp = C.upload(pc, false);
            if (C.rc) return;
            SPAQR_LAUNCH(KK_SPARSIFY, 0.0, 16.0 * tot, st, k_sparsify<real><<<(unsigned)pc.size(), NT, 16, st>>>(d, dp, 0));
            C.launched();
        }
        C.release(old_arena);
    };

    for (int k = 0; k < L; k++) {
        const StepPlan& sp = o.steps[k];
        const int ncl = (int)sp.cl.size();
        SolveLevelHost& LV = F->lv[k];
        cur_level = k;
        const int piece_begin = (int)pieces.size();
        LevelDiag& DG = F->ldiag[k];
        DG.block_entries = lay.total;
        for (int s : sp.fronts) {
            DG.n_fronts++;
            DG.front_rows += lay.H[s];
            DG.front_cols += sz[s];
            DG.max_front_rows = std::max<int>(DG.max_front_rows, (int)lay.H[s]);
            DG.max_front_cols = std::max<int>(DG.max_front_cols, (int)sz[s]);
        }
        LV.rows = lay.rows;
        LV.ws_off = ws;
        ws += lay.rows;
        auto blk = [&](int e, int j) { return arena + lay.poff[j] + lay.rowoff[e]; };

        // ---------------- (i) factor the fronts ----------------
        double fl_qr = 0, by_qr = 0, fl_ap = 0, by_ap = 0;
        std::vector<QRTask<real>> qr;
        std::vector<real*> ftau(sp.fronts.size(), nullptr), fT(sp.fronts.size(), nullptr),
            fD(sp.fronts.size(), nullptr);
        int64_t aux = 0;
        for (size_t f = 0; f < sp.fronts.size(); f++) {
            const int s = sp.fronts[f];
            aux += sz[s] + sz[s] * sz[s] + sz[s] * NB;
        }
        real* faux = C.alloc<real>(aux, true);
        if (C.rc) return C.rc;
        int tmax = 1;
        {
            int64_t a = 0;
            for (size_t f = 0; f < sp.fronts.size(); f++) {
                const int s = sp.fronts[f];
                ftau[f] = faux + a;
                a += sz[s];
                fT[f] = faux + a;
                a += sz[s] * sz[s];
                fD[f] = faux + a;
                a += sz[s] * NB;
                if (sz[s] == 0) continue;
                qr.push_back(QRTask<real>{arena + lay.poff[s], lay.H[s], (int)lay.H[s], (int)sz[s], ftau[f], fT[f], fD[f],
                                    d_flags + 2});
                tmax = std::max<int>(tmax, (int)sz[s]);
                const double fq = 2.0 * lay.H[s] * sz[s] * sz[s] - 2.0 / 3.0 * sz[s] * sz[s] * sz[s];
                flops += fq;
                fl_qr += fq;
                by_qr += 16.0 * lay.H[s] * sz[s] + 8.0 * sz[s] * sz[s];
                if (k == L - 1) F->top_size = (int)sz[s];
            }
        }
        tstart(0);
        if (!qr.empty()) {
            launch_qr<real>(C, qr, esz, KK_FRONT_QR, fl_qr, by_qr);
            if (C.rc) return C.rc;
            C.launched();
        }
        // (the application's tasks are planned while the QR runs)
        // apply: per column j, the fronts containing it (processing order,
        // sp.colf_*, with the positions of their row blocks in column j)
        std::vector<ApplyTask<real>> at;
        std::vector<ApplyFront<real>> af;
        std::vector<Seg> asg;
        size_t smem_apply = 0;
        // column chunk of a task: QAPPLY, halved while the staged work area of
        // the tallest front would not fit or the level has too few tasks to
        // give every SM two of them
        int qapply = QAPPLY;
        {
            int mm = 1;
            int64_t cols = 0;
            for (size_t f = 0; f < sp.fronts.size(); f++) mm = std::max<int>(mm, (int)lay.H[sp.fronts[f]]);
            {
                std::vector<char> used(ncl, 0);
                for (size_t f = 0; f < sp.fronts.size(); f++)
                    for (size_t t = 1; t < sp.C[f].size(); t++) used[sp.C[f][t]] = 1;
                for (int j = 0; j < ncl; j++)
                    if (used[j]) cols += sz[j];
            }
            while (qapply > 8 && ((mm + 1) / 2 + 1) * 8 + staged_smem_elems(mm, qapply) * (int64_t)esz > kSmemMax)
                qapply /= 2;
            while (qapply > 4 && cols / qapply < 2 * kNumSM) qapply /= 2;
        }
        for (int j = 0; j < ncl; j++) {
            if (sz[j] == 0) continue;
            const int fb = (int)af.size();
            int nmax = 1, mmax = 1;
            for (int q = sp.colf_ptr[j]; q < sp.colf_ptr[j + 1]; q++) {
                const int f = sp.colf_front[q];
                const int s = sp.fronts[f];
                if (sz[s] == 0) continue;
                const int* ep = sp.apply_e.data() + sp.colf_ebase[q];
                ApplyFront<real> A1;
                A1.V = arena + lay.poff[s];
                A1.T = fT[f];
                A1.ldv = lay.H[s];
                A1.m = (int)lay.H[s];
                A1.n = (int)sz[s];
                A1.seg_begin = (int)asg.size();
                int spos = 0;
                for (size_t t = 0; t < sp.R[f].size(); t++) {
                    const int i = sp.R[f][t], e = ep[t];
                    if (e < 0) { set_error("missing fill block"); return SPAQR_ERR_INVALID_ARG; }
                    if (sz[i] > 0) {
                        asg.push_back(Seg{lay.rowoff[e], (int)sz[i], spos});
                        spos += (int)sz[i];
                    }
                }
                A1.nseg = (int)asg.size() - A1.seg_begin;
                af.push_back(A1);
                nmax = std::max(nmax, A1.n);
                mmax = std::max(mmax, A1.m);
                const double fa = (4.0 * A1.m * A1.n - 2.0 * A1.n * A1.n) * sz[j];
                flops += fa;
                fl_ap += fa;
                by_ap += 16.0 * A1.m * sz[j] + 8.0 * A1.m * A1.n;
            }
            const int nfr = (int)af.size() - fb;
            if (nfr == 0) continue;
            const int q = qapply;
            for (int64_t c0 = 0; c0 < sz[j]; c0 += q) {
                ApplyTask<real> T1;
                T1.B = arena + lay.poff[j] + c0 * lay.H[j];
                T1.ldb = lay.H[j];
                T1.q = (int)std::min<int64_t>(q, sz[j] - c0);
                T1.fr_begin = fb;
                T1.nfr = nfr;
                T1.m_max = mmax;
                at.push_back(T1);
            }
            (void)nmax;
        }
        // shared memory: row map + staged work area when it fits
        int rmap_d = 0, staged = 0;
        {
            int maxm = 1;
            for (const ApplyTask<real>& T1 : at) maxm = std::max(maxm, T1.m_max);
            rmap_d = (maxm + 1) / 2 + 1;
            const int64_t need = rmap_d * 8 + staged_smem_elems(maxm, qapply) * (int64_t)esz;
            if (need <= kSmemMax) {
                staged = 1;
                smem_apply = (size_t)need;
            } else {
                smem_apply = (size_t)rmap_d * 8 + (size_t)(2 * NB * qapply + NT) * esz;
            }
        }
        if (smem_apply > (size_t)kSmemMax) { set_error("front too tall for the apply kernel"); return SPAQR_ERR_UNSUPPORTED; }
        bool tc_done = false;
        if constexpr (sizeof(real) == 4) {
            if (tcmode && !at.empty() && tc_level(sp, lay, sz)) {
                const int rc = tc_front_apply(C, sp, lay, sz, arena, ftau, tcmode == 1, d_flags + 3);
                if (rc != SPAQR_OK) return rc;
                if (C.rc) return C.rc;
                tc_done = true;
                F->tc_levels++;
            }
        }
        if (!at.empty() && !tc_done) {
            heaviest_first(at, [&](const ApplyTask<real>& T1) {
                double w = 0.0;
                for (int f = T1.fr_begin; f < T1.fr_begin + T1.nfr; f++) w += (double)af[f].m * af[f].n;
                return w * T1.q;
            });
            ApplyTask<real>* d1 = C.upload(at, false);
            ApplyFront<real>* d2 = C.upload(af, false);
            Seg* d3 = C.upload(asg, false);
            if (C.rc) return C.rc;
            SPAQR_LAUNCH(KK_FRONT_APPLY, fl_ap, by_ap, st,
                         k_front_apply<real><<<(unsigned)at.size(), NT, smem_apply, st>>>(d1, d2, d3, rmap_d, staged));
            C.launched();
        }
        tstop(0);

        // solve record of the fronts and the R_sj tiles of the backward step:
        // host planning that no launch of this level's factorisation needs, so
        // it runs while the GPU works on the level (before the rank sync)
        bool front_solve_planned = false;
        auto plan_front_solve = [&]() {
            front_solve_planned = true;
            // solve record of the fronts, grouped by colour
            LV.front_begin = (int)sfronts.size();
            LV.colour_ptr.assign(1, 0);
            {
                int cur = 0;
                LV.ff_flops.assign(1, 0.0);
                LV.ff_fixed.assign(1, 0.0);
                LV.ff_vec.assign(1, 0.0);
                for (size_t f = 0; f < sp.fronts.size(); f++) {
                    while (sp.colour[f] > cur) {
                        LV.colour_ptr.push_back((int)sfronts.size() - LV.front_begin);
                        LV.ff_flops.push_back(0.0);
                        LV.ff_fixed.push_back(0.0);
                        LV.ff_vec.push_back(0.0);
                        cur++;
                    }
                    const int s = sp.fronts[f];
                    if (sz[s] == 0) continue;
                    SolveFront<real> sf;
                    sf.V = arena + lay.poff[s];
                    sf.T = fT[f];
                    sf.Dinv = fD[f];
                    sf.ldv = lay.H[s];
                    sf.m = (int)lay.H[s];
                    sf.n = (int)sz[s];
                    sf.seg_begin = (int)ssegs.size();
                    int spos = 0;
                    for (int i : sp.R[f])
                        if (sz[i] > 0) {
                            ssegs.push_back(Seg{lay.voff[i], (int)sz[i], spos});
                            spos += (int)sz[i];
                        }
                    sf.nseg = (int)ssegs.size() - sf.seg_begin;
                    sf.rsj_begin = (int)srsj.size();
                    for (size_t t = 1; t < sp.C[f].size(); t++) {
                        const int j = sp.C[f][t];
                        if (sz[j] == 0) continue;
                        const int e = sp.find(s, j);
                        srsj.push_back(SolveRsj<real>{blk(e, j), lay.H[j], (int)sz[j], 0, lay.voff[j]});
                        rsj_cl.push_back(sp.cl[j]);
                        sflops += 2.0 * sz[s] * sz[j];
                        sbytes += 8 * sz[s] * sz[j];
                    }
                    sf.nrsj = (int)srsj.size() - sf.rsj_begin;
                    {
                        double snj = 0;
                        for (int b = sf.rsj_begin; b < (int)srsj.size(); b++) snj += srsj[b].nj;
                        const double m_ = sf.m, n_ = sf.n;
                        // applying n reflectors of m rows to one column: 4mn - 2n^2
                        LV.ff_flops.back() += 4.0 * m_ * n_ - 2.0 * n_ * n_;
                        LV.ff_fixed.back() += 8.0 * (m_ * n_ + n_ * n_);
                        LV.ff_vec.back() += 16.0 * m_;
                        LV.fb_flops += 2.0 * n_ * snj + n_ * n_;
                        LV.fb_fixed += 8.0 * (n_ * n_ + n_ * snj);
                        LV.fb_vec += 16.0 * n_ + 8.0 * snj;
                    }
                    sfronts.push_back(sf);
                    front_cl.push_back(sp.cl[s]);
                    LV.max_front_m = std::max(LV.max_front_m, sf.m);
                    LV.max_front_n = std::max(LV.max_front_n, sf.n);
                    sflops += 4.0 * sf.m * sf.n - 2.0 * sf.n * sf.n + 1.0 * sf.n * sf.n;
                    sbytes += 8 * (int64_t)sf.m * sf.n + 8 * (int64_t)sf.n * sf.n;
                }
                LV.colour_ptr.push_back((int)sfronts.size() - LV.front_begin);
                LV.nfront = (int)sfronts.size() - LV.front_begin;
                // within a colour (disjoint rows, any order), the heaviest
                // fronts first: the application's launches issue them first
                for (size_t c = 0; c + 1 < LV.colour_ptr.size(); c++) {
                    const int a = LV.front_begin + LV.colour_ptr[c], b = LV.front_begin + LV.colour_ptr[c + 1];
                    if (b - a < 2) continue;
                    std::vector<int> idx(b - a);
                    for (int u = 0; u < b - a; u++) idx[u] = a + u;
                    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
                        return (int64_t)sfronts[x].m * sfronts[x].n > (int64_t)sfronts[y].m * sfronts[y].n;
                    });
                    std::vector<SolveFront<real>> sf2(b - a);
                    std::vector<int> cl2(b - a);
                    for (int u = 0; u < b - a; u++) {
                        sf2[u] = sfronts[idx[u]];
                        cl2[u] = front_cl[idx[u]];
                    }
                    std::copy(sf2.begin(), sf2.end(), sfronts.begin() + a);
                    std::copy(cl2.begin(), cl2.end(), front_cl.begin() + a);
                }
            }
            // tallest front of every colour (shared-memory size of the staged and
            // cluster forms of the forward step)
            LV.ff_maxm.assign(LV.colour_ptr.size() - 1, 0);
            for (size_t c = 0; c + 1 < LV.colour_ptr.size(); c++) {
                const int a = LV.colour_ptr[c], b = LV.colour_ptr[c + 1];
                int mm = 0;
                for (int f = a; f < b; f++) mm = std::max(mm, sfronts[LV.front_begin + f].m);
                LV.ff_maxm[c] = mm;
            }
            // R_sj tiles of the backward step, planned for every level
            LV.bwd_tiles = LV.nfront > 0;
            if (LV.bwd_tiles) {
                LV.tile_begin = (int)tiles.size();
                LV.wf_begin = (int)wfr.size();
                int64_t zrows = 0;
                for (int f = LV.front_begin; f < LV.front_begin + LV.nfront; f++) {
                    const SolveFront<real>& sf = sfronts[f];
                    // pieces of R_sj columns filling chunks of kTileK columns
                    std::vector<std::pair<int, int>> chunks;
                    int cw = 0, cb = (int)pieces.size(), cn = 0;
                    for (int b = sf.rsj_begin; b < sf.rsj_begin + sf.nrsj; b++) {
                        const SolveRsj<real> R = srsj[b];
                        for (int u0 = 0; u0 < R.nj;) {
                            const int w = std::min(R.nj - u0, kTileK - cw);
                            pieces.push_back(SolveRsj<real>{R.R + (int64_t)u0 * R.ldr, R.ldr, w, 0, R.xoff + u0});
                            piece_src.push_back({b, u0});
                            cn++;
                            cw += w;
                            u0 += w;
                            if (cw == kTileK) {
                                chunks.push_back({cb, cn});
                                cb = (int)pieces.size();
                                cn = 0;
                                cw = 0;
                            }
                        }
                    }
                    if (cn > 0) chunks.push_back({cb, cn});
                    const int nkc = (int)chunks.size();
                    for (int kc = 0; kc < nkc; kc++)
                        for (int r0 = 0; r0 < sf.n; r0 += kTileRows)
                            tiles.push_back(RsjTile{f, r0, std::min(kTileRows, sf.n - r0), chunks[kc].first,
                                                    chunks[kc].second, kc, zrows});
                    wfr.push_back(WideFront{f, nkc, zrows});
                    zrows += (int64_t)nkc * sf.n;
                    double snj = 0;
                    for (int b = sf.rsj_begin; b < sf.rsj_begin + sf.nrsj; b++) snj += srsj[b].nj;
                    LV.rt_flops += 2.0 * sf.n * snj;
                    LV.rt_fixed += 8.0 * sf.n * snj;
                    LV.rt_vec += 8.0 * snj * ((sf.n + kTileRows - 1) / kTileRows) + 8.0 * nkc * sf.n;
                }
                LV.ntile = (int)tiles.size() - LV.tile_begin;
                // heaviest tiles first (rows x columns of their chunk)
                std::stable_sort(tiles.begin() + LV.tile_begin, tiles.end(), [&](const RsjTile& x, const RsjTile& y) {
                    auto w = [&](const RsjTile& t) {
                        int64_t c = 0;
                        for (int q = t.piece_begin; q < t.piece_begin + t.npiece; q++) c += pieces[q].nj;
                        return (int64_t)t.nrows * c;
                    };
                    return w(x) > w(y);
                });
                zp_max = std::max(zp_max, zrows);
            }
        };

        // ---------------- (ii)/(iii) scale and sparsify ----------------
        std::vector<int> rest;
        for (int i = 0; i < ncl; i++)
            if (!sp.is_front[i]) rest.push_back(i);
        const bool sparsify = (k + 1 > opt->skip) && !rest.empty();
        std::vector<int64_t> newsz(ncl, 0);
        std::vector<real*> uT(ncl, nullptr), uD(ncl, nullptr), qV(ncl, nullptr), qT(ncl, nullptr);
        std::vector<real*> uTau(ncl, nullptr), qTau(ncl, nullptr);   // scaling / CPQR Householder scalars
        std::vector<real*> hR(ncl, nullptr), hT(ncl, nullptr), hD(ncl, nullptr);   // unscaled form
        std::vector<int> hF(ncl, 0);
        std::vector<int> kmax(ncl, 0);
        if (sparsify) {
            const bool unscaled = opt->scaling == 0;
            double* sig = nullptr;
            if (!unscaled) {
                // scaling QR of every diagonal block
                int64_t ua = 0;
                for (int p : rest) ua += sz[p] + sz[p] * sz[p] + sz[p] * NB;
                real* uaux = C.alloc<real>(ua, true);
                if (C.rc) return C.rc;
                std::vector<QRTask<real>> sq;
                double fl_sq = 0, by_sq = 0, fl_sc = 0, by_sc = 0;
                int tm = 1;
                int64_t a = 0;
                for (int p : rest) {
                    real* tau = uaux + a;
                    uTau[p] = tau;
                    a += sz[p];
                    uT[p] = uaux + a;
                    a += sz[p] * sz[p];
                    uD[p] = uaux + a;
                    a += sz[p] * NB;
                    if (sz[p] == 0) continue;
                    const int e = sp.find(p, p);
                    if (e < 0) { set_error("interface without diagonal block"); return SPAQR_ERR_SINGULAR; }
                    sq.push_back(QRTask<real>{blk(e, p), lay.H[p], (int)sz[p], (int)sz[p], tau, uT[p], uD[p], d_flags + 1});
                    tm = std::max<int>(tm, (int)sz[p]);
                    flops += 4.0 / 3.0 * sz[p] * sz[p] * sz[p];
                    fl_sq += 4.0 / 3.0 * sz[p] * sz[p] * sz[p];
                    by_sq += 24.0 * sz[p] * sz[p];
                }
                // scaling of the off-diagonal blocks
                std::vector<ScaleTask<real>> sc;
                std::vector<int> sc_row;   // row interface of every task
                size_t smem_sc = 16;
                for (int j : rest) {
                    if (sz[j] == 0) continue;
                    const int ej = sp.diag[j];
                    for (int e = sp.colptr[j]; e < sp.colptr[j + 1]; e++) {
                        const int i = sp.rowidx[e];
                        if (i == j || sp.is_front[i] || sz[i] == 0) continue;
                        const int ei = sp.diag[i];
                        ScaleTask<real> t;
                        t.A = blk(e, j);
                        t.lda = lay.H[j];
                        t.mi = (int)sz[i];
                        t.nj = (int)sz[j];
                        t.Vi = blk(ei, i);
                        t.ldvi = lay.H[i];
                        t.Ti = uT[i];
                        t.Rj = blk(ej, j);
                        t.ldrj = lay.H[j];
                        t.Dj = uD[j];
                        t.q = QC;
                        smem_sc = (size_t)(2 * NB * QC + NT) * esz;
                        sc.push_back(t);
                        sc_row.push_back(i);
                        const double fs = 2.0 * sz[i] * sz[i] * sz[j] + 1.0 * sz[j] * sz[j] * sz[i];
                        flops += fs;
                        fl_sc += fs;
                        by_sc += 16.0 * sz[i] * sz[j] + 8.0 * sz[i] * sz[i] + 8.0 * sz[j] * sz[j];
                    }
                }
                tstart(1);
                if (!sq.empty()) {
                    launch_qr<real>(C, sq, esz, KK_SCALE_QR, fl_sq, by_sq);
                    if (C.rc) return C.rc;
                    C.launched();
                }
                if (!sc.empty()) {
                    // U^T over column chunks of every block, then R^{-1} over row
                    // chunks (the two products of a block are independent across
                    // columns and across rows respectively)
                    std::vector<ScalePiece> pl, pr;
                    for (int t = 0; t < (int)sc.size(); t++) {
                        for (int c0 = 0; c0 < sc[t].nj; c0 += QC) pl.push_back({t, c0, std::min(QC, sc[t].nj - c0)});
                        for (int r0 = 0; r0 < sc[t].mi; r0 += 64) pr.push_back({t, r0, std::min(64, sc[t].mi - r0)});
                    }
                    heaviest_first(pl, [&](const ScalePiece& c) { return (double)sc[c.task].mi * sc[c.task].mi * c.len; });
                    heaviest_first(pr, [&](const ScalePiece& c) { return (double)sc[c.task].nj * sc[c.task].nj * c.len; });
                    ScaleTask<real>* d = C.upload(sc, false);
                    ScalePiece* dl = C.upload(pl, false);
                    ScalePiece* dr = C.upload(pr, false);
                    if (C.rc) return C.rc;
                    bool tc_left = false;
                    if constexpr (sizeof(real) == 4) {
                        if (tcmode && tc_iface_level(rest, sz)) {
                            // rows i <- U_i^T (rows i) on the tensor cores:
                            // W = V_i^T A_ij, W <- T_i^T W, A_ij <- A_ij - V_i W,
                            // T_i the full compact-WY factor of U_i
                            tc_left = true;
                            std::vector<int64_t> toff(ncl, -1);
                            int64_t tot = 0;
                            std::vector<WySpec> ws;
                            // every row interface once
                            std::vector<char> seen(ncl, 0);
                            std::vector<int> rows_i;
                            for (int j : rest) {
                                if (sz[j] == 0) continue;
                                for (int e = sp.colptr[j]; e < sp.colptr[j + 1]; e++) {
                                    const int i = sp.rowidx[e];
                                    if (i == j || sp.is_front[i] || sz[i] == 0 || seen[i]) continue;
                                    seen[i] = 1;
                                    rows_i.push_back(i);
                                }
                            }
                            for (int i : rows_i) {
                                toff[i] = tot;
                                tot += sz[i] * sz[i] * 2 + sz[i] * NB;
                            }
                            int64_t wtot = 0;
                            for (const ScaleTask<real>& t : sc) wtot += 2 * (int64_t)t.mi * t.nj;
                            float* S = C.alloc<float>(tot + wtot, false);
                            if (C.rc) return C.rc;
                            for (int i : rows_i) {
                                const int ei = sp.find(i, i);
                                ws.push_back(WySpec{GemmOperand{blk(ei, i), lay.H[i], 1, 1, 1}, (int)sz[i], (int)sz[i],
                                                    uTau[i], S + toff[i], S + toff[i] + sz[i] * sz[i]});
                            }
                            int rc = tc_full_t(C, ws, KK_IFACE_TC, d_flags + 3);
                            if (rc != SPAQR_OK) return rc;
                            std::vector<GemmTask> g1, g2, g3;
                            int64_t wo = tot;
                            double fl_l = 0.0, by_l = 0.0;
                            for (size_t ti = 0; ti < sc.size(); ti++) {
                                const ScaleTask<real>& t = sc[ti];
                                const int i = sc_row[ti];
                                float* W = S + wo;
                                float* W2 = W + (int64_t)t.mi * t.nj;
                                wo += 2 * (int64_t)t.mi * t.nj;
                                GemmTask a{};
                                a.a = GemmOperand{t.Vi, t.ldvi, 1, 1, 1};
                                a.bt = GemmOperand{t.A, t.lda, 1, 0, 0};
                                a.c = W;
                                a.c_rs = 1;
                                a.c_cs = t.mi;
                                a.M = t.mi;
                                a.N = t.nj;
                                a.K = t.mi;
                                a.alpha = 1.0f;
                                a.beta = 0.0f;
                                g1.push_back(a);
                                a.a = GemmOperand{S + toff[i], t.mi, 1, 0, 0};
                                a.bt = GemmOperand{W, t.mi, 1, 0, 0};
                                a.c = W2;
                                g2.push_back(a);
                                a.a = GemmOperand{t.Vi, 1, t.ldvi, 1, 0};
                                a.bt = GemmOperand{W2, t.mi, 1, 0, 0};
                                a.c = t.A;
                                a.c_rs = 1;
                                a.c_cs = t.lda;
                                a.alpha = -1.0f;
                                a.beta = 1.0f;
                                g3.push_back(a);
                                fl_l += 2.0 * t.mi * t.mi * t.nj;
                                by_l += 16.0 * t.mi * t.nj + 8.0 * t.mi * t.mi;
                            }
                            rc = tc_batch(C, g1, tcmode == 1, KK_IFACE_TC, 0.0, 0.0, d_flags + 3);
                            if (rc == SPAQR_OK) rc = tc_batch(C, g2, tcmode == 1, KK_IFACE_TC, 0.0, 0.0, d_flags + 3);
                            if (rc == SPAQR_OK) rc = tc_batch(C, g3, tcmode == 1, KK_IFACE_TC, fl_l, by_l, d_flags + 3);
                            if (rc != SPAQR_OK) return rc;
                            fl_sc -= fl_l;
                            by_sc -= by_l;
                        }
                    }
                    if (!tc_left) {
                        SPAQR_LAUNCH(KK_SCALE_APPLY, fl_sc, by_sc, st,
                                     k_scale_apply<real><<<(unsigned)pl.size(), NT, smem_sc, st>>>(d, dl, 0));
                        C.launched();
                        fl_sc = 0.0;
                        by_sc = 0.0;
                    }
                    SPAQR_LAUNCH(KK_SCALE_APPLY, fl_sc, by_sc, st,
                                 k_scale_apply<real><<<(unsigned)pr.size(), NT, smem_sc, st>>>(d, dr, 1));
                    C.launched();
                }
                tstop(1);
            } else {
                // sigma_p = 1 / sigma_min(A_p), A_p = column p over all its
                // rows (Lemma 1): copy, Householder QR, Lanczos on (R^T R)^{-1}
                tstart(2);
                sig = C.alloc<double>(ncl, false);
                std::vector<int64_t> mp(ncl, 0), apo(ncl, 0);
                int64_t atot = 0, wtot = 0, qtot = 0;
                for (int p : rest) {
                    if (sz[p] == 0) continue;
                    if (sp.find(p, p) < 0) { set_error("interface without diagonal block"); return SPAQR_ERR_SINGULAR; }
                    for (int e = sp.colptr[p]; e < sp.colptr[p + 1]; e++)
                        if (!sp.is_front[sp.rowidx[e]]) mp[p] += sz[sp.rowidx[e]];
                    apo[p] = atot;
                    atot += mp[p] * sz[p];
                    wtot += (std::min<int64_t>(sz[p], kLanczosMax) + 3) * sz[p];
                    qtot += sz[p] + sz[p] * sz[p];
                }
                real* Ap = C.alloc<real>(atot, false);
                real* Aq = C.alloc<real>(qtot, false);
                double* lw = C.alloc<double>(wtot, false);
                if (C.rc) return C.rc;
                std::vector<SparsifyTask<real>> cpy;
                std::vector<QRTask<real>> aq;
                std::vector<SigmaTask<real>> sgt;
                double fl_a = 0, by_a = 0;
                int64_t qo = 0, wo = 0;
                for (int p : rest) {
                    if (sz[p] == 0) continue;
                    int64_t ro = 0;
                    for (int e = sp.colptr[p]; e < sp.colptr[p + 1]; e++) {
                        const int i = sp.rowidx[e];
                        if (sp.is_front[i] || sz[i] == 0) continue;
                        SparsifyTask<real> t;
                        std::memset(&t, 0, sizeof(t));
                        t.A = blk(e, p);
                        t.lda = lay.H[p];
                        t.mi = (int)sz[i];
                        t.nj = (int)sz[p];
                        t.D = Ap + apo[p] + ro;
                        t.ldd = mp[p];
                        t.mode = 2;
                        cpy.push_back(t);
                        ro += sz[i];
                    }
                    aq.push_back(QRTask<real>{Ap + apo[p], mp[p], (int)mp[p], (int)sz[p], Aq + qo,
                                              Aq + qo + sz[p], nullptr, d_flags + 1});
                    qo += sz[p] + sz[p] * sz[p];
                    const int km = (int)std::min<int64_t>(sz[p], kLanczosMax);
                    sgt.push_back(SigmaTask<real>{Ap + apo[p], mp[p], lw + wo, sig + p, d_flags + 1, (int)sz[p], km});
                    wo += (int64_t)(km + 3) * sz[p];
                    const double m_ = (double)mp[p], n_ = (double)sz[p];
                    flops += 2.0 * m_ * n_ * n_ - 2.0 / 3.0 * n_ * n_ * n_;
                    fl_a += 2.0 * m_ * n_ * n_ - 2.0 / 3.0 * n_ * n_ * n_;
                    by_a += 16.0 * m_ * n_;
                }
                if (!cpy.empty()) {
                    std::vector<ScalePiece> pc;
                    for (int t = 0; t < (int)cpy.size(); t++) pc.push_back({t, 0, 0});
                    SparsifyTask<real>* d = C.upload(cpy, false);
                    ScalePiece* dp = C.upload(pc, false);
                    if (C.rc) return C.rc;
                    SPAQR_LAUNCH(KK_SIGMA_QR, 0.0, by_a, st, k_sparsify<real><<<(unsigned)pc.size(), NT, 16, st>>>(d, dp, 0));
                    C.launched();
                    launch_qr<real>(C, aq, esz, KK_SIGMA_QR, fl_a, 0.0);
                    if (C.rc) return C.rc;
                    SigmaTask<real>* ds = C.upload(sgt, false);
                    if (C.rc) return C.rc;
                    SPAQR_LAUNCH(KK_SIGMA, 0.0, 0.0, st, k_sigma_min<real><<<(unsigned)sgt.size(), NT, 0, st>>>(ds));
                    C.launched();
                }
                tstop(2);
            }
            tstart(2);
            // CPQR of M_p
            std::vector<std::vector<std::pair<int, int>>> rowlist(ncl);   // row i -> (col j, entry)
            for (int j = 0; j < ncl; j++)
                for (int e = sp.colptr[j]; e < sp.colptr[j + 1]; e++) rowlist[sp.rowidx[e]].push_back({j, e});
            std::vector<CPQRTask<real>> cp, cpb;
            std::vector<GatherSeg<real>> gs;
            int nif = 0;   // interfaces of the level (CPQR units)
            for (int p : rest) nif += sz[p] > 0;
            int64_t mtot = 0, ntot = 0, vtot = 0, ttot = 0, rtot = 0, ptot = 0;
            std::vector<int> ncols(ncl, 0);
            for (int p : rest) {
                if (sz[p] == 0) continue;
                int nc = 0;
                for (int e = sp.colptr[p]; e < sp.colptr[p + 1]; e++) {
                    const int i = sp.rowidx[e];
                    if (i != p && !sp.is_front[i]) nc += (int)sz[i];
                }
                for (auto& je : rowlist[p]) {
                    const int j = je.first;
                    if (j != p && !sp.is_front[j]) {
                        nc += (int)sz[j];
                        ptot += sz[p] * sz[j];
                    }
                }
                ncols[p] = nc;
                kmax[p] = (int)std::min<int64_t>(sz[p], nc);
                mtot += sz[p] * nc;
                ntot += nc;
                vtot += sz[p] * kmax[p];
                ttot += (int64_t)kmax[p] * kmax[p] + kmax[p];
                rtot += kmax[p] + 1;
            }
            real* Mbuf = C.alloc<real>(mtot, false);
            real* Nbuf = C.alloc<real>(ntot, false);
            // unscaled form: the column-neighbour part of M_p is sigma_p A_pp^T A_pj
            real* Pbuf = unscaled ? C.alloc<real>(ptot, false) : nullptr;
            std::vector<AtbTask<real>> atb;
            int64_t po = 0;
            double fl_atb = 0, by_atb = 0;
            real* Vbuf = C.alloc<real>(vtot, true);
            real* Tbuf = C.alloc<real>(ttot, true);
            double* Rdg = C.alloc<double>(rtot, false);
            int* Rk = C.alloc<int>(ncl, false);
            if (C.rc) return C.rc;
            C.cuda(cudaMemsetAsync(Rk, 0, sizeof(int) * ncl, st));
            int64_t mo = 0, no = 0, vo = 0, to = 0, ro = 0;
            double by_cp = 16.0 * mtot;
            int kmx = 1, npmax = 1;
            std::vector<int64_t> rdg_off(ncl, 0);
            for (int p : rest) {
                if (sz[p] == 0) continue;
                CPQRTask<real> t;
                t.M = Mbuf + mo;
                t.norms = Nbuf + no;
                t.np = (int)sz[p];
                t.ncols = ncols[p];
                t.seg_begin = (int)gs.size();
                int co = 0;
                for (int e = sp.colptr[p]; e < sp.colptr[p + 1]; e++) {
                    const int i = sp.rowidx[e];
                    if (i == p || sp.is_front[i] || sz[i] == 0) continue;
                    gs.push_back(GatherSeg<real>{blk(e, p), lay.H[p], (int)sz[i], (int)sz[p], 1, co});
                    co += (int)sz[i];
                }
                const int epp = unscaled ? sp.find(p, p) : 0;
                if (epp < 0) { set_error("interface without diagonal block"); return SPAQR_ERR_SINGULAR; }
                for (auto& je : rowlist[p]) {
                    const int j = je.first;
                    if (j == p || sp.is_front[j] || sz[j] == 0) continue;
                    if (unscaled) {
                        atb.push_back(AtbTask<real>{blk(epp, p), blk(je.second, j), Pbuf + po, sig + p, lay.H[p],
                                                    lay.H[j], (int)sz[p], (int)sz[j]});
                        gs.push_back(GatherSeg<real>{Pbuf + po, sz[p], (int)sz[p], (int)sz[j], 0, co});
                        po += sz[p] * sz[j];
                        const double fa = 2.0 * sz[p] * sz[p] * sz[j];
                        flops += fa;
                        fl_atb += fa;
                        by_atb += 8.0 * (sz[p] * sz[p] + 2.0 * sz[p] * sz[j]);
                    } else {
                        gs.push_back(GatherSeg<real>{blk(je.second, j), lay.H[j], (int)sz[p], (int)sz[j], 0, co});
                    }
                    co += (int)sz[j];
                }
                t.nseg = (int)gs.size() - t.seg_begin;
                t.V = Vbuf + vo;
                t.kmax = kmax[p];
                t.tau = Tbuf + to;
                t.T = Tbuf + to + kmax[p];
                t.rdiag = Rdg + ro;
                t.rank = Rk + p;
                qV[p] = t.V;
                qT[p] = t.T;
                qTau[p] = t.tau;
                rdg_off[p] = ro;
                mo += sz[p] * ncols[p];
                no += ncols[p];
                vo += sz[p] * kmax[p];
                to += (int64_t)kmax[p] * kmax[p] + kmax[p];
                ro += kmax[p] + 1;
                kmx = std::max(kmx, kmax[p]);
                npmax = std::max(npmax, (int)sz[p]);
                // large interfaces go to the cluster kernel (cpqr_cs CTAs each),
                // and at levels with fewer interfaces than SMs every interface
                // with two or more columns per CTA of the cluster
                if (((int64_t)t.np * t.ncols >= kBigCPQR && t.ncols >= 512) ||
                    (nif <= kNumSM && t.ncols >= 2 * cpqr_cs<real>() && t.np >= 8))
                    cpb.push_back(t);
                else
                    cp.push_back(t);
            }
            if (!atb.empty()) {
                std::vector<ScalePiece> pc;
                for (int t = 0; t < (int)atb.size(); t++)
                    for (int c0 = 0; c0 < atb[t].nc; c0 += QC) pc.push_back({t, c0, std::min(QC, atb[t].nc - c0)});
                AtbTask<real>* d = C.upload(atb, false);
                ScalePiece* dp = C.upload(pc, false);
                if (C.rc) return C.rc;
                SPAQR_LAUNCH(KK_UNSCALED, fl_atb, by_atb, st, k_atb_sigma<real><<<(unsigned)pc.size(), NT, 0, st>>>(d, dp));
                C.launched();
            }
            const size_t smem_cp = (size_t)(RED + 2 * NWARP) * 8 + (size_t)(NB * NB + NB * NB / 2 + npmax) * esz;
            GatherSeg<real>* dgs = nullptr;
            if (!cp.empty() || !cpb.empty()) {
                dgs = C.upload(gs, false);
                if (C.rc) return C.rc;
            }
            if (!cpb.empty()) {
                heaviest_first(cpb, [](const CPQRTask<real>& t) { return (double)t.np * t.ncols * t.kmax; });
                CPQRTask<real>* d1 = C.upload(cpb, false);
                if (C.rc) return C.rc;
                SPAQR_LAUNCH(KK_CPQR, 0.0, by_cp, st,
                             k_cpqr_cluster<real, cpqr_cs<real>()><<<(unsigned)(cpb.size() * cpqr_cs<real>()), NT, smem_cp, st>>>(
                                 d1, dgs, opt->eps));
                C.launched();
                by_cp = 0.0;   // M_p's bytes are counted once per level
            }
            if (!cp.empty()) {
                heaviest_first(cp, [](const CPQRTask<real>& t) { return (double)t.np * t.ncols * t.kmax; });
                CPQRTask<real>* d1 = C.upload(cp, false);
                if (C.rc) return C.rc;
                SPAQR_LAUNCH(KK_CPQR, 0.0, by_cp, st,
                             k_cpqr<real><<<(unsigned)cp.size(), NT, smem_cp, st>>>(d1, dgs, opt->eps));
                C.launched();
            }
            plan_front_solve();
            // ranks back to the host (the only device->host sync of a level)
            std::vector<int> rk(ncl, 0);
            std::vector<double> rdg(std::max<int64_t>(rtot, 1), 0.0);
            C.cuda(cudaMemcpyAsync(rk.data(), Rk, sizeof(int) * ncl, cudaMemcpyDeviceToHost, st));
            if (rtot > 0) C.cuda(cudaMemcpyAsync(rdg.data(), Rdg, sizeof(double) * rtot, cudaMemcpyDeviceToHost, st));
            std::vector<double> sgh(ncl, 0.0);
            if (unscaled) C.cuda(cudaMemcpyAsync(sgh.data(), sig, sizeof(double) * ncl, cudaMemcpyDeviceToHost, st));
            tstop(2);
            C.cuda(cudaStreamSynchronize(st));
            if (C.rc) return C.rc;
            for (int p : rest) {
                newsz[p] = sz[p] == 0 ? 0 : rk[p];
                if (sz[p] == 0) continue;
                F->ranks[k].push_back({(int)sz[p], rk[p]});
                F->sigmas[k].push_back(sgh[p]);
                const double* rd = rdg.data() + rdg_off[p];
                const int r = rk[p];
                // pivot norms written by the CPQR: the r kept steps and the first rejected one
                const int npiv = kmax[p] == 0 ? 0 : (rd[0] == 0.0 ? 1 : std::min(r + 1, kmax[p]));
                F->pivots[k].insert(F->pivots[k].end(), rd, rd + npiv);
                F->pivot_off[k].push_back((int32_t)F->pivots[k].size());
                DG.n_interfaces++;
                const double rr = r < kmax[p] ? rd[r] : (r > 0 ? rd[r - 1] : 0.0);
                F->margins[k].push_back({rr, rd[0]});
                // r steps of reflection (4 (m-k)(c-k)) and norm recomputation (2 (m-k)(c-k))
                double fc = 0.0;
                for (int kk = 0; kk < r; kk++) fc += 6.0 * (double)(sz[p] - kk) * (double)(ncols[p] - kk);
                flops += fc;
                prof_add(-1, KK_CPQR, fc, 0.0);
            }
            if (unscaled) {
                // T_p = A_pp Q_p; Householder QR of its fine columns
                // T_p[:, r:] (H_p, R_ff); H_p^T on its coarse columns, whose top
                // f rows are R_fc and bottom r rows the new diagonal block
                // (Section 3.2).  T_p stays with the factor for the solve.
                tstart(2);
                int64_t tt = 0;
                for (int p : rest) {
                    if (sz[p] == 0) continue;
                    const int64_t f = sz[p] - newsz[p];
                    tt += sz[p] * sz[p] + f + f * f + f * NB;
                }
                real* tb = C.alloc<real>(tt, true);
                if (C.rc) return C.rc;
                std::vector<SparsifyTask<real>> cpy;
                std::vector<ReflTask<real>> rq, lh;
                std::vector<QRTask<real>> hq;
                std::vector<ScalePiece> prq, plh;
                double fl_t = 0, by_t = 0, fl_h = 0, by_h = 0;
                int64_t o2 = 0;
                for (int p : rest) {
                    if (sz[p] == 0) continue;
                    const int np_ = (int)sz[p], r = (int)newsz[p], f = np_ - r;
                    real* Tp = tb + o2;
                    o2 += (int64_t)np_ * np_;
                    hR[p] = Tp;
                    hT[p] = tb + o2 + f;
                    hD[p] = tb + o2 + f + (int64_t)f * f;
                    SparsifyTask<real> c;
                    std::memset(&c, 0, sizeof(c));
                    c.A = blk(sp.find(p, p), p);
                    c.lda = lay.H[p];
                    c.mi = np_;
                    c.nj = np_;
                    c.D = Tp;
                    c.ldd = np_;
                    c.mode = 2;
                    cpy.push_back(c);
                    if (r > 0) {
                        for (int r0 = 0; r0 < np_; r0 += QC) prq.push_back({(int)rq.size(), r0, std::min(QC, np_ - r0)});
                        rq.push_back(ReflTask<real>{qV[p], qT[p], Tp, np_, np_, np_, r, kmax[p], 1, 1, 0});
                        fl_t += 4.0 * np_ * np_ * r;
                        by_t += 16.0 * np_ * np_ + 8.0 * np_ * r;
                    }
                    if (f > 0) {
                        // the fine columns are often orthogonal to the first row of
                        // A_pp: a leading entry that is zero up to rounding takes
                        // beta = -norm, so that rounding does not pick the reflection
                        hq.push_back(QRTask<real>{Tp + (int64_t)r * np_, np_, np_, f, tb + o2, hT[p], hD[p], d_flags + 1,
                                                  sizeof(real) == 8 ? 1e-12 : 1e-5});
                        fl_h += 2.0 * np_ * f * f - 2.0 / 3.0 * f * f * f;
                        by_h += 16.0 * np_ * f;
                        if (r > 0) {
                            for (int c0 = 0; c0 < r; c0 += QC) plh.push_back({(int)lh.size(), c0, std::min(QC, r - c0)});
                            lh.push_back(ReflTask<real>{Tp + (int64_t)r * np_, hT[p], Tp, np_, np_, np_, f, f, 0, 0, 0});
                            fl_h += 4.0 * np_ * f * r;
                            by_h += 16.0 * np_ * r + 8.0 * np_ * f;
                        }
                    }
                    o2 += f + (int64_t)f * f + (int64_t)f * NB;
                    hF[p] = f;
                }
                flops += fl_t + fl_h;
                const size_t smem_rf = (size_t)(2 * NB * QC + NT) * esz;
                if (!cpy.empty()) {
                    std::vector<ScalePiece> pc;
                    for (int t = 0; t < (int)cpy.size(); t++) pc.push_back({t, 0, 0});
                    SparsifyTask<real>* d = C.upload(cpy, false);
                    ScalePiece* dp = C.upload(pc, false);
                    if (C.rc) return C.rc;
                    SPAQR_LAUNCH(KK_UNSCALED, 0.0, 0.0, st, k_sparsify<real><<<(unsigned)pc.size(), NT, 16, st>>>(d, dp, 0));
                    C.launched();
                }
                if (!rq.empty()) {
                    ReflTask<real>* d = C.upload(rq, false);
                    ScalePiece* dp = C.upload(prq, false);
                    if (C.rc) return C.rc;
                    SPAQR_LAUNCH(KK_UNSCALED, fl_t, by_t, st,
                                 k_refl_apply<real><<<(unsigned)prq.size(), NT, smem_rf, st>>>(d, dp));
                    C.launched();
                }
                if (!hq.empty()) {
                    launch_qr<real>(C, hq, esz, KK_UNSCALED, fl_h, by_h);
                    if (C.rc) return C.rc;
                }
                if (!lh.empty()) {
                    ReflTask<real>* d = C.upload(lh, false);
                    ScalePiece* dp = C.upload(plh, false);
                    if (C.rc) return C.rc;
                    SPAQR_LAUNCH(KK_UNSCALED, 0.0, 0.0, st,
                                 k_refl_apply<real><<<(unsigned)plh.size(), NT, smem_rf, st>>>(d, dp));
                    C.launched();
                }
                tstop(2);
            }
        } else {
            for (int p : rest) newsz[p] = sz[p];
        }

        for (int p : rest) {
            DG.n_remaining++;
            DG.remaining_size += sz[p];
            DG.interface_after += newsz[p];
            DG.max_interface = std::max<int>(DG.max_interface, (int)sz[p]);
        }

        if (!front_solve_planned) plan_front_solve();

        // ---------------- (iv) merge into the next level ----------------
        if (k < L - 1) {
            const StepPlan& sn = o.steps[k + 1];
            const int nn = (int)sn.cl.size();
            std::vector<int64_t> nsz(nn, 0), coff(ncl, 0);
            for (int p : rest) {
                const int J = sp.parent[p];
                coff[p] = nsz[J];
                nsz[J] += newsz[p];
            }
            LevelLayout nl;
            layout_of(sn, nsz, nl);
            real* narena = C.alloc<real>(nl.total, true);
            if (C.rc) return C.rc;
            tstart(3);
            C.cuda(cudaMemsetAsync(narena, 0, sizeof(real) * nl.total, st));
            std::vector<SparsifyTask<real>> sk;
            std::vector<std::pair<int, int>> sk_ij;   // (i, j) of every task
            if (sparsify) sk.reserve(sp.rowidx.size());
            int64_t scr = 0;
            double fl_sp = 0, by_sp = 0;
            if (!sparsify) {
                // copies only: per column chunk, its interface row segments
                // (adjacent ones joined)
                std::vector<CopyCol<real>> cc;
                std::vector<RowSeg> cs;
                constexpr int kCopyCols = 32;
                for (int j : rest) {
                    if (sz[j] == 0) continue;
                    const int J = sp.parent[j];
                    const int sb = (int)cs.size();
                    for (int e = sp.colptr[j]; e < sp.colptr[j + 1]; e++) {
                        const int i = sp.rowidx[e];
                        if (sp.is_front[i] || sz[i] == 0) continue;
                        const int e2 = sp.merge_e[e];
                        if (e2 < 0) { set_error("merged block missing"); return SPAQR_ERR_INVALID_ARG; }
                        const int64_t src = lay.rowoff[e], dst = nl.rowoff[e2] + coff[i];
                        if ((int)cs.size() > sb && cs.back().src + cs.back().len == src &&
                            cs.back().dst + cs.back().len == dst)
                            cs.back().len += (int)sz[i];
                        else
                            cs.push_back(RowSeg{src, dst, (int)sz[i], 0});
                        by_sp += 8.0 * sz[i] * sz[j] + 8.0;
                    }
                    const int ns = (int)cs.size() - sb;
                    if (ns == 0) continue;
                    const real* A0 = arena + lay.poff[j];
                    real* D0 = narena + nl.poff[J] + coff[j] * nl.H[J];
                    for (int64_t c0 = 0; c0 < sz[j]; c0 += kCopyCols)
                        cc.push_back(CopyCol<real>{A0 + c0 * lay.H[j], lay.H[j], D0 + c0 * nl.H[J], nl.H[J],
                                                   (int)std::min<int64_t>(kCopyCols, sz[j] - c0), sb, ns, 0});
                }
                if (!cc.empty()) {
                    CopyCol<real>* d = C.upload(cc, false);
                    RowSeg* dsg = C.upload(cs, false);
                    if (C.rc) return C.rc;
                    SPAQR_LAUNCH(KK_SPARSIFY, 0.0, by_sp, st,
                                 k_merge_copy<real><<<(unsigned)cc.size(), NT, 0, st>>>(d, dsg));
                    C.launched();
                }
            }
            for (int j : rest) {
                if (!sparsify) break;   // copies above
                for (int e = sp.colptr[j]; e < sp.colptr[j + 1]; e++) {
                    const int i = sp.rowidx[e];
                    if (sp.is_front[i]) continue;
                    const int I = sp.parent[i], J = sp.parent[j];
                    const int e2 = sp.merge_e[e];
                    if (e2 < 0) { set_error("merged block missing"); return SPAQR_ERR_INVALID_ARG; }
                    SparsifyTask<real> t;
                    std::memset(&t, 0, sizeof(t));
                    t.A = blk(e, j);
                    t.lda = lay.H[j];
                    t.mi = (int)sz[i];
                    t.nj = (int)sz[j];
                    t.D = narena + nl.poff[J] + nl.rowoff[e2] + coff[i] + coff[j] * nl.H[J];
                    t.ldd = nl.H[J];
                    if (i == j && opt->scaling == 0) {
                        // unscaled form: the coarse rows of H_p^T A_pp Q_p[:, 0:r]
                        if (newsz[i] == 0) continue;
                        t.mode = 2;
                        t.A = hR[i] + hF[i];
                        t.lda = sz[i];
                        t.mi = (int)newsz[i];
                        t.nj = (int)newsz[i];
                    } else if (i == j) {
                        if (newsz[i] == 0) continue;
                        t.mode = 1;
                        t.ri = (int)newsz[i];
                    } else {
                        if (newsz[i] == 0 || newsz[j] == 0) continue;
                        t.mode = 0;
                        if (opt->scaling == 0) {
                            // left: H_i^T (f_i reflectors), keep rows f_i..n_i
                            t.Vi = hR[i] + newsz[i] * sz[i];
                            t.Ti = hT[i];
                            t.ldti = std::max(hF[i], 1);
                            t.li = hF[i];
                            t.lkeep = hF[i];
                            t.lexp = 0;
                        } else {
                            // left: Q_i^T (r_i reflectors), keep rows 0..r_i
                            t.Vi = qV[i];
                            t.Ti = qT[i];
                            t.ldti = kmax[i];
                            t.li = (int)newsz[i];
                            t.lkeep = 0;
                            t.lexp = 1;
                        }
                        t.ri = (int)newsz[i];
                        t.Vj = qV[j];
                        t.Tj = qT[j];
                        t.rj = (int)newsz[j];
                        t.ldtj = kmax[j];
                        t.scratch = (real*)(intptr_t)scr;  // offset, fixed below
                        scr += (int64_t)t.mi * t.nj;
                        const double fp = 4.0 * t.li * t.mi * t.nj + 4.0 * t.rj * t.nj * t.ri;
                        flops += fp;
                        fl_sp += fp;
                    }
                    by_sp += 8.0 * t.mi * t.nj + 8.0 * std::max(t.ri, 1) * std::max(t.rj, 1);
                    sk.push_back(t);
                    sk_ij.push_back({i, j});
                }
            }
            bool tc_sp = false;
            if constexpr (sizeof(real) == 4) {
                if (!sk.empty() && sparsify && tcmode && opt->scaling != 0 && tc_iface_level(rest, sz)) {
                    // coarse blocks on the tensor cores: X = (Q_i^T A_ij)[0:r_i, :]
                    // as A - V_i T_i^T (V_i^T A) on the kept rows (in place in the
                    // level's arena), then X Q_j on the kept columns,
                    // X - (X V_j) T_j V_j[0:r_j, :]^T, and a copy into the merged
                    // block; T_i, T_j the full compact-WY factors of the CPQRs
                    tc_sp = true;
                    std::vector<int64_t> toff(ncl, -1);
                    int64_t tot = 0;
                    for (int q : rest)
                        if (sz[q] > 0 && newsz[q] > 0) {
                            toff[q] = tot;
                            tot += newsz[q] * newsz[q] * 2 + newsz[q] * NB;
                        }
                    int64_t wtot = 0;
                    for (const SparsifyTask<real>& t : sk)
                        if (t.mode == 0) wtot += 2 * (int64_t)t.ri * t.nj + 2 * (int64_t)t.ri * t.rj;
                    float* S = C.alloc<float>(tot + wtot, false);
                    if (C.rc) return C.rc;
                    std::vector<WySpec> ws;
                    std::vector<const float*> tq(ncl, nullptr);
                    for (int q : rest)
                        if (toff[q] >= 0) {
                            ws.push_back(WySpec{GemmOperand{qV[q], sz[q], 1, 0, 0}, (int)sz[q], (int)newsz[q], qTau[q],
                                                S + toff[q], S + toff[q] + newsz[q] * newsz[q]});
                            tq[q] = S + toff[q];
                        }
                    int rc = tc_full_t(C, ws, KK_IFACE_TC, d_flags + 3);
                    if (rc != SPAQR_OK) return rc;
                    std::vector<GemmTask> g[6];
                    std::vector<SparsifyTask<real>> rest_tasks;
                    int64_t wo = tot;
                    double fl_t = 0.0;
                    for (size_t ti = 0; ti < sk.size(); ti++) {
                        const SparsifyTask<real>& t = sk[ti];
                        if (t.mode != 0) {
                            rest_tasks.push_back(t);
                            continue;
                        }
                        // the interfaces of this block
                        const int ii = sk_ij[ti].first, jj = sk_ij[ti].second;
                        if (!tq[ii] || !tq[jj]) {
                            set_error("sparsification task without its interfaces");
                            return SPAQR_ERR_INVALID_ARG;
                        }
                        const int mi = t.mi, nj = t.nj, ri = t.ri, rj = t.rj;
                        float* W = S + wo;
                        float* W2 = W + (int64_t)ri * nj;
                        float* W3 = W2 + (int64_t)ri * nj;
                        float* W4 = W3 + (int64_t)ri * rj;
                        wo += 2 * (int64_t)ri * nj + 2 * (int64_t)ri * rj;
                        float* Ab = const_cast<float*>(t.A);
                        auto task = [](GemmOperand a, GemmOperand bt, float* c, int64_t crs, int64_t ccs, int M, int N,
                                       int K, float alpha, float beta) {
                            GemmTask x{};
                            x.a = a;
                            x.bt = bt;
                            x.c = c;
                            x.c_rs = crs;
                            x.c_cs = ccs;
                            x.M = M;
                            x.N = N;
                            x.K = K;
                            x.alpha = alpha;
                            x.beta = beta;
                            return x;
                        };
                        g[0].push_back(task({t.Vi, mi, 1, 0, 0}, {t.A, t.lda, 1, 0, 0}, W, 1, ri, ri, nj, mi, 1.f, 0.f));
                        g[1].push_back(task({tq[ii], ri, 1, 0, 0}, {W, ri, 1, 0, 0}, W2, 1, ri, ri, nj, ri, 1.f, 0.f));
                        g[2].push_back(task({t.Vi, 1, mi, 0, 0}, {W2, ri, 1, 0, 0}, Ab, 1, t.lda, ri, nj, ri, -1.f, 1.f));
                        g[3].push_back(task({t.A, 1, t.lda, 0, 0}, {t.Vj, nj, 1, 0, 0}, W3, 1, ri, ri, rj, nj, 1.f, 0.f));
                        g[4].push_back(task({W3, 1, ri, 0, 0}, {tq[jj], rj, 1, 0, 0}, W4, 1, ri, ri, rj, rj, 1.f, 0.f));
                        g[5].push_back(task({W4, 1, ri, 0, 0}, {t.Vj, 1, nj, 0, 0}, Ab, 1, t.lda, ri, rj, rj, -1.f, 1.f));
                        SparsifyTask<real> cp = t;
                        cp.mode = 2;
                        cp.mi = ri;
                        cp.nj = rj;
                        rest_tasks.push_back(cp);
                        fl_t += 4.0 * t.li * mi * nj + 4.0 * rj * nj * ri;
                    }
                    for (int b = 0; b < 6 && rc == SPAQR_OK; b++)
                        rc = tc_batch(C, g[b], tcmode == 1, KK_IFACE_TC, b == 5 ? fl_t : 0.0, 0.0, d_flags + 3);
                    if (rc != SPAQR_OK) return rc;
                    if (!rest_tasks.empty()) {
                        std::vector<ScalePiece> pc;
                        for (int t = 0; t < (int)rest_tasks.size(); t++) pc.push_back({t, 0, 0});
                        SparsifyTask<real>* d = C.upload(rest_tasks, false);
                        ScalePiece* dp = C.upload(pc, false);
                        if (C.rc) return C.rc;
                        SPAQR_LAUNCH(KK_SPARSIFY, fl_sp - fl_t, by_sp, st,
                                     k_sparsify<real><<<(unsigned)pc.size(), NT, 16, st>>>(d, dp, 0));
                        C.launched();
                    }
                }
            }
            if (!sk.empty() && !tc_sp) {
                real* sbuf = C.alloc<real>(scr, false);
                if (C.rc) return C.rc;
                for (SparsifyTask<real>& t : sk)
                    if (t.mode == 0) t.scratch = sbuf + (int64_t)(intptr_t)t.scratch;
                // Q_i^T over column chunks (copies and identities: one piece
                // each), then Q_j over chunks of the r_i coarse rows, the only
                // rows of Q_i^T A_ij the coarse block keeps
                std::vector<ScalePiece> pl, pr;
                for (int t = 0; t < (int)sk.size(); t++) {
                    if (sk[t].mode != 0) {
                        pl.push_back({t, 0, 0});
                        continue;
                    }
                    for (int c0 = 0; c0 < sk[t].nj; c0 += QC) pl.push_back({t, c0, std::min(QC, sk[t].nj - c0)});
                    for (int r0 = 0; r0 < sk[t].ri; r0 += 32) pr.push_back({t, r0, std::min(32, sk[t].ri - r0)});
                }
                heaviest_first(pl, [&](const ScalePiece& c) {
                    const SparsifyTask<real>& t = sk[c.task];
                    return t.mode == 0 ? (double)t.li * t.mi * c.len : (double)t.mi * t.nj / 16.0;
                });
                heaviest_first(pr, [&](const ScalePiece& c) { return (double)sk[c.task].rj * sk[c.task].nj * c.len; });
                SparsifyTask<real>* d = C.upload(sk, false);
                ScalePiece* dl = C.upload(pl, false);
                ScalePiece* dr = C.upload(pr, false);
                if (C.rc) return C.rc;
                const size_t smem_sp = (size_t)(2 * NB * QC + NT) * esz;
                SPAQR_LAUNCH(KK_SPARSIFY, fl_sp, by_sp, st,
                             k_sparsify<real><<<(unsigned)pl.size(), NT, smem_sp, st>>>(d, dl, 0));
                C.launched();
                if (!pr.empty()) {
                    SPAQR_LAUNCH(KK_SPARSIFY, 0.0, 0.0, st,
                                 k_sparsify<real><<<(unsigned)pr.size(), NT, smem_sp, st>>>(d, dr, 1));
                    C.launched();
                }
            }
            tstop(3);
            // solve record of the surviving clusters
            LV.ss_begin = (int)sss.size();
            for (int p : rest) {
                SolveSS<real> s;
                std::memset(&s, 0, sizeof(s));
                s.off = lay.voff[p];
                s.noff = nl.voff[sp.parent[p]] + coff[p];
                s.np = (int)sz[p];
                s.r = (int)newsz[p];
                if (sparsify && sz[p] > 0 && opt->scaling == 0) {
                    // unscaled form: forward H_p^T; backward R_ff^{-1} (y_f - R_fc x_c), then Q_p
                    const int f = hF[p];
                    s.QV = qV[p];
                    s.QT = qT[p];
                    s.ldqt = std::max(kmax[p], 1);
                    s.f = f;
                    s.HR = hR[p];
                    s.HT = hT[p];
                    s.HD = hD[p];
                    const double n_ = (double)sz[p], r_ = (double)newsz[p], f_ = (double)f;
                    sflops += 4.0 * n_ * f_ - 2.0 * f_ * f_ + 2.0 * f_ * r_ + f_ * f_ + 4.0 * n_ * r_ - 2.0 * r_ * r_;
                    sbytes += 8 * (int64_t)(n_ * f_ + f_ * r_ + f_ * f_ + n_ * r_);
                    LV.ssf_flops += 4.0 * n_ * f_ - 2.0 * f_ * f_;
                    LV.ssf_fixed += 8.0 * (n_ * f_ + f_ * f_);
                    LV.ssb_flops += 2.0 * f_ * r_ + f_ * f_ + 4.0 * n_ * r_ - 2.0 * r_ * r_;
                    LV.ssb_fixed += 8.0 * (f_ * r_ + f_ * f_ + n_ * r_ + r_ * r_);
                } else if (sparsify && sz[p] > 0) {
                    const int e = sp.find(p, p);
                    s.UV = blk(e, p);
                    s.lduv = lay.H[p];
                    s.UT = uT[p];
                    s.UD = uD[p];
                    s.QV = qV[p];
                    s.QT = qT[p];
                    s.ldqt = std::max(kmax[p], 1);
                    {
                        const double n_ = (double)sz[p], r_ = (double)newsz[p];
                        sflops += 2.0 * n_ * n_ + 2.0 * (4.0 * n_ * r_ - 2.0 * r_ * r_) + n_ * n_;
                    }
                    sbytes += 8 * (2 * sz[p] * sz[p] + sz[p] * newsz[p]);
                    const double n_ = (double)sz[p], r_ = (double)newsz[p];
                    // U_pp^T (n reflectors of n rows), then Q_pp^T (r reflectors)
                    LV.ssf_flops += 2.0 * n_ * n_ + 4.0 * n_ * r_ - 2.0 * r_ * r_;
                    LV.ssf_fixed += 8.0 * (2.0 * n_ * n_ + n_ * r_ + r_ * r_);
                    // Q_pp, then R_pp^{-1}
                    LV.ssb_flops += 4.0 * n_ * r_ - 2.0 * r_ * r_ + n_ * n_;
                    LV.ssb_fixed += 8.0 * (n_ * n_ + n_ * r_ + r_ * r_);
                }
                LV.ssf_vec += 16.0 * sz[p] + 8.0 * newsz[p];
                LV.ssb_vec += 16.0 * sz[p] + 8.0 * newsz[p];
                sss.push_back(s);
                ss_cl.push_back(sp.cl[p]);
                LV.max_ss_n = std::max(LV.max_ss_n, s.np);
                LV.max_ss_r = std::max(LV.max_ss_r, s.r);
            }
            LV.nss = (int)sss.size() - LV.ss_begin;
            {
                // heaviest interfaces first (disjoint rows: any order)
                const int a = LV.ss_begin, b = (int)sss.size();
                std::vector<int> idx(b - a);
                for (int u = 0; u < b - a; u++) idx[u] = a + u;
                std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
                    return (int64_t)sss[x].np * sss[x].np > (int64_t)sss[y].np * sss[y].np;
                });
                std::vector<SolveSS<real>> s2(b - a);
                std::vector<int> c2(b - a);
                for (int u = 0; u < b - a; u++) {
                    s2[u] = sss[idx[u]];
                    c2[u] = ss_cl[idx[u]];
                }
                std::copy(s2.begin(), s2.end(), sss.begin() + a);
                std::copy(c2.begin(), c2.end(), ss_cl.begin() + a);
            }
            compact_level(k, arena, piece_begin);
            if (C.rc) return C.rc;
            DG.factor_bytes = F->bytes;
            C.free_temps();
            sz = nsz;
            lay = nl;
            arena = narena;
        } else {
            LV.ss_begin = (int)sss.size();
            LV.nss = 0;
            compact_level(k, arena, piece_begin);
            if (C.rc) return C.rc;
            DG.factor_bytes = F->bytes;
            C.free_temps();
        }
    }
    // index of the stored blocks (final device locations, after the
    // per-level compaction)
    for (int k = 0; k < L; k++) {
        const SolveLevelHost& LVk = F->lv[k];
        for (int f = LVk.front_begin; f < LVk.front_begin + LVk.nfront; f++) {
            const SolveFront<real>& sf = sfronts[f];
            const int c = front_cl[f];
            F->blocks.push_back({k, SPAQR_BLK_FRONT, c, -1, sf.m, sf.n, sf.V, sf.ldv, 1});
            F->blocks.push_back({k, SPAQR_BLK_FRONT_TAU, c, -1, sf.n, 1, sf.T, sf.n, (int64_t)sf.n + 1});
            for (int b = sf.rsj_begin; b < sf.rsj_begin + sf.nrsj; b++)
                F->blocks.push_back({k, SPAQR_BLK_RSJ, c, rsj_cl[b], sf.n, srsj[b].nj, srsj[b].R, srsj[b].ldr, 1});
        }
        for (int q = LVk.ss_begin; q < LVk.ss_begin + LVk.nss; q++) {
            const SolveSS<real>& s = sss[q];
            const int c = ss_cl[q];
            if (s.UV) {
                F->blocks.push_back({k, SPAQR_BLK_SCALE, c, -1, s.np, s.np, s.UV, s.lduv, 1});
                F->blocks.push_back({k, SPAQR_BLK_SCALE_TAU, c, -1, s.np, 1, s.UT, s.np, (int64_t)s.np + 1});
            }
            if (s.QV && s.r > 0) {
                F->blocks.push_back({k, SPAQR_BLK_CPQR, c, -1, s.np, s.r, s.QV, s.np, 1});
                F->blocks.push_back({k, SPAQR_BLK_CPQR_TAU, c, -1, s.r, 1, s.QT, s.ldqt, (int64_t)s.ldqt + 1});
            }
            if (s.HR) {
                F->blocks.push_back({k, SPAQR_BLK_FINE, c, -1, s.np, s.np, s.HR, s.np, 1});
                if (s.f > 0)
                    F->blocks.push_back({k, SPAQR_BLK_FINE_TAU, c, -1, s.f, 1, s.HT, s.f, (int64_t)s.f + 1});
            }
        }
    }
    // upload the solve plan
    F->d_fronts = C.upload(sfronts, true);
    F->d_segs = C.upload(ssegs, true);
    F->d_rsj = C.upload(srsj, true);
    F->d_ss = C.upload(sss, true);
    F->d_tiles = C.upload(tiles, true);
    F->d_pieces = C.upload(pieces, true);
    F->d_wfronts = C.upload(wfr, true);
    F->zp_off = ws;
    F->zp_rows = zp_max;
    ws += zp_max;
    F->ws_rows = ws;
    F->flops = flops;
    F->solve_flops = sflops;
    F->solve_bytes = sbytes;
    int flags[4] = {0, 0, 0, 0};
    C.cuda(cudaMemcpyAsync(flags, d_flags, sizeof(flags), cudaMemcpyDeviceToHost, st));
    C.cuda(cudaStreamSynchronize(st));
    C.free_temps();
    C.cuda(cudaStreamSynchronize(st));
    tl_stage.grow();   // every staged copy has completed
    if (C.rc) return C.rc;
    for (Timer& t : timers) {
        float ms = 0.0f;
        if (t.ph >= 0 && cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            F->phase_ms[t.ph] += ms;
            if (t.lev >= 0) F->ldiag[t.lev].phase_ms[t.ph] += ms;
        }
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    if (flags[0]) { set_error("matrix has a zero column"); return SPAQR_ERR_SINGULAR; }
    if (flags[1]) {
        set_error(opt->scaling ? "zero diagonal in a scaling factor R_pp"
                               : "zero diagonal in R of A_p or in R_ff (unscaled sparsification)");
        return SPAQR_ERR_SINGULAR;
    }
    if (flags[2]) { set_error("zero diagonal in a separator factor R_ss"); return SPAQR_ERR_SINGULAR; }
    if (flags[3]) { set_error("a bounded tensor-core wait ran out"); return SPAQR_ERR_TIMEOUT; }
    return SPAQR_OK;
}

template int run_factor<double>(const Ordering&, const spaqr_csr*, const spaqr_opts*, spaqr_factor_s*);
template int run_factor<float>(const Ordering&, const spaqr_csr*, const spaqr_opts*, spaqr_factor_s*);

}  // namespace spaqr

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" int spaqr_factor(const spaqr_ordering* ord, const spaqr_csr* A, const spaqr_opts* opts,
                            spaqr_factor_t** out) {
    using namespace spaqr;
    if (!out) { set_error("out is NULL"); return SPAQR_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!ord || !A || !opts) { set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    if (A->n != ord->o.n || A->nnz != ord->o.nnz || !A->val) {
        set_error("matrix does not match the ordering's pattern");
        return SPAQR_ERR_INVALID_ARG;
    }
    if (check_csr_location(A) != SPAQR_OK) return SPAQR_ERR_INVALID_ARG;
    if (!(opts->eps >= 0.0) || opts->skip < 0) { set_error("eps must be >= 0 and skip >= 0"); return SPAQR_ERR_INVALID_ARG; }
    if (opts->nlevels != 0 && opts->nlevels != ord->o.L) {
        set_error("opts.nlevels differs from the ordering's level count");
        return SPAQR_ERR_INVALID_ARG;
    }
    if (opts->scaling != 0 && opts->scaling != 1) { set_error("scaling must be 0 or 1"); return SPAQR_ERR_INVALID_ARG; }
    if (opts->precision != SPAQR_FP64 && opts->precision != SPAQR_FP32 && opts->precision != SPAQR_TF32) {
        set_error("precision must be SPAQR_FP64, SPAQR_FP32 or SPAQR_TF32");
        return SPAQR_ERR_UNSUPPORTED;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        set_error("no CUDA device");
        return SPAQR_ERR_NO_DEVICE;
    }
    int curdev = 0;
    if (cudaGetDevice(&curdev) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaGetDevice failed");
        return SPAQR_ERR_CUDA;
    }
    if (check_csr_device(A, curdev) != SPAQR_OK) return SPAQR_ERR_INVALID_ARG;
    spaqr_factor_s* F = new (std::nothrow) spaqr_factor_s();
    if (!F) { set_error("host allocation failed"); return SPAQR_ERR_OOM; }
    F->device = curdev;
    keep_pool_memory(F->device);
    int rc;
    try {
        rc = opts->precision != SPAQR_FP64 ? run_factor<float>(ord->o, A, opts, F)
                                           : run_factor<double>(ord->o, A, opts, F);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        rc = SPAQR_ERR_OOM;
    }
    if (rc != SPAQR_OK) {
        cudaStreamSynchronize((cudaStream_t)opts->stream);
        spaqr_factor_destroy(F);
        return rc;
    }
    *out = F;
    return SPAQR_OK;
}

extern "C" void spaqr_factor_destroy(spaqr_factor_t* F) {
    if (!F) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(F->device);
    cudaDeviceSynchronize();
    for (void* p : F->allocs) cudaFree(p);
    cudaSetDevice(cur);
    delete F;
}

extern "C" int spaqr_factor_nblocks(const spaqr_factor_t* F, int64_t* count) {
    if (!F || !count) { spaqr::set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    *count = (int64_t)F->blocks.size();
    return SPAQR_OK;
}

extern "C" int spaqr_factor_block(const spaqr_factor_t* F, int64_t index, spaqr_block_info* info, double* out) {
    using namespace spaqr;
    if (!F || !info) { set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    if (index < 0 || index >= (int64_t)F->blocks.size()) { set_error("block index out of range"); return SPAQR_ERR_INVALID_ARG; }
    const BlockRec& b = F->blocks[(size_t)index];
    info->level = b.level;
    info->kind = b.kind;
    info->cluster = b.cluster;
    info->other = b.other;
    info->rows = b.rows;
    info->cols = b.cols;
    if (!out || b.rows == 0 || b.cols == 0) return SPAQR_OK;
    const size_t esz = (size_t)F->esz;
    std::vector<char> tmp((size_t)b.rows * b.cols * esz);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); cur = -1; }
    if (cur != F->device) cudaSetDevice(F->device);
    cudaError_t e;
    if (b.rstride == 1)
        e = cudaMemcpy2D(tmp.data(), b.rows * esz, b.ptr, (size_t)b.ld * esz, b.rows * esz, (size_t)b.cols,
                         cudaMemcpyDeviceToHost);
    else
        e = cudaMemcpy2D(tmp.data(), esz, b.ptr, (size_t)b.rstride * esz, esz, (size_t)b.rows, cudaMemcpyDeviceToHost);
    if (cur >= 0 && cur != F->device) cudaSetDevice(cur);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("CUDA: ") + cudaGetErrorString(e));
        return SPAQR_ERR_CUDA;
    }
    const size_t cnt = (size_t)b.rows * b.cols;
    if (esz == 8) {
        std::memcpy(out, tmp.data(), cnt * 8);
    } else {
        const float* f = reinterpret_cast<const float*>(tmp.data());
        for (size_t i = 0; i < cnt; i++) out[i] = (double)f[i];
    }
    return SPAQR_OK;
}

extern "C" int spaqr_factor_info(const spaqr_factor_t* F, spaqr_info* out) {
    if (!F || !out) { spaqr::set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    std::memset(out, 0, sizeof(*out));
    out->n = F->n;
    out->nlevels = F->L;
    out->skip = F->skip;
    out->eps = F->eps;
    out->factor_bytes = F->bytes;
    out->solve_bytes = F->solve_bytes + 16 * F->n;
    out->factor_flops = F->flops;
    out->solve_flops = F->solve_flops;
    for (auto& lvl : F->ranks)
        for (auto& pr : lvl) {
            out->n_interfaces_sparsified++;
            out->rank_sum += pr.second;
            out->size_sum += pr.first;
        }
    for (int i = 0; i < 4; i++) out->phase_ms[i] = F->phase_ms[i];
    out->top_size = F->top_size;
    out->peak_bytes = F->peak_bytes;
    out->workspace_rows = F->ws_rows;
    out->precision = F->precision;
    out->tc_levels = F->tc_levels;
    return SPAQR_OK;
}

extern "C" int spaqr_factor_level(const spaqr_factor_t* F, int level, spaqr_level_info* out) {
    if (!F || !out) { spaqr::set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    if (level < 0 || level >= (int)F->ldiag.size()) { spaqr::set_error("level out of range"); return SPAQR_ERR_INVALID_ARG; }
    const LevelDiag& d = F->ldiag[level];
    out->n_fronts = d.n_fronts;
    out->max_front_rows = d.max_front_rows;
    out->max_front_cols = d.max_front_cols;
    out->n_interfaces = d.n_interfaces;
    out->front_rows = d.front_rows;
    out->front_cols = d.front_cols;
    out->n_remaining = d.n_remaining;
    out->max_interface = d.max_interface;
    out->remaining_size = d.remaining_size;
    out->interface_after = d.interface_after;
    out->block_entries = d.block_entries;
    out->factor_bytes = d.factor_bytes;
    for (int i = 0; i < 4; i++) out->phase_ms[i] = d.phase_ms[i];
    return SPAQR_OK;
}

extern "C" int spaqr_factor_pivots(const spaqr_factor_t* F, int level, double* norms, int64_t cap,
                                   int32_t* offsets, int cap_offsets, int64_t* n_norms, int* n_interfaces) {
    if (!F || !n_norms || !n_interfaces) { spaqr::set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    if (level < 0 || level >= (int)F->pivots.size()) { spaqr::set_error("level out of range"); return SPAQR_ERR_INVALID_ARG; }
    const auto& P = F->pivots[level];
    const auto& O = F->pivot_off[level];
    *n_norms = (int64_t)P.size();
    *n_interfaces = (int)O.size() - 1;
    if (norms)
        for (int64_t i = 0; i < std::min<int64_t>(cap, (int64_t)P.size()); i++) norms[i] = P[i];
    if (offsets)
        for (int i = 0; i < std::min<int>(cap_offsets, (int)O.size()); i++) offsets[i] = O[i];
    return SPAQR_OK;
}

extern "C" int spaqr_factor_sigmas(const spaqr_factor_t* F, int level, double* sigma, int cap, int* count) {
    if (!F || !count) { spaqr::set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    if (level < 0 || level >= (int)F->sigmas.size()) { spaqr::set_error("level out of range"); return SPAQR_ERR_INVALID_ARG; }
    const auto& S = F->sigmas[level];
    *count = (int)S.size();
    if (sigma)
        for (int i = 0; i < std::min<int>(cap, (int)S.size()); i++) sigma[i] = S[i];
    return SPAQR_OK;
}

extern "C" int spaqr_factor_ranks(const spaqr_factor_t* F, int level, int32_t* pairs, double* margins,
                                  int cap, int* count) {
    if (!F || !count) { spaqr::set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    if (level < 0 || level >= (int)F->ranks.size()) { spaqr::set_error("level out of range"); return SPAQR_ERR_INVALID_ARG; }
    const auto& R = F->ranks[level];
    *count = (int)R.size();
    const int m = std::min<int>(cap, (int)R.size());
    for (int i = 0; i < m; i++) {
        if (pairs) { pairs[2 * i] = R[i].first; pairs[2 * i + 1] = R[i].second; }
        if (margins) { margins[2 * i] = F->margins[level][i].first; margins[2 * i + 1] = F->margins[level][i].second; }
    }
    return SPAQR_OK;
}
