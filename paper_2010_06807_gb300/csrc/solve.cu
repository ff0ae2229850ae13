// Application of the spaQR factor (Section 2.7) and right-preconditioned
// GMRES (Section 4) on the GPU.
//
// With left operations L_1..L_K (H_s^T on front rows, U_p^T, Q_p^T) and right
// operations C_1..C_K (R_s^{-1}, R_p^{-1}, Q_p) recorded in factor order,
// L_K ... L_1 A D C_1 ... C_K ~ I, so x = D C_1 (C_2 (... C_K (L_K ... L_1 b))).
//   forward  (leaves -> root): fronts (by colour), then per surviving cluster
//            y_p <- Q_p^T U_p^T y_p; the coarse part moves into the merged
//            cluster of the next level, the fine part stays (its block is I);
//   backward (root -> leaves): coarse part back, x_p <- R_p^{-1} Q_p [x_c; x_f],
//            then x_s <- R_ss^{-1} (z_s - sum_j R_sj x_j) for every front.
// Each level has its own vector (rows = sizes of its clusters), all in one
// workspace, column-major with one column per right-hand side.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>
#include <limits>

#include "dense.cuh"
#include "spaqr_internal.h"
#include "tasks.h"

#define SPAQR_LAUNCH(kind, flops, bytes, stream, ...)                            \
    do {                                                                         \
        const int rec_ = prof_begin((void*)(stream), (kind), (flops), (bytes)); \
        __VA_ARGS__;                                                             \
        prof_end((void*)(stream), rec_);                                         \
    } while (0)

namespace spaqr {

// Level-1 vector <- permuted right-hand sides (rounded to the factor's type).
template <class real>
__global__ void k_perm_in(int64_t n, int nrhs, const int64_t* __restrict__ perm, const double* __restrict__ B,
                          int64_t ldb, real* __restrict__ Y, int64_t ldy) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t g = perm[i];
    for (int c = 0; c < nrhs; c++) Y[i + c * ldy] = (real)B[g + c * ldb];
}

// X <- D (permuted back) level-1 vector, in FP64.
template <class real>
__global__ void k_perm_out(int64_t n, int nrhs, const int64_t* __restrict__ perm, const double* __restrict__ d,
                           const real* __restrict__ Y, int64_t ldy, double* __restrict__ X, int64_t ldx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t g = perm[i];
    const double s = d[g];
    for (int c = 0; c < nrhs; c++) X[g + c * ldx] = s * (double)Y[i + c * ldy];
}

// The right-hand sides of a launch are split into blockIdx.y chunks of qs
// columns, so that levels with few fronts still occupy many SMs.
__device__ __forceinline__ bool rhs_chunk(int nrhs, int qs, int& c0, int& qn) {
    c0 = blockIdx.y * qs;
    qn = nrhs - c0 < qs ? nrhs - c0 : qs;
    return qn > 0;
}

template <class real>
__global__ void __launch_bounds__(NT) k_sfront_fwd(const SolveFront<real>* __restrict__ fr,
                                                   const Seg* __restrict__ segs, real* Y, int64_t ldy, int nrhs,
                                                   int qs, int rmap_doubles, int staged) {
    extern __shared__ double sm[];
    int* rmap = reinterpret_cast<int*>(sm);
    real* W = reinterpret_cast<real*>(sm + rmap_doubles);
    int c0, qn;
    if (!rhs_chunk(nrhs, qs, c0, qn)) return;
    const SolveFront<real> F = fr[blockIdx.x];
    for (int s = threadIdx.x; s < F.nseg; s += NT) {   // a segment per thread
        const Seg g = segs[F.seg_begin + s];
        for (int r = 0; r < g.len; r++) rmap[g.pos + r] = (int)(g.off + r);
    }
    __syncthreads();
    const Mat<real> B{Y + (int64_t)c0 * ldy, 1, ldy, rmap};
    if (staged) cta_apply_q_staged(F.V, F.ldv, F.m, F.n, F.T, F.n, false, B, qn, true, W);
    else cta_apply_q(F.V, F.ldv, F.m, F.n, F.T, F.n, false, B, qn, true, W);
}

// Reverse rows [a, b) of every one of the q columns of y in place.
template <class real>
__device__ void cta_reverse_rows(real* y, int64_t ldy, int a, int b, int q) {
    const int h = (b - a) / 2;
    for (int o = threadIdx.x; o < h * q; o += NT) {
        const int i = o % h, c = o / h;
        real* col = y + (int64_t)c * ldy;
        const real x = col[a + i];
        col[a + i] = col[b - 1 - i];
        col[b - 1 - i] = x;
    }
    __syncthreads();
}

template <class real>
__global__ void __launch_bounds__(NT) k_sss_fwd(const SolveSS<real>* __restrict__ ss, real* Y, int64_t ldy, real* Yn,
                                                int64_t ldyn, int nrhs, int qs, int staged) {
    extern __shared__ double smd[];
    real* sm = reinterpret_cast<real*>(smd);
    int c0, qn;
    if (!rhs_chunk(nrhs, qs, c0, qn)) return;
    const SolveSS<real> S = ss[blockIdx.x];
    real* y = Y + S.off + (int64_t)c0 * ldy;
    const Mat<real> B{y, 1, ldy, nullptr};
    if (S.HR) {
        // unscaled form (Section 3.2): y_p <- H_p^T y_p, whose first f rows are
        // the fine entries; rotate every column so that the r coarse entries
        // come first (three reversals) and the fine ones wait at rows r..n_p
        if (S.f > 0) {
            const real* HV = S.HR + (int64_t)S.r * S.np;
            if (staged) cta_apply_q_staged(HV, S.np, S.np, S.f, S.HT, S.f, false, B, qn, true, sm);
            else cta_apply_q(HV, S.np, S.np, S.f, S.HT, S.f, false, B, qn, true, sm);
            __syncthreads();
            cta_reverse_rows(y, ldy, 0, S.f, qn);
            cta_reverse_rows(y, ldy, S.f, S.np, qn);
            cta_reverse_rows(y, ldy, 0, S.np, qn);
        }
    } else if (S.UV) {
        if (staged) cta_apply_q_staged(S.UV, S.lduv, S.np, S.np, S.UT, S.np, false, B, qn, true, sm);
        else cta_apply_q(S.UV, S.lduv, S.np, S.np, S.UT, S.np, false, B, qn, true, sm);
    }
    if (!S.HR && S.QV && S.r > 0) {
        if (staged) cta_apply_q_staged(S.QV, S.np, S.np, S.r, S.QT, S.ldqt, true, B, qn, true, sm);
        else cta_apply_q(S.QV, S.np, S.np, S.r, S.QT, S.ldqt, true, B, qn, true, sm);
    }
    for (int64_t o = threadIdx.x; o < (int64_t)S.r * qn; o += NT) {
        const int r = (int)(o % S.r), c = (int)(o / S.r);
        Yn[S.noff + r + (c0 + c) * ldyn] = y[r + c * ldy];
    }
}

template <class real>
__global__ void __launch_bounds__(NT) k_sss_bwd(const SolveSS<real>* __restrict__ ss, real* Y, int64_t ldy,
                                                const real* Yn, int64_t ldyn, int nrhs, int qs, int staged,
                                                int* singular) {
    extern __shared__ double smd[];
    real* sm = reinterpret_cast<real*>(smd);
    int c0, qn;
    if (!rhs_chunk(nrhs, qs, c0, qn)) return;
    const SolveSS<real> S = ss[blockIdx.x];
    real* y = Y + S.off + (int64_t)c0 * ldy;
    for (int64_t o = threadIdx.x; o < (int64_t)S.r * qn; o += NT) {
        const int r = (int)(o % S.r), c = (int)(o / S.r);
        y[r + c * ldy] = Yn[S.noff + r + (c0 + c) * ldyn];
    }
    __syncthreads();
    const Mat<real> B{y, 1, ldy, nullptr};
    if (S.HR && S.f > 0) {
        // unscaled form: x_f = R_ff^{-1} (y_f - R_fc x_c), fine rows at r..n_p
        const int f = S.f, r = S.r, np_ = S.np;
        for (int o = threadIdx.x; o < f * qn; o += NT) {
            const int i = o % f, c = o / f;
            const real* yc = y + (int64_t)c * ldy;
            real acc = 0;
            for (int u = 0; u < r; u++) acc += S.HR[i + (int64_t)u * np_] * yc[u];
            y[r + i + (int64_t)c * ldy] -= acc;
        }
        __syncthreads();
        cta_trsv_upper(S.HR + (int64_t)r * np_, np_, f, S.HD, Mat<real>{y + r, 1, ldy, nullptr}, qn, sm);
    }
    if (S.QV && S.r > 0) {
        if (staged) cta_apply_q_staged(S.QV, S.np, S.np, S.r, S.QT, S.ldqt, true, B, qn, false, sm);
        else cta_apply_q(S.QV, S.np, S.np, S.r, S.QT, S.ldqt, true, B, qn, false, sm);
    }
    if (S.UV) cta_trsv_upper(S.UV, S.lduv, S.np, S.UD, B, qn, sm);
    (void)singular;
}

template <class real>
__global__ void __launch_bounds__(NT) k_sfront_bwd(const SolveFront<real>* __restrict__ fr,
                                                   const Seg* __restrict__ segs, const SolveRsj<real>* __restrict__ rsj,
                                                   real* Y, int64_t ldy, int nrhs, int qs, int* singular) {
    __shared__ real P[NT];
    __shared__ real tmp[NB * 16];
    int c0, qn;
    if (!rhs_chunk(nrhs, qs, c0, qn)) return;
    const SolveFront<real> F = fr[blockIdx.x];
    const Seg s0 = segs[F.seg_begin];  // the front's own rows
    real* Yc = Y + (int64_t)c0 * ldy;
    real* xs = Yc + s0.off;
    const int n = F.n;
    // rhs = z_s - sum_j R_sj x_j; every output sum is split over G thread groups,
    // group g taking the blocks b = g, g + G, ...
    const int nout = n * qn;
    int G = 1;
    while (G < 16 && nout * G * 2 <= NT && G < F.nrsj) G *= 2;
    for (int o0 = 0; o0 < nout; o0 += NT / G) {
        const int tt = threadIdx.x;
        const int o = o0 + tt % (NT / G), gg = tt / (NT / G);
        real acc = 0;
        if (o < nout) {
            const int r = o % n, c = o / n;
            for (int b = gg; b < F.nrsj; b += G) {
                const SolveRsj<real> R = rsj[F.rsj_begin + b];
                const real* xj = Yc + R.xoff + (int64_t)c * ldy;
                const real* row = R.R + r;
                for (int u = 0; u < R.nj; u++) acc += row[(int64_t)u * R.ldr] * xj[u];
            }
        }
        if (G == 1) {
            if (o < nout) xs[(o % n) + (int64_t)(o / n) * ldy] -= acc;
        } else {
            P[tt] = acc;
            __syncthreads();
            if (tt < NT / G && o0 + tt < nout) {
                const int oo = o0 + tt;
                real s = 0;
                for (int k = 0; k < G; k++) s += P[tt + k * (NT / G)];
                xs[(oo % n) + (int64_t)(oo / n) * ldy] -= s;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    cta_trsv_upper(F.V, F.ldv, n, F.Dinv, Mat<real>{xs, 1, ldy, nullptr}, qn, tmp);
    (void)singular;
}

// ---------------------------------------------------------------------------
// Wide forms for colours / levels with few fronts: a thread-block cluster of
// CS CTAs shares one front (and one chunk of right-hand sides), every CTA
// owning a slab of the front's rows (a multiple of NB rows).
// ---------------------------------------------------------------------------

__host__ __device__ __forceinline__ int wide_slab_rows(int m, int cs) {
    const int slab = (m + cs - 1) / cs;
    return (slab + NB - 1) / NB * NB;
}

template <class real>
__device__ __forceinline__ real warp_sum_r(real v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Shared memory (bytes) of every wide kernel for slabs of `slab` rows:
// [row map | P NT | part 2 NB qs | W1 NB qs | W2 NB qs | Ts 2 NB^2 | Vs 2 ld NB | Bs ld qs]
__host__ __forceinline__ size_t wide_smem(int slab, int qs, int esz) {
    const int64_t ld = slab | 1;
    return (size_t)((slab + 1) / 2) * 8 + (size_t)(NT + 4 * NB * qs + 2 * NB * NB + 2 * ld * NB + ld * qs) * esz;
}

// Work areas of a wide kernel.  part (and, in the back substitution, the
// solved block) is read by the other CTAs of the cluster; it is indexed by
// the parity of a phase counter that runs over all cluster barriers of the
// kernel, so that a buffer is rewritten only two barriers after it was read.
template <class real>
struct WideSmem {
    int* rmap;
    real *P, *part, *W1, *W2, *Ts, *Vs, *Bs;
    int ld;
};

template <class real>
__device__ __forceinline__ WideSmem<real> wide_smem_layout(double* sm, int slab_cap, int qs) {
    WideSmem<real> w;
    w.ld = slab_cap | 1;
    w.rmap = reinterpret_cast<int*>(sm);
    w.P = reinterpret_cast<real*>(sm + (slab_cap + 1) / 2);
    w.part = w.P + NT;
    w.W1 = w.part + 2 * NB * qs;
    w.W2 = w.W1 + NB * qs;
    w.Ts = w.W2 + NB * qs;
    w.Vs = w.Ts + 2 * NB * NB;
    w.Bs = w.Vs + 2 * (int64_t)w.ld * NB;
    return w;
}

// B <- Q^T B (trans) or Q B for the t reflectors in V (rows 0..m-1, ld ldv;
// unit diagonal implied unless explicit_v) and the diagonal NB x NB blocks of
// T (ld ldt), with B's rows split over the cluster: this CTA holds rows
// [lo, hi) in w.Bs.  Per panel the partial products V_b^T B over every CTA's
// rows are added (a fixed tree over the ranks) through distributed shared
// memory, then every
// CTA updates its rows.  V rows and T block of the next panel are staged by
// cp.async while the current one is applied.
template <class real, int CS, int Q>
__device__ void cl_apply_q(cooperative_groups::cluster_group& cl, const WideSmem<real>& w, int lo, int hi,
                           const real* V, int64_t ldv, int t, const real* T, int ldt, bool explicit_v, bool trans,
                           int qn, int qs, int& ph) {
    const int ld = w.ld;
    const int nbk = (t + NB - 1) / NB;
    auto stage = [&](int k) {
        const int b = trans ? k : nbk - 1 - k;
        const int p0 = b * NB, pb = min(NB, t - p0);
        real* vs = w.Vs + (int64_t)(k & 1) * ld * NB;
        real* ts = w.Ts + (k & 1) * NB * NB;
        const int r0 = max(lo, p0), nr = hi - r0;
        for (int o = threadIdx.x; o < nr * pb; o += NT) {
            const int rr = o % nr, i = o / nr;
            const int r = r0 + rr, col = p0 + i;
            real* d = vs + (r - lo) + (int64_t)i * ld;
            if (r > col || (r == col && explicit_v)) cp_async_elem(d, V + r + (int64_t)col * ldv);
            else *d = r == col ? (real)1 : (real)0;
        }
        for (int o = threadIdx.x; o < pb * pb; o += NT)
            cp_async_elem(ts + o, T + (p0 + o % pb) + (int64_t)(p0 + o / pb) * ldt);
    };
    stage(0);
    cp_async_commit();
    for (int k = 0; k < nbk; k++, ph++) {
        const int b = trans ? k : nbk - 1 - k;
        const int p0 = b * NB, pb = min(NB, t - p0);
        if (k + 1 < nbk) stage(k + 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const real* vs = w.Vs + (int64_t)(k & 1) * ld * NB;
        real* myp = w.part + (ph & 1) * NB * qs;
        const int r0 = max(lo, p0);
        // partial W(i, c) over own rows, split into row groups added in order
        cta_small_gemv(pb, qn, myp, w.P, [&](int i, int c, int g, int G) {
            const real* vi = vs + i * ld - lo;
            const real* bc = w.Bs + c * ld - lo;
            real v = 0;
            for (int r = max(r0, p0 + i) + g; r < hi; r += G) v += vi[r] * bc[r];
            return v;
        });
        cl.sync();
        for (int o = threadIdx.x; o < pb * qn; o += NT) {
            // the CTAs' partials added as a tree over the ranks
            real v[CS];
#pragma unroll
            for (int q = 0; q < CS; q++) v[q] = cl.map_shared_rank(myp, q)[o];
#pragma unroll
            for (int h = CS / 2; h > 0; h >>= 1)
#pragma unroll
                for (int q = 0; q < h; q++) v[q] += v[q + h];
            w.W1[o] = v[0];
        }
        __syncthreads();
        cta_tblock_mul(w.Ts + (k & 1) * NB * NB, pb, 0, pb, qn, trans, w.W1, w.W2);
        for (int r = r0 + (int)threadIdx.x; r < hi; r += NT) {
            real acc[Q];
#pragma unroll
            for (int c = 0; c < Q; c++) acc[c] = 0;
            const real* vr = vs + (r - lo);
            for (int i = 0; i < pb; i++) {
                const real v = vr[i * ld];
#pragma unroll
                for (int c = 0; c < Q; c++)
                    if (c < qn) acc[c] += v * w.W2[i + c * pb];
            }
            real* br = w.Bs + (r - lo);
#pragma unroll
            for (int c = 0; c < Q; c++)
                if (c < qn) br[c * ld] -= acc[c];
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// X <- R^{-1} X for R upper n x n (ld ldr) with inverted diagonal blocks Dinv
// (n x NB, ld n), with X's rows split over the cluster in slabs of `slab`
// rows (this CTA: [lo, hi) in w.Bs).  Block back substitution from the
// bottom: the CTA owning block b forms x_b = Dinv_b x_b and publishes it in
// distributed shared memory (one barrier per block); every CTA with rows
// above b updates them with R(rows, b) x_b.  R(rows, b) and Dinv_b are staged
// by cp.async one block ahead.
template <class real, int CS, int Q>
__device__ void cl_trsv_upper(cooperative_groups::cluster_group& cl, const WideSmem<real>& w, int lo, int hi,
                              int slab, const real* R, int64_t ldr, int n, const real* Dinv, int qn, int qs,
                              int& ph) {
    const int ld = w.ld;
    real* xl = w.W1;
    const int nbk = (n + NB - 1) / NB;
    auto stage = [&](int b, int k) {
        const int b0 = b * NB, bs = min(NB, n - b0);
        real* rs = w.Vs + (int64_t)(k & 1) * ld * NB;
        const int nr = min(hi, b0) - lo;
        for (int o = threadIdx.x; o < nr * bs; o += NT) {
            const int rr = o % nr, u = o / nr;
            cp_async_elem(rs + rr + (int64_t)u * ld, R + (lo + rr) + (int64_t)(b0 + u) * ldr);
        }
        if (b0 >= lo && b0 < hi) {
            real* ds = w.Ts + (k & 1) * NB * NB;
            for (int o = threadIdx.x; o < bs * bs; o += NT)
                cp_async_elem(ds + o, Dinv + (b0 + o % bs) + (int64_t)(o / bs) * n);
        }
    };
    stage(nbk - 1, 0);
    cp_async_commit();
    for (int k = 0; k < nbk; k++, ph++) {
        const int b = nbk - 1 - k;
        const int b0 = b * NB, bs = min(NB, n - b0);
        if (b > 0) stage(b - 1, k + 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        real* buf = w.part + (ph & 1) * NB * qs;
        if (b0 >= lo && b0 < hi) {
            const real* ds = w.Ts + (k & 1) * NB * NB;
            for (int o = threadIdx.x; o < bs * qn; o += NT) {
                const int i = o % bs, c = o / bs;
                real v = 0;
                for (int u = i; u < bs; u++) v += ds[i + u * bs] * w.Bs[(b0 - lo + u) + c * ld];
                buf[i + c * bs] = v;
            }
            __syncthreads();
            for (int o = threadIdx.x; o < bs * qn; o += NT) w.Bs[(b0 - lo + o % bs) + (o / bs) * ld] = buf[o];
        }
        cl.sync();
        if (lo < b0) {
            const real* ob = cl.map_shared_rank(buf, b0 / slab);
            for (int o = threadIdx.x; o < bs * qn; o += NT) xl[o] = ob[o];
            __syncthreads();
            const real* rs = w.Vs + (int64_t)(k & 1) * ld * NB;
            const int top = min(hi, b0);
            for (int r = lo + (int)threadIdx.x; r < top; r += NT) {
                real acc[Q];
#pragma unroll
                for (int c = 0; c < Q; c++) acc[c] = 0;
                for (int u = 0; u < bs; u++) {
                    const real v = rs[(r - lo) + u * ld];
#pragma unroll
                    for (int c = 0; c < Q; c++)
                        if (c < qn) acc[c] += v * xl[u + c * bs];
                }
#pragma unroll
                for (int c = 0; c < Q; c++)
                    if (c < qn) w.Bs[(r - lo) + c * ld] -= acc[c];
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// y_R(s) <- Q_s^T y_R(s) (the forward front step), one cluster per front.
template <class real, int CS, int Q>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(NT, 1)
    k_sfront_fwd_wide(const SolveFront<real>* __restrict__ fr, const Seg* __restrict__ segs, real* Y, int64_t ldy,
                      int nrhs, int qs, int slab_cap) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double sm[];
    const WideSmem<real> w = wide_smem_layout<real>(sm, slab_cap, qs);
    int c0, qn;
    if (!rhs_chunk(nrhs, qs, c0, qn)) return;   // uniform over the cluster (same blockIdx.y)
    const int rank = (int)cl.block_rank();
    const SolveFront<real> F = fr[blockIdx.x / CS];
    const int slab = wide_slab_rows(F.m, CS);
    const int lo = min(F.m, rank * slab), hi = min(F.m, lo + slab);
    const int rows = hi - lo;
    for (int s = threadIdx.x; s < F.nseg; s += NT) {   // a segment per thread: one load each
        const Seg g = segs[F.seg_begin + s];
        const int a = max(g.pos, lo), b = min(g.pos + g.len, hi);
        for (int r = a; r < b; r++) w.rmap[r - lo] = (int)(g.off + (r - g.pos));
    }
    __syncthreads();
    real* Yc = Y + (int64_t)c0 * ldy;
    for (int o = threadIdx.x; o < rows * qn; o += NT) {
        const int r = o % rows, c = o / rows;
        cp_async_elem(w.Bs + r + (int64_t)c * w.ld, Yc + w.rmap[r] + (int64_t)c * ldy);
    }
    cp_async_commit();
    int ph = 0;
    cl_apply_q<real, CS, Q>(cl, w, lo, hi, F.V, F.ldv, F.n, F.T, F.n, false, true, qn, qs, ph);
    for (int o = threadIdx.x; o < rows * qn; o += NT) {
        const int r = o % rows, c = o / rows;
        Yc[w.rmap[r] + (int64_t)c * ldy] = w.Bs[r + c * w.ld];
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

// Partial products R_sj x_j of the backward front step: one CTA per tile
// (front, kTileRows rows, one K chunk of at most kTileK columns) and chunk of
// right-hand sides; four thread groups split the chunk's columns and are
// added in group order.  Each thread keeps eight loads of R in flight.
// Partials go to Zp rows zoff + kc * n_s + r.
template <class real, int Q>
__global__ void __launch_bounds__(NT) k_rsj_tiles(const RsjTile* __restrict__ tiles,
                                                  const SolveRsj<real>* __restrict__ pieces,
                                                  const SolveFront<real>* __restrict__ fr, const real* __restrict__ Y,
                                                  int64_t ldy, real* __restrict__ Zp, int64_t ldz, int nrhs, int qs) {
    __shared__ real xs[kTileK * kTileQ];
    __shared__ const real* colp[kTileK];   // R column of every column of the chunk (tile row 0)
    __shared__ int64_t colx[kTileK];       // its rows in the level vector
    __shared__ int pnj[kTileK];            // columns of every piece (npiece <= kTileK)
    constexpr int G = NT / kTileRows;
    constexpr int U = 8;
    int c0, qn;
    if (!rhs_chunk(nrhs, qs, c0, qn)) return;
    const RsjTile t = tiles[blockIdx.x];
    const int n = fr[t.front].n;
    // the pieces' descriptors are read in parallel (not one after the other
    // by every thread), then every column of the chunk gets its R column and
    // its rows of x in shared memory
    SolveRsj<real> P{};
    if ((int)threadIdx.x < t.npiece) {
        P = pieces[t.piece_begin + threadIdx.x];
        pnj[threadIdx.x] = P.nj;
    }
    __syncthreads();
    if ((int)threadIdx.x < t.npiece) {
        int koff = 0;
        for (int q = 0; q < (int)threadIdx.x; q++) koff += pnj[q];
        for (int u = 0; u < P.nj; u++) {
            colp[koff + u] = P.R + (int64_t)u * P.ldr + t.row0;
            colx[koff + u] = P.xoff + u;
        }
    }
    __syncthreads();
    int K = 0;
    for (int q = 0; q < t.npiece; q++) K += pnj[q];
    for (int o = threadIdx.x; o < K * qn; o += NT) {
        const int u = o % K, c = o / K;
        cp_async_elem(xs + u + c * kTileK, Y + colx[u] + (int64_t)(c0 + c) * ldy);
    }
    cp_async_commit();
    const int r = threadIdx.x % kTileRows, g = threadIdx.x / kTileRows;
    real acc[Q];
#pragma unroll
    for (int c = 0; c < Q; c++) acc[c] = 0;
    cp_async_wait<0>();
    __syncthreads();
    if (r < t.nrows) {
        // the chunk's columns with stride G, eight loads of R in flight
        int u = g;
        for (; u + (U - 1) * G < K; u += U * G) {
            real v[U];
#pragma unroll
            for (int k = 0; k < U; k++) v[k] = colp[u + k * G][r];
#pragma unroll
            for (int k = 0; k < U; k++) {
                const real* xu = xs + u + k * G;
#pragma unroll
                for (int c = 0; c < Q; c++)
                    if (c < qn) acc[c] += v[k] * xu[c * kTileK];
            }
        }
        for (; u < K; u += G) {
            const real v = colp[u][r];
            const real* xu = xs + u;
#pragma unroll
            for (int c = 0; c < Q; c++)
                if (c < qn) acc[c] += v * xu[c * kTileK];
        }
    }
    __syncthreads();
    real* red = xs;   // (c * G + g) * kTileRows + r
#pragma unroll
    for (int c = 0; c < Q; c++)
        if (c < qn) red[(c * G + g) * kTileRows + r] = acc[c];
    __syncthreads();
    for (int o = threadIdx.x; o < t.nrows * qn; o += NT) {
        const int rr = o % t.nrows, c = o / t.nrows;
        real s = 0;
#pragma unroll
        for (int k = 0; k < G; k++) s += red[(c * G + k) * kTileRows + rr];
        Zp[t.zoff + (int64_t)t.kc * n + t.row0 + rr + (int64_t)(c0 + c) * ldz] = s;
    }
}

// x_s <- R_ss^{-1} (y_s - sum of the R_sj partials), one cluster per front.
template <class real, int CS, int Q>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(NT, 1)
    k_sfront_bwd_wide(const WideFront* __restrict__ wf, const SolveFront<real>* __restrict__ fr,
                      const Seg* __restrict__ segs, real* Y, int64_t ldy, const real* __restrict__ Zp, int64_t ldz,
                      int nrhs, int qs, int slab_cap) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double sm[];
    const WideSmem<real> w = wide_smem_layout<real>(sm, slab_cap, qs);
    int c0, qn;
    if (!rhs_chunk(nrhs, qs, c0, qn)) return;   // uniform over the cluster
    const int rank = (int)cl.block_rank();
    const WideFront W = wf[blockIdx.x / CS];
    const SolveFront<real> F = fr[W.front];
    const int n = F.n;
    const int slab = wide_slab_rows(n, CS);
    const int lo = min(n, rank * slab), hi = min(n, lo + slab);
    const int rows = hi - lo;
    real* xs = Y + segs[F.seg_begin].off + (int64_t)c0 * ldy;
    for (int o = threadIdx.x; o < rows * qn; o += NT) {
        const int r = o % rows, c = o / rows;
        const real* zp = Zp + W.zoff + lo + r + (int64_t)(c0 + c) * ldz;
        real t = 0;
        for (int kc = 0; kc < W.nkc; kc++) t += zp[(int64_t)kc * n];
        w.Bs[r + c * w.ld] = xs[lo + r + (int64_t)c * ldy] - t;
    }
    int ph = 0;
    cl_trsv_upper<real, CS, Q>(cl, w, lo, hi, slab, F.V, F.ldv, n, F.Dinv, qn, qs, ph);
    for (int o = threadIdx.x; o < rows * qn; o += NT) {
        const int r = o % rows, c = o / rows;
        xs[lo + r + (int64_t)c * ldy] = w.Bs[r + c * w.ld];
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

// Forward scale + sparsify of one surviving cluster p, one cluster of CTAs
// per interface: y_p <- Q_p^T U_p^T y_p, then the coarse part moves to the
// next level's vector.
template <class real, int CS, int Q>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(NT, 1)
    k_sss_fwd_wide(const SolveSS<real>* __restrict__ ss, real* Y, int64_t ldy, real* Yn, int64_t ldyn, int nrhs,
                   int qs, int slab_cap) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double sm[];
    const WideSmem<real> w = wide_smem_layout<real>(sm, slab_cap, qs);
    int c0, qn;
    if (!rhs_chunk(nrhs, qs, c0, qn)) return;
    const int rank = (int)cl.block_rank();
    const SolveSS<real> S = ss[blockIdx.x / CS];
    const int m = S.np;
    const int slab = wide_slab_rows(m, CS);
    const int lo = min(m, rank * slab), hi = min(m, lo + slab);
    const int rows = hi - lo;
    real* y = Y + S.off + (int64_t)c0 * ldy;
    for (int o = threadIdx.x; o < rows * qn; o += NT) {
        const int r = o % rows, c = o / rows;
        cp_async_elem(w.Bs + r + (int64_t)c * w.ld, y + lo + r + (int64_t)c * ldy);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    int ph = 0;
    if (S.UV) cl_apply_q<real, CS, Q>(cl, w, lo, hi, S.UV, S.lduv, m, S.UT, m, false, true, qn, qs, ph);
    if (S.QV && S.r > 0)
        cl_apply_q<real, CS, Q>(cl, w, lo, hi, S.QV, m, S.r, S.QT, S.ldqt, true, true, qn, qs, ph);
    for (int o = threadIdx.x; o < rows * qn; o += NT) {
        const int r = o % rows, c = o / rows;
        const real v = w.Bs[r + c * w.ld];
        y[lo + r + (int64_t)c * ldy] = v;
        if (lo + r < S.r) Yn[S.noff + lo + r + (int64_t)(c0 + c) * ldyn] = v;
    }
    cl.sync();
}

// Backward scale + sparsify of one surviving cluster p: the coarse part comes
// back from the next level's vector, y_p <- Q_p y_p, then y_p <- R_pp^{-1} y_p.
template <class real, int CS, int Q>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(NT, 1)
    k_sss_bwd_wide(const SolveSS<real>* __restrict__ ss, real* Y, int64_t ldy, const real* Yn, int64_t ldyn,
                   int nrhs, int qs, int slab_cap) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double sm[];
    const WideSmem<real> w = wide_smem_layout<real>(sm, slab_cap, qs);
    int c0, qn;
    if (!rhs_chunk(nrhs, qs, c0, qn)) return;
    const int rank = (int)cl.block_rank();
    const SolveSS<real> S = ss[blockIdx.x / CS];
    const int m = S.np;
    const int slab = wide_slab_rows(m, CS);
    const int lo = min(m, rank * slab), hi = min(m, lo + slab);
    const int rows = hi - lo;
    real* y = Y + S.off + (int64_t)c0 * ldy;
    for (int o = threadIdx.x; o < rows * qn; o += NT) {
        const int r = o % rows, c = o / rows;
        const real* src = lo + r < S.r ? Yn + S.noff + lo + r + (int64_t)(c0 + c) * ldyn
                                       : y + lo + r + (int64_t)c * ldy;
        cp_async_elem(w.Bs + r + (int64_t)c * w.ld, src);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    int ph = 0;
    if (S.QV && S.r > 0)
        cl_apply_q<real, CS, Q>(cl, w, lo, hi, S.QV, m, S.r, S.QT, S.ldqt, true, false, qn, qs, ph);
    if (S.UV) cl_trsv_upper<real, CS, Q>(cl, w, lo, hi, slab, S.UV, S.lduv, m, S.UD, qn, qs, ph);
    for (int o = threadIdx.x; o < rows * qn; o += NT) {
        const int r = o % rows, c = o / rows;
        y[lo + r + (int64_t)c * ldy] = w.Bs[r + c * w.ld];
    }
    cl.sync();
}

// ---------------------------------------------------------------------------
// GMRES kernels (FP64)
//
// The operator (SpMV, factor application) acts on whole columns of length n;
// the Krylov processes are "virtual columns": with nseg segments (the
// matrices of a block-diagonal batch, rows [seg_ptr[s], seg_ptr[s+1])),
// virtual column v = c * nseg + s is segment s of right-hand-side column c.
// nseg = 1 is the plain multi-RHS case.
// ---------------------------------------------------------------------------

struct VCols {
    int nseg;                  // segments per column
    const int* seg_of;         // row -> segment (nseg > 1)
    const int64_t* seg_ptr;    // nseg + 1 row offsets (device)
    __device__ __forceinline__ int of(int64_t r, int c) const { return nseg == 1 ? c : c * nseg + seg_of[r]; }
    __device__ __forceinline__ void range(int v, int64_t n, int64_t& base, int64_t& len) const {
        if (nseg == 1) { base = (int64_t)v * n; len = n; return; }
        const int c = v / nseg, s = v % nseg;
        base = (int64_t)c * n + seg_ptr[s];
        len = seg_ptr[s + 1] - seg_ptr[s];
    }
};

// Y = A X (CSR, nrhs columns)
__global__ void k_spmv(int64_t n, int nrhs, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                       const double* __restrict__ val, const double* __restrict__ X, int64_t ldx,
                       double* __restrict__ Y, int64_t ldy) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n * nrhs) return;
    const int64_t r = o % n;
    const int c = (int)(o / n);
    double s = 0.0;
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; e++) s += val[e] * X[colind[e] + c * ldx];
    Y[r + c * ldy] = s;
}

// R = B - A X
__global__ void k_residual(int64_t n, int nrhs, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                           const double* __restrict__ val, const double* __restrict__ X, int64_t ldx,
                           const double* __restrict__ B, int64_t ldb, double* __restrict__ R) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n * nrhs) return;
    const int64_t r = o % n;
    const int c = (int)(o / n);
    double s = 0.0;
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; e++) s += val[e] * X[colind[e] + c * ldx];
    R[r + c * n] = B[r + c * ldb] - s;
}

// Partial dot products: part[(i + v * nvec) * S + s] = dot over chunk s of
// the S row chunks of U_i[v] and W[v], for i < nvec and every virtual column
// v; U_i = U + i * n * nrhs.  One CTA per (i, v, chunk), so that a few long
// dot products still spread over every SM; fixed reduction order.
__global__ void __launch_bounds__(NT) k_dots_part(int64_t n, int nrhs, VCols vc, const double* __restrict__ U,
                                                  int nvec, const double* __restrict__ W, double* __restrict__ part,
                                                  int S) {
    __shared__ double red[RED];
    const int i = blockIdx.x % nvec, v = blockIdx.x / nvec, sc = blockIdx.y;
    int64_t base, len;
    vc.range(v, n, base, len);
    const int64_t a = len * sc / S, b = len * (sc + 1) / S;
    const double* u = U + (int64_t)i * n * nrhs + base;
    const double* w = W + base;
    // four independent partial sums per thread (loads in flight), added in a
    // fixed order
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t r = a + threadIdx.x;
    for (; r + 3 * NT < b; r += 4 * NT) {
        s0 += u[r] * w[r];
        s1 += u[r + NT] * w[r + NT];
        s2 += u[r + 2 * NT] * w[r + 2 * NT];
        s3 += u[r + 3 * NT] * w[r + 3 * NT];
    }
    for (; r < b; r += NT) s0 += u[r] * w[r];
    const double s = block_sum((s0 + s1) + (s2 + s3), red);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * S + sc] = s;
}

// out[i + v * nout] = the S partials of (i, v) added in chunk order.
__global__ void k_dots_sum(int nvec, int nv, const double* __restrict__ part, int S, double* __restrict__ out,
                           int nout) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nvec * nv) return;
    const int i = o % nvec, v = o / nvec;
    const double* p = part + (int64_t)o * S;
    double s = 0.0;
    for (int c = 0; c < S; c++) s += p[c];
    out[i + (int64_t)v * nout] = s;
}

// Row chunks of a dot product of len rows: about 4096 rows each, at most 32.
static inline int dot_chunks(int64_t len) { return (int)std::max<int64_t>(1, std::min<int64_t>(32, len / 4096)); }

// W[:, v] -= sum_i U_i[:, v] h[i, v]  (active virtual columns only)
__global__ void k_orth_update(int64_t n, int nrhs, VCols vc, const double* __restrict__ U, int nvec,
                              const double* __restrict__ h, int nh, double* __restrict__ W,
                              const int* __restrict__ active) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n * nrhs) return;
    const int64_t r = o % n;
    const int v = vc.of(r, (int)(o / n));
    if (!active[v]) return;
    double s = 0.0;
    for (int i = 0; i < nvec; i++) s += U[(int64_t)i * n * nrhs + o] * h[i + (int64_t)v * nh];
    W[o] -= s;
}

// U_{j+1} = W / hn[v] (zero for inactive virtual columns or hn = 0)
__global__ void k_normalize(int64_t n, int nrhs, VCols vc, const double* __restrict__ W,
                            const double* __restrict__ hn, double* __restrict__ Unext, const int* __restrict__ active) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n * nrhs) return;
    const int v = vc.of(o % n, (int)(o / n));
    const double h = hn[v];
    Unext[o] = (active[v] && h != 0.0) ? W[o] / h : 0.0;
}

// Givens update of column j of every active Hessenberg matrix (one thread per
// virtual column).  H_v is (ldh x maxit) column-major; cs/sn/g per column.
__global__ void k_givens(int nv, int j, double* H, int ldh, int64_t hstride, const double* h1,
                         const double* h2, const double* hn, double* cs, double* sn, double* g, int ldg,
                         const double* bnorm, double* est, const int* active) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nv) return;
    double* Hc = H + c * hstride;
    double* col = Hc + (int64_t)j * ldh;
    double* csc = cs + (int64_t)c * ldg;
    double* snc = sn + (int64_t)c * ldg;
    double* gc = g + (int64_t)c * ldg;
    if (!active[c]) { est[c] = 0.0; return; }
    for (int i = 0; i <= j; i++) col[i] = h1[i + (int64_t)c * ldh] + h2[i + (int64_t)c * ldh];
    col[j + 1] = hn[c];
    for (int i = 0; i < j; i++) {
        const double t = csc[i] * col[i] + snc[i] * col[i + 1];
        col[i + 1] = -snc[i] * col[i] + csc[i] * col[i + 1];
        col[i] = t;
    }
    const double den = hypot(col[j], col[j + 1]);
    double cj = 1.0, sj = 0.0;
    if (den != 0.0) { cj = col[j] / den; sj = col[j + 1] / den; }
    csc[j] = cj;
    snc[j] = sj;
    col[j] = den;
    col[j + 1] = 0.0;
    gc[j + 1] = -sj * gc[j];
    gc[j] = cj * gc[j];
    est[c] = fabs(gc[j + 1]) / bnorm[c];
}

// y_v = H_v(0:j+1, 0:j+1)^{-1} g_v(0:j+1) for virtual columns with want[v].
__global__ void k_hsolve(int nv, int j, const double* H, int ldh, int64_t hstride, const double* g, int ldg,
                         double* y, const int* want) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nv) return;
    double* yc = y + (int64_t)c * ldg;
    if (!want[c]) {
        for (int i = 0; i <= j; i++) yc[i] = 0.0;
        return;
    }
    const double* Hc = H + c * hstride;
    for (int i = j; i >= 0; i--) {
        double s = g[(int64_t)c * ldg + i];
        for (int k = i + 1; k <= j; k++) s -= Hc[i + (int64_t)k * ldh] * yc[k];
        const double d = Hc[i + (int64_t)i * ldh];
        yc[i] = d != 0.0 ? s / d : 0.0;
    }
}

// out = sum_i U_i y_i (per virtual column)
__global__ void k_combine(int64_t n, int nrhs, VCols vc, const double* __restrict__ U, int nvec,
                          const double* __restrict__ y, int ldy, double* __restrict__ out) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n * nrhs) return;
    const int v = vc.of(o % n, (int)(o / n));
    double s = 0.0;
    for (int i = 0; i < nvec; i++) s += U[(int64_t)i * n * nrhs + o] * y[i + (int64_t)v * ldy];
    out[o] = s;
}

// X = X0 + Z where take[v] (the other entries keep X)
__global__ void k_accept(int64_t n, int nrhs, VCols vc, const double* __restrict__ X0, int64_t ldx0,
                         const double* __restrict__ Z, double* __restrict__ X, int64_t ldx,
                         const int* __restrict__ take) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n * nrhs) return;
    const int64_t r = o % n;
    const int c = (int)(o / n);
    if (!take[vc.of(r, c)]) return;
    X[r + c * ldx] = X0[r + c * ldx0] + Z[r + c * n];
}

__global__ void k_copy_cols(int64_t n, int nrhs, const double* __restrict__ S, int64_t lds, double* __restrict__ D,
                            int64_t ldd) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n * nrhs) return;
    const int64_t r = o % n;
    const int c = (int)(o / n);
    D[r + c * ldd] = S[r + c * lds];
}

// D[:, c] = S[:, c] for rows of accepted virtual columns (take[v])
__global__ void k_copy_taken(int64_t n, int nrhs, VCols vc, const double* __restrict__ S, int64_t lds,
                             double* __restrict__ D, int64_t ldd, const int* __restrict__ take) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n * nrhs) return;
    const int64_t r = o % n;
    const int c = (int)(o / n);
    if (take[vc.of(r, c)]) D[r + c * ldd] = S[r + c * lds];
}

__global__ void k_sqrtv(int nv, double* v) {
    for (int c = threadIdx.x; c < nv; c += blockDim.x) v[c] = sqrt(v[c]);
}

__global__ void k_scale_cols(int64_t n, int nrhs, VCols vc, double* __restrict__ U, const double* __restrict__ s) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n * nrhs) return;
    const double v = s[vc.of(o % n, (int)(o / n))];
    U[o] = v != 0.0 ? U[o] / v : 0.0;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

const int kSmemMax = 200 * 1024;

struct SCtx {
    cudaStream_t st;
    std::vector<void*> temps;
    int rc = SPAQR_OK;
    template <class T>
    T* alloc(int64_t count) {
        if (rc != SPAQR_OK) return nullptr;
        void* p = nullptr;
        size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
        if (fail_this_alloc() || cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            set_error("device allocation failed");
            rc = SPAQR_ERR_OOM;
            return nullptr;
        }
        temps.push_back(p);
        return (T*)p;
    }
    void cuda(cudaError_t e) {
        if (e != cudaSuccess && rc == SPAQR_OK) {
            set_error(std::string("CUDA: ") + cudaGetErrorString(e));
            rc = SPAQR_ERR_CUDA;
        }
    }
    void launched() { cuda(cudaGetLastError()); }
    void release(void* p) {
        for (auto it = temps.begin(); it != temps.end(); ++it)
            if (*it == p) { cudaFreeAsync(p, st); temps.erase(it); return; }
    }
    ~SCtx() {
        for (void* p : temps) cudaFreeAsync(p, st);
    }
};

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Calls f(std::integral_constant<int, Q>) with Q the smallest of 1, 2, 4, 8,
// 16 that is >= q: the wide kernels unroll their column loops to Q.
template <class Fn>
static void with_q(int q, Fn f) {
    if (q <= 1) f(std::integral_constant<int, 1>());
    else if (q <= 2) f(std::integral_constant<int, 2>());
    else if (q <= 4) f(std::integral_constant<int, 4>());
    else if (q <= 8) f(std::integral_constant<int, 8>());
    else f(std::integral_constant<int, 16>());
}

template <class real>
void set_solve_attrs() {
    static std::once_flag once;
    std::call_once(once, [] {
    cudaFuncSetAttribute(k_sfront_fwd<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    cudaFuncSetAttribute(k_sss_fwd<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    cudaFuncSetAttribute(k_sss_bwd<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    for (int q : {1, 2, 4, 8, 16})
        with_q(q, [](auto QC) {
            cudaFuncSetAttribute(k_sfront_fwd_wide<real, 1, QC.value>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemMax);
            cudaFuncSetAttribute(k_sfront_bwd_wide<real, 1, QC.value>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemMax);
            cudaFuncSetAttribute(k_sss_fwd_wide<real, 1, QC.value>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemMax);
            cudaFuncSetAttribute(k_sss_bwd_wide<real, 1, QC.value>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemMax);
            cudaFuncSetAttribute(k_sfront_fwd_wide<real, kWideCS, QC.value>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
            cudaFuncSetAttribute(k_sfront_bwd_wide<real, kWideCS, QC.value>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
            cudaFuncSetAttribute(k_sss_fwd_wide<real, kWideCS, QC.value>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
            cudaFuncSetAttribute(k_sss_bwd_wide<real, kWideCS, QC.value>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
        });
    });
}

}  // namespace

// X = M^{-1} B with B, X device pointers (n x nrhs, leading dims).  `singular`
// is a device int (may be null).  Stream-ordered, no synchronisation.
// RHS split of a launch with `blocks` CTAs: enough chunks to give every SM
// about two CTAs, between 1 and 16 columns per chunk.
static int rhs_split(int blocks, int nrhs) {
    int split = (2 * 152 + blocks - 1) / std::max(blocks, 1);
    split = std::max(1, std::min(split, nrhs));
    split = std::max(split, (nrhs + 15) / 16);   // at most 16 columns per CTA
    return split;
}

constexpr int kNumSM = 152;


// CTAs of the one-CTA-per-unit form of a launch; the wide (cluster) forms
// are used where this leaves SMs idle.
static int narrow_ctas(int units, int nrhs) { return units * rhs_split(units, nrhs); }

// Right-hand-side chunks of a wide launch over `units` clusters: about two
// CTAs per SM, at most kTileQ columns per chunk, and the chunk's shared
// memory (smem(q) bytes) within the limit.  False if one column does not fit.
template <class Smem>
static bool wide_split(int units, int nrhs, Smem smem, int& qs, int& split, int cs = kWideCS) {
    int qmax = kTileQ;
    while (qmax > 0 && smem(qmax) > (size_t)kSmemMax) qmax--;
    if (qmax == 0) return false;
    split = std::max((nrhs + qmax - 1) / qmax,
                     std::min(nrhs, (2 * kNumSM + units * cs - 1) / (units * cs)));
    qs = (nrhs + split - 1) / split;
    split = (nrhs + qs - 1) / qs;
    return true;
}

// Launch forms of a unit: the rule's choice, one CTA per front / interface
// (the original kernels), a thread-block cluster of kWideCS CTAs per front /
// interface, or the cluster kernels with one CTA (cp.async-staged panels,
// column loops unrolled to the chunk width).
enum { kChoiceRule = 0, kChoiceNarrow = 1, kChoiceWide = 2, kChoiceSingle = 3 };

// Calls f(std::integral_constant<int, CS>) for CS = cs (1 or kWideCS).
template <class Fn>
static void with_cs(int cs, Fn f) {
    if (cs == 1) f(std::integral_constant<int, 1>());
    else f(std::integral_constant<int, kWideCS>());
}

// One application in flight: the factor, right-hand-side count, stream and
// workspace.
template <class real>
struct ApplyCtx {
    const spaqr_factor_s* F;
    int nrhs;
    cudaStream_t st;
    real* ws;
    int* singular;
    int64_t esz;
    const SolveFront<real>* dfr;
    const SolveSS<real>* dss;
    const SolveRsj<real>* drsj;
    ApplyCtx(const spaqr_factor_s* F_, int nrhs_, cudaStream_t st_, real* ws_, int* sg)
        : F(F_), nrhs(nrhs_), st(st_), ws(ws_), singular(sg), esz((int64_t)sizeof(real)),
          dfr(static_cast<const SolveFront<real>*>(F_->d_fronts)), dss(static_cast<const SolveSS<real>*>(F_->d_ss)),
          drsj(static_cast<const SolveRsj<real>*>(F_->d_rsj)) {}
    real* level(int k) const { return ws + F->lv[k].ws_off * nrhs; }
};

// Forward fronts of colour c at level k.
template <class real>
void launch_ff(const ApplyCtx<real>& A, int k, int c, int choice) {
    const spaqr_factor_s* F = A.F;
    const SolveLevelHost& LV = F->lv[k];
    const int a = LV.colour_ptr[c], b = LV.colour_ptr[c + 1];
    if (b <= a) return;
    const int nrhs = A.nrhs;
    const int64_t esz = A.esz;
    cudaStream_t st = A.st;
    real* Y = A.level(k);
    const int64_t ldy = LV.rows;
    int form = choice;
    if (form == kChoiceRule) {
        // rule (from autotuned choices on 2D and 3D grids): a cluster per
        // front where one CTA per front leaves SMs idle and the fronts are
        // tall, the staged one-CTA form otherwise
        const int units = b - a;
        if (narrow_ctas(units, nrhs) < kNumSM && LV.ff_maxm[c] >= kWideMinM) form = kChoiceWide;
        else if (units <= 64 && LV.ff_maxm[c] >= 4 * kWideMinM) form = kChoiceWide;
        else form = kChoiceSingle;
    }
    if (form == kChoiceWide || form == kChoiceSingle) {
        const int cs = form == kChoiceWide ? kWideCS : 1;
        const int slab = wide_slab_rows(LV.ff_maxm[c], cs);
        int qs, split;
        if (wide_split(b - a, nrhs, [&](int q) { return wide_smem(slab, q, (int)esz); }, qs, split, cs)) {
            SPAQR_LAUNCH(KK_SOLVE_FRONT_FWD, LV.ff_flops[c] * nrhs, LV.ff_fixed[c] * split + LV.ff_vec[c] * nrhs, st,
                         with_cs(cs, [&](auto CSC) {
                             with_q(qs, [&](auto QC) {
                                 k_sfront_fwd_wide<real, CSC.value, QC.value>
                                     <<<dim3((b - a) * CSC.value, split), NT, wide_smem(slab, qs, (int)esz), st>>>(
                                         A.dfr + LV.front_begin + a, F->d_segs, Y, ldy, nrhs, qs, slab);
                             });
                         }));
            return;
        }
    }
    const int rmap_d = (LV.max_front_m + 1) / 2 + 1;
    const int split = rhs_split(b - a, nrhs);
    const int qs = (nrhs + split - 1) / split;
    const int staged = rmap_d * 8 + staged_smem_elems(LV.max_front_m, qs) * esz <= kSmemMax;
    const size_t smem =
        (size_t)rmap_d * 8 + (size_t)(staged ? staged_smem_elems(LV.max_front_m, qs) : 2 * NB * qs + NT) * esz;
    SPAQR_LAUNCH(KK_SOLVE_FRONT_FWD, LV.ff_flops[c] * nrhs, LV.ff_fixed[c] * split + LV.ff_vec[c] * nrhs, st,
                 k_sfront_fwd<real><<<dim3(b - a, split), NT, smem, st>>>(A.dfr + LV.front_begin + a, F->d_segs, Y,
                                                                          ldy, nrhs, qs, rmap_d, staged));
}

// Scale + sparsify of level k's surviving clusters, forward (fwd) or backward.
template <class real>
void launch_ss(const ApplyCtx<real>& A, int k, bool fwd, int choice) {
    const spaqr_factor_s* F = A.F;
    const SolveLevelHost& LV = F->lv[k];
    if (LV.nss <= 0) return;
    const SolveLevelHost& LN = F->lv[k + 1];
    const int nrhs = A.nrhs;
    const int64_t esz = A.esz;
    cudaStream_t st = A.st;
    real* Y = A.level(k);
    real* Yn = A.level(k + 1);
    const int64_t ldy = LV.rows;
    const double fl = fwd ? LV.ssf_flops : LV.ssb_flops, fx = fwd ? LV.ssf_fixed : LV.ssb_fixed,
                 fv = fwd ? LV.ssf_vec : LV.ssb_vec;
    const int kind = fwd ? KK_SOLVE_SS_FWD : KK_SOLVE_SS_BWD;
    int form = choice;
    if (F->unscaled) form = kChoiceNarrow;   // the cluster forms carry the scaled steps only
    if (form == kChoiceRule) {
        // many interfaces: one CTA each; a few hundred large ones: the staged
        // one-CTA form; the last few: a cluster each
        if (LV.nss <= 8 && LV.max_ss_n >= kWideMinN) form = kChoiceWide;
        else if (LV.nss <= 40 || (LV.nss <= 400 && LV.max_ss_n >= 3 * kWideMinN)) form = kChoiceSingle;
        else form = kChoiceNarrow;
    }
    if (form == kChoiceWide || form == kChoiceSingle) {
        const int cs = form == kChoiceWide ? kWideCS : 1;
        const int slab = wide_slab_rows(LV.max_ss_n, cs);
        int qs, split;
        if (wide_split(LV.nss, nrhs, [&](int q) { return wide_smem(slab, q, (int)esz); }, qs, split, cs)) {
            const size_t smem = wide_smem(slab, qs, (int)esz);
            SPAQR_LAUNCH(kind, fl * nrhs, fx * split + fv * nrhs, st, with_cs(cs, [&](auto CSC) {
                             with_q(qs, [&](auto QC) {
                                 if (fwd)
                                     k_sss_fwd_wide<real, CSC.value, QC.value>
                                         <<<dim3(LV.nss * CSC.value, split), NT, smem, st>>>(
                                             A.dss + LV.ss_begin, Y, ldy, Yn, LN.rows, nrhs, qs, slab);
                                 else
                                     k_sss_bwd_wide<real, CSC.value, QC.value>
                                         <<<dim3(LV.nss * CSC.value, split), NT, smem, st>>>(
                                             A.dss + LV.ss_begin, Y, ldy, Yn, LN.rows, nrhs, qs, slab);
                             });
                         }));
            return;
        }
    }
    const int split = rhs_split(LV.nss, nrhs);
    const int qs = (nrhs + split - 1) / split;
    const int staged = staged_smem_elems(LV.max_ss_n, qs) * esz <= kSmemMax;
    const size_t smem = (size_t)(staged ? staged_smem_elems(LV.max_ss_n, qs) : 2 * NB * qs + NT) * esz;
    if (fwd)
        SPAQR_LAUNCH(kind, fl * nrhs, fx * split + fv * nrhs, st,
                     k_sss_fwd<real><<<dim3(LV.nss, split), NT, smem, st>>>(A.dss + LV.ss_begin, Y, ldy, Yn, LN.rows,
                                                                            nrhs, qs, staged));
    else
        SPAQR_LAUNCH(kind, fl * nrhs, fx * split + fv * nrhs, st,
                     k_sss_bwd<real><<<dim3(LV.nss, split), NT, smem, st>>>(A.dss + LV.ss_begin, Y, ldy, Yn, LN.rows,
                                                                            nrhs, qs, staged, A.singular));
}

// Backward fronts of level k.
template <class real>
void launch_fb(const ApplyCtx<real>& A, int k, int choice) {
    const spaqr_factor_s* F = A.F;
    const SolveLevelHost& LV = F->lv[k];
    if (LV.nfront <= 0) return;
    const int nrhs = A.nrhs;
    const int64_t esz = A.esz;
    cudaStream_t st = A.st;
    real* Y = A.level(k);
    const int64_t ldy = LV.rows;
    int form = choice;
    if (form == kChoiceRule)
        form = LV.nfront <= 8 || (LV.nfront <= 32 && nrhs <= 4) ? kChoiceWide : kChoiceSingle;
    if (LV.bwd_tiles && (form == kChoiceWide || form == kChoiceSingle)) {
        const int cs = form == kChoiceWide ? kWideCS : 1;
        const int slab = wide_slab_rows(LV.max_front_n, cs);
        int qs, split;
        if (wide_split(LV.nfront, nrhs, [&](int q) { return wide_smem(slab, q, (int)esz); }, qs, split, cs)) {
            real* Zp = A.ws + F->zp_off * nrhs;
            const int64_t ldz = F->zp_rows;
            if (LV.ntile > 0) {
                int tsplit = std::max((nrhs + kTileQ - 1) / kTileQ,
                                      std::min(nrhs, (2 * kNumSM + LV.ntile - 1) / LV.ntile));
                const int tq = (nrhs + tsplit - 1) / tsplit;
                tsplit = (nrhs + tq - 1) / tq;
                SPAQR_LAUNCH(KK_SOLVE_RSJ, LV.rt_flops * nrhs, LV.rt_fixed * tsplit + LV.rt_vec * nrhs, st,
                             with_q(tq, [&](auto QC) {
                                 k_rsj_tiles<real, QC.value><<<dim3(LV.ntile, tsplit), NT, 0, st>>>(
                                     static_cast<const RsjTile*>(F->d_tiles) + LV.tile_begin,
                                     static_cast<const SolveRsj<real>*>(F->d_pieces), A.dfr, Y, ldy, Zp, ldz, nrhs,
                                     tq);
                             }));
            }
            SPAQR_LAUNCH(KK_SOLVE_FRONT_BWD, (LV.fb_flops - LV.rt_flops) * nrhs,
                         (LV.fb_fixed - LV.rt_fixed) * split + LV.fb_vec * nrhs, st, with_cs(cs, [&](auto CSC) {
                             with_q(qs, [&](auto QC) {
                                 k_sfront_bwd_wide<real, CSC.value, QC.value>
                                     <<<dim3(LV.nfront * CSC.value, split), NT, wide_smem(slab, qs, (int)esz), st>>>(
                                         static_cast<const WideFront*>(F->d_wfronts) + LV.wf_begin, A.dfr,
                                         F->d_segs, Y, ldy, Zp, ldz, nrhs, qs, slab);
                             });
                         }));
            return;
        }
    }
    const int split = rhs_split(LV.nfront, nrhs);
    const int qs = (nrhs + split - 1) / split;
    SPAQR_LAUNCH(KK_SOLVE_FRONT_BWD, LV.fb_flops * nrhs, LV.fb_fixed * split + LV.fb_vec * nrhs, st,
                 k_sfront_bwd<real><<<dim3(LV.nfront, split), NT, 0, st>>>(A.dfr + LV.front_begin, F->d_segs, A.drsj,
                                                                           Y, ldy, nrhs, qs, A.singular));
}

// X = M^{-1} B: forward over the levels, then backward, with the launch
// forms of `tt` (null: the rules).
template <class real>
int apply_device_t(const spaqr_factor_s* F, int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                   cudaStream_t st, real* ws, int* singular, const TuneTable* tt) {
    set_solve_attrs<real>();
    const ApplyCtx<real> A(F, nrhs, st, ws, singular);
    const int64_t n = F->n;
    const unsigned nb = (unsigned)((n + 255) / 256);
    real* Y0 = A.level(0);
    SPAQR_LAUNCH(KK_SOLVE_PERM, 0.0, 8.0 * n + 16.0 * n * nrhs, st,
                 k_perm_in<real><<<nb, 256, 0, st>>>(n, nrhs, F->d_rperm, B, ldb, Y0, F->lv[0].rows));
    const int L = F->L;
    for (int k = 0; k < L; k++) {
        const SolveLevelHost& LV = F->lv[k];
        for (size_t c = 0; c + 1 < LV.colour_ptr.size(); c++) launch_ff(A, k, (int)c, tt ? tt->ff[k][c] : 0);
        launch_ss(A, k, true, tt ? tt->ssf[k] : 0);
    }
    for (int k = L - 1; k >= 0; k--) {
        launch_ss(A, k, false, tt ? tt->ssb[k] : 0);
        launch_fb(A, k, tt ? tt->fb[k] : 0);
    }
    SPAQR_LAUNCH(KK_SOLVE_PERM, 1.0 * n * nrhs, 16.0 * n + 16.0 * n * nrhs, st,
                 k_perm_out<real><<<nb, 256, 0, st>>>(n, nrhs, F->d_perm, F->d_scale, Y0, F->lv[0].rows, X, ldx));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("CUDA: ") + cudaGetErrorString(e));
        return SPAQR_ERR_CUDA;
    }
    return SPAQR_OK;
}

// Times the application's units one at a time on this factor (each form of a
// unit three times from the same workspace snapshot, the fastest kept) and
// returns the table of the fastest forms.  The workspace must hold the level
// vectors of a completed application.
template <class real>
int autotune_t(const spaqr_factor_s* F, int nrhs, cudaStream_t st, real* ws, real* snap, int* singular,
               TuneTable& tt) {
    set_solve_attrs<real>();
    const ApplyCtx<real> A(F, nrhs, st, ws, singular);
    const size_t wbytes = (size_t)F->ws_rows * nrhs * sizeof(real);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SPAQR_ERR_CUDA;
    auto time_unit = [&](auto&& launch) {
        float best = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
            cudaMemcpyAsync(ws, snap, wbytes, cudaMemcpyDeviceToDevice, st);
            cudaEventRecord(e0, st);
            launch();
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            if (cudaGetLastError() != cudaSuccess) return 1e30f;   // form not launchable here
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        return best;
    };
    auto pick = [&](auto&& launch_with) {
        uint8_t best = kChoiceNarrow;
        float tb = time_unit([&] { launch_with(kChoiceNarrow); });
        for (int form : {kChoiceWide, kChoiceSingle}) {
            const float t = time_unit([&] { launch_with(form); });
            if (t < tb) {
                tb = t;
                best = (uint8_t)form;
            }
        }
        return best;
    };
    const int L = F->L;
    tt.nrhs = nrhs;
    tt.ff.assign(L, {});
    tt.ssf.assign(L, 0);
    tt.ssb.assign(L, 0);
    tt.fb.assign(L, 0);
    for (int k = 0; k < L; k++) {
        const SolveLevelHost& LV = F->lv[k];
        tt.ff[k].assign(LV.colour_ptr.size() > 0 ? LV.colour_ptr.size() - 1 : 0, 0);
        for (size_t c = 0; c + 1 < LV.colour_ptr.size(); c++)
            tt.ff[k][c] = pick([&](int ch) { launch_ff(A, k, (int)c, ch); });
        if (LV.nss > 0) {
            tt.ssf[k] = pick([&](int ch) { launch_ss(A, k, true, ch); });
            tt.ssb[k] = pick([&](int ch) { launch_ss(A, k, false, ch); });
        }
        if (LV.nfront > 0) tt.fb[k] = pick([&](int ch) { launch_fb(A, k, ch); });
    }
    cudaMemcpyAsync(ws, snap, wbytes, cudaMemcpyDeviceToDevice, st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cudaGetLastError() == cudaSuccess ? SPAQR_OK : SPAQR_ERR_CUDA;
}

// X = M^{-1} B with B, X device pointers (FP64, n x nrhs, leading dims) in the
// factor's precision; `ws` holds ws_rows * nrhs elements of that type.
// Stream-ordered, no synchronisation.
int apply_with(const spaqr_factor_s* F, int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
               cudaStream_t st, void* ws, int* singular, const TuneTable* tt) {
    if (F->precision == SPAQR_FP32)
        return apply_device_t<float>(F, nrhs, B, ldb, X, ldx, st, static_cast<float*>(ws), singular, tt);
    return apply_device_t<double>(F, nrhs, B, ldb, X, ldx, st, static_cast<double*>(ws), singular, tt);
}

__global__ void k_fill_pattern(int64_t m, double* B) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
    B[i] = (double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0;   // in [-1, 1)
}

int apply_device(const spaqr_factor_s* F, int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                 cudaStream_t st, void* ws, int* singular) {
    const std::shared_ptr<const TuneTable> tt = F->tune_for(nrhs);
    if (F->precision == SPAQR_FP32)
        return apply_device_t<float>(F, nrhs, B, ldb, X, ldx, st, static_cast<float*>(ws), singular, tt.get());
    return apply_device_t<double>(F, nrhs, B, ldb, X, ldx, st, static_cast<double*>(ws), singular, tt.get());
}

// Makes the factor's device current for the scope of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace spaqr

using namespace spaqr;

extern "C" int spaqr_solve(const spaqr_factor_t* F, int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx,
                           void* stream) {
    if (!F || !B || !X) { set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    if (nrhs < 0 || ldb < F->n || ldx < F->n) { set_error("bad nrhs or leading dimension"); return SPAQR_ERR_INVALID_ARG; }
    if (nrhs == 0) return SPAQR_OK;
    if (B != X) {
        const char* b0 = (const char*)B;
        const char* b1 = (const char*)(B + (ldb * (nrhs - 1) + F->n));
        const char* x0 = (const char*)X;
        const char* x1 = (const char*)(X + (ldx * (nrhs - 1) + F->n));
        if (b0 < x1 && x0 < b1) { set_error("B and X overlap"); return SPAQR_ERR_INVALID_ARG; }
    } else if (ldb != ldx) {
        set_error("aliased B and X need the same leading dimension");
        return SPAQR_ERR_INVALID_ARG;
    }
    if (check_on_device(B, F->device, "B") != SPAQR_OK || check_on_device(X, F->device, "X") != SPAQR_OK)
        return SPAQR_ERR_INVALID_ARG;
    const bool bdev = is_device_ptr(B), xdev = is_device_ptr(X);
    if (bdev != xdev) { set_error("B and X must both be host or both be device memory"); return SPAQR_ERR_INVALID_ARG; }
    DeviceGuard dg(F->device);   // outlives C, whose frees run on the factor's device
    SCtx C;
    C.st = (cudaStream_t)stream;
    const int64_t n = F->n;
    const double* dB = B;
    double* dX = X;
    int64_t lb = ldb, lx = ldx;
    if (!bdev) {
        double* t = C.alloc<double>(n * nrhs);
        if (C.rc) return C.rc;
        C.cuda(cudaMemcpy2DAsync(t, n * 8, B, ldb * 8, n * 8, nrhs, cudaMemcpyHostToDevice, C.st));
        dB = t;
        dX = t;
        lb = lx = n;
    }
    double* ws = C.alloc<double>((F->ws_rows * nrhs * F->esz + 7) / 8);
    int* flag = C.alloc<int>(1);
    if (C.rc) return C.rc;
    C.cuda(cudaMemsetAsync(flag, 0, sizeof(int), C.st));
    C.cuda((cudaError_t)0);
    const int rc = apply_device(F, nrhs, dB, lb, dX, lx, C.st, ws, flag);
    if (rc != SPAQR_OK) return C.rc ? C.rc : rc;
    if (!bdev) C.cuda(cudaMemcpy2DAsync(X, ldx * 8, dX, n * 8, n * 8, nrhs, cudaMemcpyDeviceToHost, C.st));
    int hflag = 0;
    C.cuda(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, C.st));
    C.cuda(cudaStreamSynchronize(C.st));
    if (C.rc) return C.rc;
    if (hflag) { set_error("zero diagonal in an R factor"); return SPAQR_ERR_SINGULAR; }
    return SPAQR_OK;
}

namespace {

// The factor application of one GMRES iteration as a CUDA graph: captured
// once per GMRES call with fixed input / output buffers, replayed every
// iteration (the launches it holds are counted at every replay).
struct ApplyGraph {
    cudaGraphExec_t exec = nullptr;
    LaunchTally tally;
    ~ApplyGraph() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

bool capture_apply(const spaqr_factor_s* F, int nrhs, const double* Vin, double* Zout, cudaStream_t st, void* ws,
                   int* flag, ApplyGraph& g) {
    if (F->precision == SPAQR_FP32) set_solve_attrs<float>();
    else set_solve_attrs<double>();
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    prof_capture_begin(&g.tally);
    const int rc = apply_device(F, nrhs, Vin, F->n, Zout, F->n, st, ws, flag);
    prof_capture_end();
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    bool ok = rc == SPAQR_OK && e == cudaSuccess && graph != nullptr;
    if (ok) ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        g.exec = nullptr;
    }
    return ok;
}

// A private non-blocking stream for one call, ordered after the caller's
// stream: graphs cannot be captured on the legacy default stream.
struct PrivateStream {
    cudaStream_t s = nullptr;
    bool init(cudaStream_t user) {
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            s = nullptr;
            return false;
        }
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); return false; }
        cudaEventRecord(ev, user);
        cudaStreamWaitEvent(s, ev, 0);
        cudaEventDestroy(ev);
        return true;
    }
    ~PrivateStream() {
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
};

// Right-preconditioned flexible GMRES over virtual columns (see VCols):
// nseg = 1 for one matrix, nseg = count for a block-diagonal batch with
// segment row offsets seg_ptr (host).  iters / relres per virtual column
// v = c * nseg + s.
// hist (host, may be null): nv x maxit, hist[v * maxit + j] = the Arnoldi
// estimate of virtual column v's relative residual after iteration j + 1, NaN
// once the column has stopped.
int gmres_impl(const spaqr_factor_t* F, const spaqr_csr* A, int nrhs, int nseg, const int64_t* seg_ptr,
               const double* B, int64_t ldb, double* X, int64_t ldx, double tol, int maxit, int* iters,
               double* relres, void* stream, double* hist = nullptr) {
    if (!F || !A || !B || !X) { set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    if (A->n != F->n || nrhs < 0 || ldb < F->n || ldx < F->n || maxit < 1 || !(tol >= 0.0)) {
        set_error("bad size, leading dimension, tol or maxit");
        return SPAQR_ERR_INVALID_ARG;
    }
    // A must be the factored matrix: its pattern has as many entries, and a
    // host CSR is checked in full before any kernel reads it (a device CSR
    // is trusted: checking it would cost a pass and a synchronisation)
    if (A->nnz != F->nnz || !A->rowptr || !A->colind || !A->val) {
        set_error("A does not match the factored pattern (nnz) or has NULL arrays");
        return SPAQR_ERR_INVALID_ARG;
    }
    if (check_csr_location(A) != SPAQR_OK || check_csr_device(A, F->device) != SPAQR_OK ||
        check_on_device(B, F->device, "B") != SPAQR_OK || check_on_device(X, F->device, "X") != SPAQR_OK)
        return SPAQR_ERR_INVALID_ARG;
    if (!A->on_device) {
        if (A->rowptr[0] != 0 || A->rowptr[A->n] != A->nnz) { set_error("bad CSR rowptr"); return SPAQR_ERR_INVALID_ARG; }
        for (int64_t r = 0; r < A->n; r++)
            if (A->rowptr[r + 1] < A->rowptr[r]) { set_error("bad CSR rowptr (decreasing)"); return SPAQR_ERR_INVALID_ARG; }
        for (int64_t e = 0; e < A->nnz; e++)
            if (A->colind[e] < 0 || A->colind[e] >= A->n) { set_error("column index out of range"); return SPAQR_ERR_INVALID_ARG; }
    }
    if (nrhs == 0) return SPAQR_OK;
    if (hist) std::fill(hist, hist + (int64_t)nrhs * nseg * maxit, std::numeric_limits<double>::quiet_NaN());
    DeviceGuard dg(F->device);   // outlives the stream and allocations below
    keep_pool_memory(F->device);
    const bool graphs = graphs_on() && !prof_on();
    PrivateStream ps;   // destroyed after C, whose frees are ordered on it
    if (graphs && !ps.init((cudaStream_t)stream)) { set_error("stream creation failed"); return SPAQR_ERR_CUDA; }
    SCtx C;
    C.st = graphs ? ps.s : (cudaStream_t)stream;
    cudaStream_t st = C.st;
    const int64_t n = F->n, nnz = A->nnz;
    const int nv = nrhs * nseg;
    const bool bdev = is_device_ptr(B), xdev = is_device_ptr(X);
    if (bdev != xdev) { set_error("B and X must both be host or both be device memory"); return SPAQR_ERR_INVALID_ARG; }
    // virtual columns
    VCols vc{nseg, nullptr, nullptr};
    if (nseg > 1) {
        std::vector<int> so(n);
        for (int sg = 0; sg < nseg; sg++)
            for (int64_t r = seg_ptr[sg]; r < seg_ptr[sg + 1]; r++) so[r] = sg;
        int* d_so = C.alloc<int>(n);
        int64_t* d_sp = C.alloc<int64_t>(nseg + 1);
        if (C.rc) return C.rc;
        C.cuda(cudaMemcpyAsync(d_so, so.data(), 4 * n, cudaMemcpyHostToDevice, st));
        C.cuda(cudaMemcpyAsync(d_sp, seg_ptr, 8 * (nseg + 1), cudaMemcpyHostToDevice, st));
        vc.seg_of = d_so;
        vc.seg_ptr = d_sp;
    }
    auto seg_base = [&](int v) { return nseg == 1 ? (int64_t)0 : seg_ptr[v % nseg]; };
    auto seg_len = [&](int v) { return nseg == 1 ? n : seg_ptr[v % nseg + 1] - seg_ptr[v % nseg]; };
    // matrix on the device
    const int64_t* rp = A->rowptr;
    const int32_t* ci = A->colind;
    const double* va = A->val;
    if (!A->on_device) {
        int64_t* a = C.alloc<int64_t>(n + 1);
        int32_t* b = C.alloc<int32_t>(nnz);
        double* v = C.alloc<double>(nnz);
        if (C.rc) return C.rc;
        C.cuda(cudaMemcpyAsync(a, A->rowptr, 8 * (n + 1), cudaMemcpyHostToDevice, st));
        C.cuda(cudaMemcpyAsync(b, A->colind, 4 * nnz, cudaMemcpyHostToDevice, st));
        C.cuda(cudaMemcpyAsync(v, A->val, 8 * nnz, cudaMemcpyHostToDevice, st));
        rp = a;
        ci = b;
        va = v;
    }
    // B, X on the device (column-major n x nrhs, ld n for temporaries)
    const double* dB = B;
    double* dX = X;
    int64_t lb = ldb, lx = ldx;
    if (!bdev) {
        double* tb = C.alloc<double>(n * nrhs);
        double* tx = C.alloc<double>(n * nrhs);
        if (C.rc) return C.rc;
        C.cuda(cudaMemcpy2DAsync(tb, n * 8, B, ldb * 8, n * 8, nrhs, cudaMemcpyHostToDevice, st));
        C.cuda(cudaMemcpy2DAsync(tx, n * 8, X, ldx * 8, n * 8, nrhs, cudaMemcpyHostToDevice, st));
        dB = tb;
        dX = tx;
        lb = lx = n;
    }
    const unsigned nbl = (unsigned)((n * nrhs + 255) / 256);
    const unsigned nbv = (unsigned)((nv + 31) / 32);
    const int ldh = maxit + 1;
    const int64_t hstride = (int64_t)ldh * maxit;
    double* X0 = C.alloc<double>(n * nrhs);
    double* Wv = C.alloc<double>(n * nrhs);
    double* Zv = C.alloc<double>(n * nrhs);
    double* ws = C.alloc<double>((F->ws_rows * nrhs * F->esz + 7) / 8);
    double* H = C.alloc<double>(hstride * nv);
    double* h1 = C.alloc<double>((int64_t)ldh * nv);
    double* h2 = C.alloc<double>((int64_t)ldh * nv);
    double* hn = C.alloc<double>(nv);
    double* cs = C.alloc<double>((int64_t)ldh * nv);
    double* sn = C.alloc<double>((int64_t)ldh * nv);
    double* g = C.alloc<double>((int64_t)ldh * nv);
    double* ycoef = C.alloc<double>((int64_t)ldh * nv);
    double* bn = C.alloc<double>(nv);
    double* est = C.alloc<double>(nv);
    double* rn = C.alloc<double>(nv);
    int* active = C.alloc<int>(nv);
    int* want = C.alloc<int>(nv);
    int* taken = C.alloc<int>(nv);
    int* flag = C.alloc<int>(1);
    if (C.rc) return C.rc;
    int cap = std::min(maxit, 48) + 1;
    double* Vb = C.alloc<double>((int64_t)cap * n * nrhs);
    double* Zb = C.alloc<double>((int64_t)cap * n * nrhs);   // Z_j = M^{-1} V_j (flexible GMRES)
    const int dS = dot_chunks(n / nseg);                       // row chunks of a dot product
    double* dpart = C.alloc<double>((int64_t)cap * nv * dS);   // their partial sums
    // out[i + v * nout] = dot(U_i[v], W[v]) for i < nvec, every virtual column v
    auto dots = [&](const double* U, int nvec, const double* W, double* out, int nout, double fl, double by) {
        SPAQR_LAUNCH(KK_GMRES_ORTH, fl, by, st,
                     k_dots_part<<<dim3((unsigned)(nvec * nv), (unsigned)dS), NT, 0, st>>>(n, nrhs, vc, U, nvec, W,
                                                                                        dpart, dS));
        SPAQR_LAUNCH(KK_GMRES_ORTH, 0.0, 8.0 * nvec * nv * dS, st,
                     k_dots_sum<<<(unsigned)((nvec * nv + 255) / 256), 256, 0, st>>>(nvec, nv, dpart, dS, out, nout));
    };
    if (C.rc) return C.rc;
    C.cuda(cudaMemsetAsync(flag, 0, sizeof(int), st));
    ApplyGraph ag;
    double* Vin = nullptr;
    double* Zout = nullptr;
    bool use_graph = false;
    if (graphs) {
        Vin = C.alloc<double>(n * nrhs);
        Zout = C.alloc<double>(n * nrhs);
        if (C.rc) return C.rc;
        use_graph = capture_apply(F, nrhs, Vin, Zout, st, ws, flag, ag);
    }
    C.cuda(cudaMemsetAsync(H, 0, sizeof(double) * hstride * nv, st));
    C.cuda(cudaMemsetAsync(g, 0, sizeof(double) * ldh * nv, st));
    // X0 = X; r0 = B - A X0 (into V_0); beta = ||r0||; ||b||
    SPAQR_LAUNCH(KK_GMRES_SMALL, 0.0, 16.0 * n * nrhs, st, k_copy_cols<<<nbl, 256, 0, st>>>(n, nrhs, dX, lx, X0, n));
    SPAQR_LAUNCH(KK_SPMV, 2.0 * nnz * nrhs, 12.0 * nnz + (8.0 * nnz + 16.0 * n) * nrhs, st,
                 k_residual<<<nbl, 256, 0, st>>>(n, nrhs, rp, ci, va, X0, n, dB, lb, Vb));
    SPAQR_LAUNCH(KK_GMRES_SMALL, 0.0, 16.0 * n * nrhs, st, k_copy_cols<<<nbl, 256, 0, st>>>(n, nrhs, dB, lb, Wv, n));
    dots(Wv, 1, Wv, bn, 1, 2.0 * n * nrhs, 16.0 * n * nrhs);   // ||b||^2
    dots(Vb, 1, Vb, hn, 1, 2.0 * n * nrhs, 16.0 * n * nrhs);   // ||r0||^2
    C.launched();
    std::vector<double> hb(nv), hr(nv), hest(nv), hres(nv, 1.0);
    std::vector<int> hact(nv, 1), hit(nv, 0), hwant(nv, 0);
    C.cuda(cudaMemcpyAsync(hb.data(), bn, 8 * nv, cudaMemcpyDeviceToHost, st));
    C.cuda(cudaMemcpyAsync(hr.data(), hn, 8 * nv, cudaMemcpyDeviceToHost, st));
    C.cuda(cudaStreamSynchronize(st));
    if (C.rc) return C.rc;
    std::vector<double> hg((size_t)ldh * nv, 0.0);
    for (int v = 0; v < nv; v++) {
        hb[v] = std::sqrt(hb[v]);
        hr[v] = std::sqrt(hr[v]);
        if (hb[v] == 0.0) {
            // b = 0: x = 0
            hact[v] = 0;
            hres[v] = 0.0;
            C.cuda(cudaMemsetAsync(dX + (int64_t)(v / nseg) * lx + seg_base(v), 0, 8 * seg_len(v), st));
        } else if (hr[v] / hb[v] <= tol) {
            hact[v] = 0;  // the initial guess already satisfies tol
            hres[v] = hr[v] / hb[v];
        }
        hg[(int64_t)v * ldh] = hr[v];
    }
    C.cuda(cudaMemcpyAsync(bn, hb.data(), 8 * nv, cudaMemcpyHostToDevice, st));
    C.cuda(cudaMemcpyAsync(g, hg.data(), 8 * ldh * nv, cudaMemcpyHostToDevice, st));
    C.cuda(cudaMemcpyAsync(hn, hr.data(), 8 * nv, cudaMemcpyHostToDevice, st));
    C.cuda(cudaMemcpyAsync(active, hact.data(), 4 * nv, cudaMemcpyHostToDevice, st));
    SPAQR_LAUNCH(KK_GMRES_SMALL, 1.0 * n * nrhs, 16.0 * n * nrhs, st,
                 k_scale_cols<<<nbl, 256, 0, st>>>(n, nrhs, vc, Vb, hn));  // V_0 = r0 / beta
    C.launched();
    int nact = 0;
    for (int v = 0; v < nv; v++) nact += hact[v];
    std::vector<double> hnv(nv), hrn(nv);
    std::vector<int> take(nv, 0);
    int j = 0;
    for (; j < maxit && nact > 0 && C.rc == SPAQR_OK; j++) {
        if (j + 1 >= cap) {
            const int ncap = std::min(maxit, 2 * cap) + 1;
            double* nvb = C.alloc<double>((int64_t)ncap * n * nrhs);
            double* nzb = C.alloc<double>((int64_t)ncap * n * nrhs);
            if (C.rc) break;
            C.cuda(cudaMemcpyAsync(nvb, Vb, sizeof(double) * cap * n * nrhs, cudaMemcpyDeviceToDevice, st));
            C.cuda(cudaMemcpyAsync(nzb, Zb, sizeof(double) * cap * n * nrhs, cudaMemcpyDeviceToDevice, st));
            C.release(Vb);
            C.release(Zb);
            C.release(dpart);
            Vb = nvb;
            Zb = nzb;
            cap = ncap;
            dpart = C.alloc<double>((int64_t)cap * nv * dS);
            if (C.rc) break;
        }
        double* Vj = Vb + (int64_t)j * n * nrhs;
        double* Zj = Zb + (int64_t)j * n * nrhs;
        // z_j = M^{-1} v_j (kept: flexible GMRES) ; w = A z_j
        if (use_graph) {
            C.cuda(cudaMemcpyAsync(Vin, Vj, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, st));
            C.cuda(cudaGraphLaunch(ag.exec, st));
            C.cuda(cudaMemcpyAsync(Zj, Zout, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, st));
            prof_add_tally(ag.tally, 1);
        } else {
            int rc = apply_device(F, nrhs, Vj, n, Zj, n, st, ws, flag);
            if (rc != SPAQR_OK) { C.cuda(cudaGetLastError()); break; }
        }
        SPAQR_LAUNCH(KK_SPMV, 2.0 * nnz * nrhs, 12.0 * nnz + (8.0 * nnz + 8.0 * n) * nrhs, st,
                     k_spmv<<<nbl, 256, 0, st>>>(n, nrhs, rp, ci, va, Zj, n, Wv, n));
        // classical Gram-Schmidt, twice
        const double fo = 2.0 * n * (j + 1) * nrhs;
        dots(Vb, j + 1, Wv, h1, ldh, fo, 8.0 * n * (j + 2) * nrhs);
        SPAQR_LAUNCH(KK_GMRES_ORTH, fo, 8.0 * n * (j + 3) * nrhs, st,
                     k_orth_update<<<nbl, 256, 0, st>>>(n, nrhs, vc, Vb, j + 1, h1, ldh, Wv, active));
        dots(Vb, j + 1, Wv, h2, ldh, fo, 8.0 * n * (j + 2) * nrhs);
        SPAQR_LAUNCH(KK_GMRES_ORTH, fo, 8.0 * n * (j + 3) * nrhs, st,
                     k_orth_update<<<nbl, 256, 0, st>>>(n, nrhs, vc, Vb, j + 1, h2, ldh, Wv, active));
        dots(Wv, 1, Wv, hn, 1, 2.0 * n * nrhs, 16.0 * n * nrhs);
        SPAQR_LAUNCH(KK_GMRES_SMALL, 1.0 * nv, 16.0 * nv, st, k_sqrtv<<<1, 32, 0, st>>>(nv, hn));
        C.launched();
        SPAQR_LAUNCH(KK_GMRES_SMALL, 1.0 * n * nrhs, 16.0 * n * nrhs, st,
                     k_normalize<<<nbl, 256, 0, st>>>(n, nrhs, vc, Wv, hn, Vb + (int64_t)(j + 1) * n * nrhs, active));
        SPAQR_LAUNCH(KK_GMRES_SMALL, 6.0 * (j + 1) * nv, 16.0 * (j + 2) * nv, st,
                     k_givens<<<nbv, 32, 0, st>>>(nv, j, H, ldh, hstride, h1, h2, hn, cs, sn, g, ldh, bn, est,
                                                  active));
        C.launched();
        C.cuda(cudaMemcpyAsync(hest.data(), est, 8 * nv, cudaMemcpyDeviceToHost, st));
        C.cuda(cudaMemcpyAsync(hnv.data(), hn, 8 * nv, cudaMemcpyDeviceToHost, st));
        C.cuda(cudaStreamSynchronize(st));
        if (C.rc) break;
        bool anyw = false;
        for (int v = 0; v < nv; v++) {
            hwant[v] = 0;
            if (!hact[v]) continue;
            hit[v] = j + 1;
            if (hist) hist[(int64_t)v * maxit + j] = hest[v];
            if (hest[v] <= tol || hnv[v] == 0.0 || j == maxit - 1) { hwant[v] = 1; anyw = true; }
        }
        if (!anyw) continue;
        // candidate x = x0 + Z y for the wanted columns; keep it if the
        // recomputed residual meets tol
        C.cuda(cudaMemcpyAsync(want, hwant.data(), 4 * nv, cudaMemcpyHostToDevice, st));
        SPAQR_LAUNCH(KK_GMRES_SMALL, 1.0 * (j + 1) * (j + 1) * nv, 8.0 * (j + 1) * (j + 1) * nv, st,
                     k_hsolve<<<nbv, 32, 0, st>>>(nv, j, H, ldh, hstride, g, ldh, ycoef, want));
        SPAQR_LAUNCH(KK_GMRES_ORTH, 2.0 * n * (j + 1) * nrhs, 8.0 * n * (j + 2) * nrhs, st,
                     k_combine<<<nbl, 256, 0, st>>>(n, nrhs, vc, Zb, j + 1, ycoef, ldh, Zv));
        // trial X into Wv: Wv = X0 + Zv (wanted columns), residual into Zv
        SPAQR_LAUNCH(KK_GMRES_SMALL, 1.0 * n * nrhs, 24.0 * n * nrhs, st,
                     k_accept<<<nbl, 256, 0, st>>>(n, nrhs, vc, X0, n, Zv, Wv, n, want));
        SPAQR_LAUNCH(KK_SPMV, 2.0 * nnz * nrhs, 12.0 * nnz + (8.0 * nnz + 16.0 * n) * nrhs, st,
                     k_residual<<<nbl, 256, 0, st>>>(n, nrhs, rp, ci, va, Wv, n, dB, lb, Zv));
        dots(Zv, 1, Zv, rn, 1, 2.0 * n * nrhs, 16.0 * n * nrhs);
        C.launched();
        C.cuda(cudaMemcpyAsync(hrn.data(), rn, 8 * nv, cudaMemcpyDeviceToHost, st));
        C.cuda(cudaStreamSynchronize(st));
        if (C.rc) break;
        bool anyt = false;
        for (int v = 0; v < nv; v++) {
            take[v] = 0;
            if (!hwant[v]) continue;
            const double rr = std::sqrt(hrn[v]) / hb[v];
            hres[v] = rr;
            if (rr <= tol || hnv[v] == 0.0 || j == maxit - 1) {
                take[v] = 1;
                anyt = true;
                hact[v] = 0;
                nact--;
            }
        }
        if (anyt) {
            // X[:, v] = Wv[:, v] for accepted virtual columns
            C.cuda(cudaMemcpyAsync(taken, take.data(), 4 * nv, cudaMemcpyHostToDevice, st));
            SPAQR_LAUNCH(KK_GMRES_SMALL, 0.0, 16.0 * n * nrhs, st,
                         k_copy_taken<<<nbl, 256, 0, st>>>(n, nrhs, vc, Wv, n, dX, lx, taken));
            C.cuda(cudaMemcpyAsync(active, hact.data(), 4 * nv, cudaMemcpyHostToDevice, st));
        }
    }
    if (!bdev) C.cuda(cudaMemcpy2DAsync(X, ldx * 8, dX, n * 8, n * 8, nrhs, cudaMemcpyDeviceToHost, st));
    int hflag = 0;
    C.cuda(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    C.cuda(cudaStreamSynchronize(st));
    if (C.rc) return C.rc;
    if (hflag) { set_error("zero diagonal in an R factor"); return SPAQR_ERR_SINGULAR; }
    bool ok = true;
    for (int v = 0; v < nv; v++) {
        if (iters) iters[v] = hit[v];
        if (relres) relres[v] = hres[v];
        if (!(hres[v] <= tol)) ok = false;
    }
    if (!ok) { set_error("GMRES did not reach tol within maxit"); return SPAQR_ERR_NOT_CONVERGED; }
    return SPAQR_OK;
}

}  // namespace

extern "C" int spaqr_gmres(const spaqr_factor_t* F, const spaqr_csr* A, int nrhs, const double* B, int64_t ldb,
                           double* X, int64_t ldx, double tol, int maxit, int* iters, double* relres, void* stream) {
    return gmres_impl(F, A, nrhs, 1, nullptr, B, ldb, X, ldx, tol, maxit, iters, relres, stream);
}

extern "C" int spaqr_gmres_history(const spaqr_factor_t* F, const spaqr_csr* A, int nrhs, const double* B,
                                   int64_t ldb, double* X, int64_t ldx, double tol, int maxit, int* iters,
                                   double* relres, double* history, void* stream) {
    using namespace spaqr;
    if (!history) { set_error("history is NULL (use spaqr_gmres)"); return SPAQR_ERR_INVALID_ARG; }
    return gmres_impl(F, A, nrhs, 1, nullptr, B, ldb, X, ldx, tol, maxit, iters, relres, stream, history);
}

extern "C" int spaqr_gmres_batch(const spaqr_factor_t* F, const spaqr_csr* A, int count, const int64_t* part_ptr,
                                 int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx, double tol,
                                 int maxit, int* iters, double* relres, void* stream) {
    if (!F || !part_ptr || count < 1) { set_error("null argument or count < 1"); return SPAQR_ERR_INVALID_ARG; }
    if (part_ptr[0] != 0 || part_ptr[count] != F->n) {
        set_error("part_ptr must run from 0 to the batch's n");
        return SPAQR_ERR_INVALID_ARG;
    }
    for (int s = 0; s < count; s++)
        if (part_ptr[s + 1] <= part_ptr[s]) { set_error("empty or decreasing part"); return SPAQR_ERR_INVALID_ARG; }
    return gmres_impl(F, A, nrhs, count, part_ptr, B, ldb, X, ldx, tol, maxit, iters, relres, stream);
}

extern "C" int spaqr_autotune(spaqr_factor_t* F, int nrhs, void* stream, double* ms_rule, double* ms_tuned) {
    if (!F || nrhs < 1) { set_error("null factor or nrhs < 1"); return SPAQR_ERR_INVALID_ARG; }
    if (prof_on()) { set_error("autotuning needs profiling off"); return SPAQR_ERR_INVALID_ARG; }
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != F->device) cudaSetDevice(F->device);
    SCtx C;
    C.st = (cudaStream_t)stream;
    cudaStream_t st = C.st;
    const int64_t n = F->n;
    const int64_t wdbl = (F->ws_rows * nrhs * F->esz + 7) / 8;
    double* ws = C.alloc<double>(wdbl);
    double* snap = C.alloc<double>(wdbl);
    double* B = C.alloc<double>(n * nrhs);
    double* X = C.alloc<double>(n * nrhs);
    int* flag = C.alloc<int>(1);
    if (C.rc) return C.rc;
    C.cuda(cudaMemsetAsync(flag, 0, sizeof(int), st));
    k_fill_pattern<<<(unsigned)((n * nrhs + 255) / 256), 256, 0, st>>>(n * nrhs, B);
    C.launched();
    // one application by the rules fills the level vectors
    int rc = apply_with(F, nrhs, B, n, X, n, st, ws, flag, nullptr);
    if (rc != SPAQR_OK) { C.cuda(cudaGetLastError()); return C.rc ? C.rc : rc; }
    C.cuda(cudaMemcpyAsync(snap, ws, sizeof(double) * wdbl, cudaMemcpyDeviceToDevice, st));
    auto tt = std::make_shared<TuneTable>();
    rc = F->precision == SPAQR_FP32
             ? autotune_t<float>(F, nrhs, st, (float*)ws, (float*)snap, flag, *tt)
             : autotune_t<double>(F, nrhs, st, ws, snap, flag, *tt);
    if (rc != SPAQR_OK) { set_error("autotuning launch failed"); return rc; }
    // whole applications, rules vs table (best of three)
    cudaEvent_t e0, e1;
    C.cuda(cudaEventCreate(&e0));
    C.cuda(cudaEventCreate(&e1));
    if (C.rc) return C.rc;
    auto time_apply = [&](const TuneTable* t) {
        float best = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
            cudaEventRecord(e0, st);
            apply_with(F, nrhs, B, n, X, n, st, ws, flag, t);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        return (double)best;
    };
    tt->ms_rule = time_apply(nullptr);
    tt->ms_tuned = time_apply(tt.get());
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    C.cuda(cudaStreamSynchronize(st));
    if (cur != F->device) cudaSetDevice(cur);
    if (C.rc) return C.rc;
    if (ms_rule) *ms_rule = tt->ms_rule;
    if (ms_tuned) *ms_tuned = tt->ms_tuned;
    {
        std::lock_guard<std::mutex> lk(F->tune_mu);
        auto& v = F->tunes;
        v.erase(std::remove_if(v.begin(), v.end(), [&](const std::shared_ptr<const TuneTable>& t) {
                    return t->nrhs == nrhs;
                }),
                v.end());
        if (tt->ms_tuned < tt->ms_rule) v.push_back(tt);   // keep the rules where tuning does not pay
    }
    return SPAQR_OK;
}

extern "C" int spaqr_factor_tuning(const spaqr_factor_t* F, int nrhs, int32_t* forms, int cap, int* count) {
    if (!F || !count || (cap > 0 && !forms)) { set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    const std::shared_ptr<const TuneTable> tt = F->tune_exact(nrhs);
    std::vector<int32_t> v;
    if (tt) {
        for (int k = 0; k < F->L; k++) {
            for (uint8_t f : tt->ff[k]) v.push_back(f);
            v.push_back(tt->ssf[k]);
            v.push_back(tt->ssb[k]);
            v.push_back(tt->fb[k]);
        }
    }
    *count = (int)v.size();
    for (int i = 0; i < (int)v.size() && i < cap; i++) forms[i] = v[i];
    return SPAQR_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free solve.  The level vectors live in one file-scope device
// array instead of a per-call cudaMallocAsync; its last 32 doubles hold the
// singular flag.  Host code may not pass the symbol itself to a kernel (in
// host code it names a host-side stand-in), so its device address is looked up
// once per device with cudaGetSymbolAddress and cached.
// ---------------------------------------------------------------------------

static __device__ __align__(256) double g_noalloc_scratch[SPAQR_NOALLOC_SCRATCH_DOUBLES + 32];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[128] = {nullptr};
}  // namespace

extern "C" int spaqr_solve_noalloc(const spaqr_factor_t* F, int nrhs, const double* B, int64_t ldb, double* X,
                                   int64_t ldx, void* stream) {
    if (!F || !B || !X) { set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    if (nrhs < 0 || ldb < F->n || ldx < F->n) { set_error("bad nrhs or leading dimension"); return SPAQR_ERR_INVALID_ARG; }
    if (nrhs == 0) return SPAQR_OK;
    if (B != X) {
        const char* b0 = (const char*)B;
        const char* b1 = (const char*)(B + (ldb * (nrhs - 1) + F->n));
        const char* x0 = (const char*)X;
        const char* x1 = (const char*)(X + (ldx * (nrhs - 1) + F->n));
        if (b0 < x1 && x0 < b1) { set_error("B and X overlap"); return SPAQR_ERR_INVALID_ARG; }
    } else if (ldb != ldx) {
        set_error("aliased B and X need the same leading dimension");
        return SPAQR_ERR_INVALID_ARG;
    }
    const int64_t need = (F->ws_rows * (int64_t)nrhs * F->esz + 7) / 8;
    if (need > (int64_t)SPAQR_NOALLOC_SCRATCH_DOUBLES) {
        set_error("spaqr_solve_noalloc: needs " + std::to_string(need) + " scratch doubles, the fixed array holds " +
                  std::to_string((int64_t)SPAQR_NOALLOC_SCRATCH_DOUBLES) + "; use fewer right-hand sides per call");
        return SPAQR_ERR_INVALID_ARG;
    }
    if (!is_device_ptr(B) || !is_device_ptr(X)) {
        set_error("spaqr_solve_noalloc takes device pointers only");
        return SPAQR_ERR_INVALID_ARG;
    }
    const int dev = F->device;
    if (dev < 0 || dev >= 128) { set_error("device index out of range"); return SPAQR_ERR_INVALID_ARG; }
    if (check_on_device(B, dev, "B") != SPAQR_OK || check_on_device(X, dev, "X") != SPAQR_OK)
        return SPAQR_ERR_INVALID_ARG;
    DeviceGuard dg(dev);   // the caller's device is current again on every return
    double* ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                set_error(std::string("cudaGetSymbolAddress of the solve scratch failed: ") + cudaGetErrorString(e));
                return SPAQR_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = (double*)p;
        }
        ws = g_noalloc_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    int* flag = reinterpret_cast<int*>(ws + SPAQR_NOALLOC_SCRATCH_DOUBLES);
    // the flag must start at zero; the level vectors are written before read
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("CUDA: ") + cudaGetErrorString(e));
        return SPAQR_ERR_CUDA;
    }
    const int rc = apply_device(F, nrhs, B, ldb, X, ldx, st, ws, flag);   // sets the message on failure
    if (rc != SPAQR_OK) return rc;
    int hflag = 0;
    e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("CUDA: ") + cudaGetErrorString(e));
        return SPAQR_ERR_CUDA;
    }
    if (hflag) { set_error("zero diagonal in an R factor"); return SPAQR_ERR_SINGULAR; }
    return SPAQR_OK;
}
