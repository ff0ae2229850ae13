// Task descriptors handed from the host orchestration to the kernels, and the
// factor object.  Plain structs (device arrays of them are uploaded per launch).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <mutex>
#include <vector>

#include "spaqr_internal.h"

namespace spaqr {

// Householder QR of an m x n block in place (front of a separator, Section
// 2.4, or diagonal block of an interface, Section 2.5).
template <class real>
struct QRTask {
    real* A;
    int64_t lda;
    int m, n;
    real* tau;   // min(m, n)
    real* T;     // t x t block-diagonal T, ld = t
    real* Dinv;  // inverted diagonal blocks of R (t x NB, ld t), or null
    int* singular; // set on a zero diagonal of R
    double sign_tol;  // reflector sign: alpha < -sign_tol |column| counts as negative (0: alpha < 0)
};

// Rows of a front inside another column panel (or inside a solve vector).
struct Seg {
    int64_t off;   // first row
    int len;
    int pos;       // first row of the segment within the list's rows (sum of the earlier lengths)
};

// One front applied to one column panel (Section 2.4: H_s^T on the columns
// C(s) restricted to the rows R(s)).
template <class real>
struct ApplyFront {
    const real* V;   // front panel (reflectors below the diagonal)
    const real* T;
    int64_t ldv;
    int m, n;          // front rows, reflectors
    int seg_begin, nseg;
};

// A chunk of columns of panel j, with the fronts to apply in order.
template <class real>
struct ApplyTask {
    real* B;         // first column of the chunk
    int64_t ldb;
    int q;             // chunk width
    int fr_begin, nfr;
    int m_max;         // largest front in the list (row map size)
};

// Block (i, j) <- U_i^T A_ij R_j^{-1} (Section 2.5).
template <class real>
struct ScaleTask {
    real* A;
    int64_t lda;
    int mi, nj;
    const real* Vi;   // diagonal block i after its QR (reflectors below the diagonal)
    int64_t ldvi;
    const real* Ti;   // n_i x n_i, ld n_i
    const real* Rj;   // diagonal block j (R on and above the diagonal)
    int64_t ldrj;
    const real* Dj;   // inverted diagonal NB blocks of R_j (n_j x NB, ld n_j)
    int q;              // column chunk for the U^T product
};

// A piece of a ScaleTask: columns [off, off + len) for the U^T product, or
// rows [off, off + len) for the R^{-1} product.
struct ScalePiece {
    int task;
    int off, len;
};

// Merge of a level that is not sparsified (Section 2.6): the interface rows
// of a chunk of columns of one column panel are copied into the merged
// panel of the next level, row segment by row segment.
template <class real>
struct CopyCol {
    const real* A;    // first column of the chunk in the level's panel
    int64_t lda;
    real* D;          // the same column in the merged panel
    int64_t ldd;
    int ncols;
    int seg_begin, nseg;
    int pad;
};
struct RowSeg {
    int64_t src, dst;   // first row in the panel / in the merged panel
    int len;
    int pad;
};

// Column segment of M_p = [A_{k p}^T ... | A_{p j} ...] (Section 2.5).
template <class real>
struct GatherSeg {
    const real* src;
    int64_t ld;
    int rows, cols;     // of the source block
    int transpose;      // 1: src is A_{k p} (n_k x n_p) and enters as its transpose
    int col_off;        // first column in M_p
};

// Truncated column-pivoted QR of M_p (rank rule of Section 4).
template <class real>
struct CPQRTask {
    real* M;          // scratch n_p x ncols, ld n_p
    real* norms;      // scratch ncols
    int np, ncols;
    int seg_begin, nseg;
    real* V;          // out: n_p x kmax explicit reflectors, ld n_p
    real* tau;        // out: kmax
    real* T;          // out: r x r compact-WY, ld kmax
    double* rdiag;    // out: pivot norms (FP64), kmax + 1 entries
    int* rank;          // out
    int kmax;           // min(n_p, ncols)
};

// New block (r_i x r_j) = [L_i^T A_ij Q_j](keep rows, 0:r_j) (coarse rows and
// columns), written at its place in the merged block of the next level
// (Section 2.6); or a plain copy when the level is not sparsified.  The left
// reflectors L_i are Q_i (scaled form, Section 2.5: keep rows 0..r_i) or the
// Householder H_i of the fine columns (unscaled form, Section 3.2: keep rows
// f_i..n_i).
template <class real>
struct SparsifyTask {
    const real* A;
    int64_t lda;
    int mi, nj;
    const real* Vi;   // left reflectors, n_i rows, ld n_i
    const real* Ti;   // ld ldti
    int ri, ldti;     // kept rows, T leading dimension
    int li, lkeep;    // left reflectors, first kept row
    int lexp, pad;    // Vi holds its unit diagonal explicitly
    const real* Vj;
    const real* Tj;
    int rj, ldtj;
    real* D;
    int64_t ldd;
    real* scratch;    // n_i x n_j
    int mode;           // 0 sparsify, 1 identity r_i, 2 copy
};

// Reflectors applied to a block: B <- Q^T B over a chunk of columns (left) or
// B <- B Q over a chunk of rows (right); pieces are ScalePiece ranges.
template <class real>
struct ReflTask {
    const real* V;    // m rows, ld ldv
    const real* T;    // ld ldt
    real* B;
    int64_t ldv, ldb;
    int m, t, ldt;
    int vexp;           // V holds its unit diagonal explicitly
    int right;
    int pad;
};

// sigma_p = 1 / sigma_min(A_p) from R of A_p = Q R (Lemma 1).
template <class real>
struct SigmaTask {
    const real* R;    // n x n upper triangular, ld ldr
    int64_t ldr;
    double* work;     // (kmax + 3) * n doubles
    double* sigma;    // out
    int* singular;      // set on a zero diagonal of R
    int n, kmax;
};

// C = sigma A^T B for the unscaled M_p (n x n A_pp, n x nc A_pj; C ld n).
template <class real>
struct AtbTask {
    const real* A;
    const real* B;
    real* C;
    const double* sigma;
    int64_t lda, ldb;
    int n, nc;
};

// ---------------------------------------------------------------------------
// solve descriptors
// ---------------------------------------------------------------------------

template <class real>
struct SolveFront {
    const real* V;   // front panel: reflectors below the diagonal, R_ss on top
    const real* T;
    const real* Dinv;  // inverted diagonal blocks of R_ss (n x NB, ld n)
    int64_t ldv;
    int m, n;
    int seg_begin, nseg;   // rows R(s) in the level vector (first segment = s)
    int rsj_begin, nrsj;
};

template <class real>
struct SolveRsj {
    const real* R;   // n_s x n_j block of row s in column j
    int64_t ldr;
    int nj;
    int pad;
    int64_t xoff;      // rows of j in the level vector
};

// Launch shapes of the wide solve forms.
constexpr int kWideCS = 8;        // CTAs per thread-block cluster
constexpr int kWideMinM = 128;    // rows of a front from which a cluster per front can pay (forward)
constexpr int kWideMinN = 32;     // size of an interface from which a cluster can pay
constexpr int kTileRows = 64;     // rows of an R_sj tile
constexpr int kTileK = 256;       // columns of an R_sj tile chunk
constexpr int kTileQ = 16;        // right-hand sides per R_sj tile

// Wide form of the backward front step, for levels with few fronts: the
// products R_sj x_j run as tiles over (front, row block, K chunk) and write
// partial sums, which the cluster back substitution adds in chunk order.
// A piece is a column range of one R_sj block (a SolveRsj with R and xoff
// advanced to the range).
struct RsjTile {
    int front;          // index into the device SolveFront array
    int row0, nrows;    // rows of R_s* (within the front's n_s)
    int piece_begin, npiece;
    int kc;             // chunk index within the front
    int64_t zoff;       // the front's partials: rows zoff + kc * n_s + r
};

struct WideFront {
    int front;          // index into the device SolveFront array
    int nkc;            // K chunks (0: no R_sj blocks)
    int64_t zoff;
};

// Scaling + sparsification (or plain carry-over) of one cluster that survives
// a level.
template <class real>
struct SolveSS {
    int64_t off;       // rows in this level's vector
    int64_t noff;      // rows of its coarse part in the next level's vector
    int np, r;
    const real* UV;  // diagonal block after the scaling QR (null: not scaled)
    int64_t lduv;
    const real* UT;  // n_p x n_p
    const real* UD;  // inverted diagonal blocks of R_pp (n_p x NB, ld n_p)
    const real* QV;  // n_p x r explicit
    const real* QT;  // ld kmax
    int ldqt;
    int f;             // unscaled form: fine unknowns (0: scaled form)
    // unscaled form (Section 3.2): H_p of the fine columns (reflectors below
    // the diagonal of HR[:, r:], T blocks HT ld f) with R_ff on top of them,
    // R_fc = HR[0:f, 0:r], inverted diagonal blocks of R_ff in HD (f x NB)
    const real* HR;
    const real* HT;
    const real* HD;
};

}  // namespace spaqr

// ---------------------------------------------------------------------------
// factor object
// ---------------------------------------------------------------------------

struct SolveLevelHost {
    int64_t rows = 0;         // length of the level vector
    int64_t ws_off = 0;       // offset (in doubles, per RHS column) in the solve workspace
    std::vector<int> colour_ptr;   // fronts grouped by colour: [colour_ptr[c], colour_ptr[c+1])
    int front_begin = 0, nfront = 0;  // into the device SolveFront array
    int ss_begin = 0, nss = 0;        // into the device SolveSS array
    int max_front_m = 0, max_front_n = 0, max_ss_n = 0, max_ss_r = 0;
    // algorithmic work of the level's solve launches: flops per RHS, bytes of
    // factor data read once plus vector bytes per RHS
    std::vector<double> ff_flops, ff_fixed, ff_vec;   // forward fronts, per colour
    double ssf_flops = 0, ssf_fixed = 0, ssf_vec = 0; // forward scale/sparsify
    double ssb_flops = 0, ssb_fixed = 0, ssb_vec = 0; // backward scale/sparsify
    double fb_flops = 0, fb_fixed = 0, fb_vec = 0;    // backward fronts
    // staged / cluster forms: tallest front per forward colour; the R_sj
    // tiles of the backward step (bwd_tiles: planned for this level)
    std::vector<int> ff_maxm;
    bool bwd_tiles = false;
    int tile_begin = 0, ntile = 0, wf_begin = 0;
    double rt_flops = 0, rt_fixed = 0, rt_vec = 0;     // R_sj tiles
};

// Launch forms chosen by spaqr_autotune for one right-hand-side count:
// per unit of the application (forward colour, forward / backward
// scale-sparsify, backward fronts of a level) 0 = rule, 1 = one CTA per
// front / interface, 2 = thread-block cluster per front / interface.
struct TuneTable {
    int nrhs = 0;
    std::vector<std::vector<uint8_t>> ff;
    std::vector<uint8_t> ssf, ssb, fb;
    double ms_rule = 0.0, ms_tuned = 0.0;
};

// Per-level diagnostics of a factorisation (spaqr_factor_level).
struct LevelDiag {
    int n_fronts = 0, max_front_rows = 0, max_front_cols = 0, n_interfaces = 0;
    int64_t front_rows = 0, front_cols = 0;
    int n_remaining = 0, max_interface = 0;
    int64_t remaining_size = 0, interface_after = 0;
    int64_t block_entries = 0, factor_bytes = 0;
    double phase_ms[4] = {0, 0, 0, 0};
};

// One stored block of the factor (spaqr_factor_block): device location and
// the clusters (first atoms) it belongs to.  Rows are read with stride
// `rstride` elements and columns with stride `ld` (a diagonal is read as a
// column with rstride = ld + 1).
struct BlockRec {
    int level, kind, cluster, other, rows, cols;
    const void* ptr;
    int64_t ld, rstride;
};

struct spaqr_factor_s {
    int device = 0;
    int64_t n = 0;
    int64_t nnz = 0;               // entries of the factored pattern
    int L = 0, skip = 0;
    double eps = 0.0;
    std::vector<void*> allocs;     // device allocations owned by the factor
    int64_t bytes = 0;
    int precision = SPAQR_FP64;    // storage/arithmetic of the factor and its application
    int esz = 8;                   // bytes per element of that type
    double* d_scale = nullptr;     // column scaling D (n), FP64
    int64_t* d_perm = nullptr;     // new -> old
    int64_t* d_rperm = nullptr;    // new -> old row (= d_perm unless rows were matched)
    // solve plan (device arrays of SolveFront<real>, SolveRsj<real>, SolveSS<real>)
    std::vector<SolveLevelHost> lv;
    void* d_fronts = nullptr;
    spaqr::Seg* d_segs = nullptr;
    void* d_rsj = nullptr;
    void* d_ss = nullptr;
    int64_t ws_rows = 0;           // total rows of all level vectors + the R_sj partials
    int64_t zp_off = 0, zp_rows = 0;   // R_sj partial sums of a wide level (rows per RHS)
    void* d_tiles = nullptr;       // RsjTile[]
    void* d_pieces = nullptr;      // SolveRsj<real>[] of the tiles
    void* d_wfronts = nullptr;     // WideFront[]
    // autotuned launch forms, one table per right-hand-side count
    mutable std::mutex tune_mu;
    std::vector<std::shared_ptr<const TuneTable>> tunes;
    // the table for nrhs, else the one tuned for the nearest count (by ratio)
    std::shared_ptr<const TuneTable> tune_for(int nrhs) const {
        std::lock_guard<std::mutex> lk(tune_mu);
        std::shared_ptr<const TuneTable> best;
        double bd = 1e30;
        for (const auto& t : tunes) {
            const double d = t->nrhs > nrhs ? (double)t->nrhs / nrhs : (double)nrhs / t->nrhs;
            if (d < bd) { bd = d; best = t; }
        }
        return best;
    }
    std::shared_ptr<const TuneTable> tune_exact(int nrhs) const {
        std::lock_guard<std::mutex> lk(tune_mu);
        for (const auto& t : tunes)
            if (t->nrhs == nrhs) return t;
        return nullptr;
    }
    // diagnostics
    std::vector<std::vector<std::pair<int, int>>> ranks;   // per level: (size, rank)
    std::vector<std::vector<std::pair<double, double>>> margins;
    std::vector<std::vector<double>> sigmas;               // per level: sigma_p (unscaled form), else 0
    std::vector<std::vector<double>> pivots;               // per level: CPQR pivot norms |R_kk|, interfaces concatenated
    std::vector<std::vector<int32_t>> pivot_off;           // per level: offsets of each interface's norms (n + 1)
    std::vector<LevelDiag> ldiag;
    double phase_ms[4] = {0, 0, 0, 0};
    double flops = 0.0;
    double solve_flops = 0.0;
    int64_t solve_bytes = 0;
    int top_size = 0;
    bool unscaled = false;         // unscaled variant (Section 3.2): narrow solve forms only
    int64_t peak_bytes = 0;        // most device bytes the factorisation held at once
    std::vector<BlockRec> blocks;  // every stored block, level by level (spaqr_factor_block)
    int tc_levels = 0;             // levels whose fronts were applied on the tensor cores
};
