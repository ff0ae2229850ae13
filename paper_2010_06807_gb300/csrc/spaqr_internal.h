// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/spaqr.h"

namespace spaqr {

void set_error(const std::string& msg);

// ---------------------------------------------------------------------------
// Ordering and symbolic plan (host, integer).  Built once per pattern.
// ---------------------------------------------------------------------------

struct NDNode {
    int id = 0, depth = 0, parent = -1, left = -1, right = -1;
    int cut_dim = -1, cut_m = -1, size = 1;  // size = preorder subtree size
    int lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
};

// One level of Algorithm 2 in symbolic form.  Cluster "indices" below are
// positions in `cl` (the active clusters at the start of the level, ascending
// by first atom).
struct StepPlan {
    int level = 0;
    std::vector<int> cl;        // first atom of every active cluster
    std::vector<int> cl_node;   // nested-dissection node of every cluster
    std::vector<char> is_front; // factored at this level
    // block pattern including this level's fill, CSC over cluster indices:
    // column j holds rows rowidx[colptr[j] .. colptr[j+1]) (ascending)
    std::vector<int> colptr, rowidx;
    // fronts in processing order (colour, id)
    std::vector<int> fronts, colour;
    std::vector<std::vector<int>> R, C;   // per front (same order), cluster indices
    // merge: for every non-front cluster, its parent index in the next level's
    // cl (-1 when there is no next level)
    std::vector<int> parent;
    int n_next = 0;
    // position of block (i, j) within the CSC arrays: lookup helper
    int find(int i, int j) const;
    // Lookups derived from the pattern once per ordering (index_plan), so
    // that a factorisation does not search for blocks:
    //  diag[j]: position of block (j, j) (-1 if absent);
    //  per column j, the fronts applied to it in processing order
    //  (colf_front[colf_ptr[j] ..]), each with apply_e[colf_ebase[..] + t] =
    //  position of block (R(s)[t], j) (-1 if absent);
    //  the same bases per front and column C(s)[t], t >= 1:
    //  fcol_ebase[fcol_ptr[f] + t - 1];
    //  merge_e[e]: for a block (i, j) of two non-front clusters, the position
    //  of block (parent[i], parent[j]) in the next level (-1 otherwise).
    std::vector<int> diag;
    std::vector<int> colf_ptr, colf_front, colf_ebase, apply_e;
    std::vector<int> fcol_ptr, fcol_ebase;
    std::vector<int> merge_e;
};

struct Ordering {
    int dim = 2;
    int dims[3] = {1, 1, 1};
    int64_t n = 0, nnz = 0;
    int L = 1;
    std::vector<NDNode> nodes;
    std::vector<int64_t> perm;       // new -> old
    std::vector<int64_t> iperm;      // old -> new
    // general matrices: row r sits with column rowcol[r] (a matching of rows
    // to columns); rperm[new] = old row.  Both empty: rows ordered as columns.
    std::vector<int64_t> rowcol;
    std::vector<int64_t> rperm;
    std::vector<int64_t> atom_ptr;
    std::vector<int32_t> atom_node;
    std::vector<int32_t> atom_of;    // new index -> atom
    std::vector<StepPlan> steps;
    // pattern copies for the numeric phase
    std::vector<int64_t> rowptr;
    std::vector<int32_t> colind;
    // CSC traversal of the CSR entries (deterministic column sums)
    std::vector<int64_t> csc_ptr;    // n + 1
    std::vector<int64_t> csc_entry;  // nnz: CSR entry index, rows ascending per column
    // CSR entry -> offset in the level-1 block arena (column panels)
    std::vector<int64_t> gather_off;
    int64_t arena1_size = 0;
    std::vector<int32_t> plan_code;  // encoded plan (spaqr_ordering_get)
    bool related(int na, int nb) const {
        if (na > nb) { int t = na; na = nb; nb = t; }
        return nb < na + nodes[na].size;
    }
};

int build_ordering_batch(int count, const int64_t* const* rowptrs, const int32_t* const* colinds,
                         const int64_t* ns, const int64_t* nnzs, const int* dims_list, Ordering& o);
int build_ordering(const int64_t* rowptr, const int32_t* colind, int64_t n, int64_t nnz,
                   int dim, const int* dims, int nlevels, Ordering& out);
int build_ordering_general(const int64_t* rowptr, const int32_t* colind, const double* val, int64_t n,
                           int64_t nnz, int nlevels, int matching, Ordering& out);

int num_levels(int64_t n);

// ---------------------------------------------------------------------------
// launch accounting (spaqr_stats)
// ---------------------------------------------------------------------------
enum KernelKind {
    KK_COLSCALE = 0, KK_GATHER, KK_FRONT_QR, KK_FRONT_APPLY, KK_SCALE_QR, KK_SCALE_APPLY, KK_CPQR,
    KK_SPARSIFY, KK_SOLVE_PERM, KK_SOLVE_FRONT_FWD, KK_SOLVE_SS_FWD, KK_SOLVE_SS_BWD, KK_SOLVE_FRONT_BWD,
    KK_SPMV, KK_GMRES_ORTH, KK_GMRES_SMALL, KK_SOLVE_RSJ, KK_SIGMA, KK_UNSCALED, KK_SIGMA_QR, KK_FRONT_APPLY_TC,
    KK_IFACE_TC, KK_COUNT
};
// Call immediately before a launch; returns a record id (or -1).
int prof_begin(void* stream, int kind, double flops, double bytes);
// Call immediately after the launch.
void prof_end(void* stream, int rec);
// Add algorithmic flops to a record known only later (e.g. after ranks).
void prof_add(int rec, int kind, double flops, double bytes);
// Launch tallies: a CUDA-graph capture takes back the launches it recorded
// (nothing ran) and every replay adds them again.
struct LaunchTally {
    int64_t count[KK_COUNT];
    double flops[KK_COUNT], bytes[KK_COUNT];
};
void prof_capture_begin(LaunchTally* t);   // this thread's launches go to *t only
void prof_capture_end();
void prof_add_tally(const LaunchTally& t, int sign);
bool prof_on();
void keep_pool_memory(int device);
bool graphs_on();
bool tensor_cores_on();   // spaqr_use_tensor_cores
bool fail_this_alloc();   // fault injection (spaqr_test_fail_alloc)
int check_csr_location(const spaqr_csr* A);   // A->on_device against where the arrays are
// INVALID_ARG (with the message) when p is device memory of a GPU other than
// dev; host, pinned and managed memory pass.  Kernels on dev would otherwise
// reach another GPU's memory through unified addressing.
int check_on_device(const void* p, int dev, const char* what);
int check_csr_device(const spaqr_csr* A, int dev);   // check_on_device on a device CSR's arrays

}  // namespace spaqr

struct spaqr_ordering {
    spaqr::Ordering o;
};
