// C ABI entry points that need no kernels: errors, options, ordering.
#include <cuda_runtime.h>

#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "spaqr_internal.h"

namespace spaqr {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
}  // namespace spaqr

extern "C" const char* spaqr_last_error(void) { return spaqr::g_last_error.c_str(); }

extern "C" void spaqr_opts_default(spaqr_opts* o) {
    if (!o) return;
    o->eps = 1e-2;
    o->nlevels = 0;
    o->skip = 2;
    o->scaling = 1;
    o->precision = SPAQR_FP64;
    o->col_normalize = 1;
    o->stream = nullptr;
}

namespace spaqr {
// A->on_device must say where the arrays are: device memory flagged as host
// would be read by the host, plain host memory flagged as device by the
// kernels.  Pinned and managed memory are readable from both sides.
int check_csr_location(const spaqr_csr* A) {
    const void* ps[3] = {A->rowptr, A->colind, A->val};
    for (const void* p : ps) {
        if (!p) continue;
        cudaPointerAttributes a;
        cudaMemoryType t = cudaMemoryTypeUnregistered;
        if (cudaPointerGetAttributes(&a, p) == cudaSuccess)
            t = a.type;
        else
            cudaGetLastError();
        if (A->on_device ? t == cudaMemoryTypeUnregistered : t == cudaMemoryTypeDevice) {
            set_error(A->on_device ? "A->on_device is set but an array is plain host memory"
                                   : "A->on_device is 0 but an array is device memory");
            return SPAQR_ERR_INVALID_ARG;
        }
    }
    return SPAQR_OK;
}

int check_on_device(const void* p, int dev, const char* what) {
    if (!p) return SPAQR_OK;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return SPAQR_OK;
    }
    if (a.type == cudaMemoryTypeDevice && a.device != dev) {
        set_error(std::string(what) + " is device memory of GPU " + std::to_string(a.device) +
                  ", the call runs on GPU " + std::to_string(dev));
        return SPAQR_ERR_INVALID_ARG;
    }
    return SPAQR_OK;
}

int check_csr_device(const spaqr_csr* A, int dev) {
    if (!A->on_device) return SPAQR_OK;
    if (check_on_device(A->rowptr, dev, "A->rowptr") != SPAQR_OK ||
        check_on_device(A->colind, dev, "A->colind") != SPAQR_OK ||
        check_on_device(A->val, dev, "A->val") != SPAQR_OK)
        return SPAQR_ERR_INVALID_ARG;
    return SPAQR_OK;
}
}  // namespace spaqr

namespace {
int order_impl(const spaqr_csr* A, const spaqr_grid* g, int nlevels, int matching, spaqr_ordering** out) {
    if (!out) { spaqr::set_error("out is NULL"); return SPAQR_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!A) { spaqr::set_error("A is NULL"); return SPAQR_ERR_INVALID_ARG; }
    if (A->n <= 0 || A->nnz < A->n || !A->rowptr || !A->colind) {
        spaqr::set_error("bad CSR sizes or pointers");
        return SPAQR_ERR_INVALID_ARG;
    }
    if (nlevels < 0 || nlevels > 40) { spaqr::set_error("nlevels out of range"); return SPAQR_ERR_INVALID_ARG; }
    if (spaqr::check_csr_location(A) != SPAQR_OK) return SPAQR_ERR_INVALID_ARG;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    const int64_t* rowptr = A->rowptr;
    const int32_t* colind = A->colind;
    if (A->on_device) {
        rp.resize(A->n + 1);
        ci.resize(A->nnz);
        if (cudaMemcpy(rp.data(), A->rowptr, sizeof(int64_t) * (A->n + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(ci.data(), A->colind, sizeof(int32_t) * A->nnz, cudaMemcpyDeviceToHost) != cudaSuccess) {
            spaqr::set_error("copying the device pattern failed");
            return SPAQR_ERR_CUDA;
        }
        rowptr = rp.data();
        colind = ci.data();
    }
    // general matrices (no grid): the row matching uses |a_ij| when values are given
    std::vector<double> vh;
    const double* val = A->val;
    if (!g && val && A->on_device) {
        vh.resize(A->nnz);
        if (cudaMemcpy(vh.data(), A->val, sizeof(double) * A->nnz, cudaMemcpyDeviceToHost) != cudaSuccess) {
            spaqr::set_error("copying the device values failed");
            return SPAQR_ERR_CUDA;
        }
        val = vh.data();
    }
    spaqr_ordering* ord = new (std::nothrow) spaqr_ordering();
    if (!ord) { spaqr::set_error("host allocation failed"); return SPAQR_ERR_OOM; }
    int rc;
    try {
        if (g) {
            int dims[3] = {g->nx, g->ny, g->dim == 3 ? g->nz : 1};
            rc = spaqr::build_ordering(rowptr, colind, A->n, A->nnz, g->dim, dims, nlevels, ord->o);
        } else {
            rc = spaqr::build_ordering_general(rowptr, colind, val, A->n, A->nnz, nlevels, matching, ord->o);
        }
    } catch (const std::bad_alloc&) {
        spaqr::set_error("host allocation failed");
        rc = SPAQR_ERR_OOM;
    } catch (const std::exception& e) {
        spaqr::set_error(std::string("ordering failed: ") + e.what());
        rc = SPAQR_ERR_INVALID_ARG;
    }
    if (rc != SPAQR_OK) { delete ord; return rc; }
    *out = ord;
    return SPAQR_OK;
}
}  // namespace

extern "C" int spaqr_order(const spaqr_csr* A, const spaqr_grid* g, int nlevels, spaqr_ordering** out) {
    return order_impl(A, g, nlevels, SPAQR_MATCH_MAX_PRODUCT, out);
}

extern "C" int spaqr_order_general(const spaqr_csr* A, int nlevels, int matching, spaqr_ordering** out) {
    if (matching != SPAQR_MATCH_GREEDY && matching != SPAQR_MATCH_MAX_PRODUCT) {
        if (out) *out = nullptr;
        spaqr::set_error("matching must be SPAQR_MATCH_GREEDY or SPAQR_MATCH_MAX_PRODUCT");
        return SPAQR_ERR_INVALID_ARG;
    }
    return order_impl(A, nullptr, nlevels, matching, out);
}

extern "C" int spaqr_order_batch(int count, const spaqr_csr* A, const spaqr_grid* g, spaqr_ordering** out) {
    if (!out) { spaqr::set_error("out is NULL"); return SPAQR_ERR_INVALID_ARG; }
    *out = nullptr;
    if (count < 1 || !A || !g) { spaqr::set_error("count < 1 or NULL arrays"); return SPAQR_ERR_INVALID_ARG; }
    std::vector<std::vector<int64_t>> rps(count);
    std::vector<std::vector<int32_t>> cis(count);
    std::vector<const int64_t*> rowptrs(count);
    std::vector<const int32_t*> colinds(count);
    std::vector<int64_t> ns(count), nnzs(count);
    std::vector<int> dims(4 * (size_t)count);
    for (int i = 0; i < count; i++) {
        const spaqr_csr& Ai = A[i];
        if (Ai.n <= 0 || Ai.nnz < Ai.n || !Ai.rowptr || !Ai.colind) {
            spaqr::set_error("bad CSR sizes or pointers of matrix " + std::to_string(i));
            return SPAQR_ERR_INVALID_ARG;
        }
        if (spaqr::check_csr_location(&Ai) != SPAQR_OK) return SPAQR_ERR_INVALID_ARG;
        rowptrs[i] = Ai.rowptr;
        colinds[i] = Ai.colind;
        if (Ai.on_device) {
            rps[i].resize(Ai.n + 1);
            cis[i].resize(Ai.nnz);
            if (cudaMemcpy(rps[i].data(), Ai.rowptr, sizeof(int64_t) * (Ai.n + 1), cudaMemcpyDeviceToHost) !=
                    cudaSuccess ||
                cudaMemcpy(cis[i].data(), Ai.colind, sizeof(int32_t) * Ai.nnz, cudaMemcpyDeviceToHost) != cudaSuccess) {
                spaqr::set_error("copying the device pattern failed");
                return SPAQR_ERR_CUDA;
            }
            rowptrs[i] = rps[i].data();
            colinds[i] = cis[i].data();
        }
        ns[i] = Ai.n;
        nnzs[i] = Ai.nnz;
        dims[4 * i] = g[i].dim;
        dims[4 * i + 1] = g[i].nx;
        dims[4 * i + 2] = g[i].ny;
        dims[4 * i + 3] = g[i].dim == 3 ? g[i].nz : 1;
    }
    spaqr_ordering* ord = new (std::nothrow) spaqr_ordering();
    if (!ord) { spaqr::set_error("host allocation failed"); return SPAQR_ERR_OOM; }
    int rc;
    try {
        rc = spaqr::build_ordering_batch(count, rowptrs.data(), colinds.data(), ns.data(), nnzs.data(), dims.data(),
                                         ord->o);
    } catch (const std::bad_alloc&) {
        spaqr::set_error("host allocation failed");
        rc = SPAQR_ERR_OOM;
    } catch (const std::exception& e) {
        spaqr::set_error(std::string("ordering failed: ") + e.what());
        rc = SPAQR_ERR_INVALID_ARG;
    }
    if (rc != SPAQR_OK) { delete ord; return rc; }
    *out = ord;
    return SPAQR_OK;
}

// ---------------------------------------------------------------------------
// launch accounting
// ---------------------------------------------------------------------------
namespace spaqr {
namespace {
const char* kKindNames[KK_COUNT] = {
    "colscale", "gather", "front_qr", "front_apply", "scale_qr", "scale_apply", "cpqr",
    "sparsify_merge", "solve_perm", "solve_front_fwd", "solve_ss_fwd", "solve_ss_bwd",
    "solve_front_bwd", "spmv", "gmres_orth", "gmres_small", "solve_rsj", "sigma_min",
    "unscaled_sparsify", "sigma_qr", "front_apply_tc", "interface_tc"};
struct Rec { int kind; cudaEvent_t a, b; void* stream; };
std::mutex g_mu;
bool g_prof = false;
int64_t g_launches = 0;
int64_t g_count[KK_COUNT];
double g_ms[KK_COUNT], g_flops[KK_COUNT], g_bytes[KK_COUNT], g_idle[KK_COUNT];
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}
}  // namespace

// The device's default memory pool (cudaMallocAsync) keeps freed memory for
// reuse instead of returning it to the system at every synchronisation: a
// factorisation allocates and frees tens of megabytes of temporaries per
// level around a host synchronisation, and re-mapping them each time left the
// GPU waiting on the host.  Done once per device.
void keep_pool_memory(int device) {
    static std::mutex mu;
    static std::vector<char> done;
    std::lock_guard<std::mutex> lk(mu);
    if (device < 0) return;
    if ((int)done.size() <= device) done.resize(device + 1, 0);
    if (done[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[device] = 1;
}

thread_local LaunchTally* tl_capture = nullptr;

void prof_capture_begin(LaunchTally* t) {
    std::memset(t, 0, sizeof(*t));
    tl_capture = t;
}

void prof_capture_end() { tl_capture = nullptr; }

int prof_begin(void* stream, int kind, double flops, double bytes) {
    if (tl_capture) {   // recorded into a graph: counted when it is replayed
        tl_capture->count[kind]++;
        tl_capture->flops[kind] += flops;
        tl_capture->bytes[kind] += bytes;
        return -1;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_launches++;
    g_count[kind]++;
    g_flops[kind] += flops;
    g_bytes[kind] += bytes;
    if (!g_prof) return -1;
    Rec r;
    r.kind = kind;
    r.stream = stream;
    r.a = get_event();
    r.b = get_event();
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, (cudaStream_t)stream);
    g_recs.push_back(r);
    return (int)g_recs.size() - 1;
}

void prof_end(void* stream, int rec) {
    if (rec < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (rec < (int)g_recs.size()) cudaEventRecord(g_recs[rec].b, (cudaStream_t)stream);
}


void prof_add_tally(const LaunchTally& t, int sign) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (int k = 0; k < KK_COUNT; k++) {
        g_count[k] += sign * t.count[k];
        g_launches += sign * t.count[k];
        g_flops[k] += sign * t.flops[k];
        g_bytes[k] += sign * t.bytes[k];
    }
}

bool prof_on() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_prof;
}

std::atomic<bool> g_graphs{true};
bool graphs_on() { return g_graphs.load(); }

std::atomic<bool> g_tensor_cores{true};
bool tensor_cores_on() { return g_tensor_cores.load(); }

// Host-side fault injection: the allocation that finds the countdown at 0
// reports failure (as a failed cudaMallocAsync would), once; -1 = off.
std::atomic<int64_t> g_fail_alloc{-1};
bool fail_this_alloc() {
    int64_t v = g_fail_alloc.load();
    while (v >= 0)
        if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return v == 0;
    return false;
}

void prof_add(int rec, int kind, double flops, double bytes) {
    (void)rec;
    std::lock_guard<std::mutex> lk(g_mu);
    g_flops[kind] += flops;
    g_bytes[kind] += bytes;
}
}  // namespace spaqr

extern "C" void spaqr_stats_reset(void) {
    using namespace spaqr;
    std::lock_guard<std::mutex> lk(g_mu);
    for (Rec& r : g_recs) {
        cudaEventSynchronize(r.b);
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    g_launches = 0;
    for (int k = 0; k < KK_COUNT; k++) { g_count[k] = 0; g_ms[k] = g_flops[k] = g_bytes[k] = g_idle[k] = 0.0; }
}

extern "C" void spaqr_use_graphs(int on) { spaqr::g_graphs.store(on != 0); }
extern "C" void spaqr_use_tensor_cores(int on) { spaqr::g_tensor_cores.store(on != 0); }

extern "C" void spaqr_test_fail_alloc(int64_t after) { spaqr::g_fail_alloc.store(after < 0 ? -1 : after); }

extern "C" void spaqr_profile(int on) {
    std::lock_guard<std::mutex> lk(spaqr::g_mu);
    spaqr::g_prof = on != 0;
}

extern "C" int spaqr_stats(spaqr_kernel_stat* out, int cap, int* count, int64_t* total_launches) {
    using namespace spaqr;
    if ((cap > 0 && !out) || !count) { set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    std::lock_guard<std::mutex> lk(g_mu);
    // idle gaps: from the end of the previous record on the same stream to
    // the start of this one
    std::vector<std::pair<void*, cudaEvent_t>> last;
    for (Rec& r : g_recs) {
        float ms = 0.0f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            set_error("event timing failed");
            return SPAQR_ERR_CUDA;
        }
        g_ms[r.kind] += ms;
        cudaEvent_t* prev = nullptr;
        for (auto& l : last)
            if (l.first == r.stream) prev = &l.second;
        if (prev) {
            float gap = 0.0f;
            if (cudaEventElapsedTime(&gap, *prev, r.a) == cudaSuccess && gap > 0.0f) g_idle[r.kind] += gap;
            cudaGetLastError();
            *prev = r.b;
        } else {
            last.push_back({r.stream, r.b});
        }
    }
    for (Rec& r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    *count = KK_COUNT;
    if (total_launches) *total_launches = g_launches;
    for (int k = 0; k < KK_COUNT && k < cap; k++) {
        std::memset(out[k].name, 0, sizeof(out[k].name));
        std::strncpy(out[k].name, kKindNames[k], sizeof(out[k].name) - 1);
        out[k].launches = g_count[k];
        out[k].total_ms = g_ms[k];
        out[k].flops = g_flops[k];
        out[k].bytes = g_bytes[k];
        out[k].idle_ms = g_idle[k];
    }
    return SPAQR_OK;
}
