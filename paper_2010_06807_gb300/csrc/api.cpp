// C ABI entry points that need no kernels: errors, options, ordering.
#include <cuda_runtime.h>

#include <cstring>
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

extern "C" int spaqr_order(const spaqr_csr* A, const spaqr_grid* g, int nlevels, spaqr_ordering** out) {
    if (!out) { spaqr::set_error("out is NULL"); return SPAQR_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!A) { spaqr::set_error("A is NULL"); return SPAQR_ERR_INVALID_ARG; }
    if (!g) {
        spaqr::set_error("no grid given: hypergraph ordering of general matrices is not built");
        return SPAQR_ERR_UNSUPPORTED;
    }
    if (A->n <= 0 || A->nnz < A->n || !A->rowptr || !A->colind) {
        spaqr::set_error("bad CSR sizes or pointers");
        return SPAQR_ERR_INVALID_ARG;
    }
    if (nlevels < 0 || nlevels > 40) { spaqr::set_error("nlevels out of range"); return SPAQR_ERR_INVALID_ARG; }
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
    int dims[3] = {g->nx, g->ny, g->dim == 3 ? g->nz : 1};
    spaqr_ordering* ord = new (std::nothrow) spaqr_ordering();
    if (!ord) { spaqr::set_error("host allocation failed"); return SPAQR_ERR_OOM; }
    int rc;
    try {
        rc = spaqr::build_ordering(rowptr, colind, A->n, A->nnz, g->dim, dims, nlevels, ord->o);
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
