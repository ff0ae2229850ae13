// Host-only check of the block lookups an ordering indexes once for the
// factorisation (StepPlan::diag, colf_*, apply_e, fcol_*, merge_e): every
// entry equals the search it replaces.  Built and run by test_plan_index.py.
#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "spaqr_internal.h"

namespace spaqr {
void set_error(const std::string&) {}
}
using namespace spaqr;

static void grid(int dim, const int* n, std::vector<int64_t>& rp, std::vector<int32_t>& ci, std::vector<double>& va) {
    int64_t N = 1;
    for (int d = 0; d < dim; d++) N *= n[d];
    rp.assign(N + 1, 0);
    ci.clear();
    va.clear();
    const int64_t st[3] = {1, n[0], (int64_t)n[0] * n[1]};
    for (int64_t r = 0; r < N; r++) {
        const int64_t c[3] = {r % n[0], (r / n[0]) % n[1], dim == 3 ? r / ((int64_t)n[0] * n[1]) : 0};
        std::vector<int64_t> nb{r};
        for (int d = 0; d < dim; d++) {
            if (c[d] > 0) nb.push_back(r - st[d]);
            if (c[d] < n[d] - 1) nb.push_back(r + st[d]);
        }
        std::sort(nb.begin(), nb.end());
        for (int64_t x : nb) {
            ci.push_back((int32_t)x);
            va.push_back(x == r ? 4.0 + dim : -1.0 - 0.01 * (double)((r + x) % 7));
        }
        rp[r + 1] = (int64_t)ci.size();
    }
}

static int check(const Ordering& o, const char* what) {
    int bad = 0;
    for (size_t k = 0; k < o.steps.size(); k++) {
        const StepPlan& sp = o.steps[k];
        const int ncl = (int)sp.cl.size();
        for (int j = 0; j < ncl; j++)
            if (sp.diag[j] != sp.find(j, j)) bad++;
        // fronts per column, in processing order, with their row blocks
        for (int j = 0; j < ncl; j++) {
            std::vector<int> want;
            for (size_t f = 0; f < sp.fronts.size(); f++)
                for (size_t t = 1; t < sp.C[f].size(); t++)
                    if (sp.C[f][t] == j) want.push_back((int)f);
            std::vector<int> got(sp.colf_front.begin() + sp.colf_ptr[j], sp.colf_front.begin() + sp.colf_ptr[j + 1]);
            if (got != want) bad++;
            for (int q = sp.colf_ptr[j]; q < sp.colf_ptr[j + 1]; q++) {
                const int f = sp.colf_front[q];
                for (size_t t = 0; t < sp.R[f].size(); t++)
                    if (sp.apply_e[sp.colf_ebase[q] + t] != sp.find(sp.R[f][t], j)) bad++;
            }
        }
        for (size_t f = 0; f < sp.fronts.size(); f++)
            for (size_t t = 1; t < sp.C[f].size(); t++) {
                const int j = sp.C[f][t], base = sp.fcol_ebase[sp.fcol_ptr[f] + t - 1];
                for (size_t u = 0; u < sp.R[f].size(); u++)
                    if (sp.apply_e[base + u] != sp.find(sp.R[f][u], j)) bad++;
            }
        if (k + 1 < o.steps.size()) {
            const StepPlan& sn = o.steps[k + 1];
            for (int j = 0; j < ncl; j++)
                for (int e = sp.colptr[j]; e < sp.colptr[j + 1]; e++) {
                    const int i = sp.rowidx[e];
                    int want = -1;
                    if (!sp.is_front[i] && !sp.is_front[j] && sp.parent[i] >= 0 && sp.parent[j] >= 0)
                        want = sn.find(sp.parent[i], sp.parent[j]);
                    if (sp.merge_e[e] != want) bad++;
                    if (!sp.is_front[i] && !sp.is_front[j] && want < 0) bad++;   // every merged block exists
                }
        }
    }
    std::printf("%s: %d levels, %d mismatches\n", what, (int)o.steps.size(), bad);
    return bad;
}

int main() {
    int bad = 0;
    const int cases[][4] = {{2, 64, 64, 1}, {2, 50, 37, 1}, {3, 12, 12, 12}, {3, 9, 14, 7}};
    for (const auto& c : cases) {
        std::vector<int64_t> rp;
        std::vector<int32_t> ci;
        std::vector<double> va;
        const int dims[3] = {c[1], c[2], c[3]};
        grid(c[0], dims, rp, ci, va);
        Ordering o;
        if (build_ordering(rp.data(), ci.data(), (int64_t)rp.size() - 1, (int64_t)ci.size(), c[0], dims, 0, o) !=
            SPAQR_OK) {
            std::printf("grid ordering failed\n");
            return 1;
        }
        char name[64];
        std::snprintf(name, sizeof(name), "grid %dD %dx%dx%d", c[0], c[1], c[2], c[3]);
        bad += check(o, name);
        Ordering g;
        if (build_ordering_general(rp.data(), ci.data(), va.data(), (int64_t)rp.size() - 1, (int64_t)ci.size(), 0,
                                   SPAQR_MATCH_MAX_PRODUCT, g) != SPAQR_OK) {
            std::printf("general ordering failed\n");
            return 1;
        }
        std::snprintf(name, sizeof(name), "grid-free %dD %dx%dx%d", c[0], c[1], c[2], c[3]);
        bad += check(g, name);
    }
    std::printf(bad ? "FAIL\n" : "ok\n");
    return bad ? 1 : 0;
}
