/* A plain C99 user of the C ABI (include/spaqr.h), host-only calls:
 *   - the geometric ordering of a 5-point pattern on a 40 x 40 grid;
 *   - the general ordering (maximum-product row matching) of the same matrix
 *     with its rows reversed, whose matching must undo the reversal;
 *   - error codes for a bad argument.
 * Prints "ok ..." and returns 0 when every check holds. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "spaqr.h"

static int is_perm(const int64_t* p, int64_t n) {
    char* seen = calloc((size_t)n, 1);
    int ok = seen != NULL;
    for (int64_t i = 0; ok && i < n; i++) {
        if (p[i] < 0 || p[i] >= n || seen[p[i]]) ok = 0;
        else seen[p[i]] = 1;
    }
    free(seen);
    return ok;
}

/* row r of the 5-point matrix: 4 on the diagonal, -1 for each neighbour */
static int64_t stencil_row(int s, int64_t r, int32_t* ci, double* v) {
    const int x = (int)(r % s), y = (int)(r / s);
    int64_t k = 0;
    if (y > 0) { ci[k] = (int32_t)(r - s); v[k++] = -1.0; }
    if (x > 0) { ci[k] = (int32_t)(r - 1); v[k++] = -1.0; }
    ci[k] = (int32_t)r; v[k++] = 4.0;
    if (x < s - 1) { ci[k] = (int32_t)(r + 1); v[k++] = -1.0; }
    if (y < s - 1) { ci[k] = (int32_t)(r + s); v[k++] = -1.0; }
    return k;
}

#define CHECK(cond, what) do { if (!(cond)) { fprintf(stderr, "failed: %s (%s)\n", what, spaqr_last_error()); return 1; } } while (0)

int main(void) {
    const int s = 40;
    const int64_t n = (int64_t)s * s;
    int64_t* rp = malloc((size_t)(n + 1) * sizeof *rp);
    int64_t* rpb = malloc((size_t)(n + 1) * sizeof *rpb);
    int32_t* ci = malloc((size_t)(5 * n) * sizeof *ci);
    int32_t* cib = malloc((size_t)(5 * n) * sizeof *cib);
    double* v = malloc((size_t)(5 * n) * sizeof *v);
    double* vb = malloc((size_t)(5 * n) * sizeof *vb);
    int64_t* perm = malloc((size_t)n * sizeof *perm);
    int64_t* rperm = malloc((size_t)n * sizeof *rperm);
    CHECK(rp && rpb && ci && cib && v && vb && perm && rperm, "host allocation");

    rp[0] = 0;
    for (int64_t r = 0; r < n; r++) rp[r + 1] = rp[r] + stencil_row(s, r, ci + rp[r], v + rp[r]);
    const int64_t nnz = rp[n];
    /* B: row r of B is row n-1-r of A */
    rpb[0] = 0;
    for (int64_t r = 0; r < n; r++) rpb[r + 1] = rpb[r] + stencil_row(s, n - 1 - r, cib + rpb[r], vb + rpb[r]);

    spaqr_opts opts;
    spaqr_opts_default(&opts);
    CHECK(opts.eps == 1e-2 && opts.skip == 2 && opts.precision == SPAQR_FP64, "default options");

    spaqr_csr A;
    A.n = n; A.nnz = nnz; A.rowptr = rp; A.colind = ci; A.val = v; A.on_device = 0;
    spaqr_grid g;
    g.dim = 2; g.nx = s; g.ny = s; g.nz = 1;
    spaqr_ordering* o = NULL;
    CHECK(spaqr_order(&A, &g, 0, &o) == SPAQR_OK && o != NULL, "grid ordering");
    spaqr_ordering_info_t info;
    CHECK(spaqr_ordering_info(o, &info) == SPAQR_OK && info.n == n && info.nnz == nnz, "ordering info");
    CHECK(spaqr_ordering_get(o, perm, NULL, NULL, NULL, NULL) == SPAQR_OK && is_perm(perm, n), "grid perm");
    CHECK(spaqr_ordering_rows(o, rperm) == SPAQR_OK && memcmp(perm, rperm, (size_t)n * sizeof *perm) == 0,
          "grid rows follow the columns");
    const int atoms = info.n_atoms, levels = info.nlevels;
    spaqr_ordering_destroy(o);

    spaqr_csr B = A;
    B.rowptr = rpb; B.colind = cib; B.val = vb;
    o = NULL;
    CHECK(spaqr_order_general(&B, 0, SPAQR_MATCH_MAX_PRODUCT, &o) == SPAQR_OK && o != NULL, "general ordering");
    CHECK(spaqr_ordering_get(o, perm, NULL, NULL, NULL, NULL) == SPAQR_OK && is_perm(perm, n), "general perm");
    CHECK(spaqr_ordering_rows(o, rperm) == SPAQR_OK && is_perm(rperm, n), "general rperm");
    /* the diagonal of row r of B sits in column n-1-r: the matching undoes the reversal */
    for (int64_t k = 0; k < n; k++) CHECK(rperm[k] == n - 1 - perm[k], "matched rows");
    spaqr_ordering_destroy(o);

    o = (spaqr_ordering*)&B;   /* must be reset to NULL on error */
    CHECK(spaqr_order_general(&B, 0, 9, &o) == SPAQR_ERR_INVALID_ARG && o == NULL, "bad matching code");
    CHECK(strlen(spaqr_last_error()) > 0, "error message");
    CHECK(spaqr_order(NULL, &g, 0, &o) == SPAQR_ERR_INVALID_ARG, "NULL matrix");

    printf("ok n=%lld nnz=%lld atoms=%d levels=%d\n", (long long)n, (long long)nnz, atoms, levels);
    free(rp); free(rpb); free(ci); free(cib); free(v); free(vb); free(perm); free(rperm);
    return 0;
}
