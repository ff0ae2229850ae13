// Geometric modified nested dissection and the symbolic spaQR plan (host).
//
// Paper: Section 2.1 (nested dissection on G(A^T A) gives the column
// partition), Section 2.3 (modified nested dissection: the recursion on
// interior + boundary splits separators into interfaces; rows ordered like
// columns for diagonally dominant matrices), Section 2.6 (merge along the
// cluster hierarchy), Section 4 (L = ceil(log2(N/64))).
//
// Readings where the paper is silent:
//  * a separator of G(A^T A) for 5/7-point stencils is two grid planes thick;
//  * cut the longest extent (ties x, y, z) at m = lo + max(0, (ext-2)/2);
//    separator planes [m, m+2), children [lo, m) and [m+2, hi);
//  * the cut of a non-leaf descendant box D splits separator S of box B when D
//    touches S along B's cut dimension and D cuts a tangent dimension; it
//    applies to the nodes of S that, in the remaining tangent dimension(s), lie
//    within D's extent widened by two planes; it classifies them as below,
//    inside or above D's slab;
//  * interfaces after eliminating level l are the classes under cuts of depth
//    <= l-1, the merge after level l removes depth l-1 cuts;
//  * order: nodes by level (leaves first), then preorder; inside a separator
//    atoms in hierarchical order (coarser classes first, classes by their
//    smallest grid index); inside an atom by grid index.
//  * blocks exist only between clusters whose nodes are equal or ancestor /
//    descendant (Section 2.1, Theorem 2.1); a front's rows R(s) are the
//    clusters with a block in column s, its columns C(s) the related clusters
//    with a block in a row of R(s), both taken at the start of the level;
//    fronts sharing a row cluster are ordered by a greedy colouring.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <queue>
#include <set>
#include <system_error>
#include <thread>
#include <exception>
#include <string>
#include <tuple>
#include <unordered_map>

#include "spaqr_internal.h"

namespace spaqr {

int num_levels(int64_t n) {
    if (n <= 64) return 1;
    double v = std::log2((double)n / 64.0);
    int L = (int)std::ceil(v - 1e-12);
    return L < 1 ? 1 : L;
}

// The lookups of StepPlan that a factorisation needs, from the pattern.
static void index_plan(Ordering& o) {
    for (size_t k = 0; k < o.steps.size(); k++) {
        StepPlan& sp = o.steps[k];
        const int ncl = (int)sp.cl.size();
        sp.diag.assign(ncl, -1);
        for (int j = 0; j < ncl; j++) sp.diag[j] = sp.find(j, j);
        sp.colf_ptr.assign(ncl + 1, 0);
        for (size_t f = 0; f < sp.fronts.size(); f++)
            for (size_t t = 1; t < sp.C[f].size(); t++) sp.colf_ptr[sp.C[f][t] + 1]++;
        for (int j = 0; j < ncl; j++) sp.colf_ptr[j + 1] += sp.colf_ptr[j];
        sp.colf_front.assign(sp.colf_ptr[ncl], 0);
        sp.colf_ebase.assign(sp.colf_ptr[ncl], 0);
        std::vector<int> fill(sp.colf_ptr.begin(), sp.colf_ptr.end() - 1);
        std::vector<int> slot;   // (f, t) in front order -> position in colf
        sp.fcol_ptr.assign(sp.fronts.size() + 1, 0);
        for (size_t f = 0; f < sp.fronts.size(); f++) {
            for (size_t t = 1; t < sp.C[f].size(); t++) {
                const int q = fill[sp.C[f][t]]++;
                sp.colf_front[q] = (int)f;
                slot.push_back(q);
            }
            sp.fcol_ptr[f + 1] = (int)slot.size();
        }
        sp.apply_e.clear();
        for (int j = 0; j < ncl; j++)
            for (int q = sp.colf_ptr[j]; q < sp.colf_ptr[j + 1]; q++) {
                sp.colf_ebase[q] = (int)sp.apply_e.size();
                for (int i : sp.R[sp.colf_front[q]]) sp.apply_e.push_back(sp.find(i, j));
            }
        sp.fcol_ebase.assign(slot.size(), 0);
        for (size_t u = 0; u < slot.size(); u++) sp.fcol_ebase[u] = sp.colf_ebase[slot[u]];
        sp.merge_e.assign(sp.rowidx.size(), -1);
        if (k + 1 < o.steps.size() && !sp.parent.empty()) {
            const StepPlan& sn = o.steps[k + 1];
            for (int j = 0; j < ncl; j++) {
                if (sp.is_front[j] || sp.parent[j] < 0) continue;
                for (int e = sp.colptr[j]; e < sp.colptr[j + 1]; e++) {
                    const int i = sp.rowidx[e];
                    if (sp.is_front[i] || sp.parent[i] < 0) continue;
                    sp.merge_e[e] = sn.find(sp.parent[i], sp.parent[j]);
                }
            }
        }
    }
}

int StepPlan::find(int i, int j) const {
    auto b = rowidx.begin() + colptr[j], e = rowidx.begin() + colptr[j + 1];
    auto it = std::lower_bound(b, e, i);
    if (it == e || *it != i) return -1;
    return (int)(it - rowidx.begin());
}

namespace {

struct Builder {
    int dim;
    int dims[3];
    int L;
    std::vector<NDNode> nodes;

    int build(const int* lo, const int* hi, int depth, int parent) {
        int id = (int)nodes.size();
        nodes.push_back(NDNode());
        {
            NDNode& nd = nodes[id];
            nd.id = id;
            nd.depth = depth;
            nd.parent = parent;
            for (int k = 0; k < 3; k++) { nd.lo[k] = lo[k]; nd.hi[k] = hi[k]; }
        }
        if (depth < L - 1) {
            int ext[3];
            for (int k = 0; k < 3; k++) ext[k] = hi[k] - lo[k];
            int c = 0;
            for (int k = 1; k < dim; k++)
                if (ext[k] > ext[c]) c = k;
            int m = lo[c] + (ext[c] >= 2 ? (ext[c] - 2) / 2 : 0);
            int llo[3], lhi[3], rlo[3], rhi[3];
            for (int k = 0; k < 3; k++) { llo[k] = lo[k]; lhi[k] = hi[k]; rlo[k] = lo[k]; rhi[k] = hi[k]; }
            lhi[c] = m;
            rlo[c] = std::min(m + 2, hi[c]);
            int l = build(llo, lhi, depth + 1, id);
            int r = build(rlo, rhi, depth + 1, id);
            NDNode& nd = nodes[id];
            nd.cut_dim = c;
            nd.cut_m = m;
            nd.left = l;
            nd.right = r;
            nd.size = 1 + nodes[l].size + nodes[r].size;
        }
        return id;
    }
};

struct Key {
    int depth, node, k;
    bool operator==(const Key& o) const { return depth == o.depth && node == o.node && k == o.k; }
    bool operator!=(const Key& o) const { return !(*this == o); }
};

bool prefix_equal(const std::vector<Key>& a, const std::vector<Key>& b, int stage) {
    size_t i = 0, j = 0;
    while (true) {
        while (i < a.size() && a[i].depth > stage) i++;
        while (j < b.size() && b[j].depth > stage) j++;
        if (i == a.size() || j == b.size()) return i == a.size() && j == b.size();
        if (a[i] != b[j]) return false;
        i++;
        j++;
    }
}

}  // namespace

namespace {

struct Atom {
    std::vector<int64_t> pts;
    std::vector<Key> key;
};

// Atoms of one separator in hierarchical order (coarser classes first, each
// class by its smallest index), points by index.
void order_atoms(const std::vector<int64_t>& gidx, const std::vector<std::vector<Key>>& keys,
                 std::vector<Atom>& atoms) {
    const size_t np = gidx.size();
    std::vector<int> depths;
    for (auto& kk : keys)
        for (const Key& k : kk) depths.push_back(k.depth);
    std::sort(depths.begin(), depths.end());
    depths.erase(std::unique(depths.begin(), depths.end()), depths.end());
    std::vector<std::vector<int64_t>> scol(depths.size(), std::vector<int64_t>(np));
    for (size_t si = 0; si < depths.size(); si++) {
        const int s = depths[si];
        std::map<std::vector<std::tuple<int, int, int>>, int64_t> minidx;
        std::vector<std::vector<std::tuple<int, int, int>>> cls(np);
        for (size_t i = 0; i < np; i++) {
            for (const Key& kk : keys[i])
                if (kk.depth <= s) cls[i].push_back(std::make_tuple(kk.depth, kk.node, kk.k));
            auto it = minidx.find(cls[i]);
            if (it == minidx.end() || gidx[i] < it->second) minidx[cls[i]] = gidx[i];
        }
        for (size_t i = 0; i < np; i++) scol[si][i] = minidx[cls[i]];
    }
    std::vector<size_t> ord(np);
    for (size_t i = 0; i < np; i++) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) {
        for (size_t si = 0; si < depths.size(); si++)
            if (scol[si][a] != scol[si][b]) return scol[si][a] < scol[si][b];
        return gidx[a] < gidx[b];
    });
    for (size_t t = 0; t < np; t++) {
        const size_t i = ord[t];
        if (atoms.empty() || atoms.back().key != keys[i]) {
            Atom a;
            a.key = keys[i];
            atoms.push_back(std::move(a));
        }
        atoms.back().pts.push_back(gidx[i]);
    }
}

// Geometric nested dissection of one grid with L levels: the tree (depth 0 =
// root) and the atoms of every node, their points as grid indices.
int nd_grid(int dim, const int* dims3, int L, std::vector<NDNode>& nodes_out,
            std::vector<std::vector<Atom>>& node_atoms) {
    Builder b;
    b.dim = dim;
    for (int k = 0; k < 3; k++) b.dims[k] = dims3[k];
    b.L = L;
    int lo0[3] = {0, 0, 0}, hi0[3] = {dims3[0], dims3[1], dims3[2]};
    b.build(lo0, hi0, 0, -1);
    nodes_out = b.nodes;
    const std::vector<NDNode>& nodes = nodes_out;
    const int nn = (int)nodes.size();
    const int64_t stride[3] = {1, dims3[0], (int64_t)dims3[0] * dims3[1]};
    node_atoms.assign(nn, {});
    for (int id = 0; id < nn; id++) {
        const NDNode& nd = nodes[id];
        int lo[3], hi[3];
        for (int k = 0; k < 3; k++) { lo[k] = nd.lo[k]; hi[k] = nd.hi[k]; }
        if (nd.cut_dim >= 0) {
            lo[nd.cut_dim] = nd.cut_m;
            hi[nd.cut_dim] = std::min(nd.cut_m + 2, nd.hi[nd.cut_dim]);
        }
        bool empty = false;
        for (int k = 0; k < 3; k++) if (hi[k] <= lo[k]) empty = true;
        if (empty) continue;
        // points in index order (x fastest)
        std::vector<std::array<int, 3>> pts;
        for (int z = lo[2]; z < hi[2]; z++)
            for (int y = lo[1]; y < hi[1]; y++)
                for (int x = lo[0]; x < hi[0]; x++) pts.push_back({x, y, z});
        const size_t np = pts.size();
        std::vector<int64_t> gidx(np);
        for (size_t i = 0; i < np; i++)
            gidx[i] = pts[i][0] * stride[0] + pts[i][1] * stride[1] + pts[i][2] * stride[2];
        if (nd.cut_dim < 0) {
            Atom a;
            a.pts = gidx;
            node_atoms[id].push_back(std::move(a));
            continue;
        }
        const int c = nd.cut_dim;
        const int left_hi = nodes[nd.left].hi[c];
        const int right_lo = nodes[nd.right].lo[c];
        std::vector<int> cuts;
        for (int d = id + 1; d < id + nd.size; d++) {
            const NDNode& D = nodes[d];
            if (D.cut_dim < 0 || D.cut_dim == c) continue;
            bool dempty = false;
            for (int k = 0; k < 3; k++) if (D.hi[k] <= D.lo[k]) dempty = true;
            if (dempty) continue;
            if (!(D.hi[c] == left_hi || D.lo[c] == right_lo)) continue;
            cuts.push_back(d);
        }
        std::sort(cuts.begin(), cuts.end(), [&](int a, int bb) {
            if (nodes[a].depth != nodes[bb].depth) return nodes[a].depth < nodes[bb].depth;
            return a < bb;
        });
        std::vector<std::vector<Key>> keys(np);
        for (int d : cuts) {
            const NDNode& D = nodes[d];
            const int cd = D.cut_dim;
            for (size_t i = 0; i < np; i++) {
                bool ok = true;
                for (int e = 0; e < dim; e++) {
                    if (e == c || e == cd) continue;
                    if (pts[i][e] < D.lo[e] - 2 || pts[i][e] >= D.hi[e] + 2) { ok = false; break; }
                }
                if (!ok) continue;
                int v = pts[i][cd];
                int kv = v < D.cut_m ? 0 : (v < D.cut_m + 2 ? 1 : 2);
                keys[i].push_back(Key{D.depth, d, kv});
            }
        }
        order_atoms(gidx, keys, node_atoms[id]);
    }

    return SPAQR_OK;
}

// Order, pattern, symbolic plan and gather map of a forest of nested-dissection
// trees (o.nodes in preorder, every tree's leaves at depth o.L - 1) with the
// atoms of every node and the CSR pattern of the whole matrix.
int plan_forest(Ordering& o, const int64_t* rowptr, const int32_t* colind,
                std::vector<std::vector<Atom>>& node_atoms) {
    const std::vector<NDNode>& nodes = o.nodes;
    const int nn = (int)nodes.size();
    const int64_t n = o.n, nnz = o.nnz;
    const int L = o.L;
    // ---- global order ----------------------------------------------------
    std::vector<int> norder(nn);
    for (int i = 0; i < nn; i++) norder[i] = i;
    std::sort(norder.begin(), norder.end(), [&](int a, int bb) {
        if (nodes[a].depth != nodes[bb].depth) return nodes[a].depth > nodes[bb].depth;
        return a < bb;
    });
    o.perm.clear();
    o.atom_ptr.assign(1, 0);
    o.atom_node.clear();
    std::vector<std::vector<Key>> atom_keys;
    for (int id : norder) {
        for (Atom& a : node_atoms[id]) {
            for (int64_t g : a.pts) o.perm.push_back(g);
            o.atom_ptr.push_back((int64_t)o.perm.size());
            o.atom_node.push_back(id);
            atom_keys.push_back(a.key);
        }
    }
    if ((int64_t)o.perm.size() != n) { set_error("ordering lost points"); return SPAQR_ERR_INVALID_ARG; }
    const int na = (int)o.atom_node.size();
    o.iperm.assign(n, 0);
    for (int64_t i = 0; i < n; i++) o.iperm[o.perm[i]] = i;
    o.atom_of.assign(n, 0);
    for (int a = 0; a < na; a++)
        for (int64_t i = o.atom_ptr[a]; i < o.atom_ptr[a + 1]; i++) o.atom_of[i] = a;

    auto stage_first = [&](int stage) {
        std::vector<int> f(na);
        for (int a = 0; a < na; a++) {
            if (a > 0 && o.atom_node[a] == o.atom_node[a - 1] &&
                prefix_equal(atom_keys[a], atom_keys[a - 1], stage))
                f[a] = f[a - 1];
            else
                f[a] = a;
        }
        return f;
    };

    // ---- pattern copies, CSC traversal ------------------------------------
    o.rowptr.assign(rowptr, rowptr + n + 1);
    o.colind.assign(colind, colind + nnz);
    for (int64_t e = 0; e < nnz; e++)
        if (colind[e] < 0 || colind[e] >= n) { set_error("column index out of range"); return SPAQR_ERR_INVALID_ARG; }
    o.csc_ptr.assign(n + 1, 0);
    for (int64_t e = 0; e < nnz; e++) o.csc_ptr[colind[e] + 1]++;
    for (int64_t i = 0; i < n; i++) o.csc_ptr[i + 1] += o.csc_ptr[i];
    o.csc_entry.assign(nnz, 0);
    {
        std::vector<int64_t> fill(o.csc_ptr.begin(), o.csc_ptr.end() - 1);
        for (int64_t r = 0; r < n; r++)
            for (int64_t e = rowptr[r]; e < rowptr[r + 1]; e++) o.csc_entry[fill[colind[e]]++] = e;
    }

    // ---- symbolic plan -------------------------------------------------
    // a row sits at the position of its matched column (rows = columns when
    // there is no matching)
    auto rowpos = [&](int64_t r) { return o.rowcol.empty() ? o.iperm[r] : o.iperm[o.rowcol[r]]; };
    // block pattern: (row cluster, col cluster) by first atom as the key
    // row * na + col, kept sorted and unique (row, then column)
    std::vector<uint64_t> P;
    const uint64_t NA = (uint64_t)na;
    auto key = [NA](int r, int c) { return (uint64_t)r * NA + (uint64_t)c; };
    auto krow = [NA](uint64_t k) { return (int)(k / NA); };
    auto kcol = [NA](uint64_t k) { return (int)(k % NA); };
    int kbits = 1;
    while (kbits < 64 && (NA * NA) >> kbits) kbits++;
    std::vector<uint64_t> ktmp;
    auto normalise = [&](std::vector<uint64_t>& v) {
        if (v.size() < 4096) {
            std::sort(v.begin(), v.end());
        } else {  // least-significant-digit radix sort, 11-bit digits
            ktmp.resize(v.size());
            for (int sh = 0; sh < kbits; sh += 11) {
                std::vector<size_t> cnt(2049, 0);
                for (uint64_t k : v) cnt[((k >> sh) & 2047) + 1]++;
                for (int d = 0; d < 2048; d++) cnt[d + 1] += cnt[d];
                for (uint64_t k : v) ktmp[cnt[(k >> sh) & 2047]++] = k;
                v.swap(ktmp);
            }
        }
        v.erase(std::unique(v.begin(), v.end()), v.end());
    };
    for (int64_t r = 0; r < n; r++) {
        int ar = o.atom_of[rowpos(r)];
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; e++) {
            int ac = o.atom_of[o.iperm[colind[e]]];
            if (!o.related(o.atom_node[ar], o.atom_node[ac])) {
                set_error("matrix pattern couples separated subdomains (not a 5/7-point stencil on this grid?)");
                return SPAQR_ERR_UNSUPPORTED;
            }
            P.push_back(key(ar, ac));
        }
    }
    normalise(P);
    std::vector<int> idx(na, -1);   // local index of an active cluster
    std::vector<int> active(na);
    std::vector<int> cnode(na), cend(na);
    for (int a = 0; a < na; a++) { active[a] = a; cnode[a] = o.atom_node[a]; cend[a] = a + 1; }
    o.steps.clear();
    o.plan_code.clear();
    for (int k = 1; k <= L; k++) {
        const int lev = L - k + 1;
        StepPlan sp;
        sp.level = lev;
        sp.cl = active;  // sorted
        const int ncl = (int)active.size();
        for (int i = 0; i < ncl; i++) idx[active[i]] = i;
        sp.cl_node.resize(ncl);
        sp.is_front.assign(ncl, 0);
        for (int i = 0; i < ncl; i++) {
            sp.cl_node[i] = cnode[active[i]];
            if (nodes[sp.cl_node[i]].depth + 1 == lev) sp.is_front[i] = 1;
        }
        std::vector<std::vector<int>> col_rows(ncl), row_cols(ncl);
        for (uint64_t pk : P) {
            int i = idx[krow(pk)], j = idx[kcol(pk)];
            col_rows[j].push_back(i);
            row_cols[i].push_back(j);
        }
        std::vector<int> fr;
        for (int i = 0; i < ncl; i++) if (sp.is_front[i]) fr.push_back(i);
        {
            std::set<int> seen;
            for (int f : fr) {
                if (seen.count(sp.cl_node[f])) { set_error("separator not merged at its level"); return SPAQR_ERR_INVALID_ARG; }
                seen.insert(sp.cl_node[f]);
            }
        }
        std::vector<std::vector<int>> Rf(fr.size()), Cf(fr.size());
        std::vector<int> seen_by(ncl, -1);   // front that last took column cluster j
        for (size_t t = 0; t < fr.size(); t++) {
            int s = fr[t];
            Rf[t] = col_rows[s];  // ascending (pattern order)
            std::vector<int>& cs = Cf[t];
            for (int i : Rf[t])
                for (int j : row_cols[i])
                    if (seen_by[j] != (int)t && o.related(sp.cl_node[j], sp.cl_node[s])) {
                        seen_by[j] = (int)t;
                        cs.push_back(j);
                    }
            std::sort(cs.begin(), cs.end());
            if (Rf[t].empty() || Rf[t][0] != s || Cf[t][0] != s) {
                set_error("front without its diagonal block");
                return SPAQR_ERR_SINGULAR;
            }
        }
        // greedy colouring in ascending id: conflict = a shared row cluster
        // (the earlier fronts of every row cluster are listed as we go)
        std::vector<int> col(fr.size(), 0);
        {
            std::vector<std::vector<int>> fronts_of_row(ncl);
            for (size_t t = 0; t < fr.size(); t++) {
                std::set<int> used;
                for (int i : Rf[t])
                    for (int u : fronts_of_row[i]) used.insert(col[u]);
                int c = 0;
                while (used.count(c)) c++;
                col[t] = c;
                for (int i : Rf[t]) fronts_of_row[i].push_back((int)t);
            }
        }
        std::vector<size_t> seq(fr.size());
        for (size_t t = 0; t < fr.size(); t++) seq[t] = t;
        std::stable_sort(seq.begin(), seq.end(), [&](size_t a, size_t bb) {
            if (col[a] != col[bb]) return col[a] < col[bb];
            return fr[a] < fr[bb];
        });
        for (size_t t : seq) {
            sp.fronts.push_back(fr[t]);
            sp.colour.push_back(col[t]);
            sp.R.push_back(Rf[t]);
            sp.C.push_back(Cf[t]);
        }
        // fill of this level
        for (size_t t = 0; t < fr.size(); t++)
            for (int i : Rf[t])
                for (int j : Cf[t]) P.push_back(key(active[i], active[j]));
        normalise(P);
        // CSC of the pattern with fill
        sp.colptr.assign(ncl + 1, 0);
        for (uint64_t pk : P) sp.colptr[idx[kcol(pk)] + 1]++;
        for (int j = 0; j < ncl; j++) sp.colptr[j + 1] += sp.colptr[j];
        sp.rowidx.assign(sp.colptr[ncl], 0);
        {
            std::vector<int> fillp(sp.colptr.begin(), sp.colptr.end() - 1);
            // P iterates by row then column; rows ascending within each column
            for (uint64_t pk : P) sp.rowidx[fillp[idx[kcol(pk)]]++] = idx[krow(pk)];
        }
        // encode
        o.plan_code.push_back(lev);
        o.plan_code.push_back(ncl);
        for (int i = 0; i < ncl; i++) o.plan_code.push_back(active[i]);
        o.plan_code.push_back((int)sp.fronts.size());
        for (size_t t = 0; t < sp.fronts.size(); t++) {
            o.plan_code.push_back(active[sp.fronts[t]]);
            o.plan_code.push_back(sp.colour[t]);
            o.plan_code.push_back((int)sp.R[t].size());
            for (int i : sp.R[t]) o.plan_code.push_back(active[i]);
            o.plan_code.push_back((int)sp.C[t].size());
            for (int j : sp.C[t]) o.plan_code.push_back(active[j]);
        }
        // eliminate the fronts
        P.erase(std::remove_if(P.begin(), P.end(),
                               [&](uint64_t pk) {
                                   return sp.is_front[idx[krow(pk)]] || sp.is_front[idx[kcol(pk)]];
                               }),
                P.end());
        std::vector<int> rest;
        for (int i = 0; i < ncl; i++) if (!sp.is_front[i]) rest.push_back(active[i]);
        sp.parent.assign(ncl, -1);
        if (k < L && !rest.empty()) {
            std::vector<int> f = stage_first(L - k - 1);
            std::map<int, int> newid;  // parent first atom -> new end
            for (int c : rest) {
                int g = f[c];
                if (f[cend[c] - 1] != g) { set_error("merge hierarchy not nested"); return SPAQR_ERR_INVALID_ARG; }
                auto it = newid.find(g);
                if (it == newid.end()) newid[g] = cend[c];
                else it->second = std::max(it->second, cend[c]);
            }
            std::vector<int> nxt;
            for (auto& kv : newid) nxt.push_back(kv.first);
            std::unordered_map<int, int> nidx;
            for (size_t i = 0; i < nxt.size(); i++) nidx[nxt[i]] = (int)i;
            for (int i = 0; i < ncl; i++)
                if (!sp.is_front[i]) sp.parent[i] = nidx.at(f[active[i]]);
            sp.n_next = (int)nxt.size();
            for (uint64_t& pk : P) pk = key(f[krow(pk)], f[kcol(pk)]);
            normalise(P);
            for (int g : nxt) {
                cnode[g] = o.atom_node[g];
                cend[g] = newid[g];
            }
            active = nxt;
        } else {
            active = rest;
        }
        o.steps.push_back(std::move(sp));
    }
    if (!active.empty() || !P.empty()) { set_error("plan left active clusters"); return SPAQR_ERR_INVALID_ARG; }
    index_plan(o);

    // ---- gather map into the level-1 arena --------------------------------
    {
        const StepPlan& s1 = o.steps[0];
        const int ncl = (int)s1.cl.size();  // == na
        std::vector<int64_t> H(ncl, 0), poff(ncl + 1, 0), rowoff(s1.rowidx.size());
        for (int j = 0; j < ncl; j++) {
            int64_t h = 0;
            for (int e = s1.colptr[j]; e < s1.colptr[j + 1]; e++) {
                rowoff[e] = h;
                int i = s1.rowidx[e];
                h += o.atom_ptr[i + 1] - o.atom_ptr[i];
            }
            H[j] = h;
            poff[j + 1] = poff[j] + h * (o.atom_ptr[j + 1] - o.atom_ptr[j]);
        }
        o.arena1_size = poff[ncl];
        o.gather_off.assign(nnz, 0);
        for (int64_t r = 0; r < n; r++) {
            int64_t nr = rowpos(r);
            int ar = o.atom_of[nr];
            for (int64_t e = rowptr[r]; e < rowptr[r + 1]; e++) {
                int64_t nc = o.iperm[colind[e]];
                int ac = o.atom_of[nc];
                int pos = s1.find(ar, ac);
                o.gather_off[e] = poff[ac] + rowoff[pos] + (nr - o.atom_ptr[ar]) +
                                  (nc - o.atom_ptr[ac]) * H[ac];
            }
        }
    }
    return SPAQR_OK;
}

// ---------------------------------------------------------------------------
// General sparse matrices: modified nested dissection on G(A^T A) and a row
// matching (Section 2.3 orders such matrices with a hypergraph partitioner and
// MC64; this is our restatement).  Readings:
//  * G(A^T A): columns i != j adjacent when a row holds nonzeros in both;
//  * separator of a node's column set V: a breadth-first level.  Components
//    of G restricted to V are taken by their smallest column; each is
//    searched from a pseudo-peripheral column (start at the smallest column;
//    repeatedly search, take the last level's column with the fewest
//    neighbours in V, ties to the smallest index, and move there while the
//    number of levels grows); the levels of all components are concatenated
//    and the separator is the first level whose cumulative size reaches half
//    of |V|, the left child gets the levels before it, the right child those
//    after it; the separator keeps only its columns adjacent to the right
//    side, the others join the left side;
//  * a separator column x gets, for every non-leaf strict descendant D of its
//    node that x is adjacent to, the key (depth D, D, k): k = 1 when x touches
//    D's separator or both of D's child subtrees, 0 when only the left one,
//    2 when only the right one; atoms and their order as for grids, with the
//    column index as the index;
//  * rows: entries by decreasing |a_ij| (ties: row, column) matched greedily,
//    then every unmatched row (ascending) by an augmenting path (columns of a
//    row in ascending order, depth first), or the maximum-product matching
//    (row_matching_max_product); row r sits with its column.
// ---------------------------------------------------------------------------
// G(A^T A) restricted to a column set: local vertices in ascending global
// order, each with its neighbours inside the set (ascending).  Because the
// local order is the global one, searches and tie-breaks on a subgraph give
// what they give on the whole graph restricted to the set, with the set's
// own compact arrays in cache.
struct SubGraph {
    std::vector<int64_t> gid;   // global column of every local vertex
    std::vector<int64_t> xp;    // local CSR
    std::vector<int32_t> adj;
    int64_t size() const { return (int64_t)gid.size(); }
    int64_t degree(int64_t v) const { return xp[v + 1] - xp[v]; }
};

struct GeneralND {
    int64_t n = 0;
    int L = 1;
    SubGraph root;                      // the whole G(A^T A); kept for the interfaces
    std::vector<NDNode> nodes;
    std::vector<std::vector<int64_t>> pts;
    // breadth-first levels: vertices in visiting order, level l holding
    // ord[lptr[l] .. lptr[l+1])
    struct Levels {
        std::vector<int32_t> ord;
        std::vector<int64_t> lptr;
        size_t count() const { return lptr.empty() ? 0 : lptr.size() - 1; }
    };

    void graph(const int64_t* rp, const int32_t* ci) {
        std::vector<int64_t> cp(n + 1, 0), ri(rp[n]);
        for (int64_t e = 0; e < rp[n]; e++) cp[ci[e] + 1]++;
        for (int64_t j = 0; j < n; j++) cp[j + 1] += cp[j];
        {
            std::vector<int64_t> f(cp.begin(), cp.end() - 1);
            for (int64_t r = 0; r < n; r++)
                for (int64_t e = rp[r]; e < rp[r + 1]; e++) ri[f[ci[e]]++] = r;
        }
        std::vector<int32_t> mark(n, -1);
        root.gid.resize(n);
        root.xp.assign(n + 1, 0);
        root.adj.clear();
        std::vector<int32_t> tmp;
        for (int64_t j = 0; j < n; j++) {
            root.gid[j] = j;
            tmp.clear();
            mark[j] = (int32_t)j;
            for (int64_t e = cp[j]; e < cp[j + 1]; e++) {
                const int64_t r = ri[e];
                for (int64_t f = rp[r]; f < rp[r + 1]; f++) {
                    const int32_t c = ci[f];
                    if (mark[c] != (int32_t)j) {
                        mark[c] = (int32_t)j;
                        tmp.push_back(c);
                    }
                }
            }
            std::sort(tmp.begin(), tmp.end());
            root.adj.insert(root.adj.end(), tmp.begin(), tmp.end());
            root.xp[j + 1] = (int64_t)root.adj.size();
        }
    }
    // levels of the component of `r` (stamp: seen[v] == id marks a visit)
    static void bfs(const SubGraph& G, int32_t r, std::vector<int32_t>& seen, int32_t id, Levels& lv) {
        lv.ord.assign(1, r);
        lv.lptr.assign(1, 0);
        seen[r] = id;
        int64_t b = 0;
        while (b < (int64_t)lv.ord.size()) {
            const int64_t e0 = (int64_t)lv.ord.size();
            lv.lptr.push_back(e0);
            for (int64_t i = b; i < e0; i++) {
                const int32_t x = lv.ord[i];
                for (int64_t e = G.xp[x]; e < G.xp[x + 1]; e++) {
                    const int32_t y = G.adj[e];
                    if (seen[y] != id) {
                        seen[y] = id;
                        lv.ord.push_back(y);
                    }
                }
            }
            b = e0;
        }
    }
    // all levels of G, component by component (smallest vertex first), each
    // component searched from a pseudo-peripheral vertex
    static Levels level_structure(const SubGraph& G) {
        const int64_t m = G.size();
        std::vector<int32_t> seen(m, 0);
        std::vector<char> done(m, 0);
        int32_t id = 0;
        Levels all, lv, lv2;
        all.lptr.assign(1, 0);
        for (int64_t s = 0; s < m; s++) {
            if (done[s]) continue;
            bfs(G, (int32_t)s, seen, ++id, lv);
            while (true) {
                int32_t cand = -1;
                int64_t bd = 0;
                for (int64_t i = lv.lptr[lv.count() - 1]; i < lv.lptr[lv.count()]; i++) {
                    const int32_t v = lv.ord[i];
                    const int64_t d = G.degree(v);
                    if (cand < 0 || d < bd || (d == bd && v < cand)) { bd = d; cand = v; }
                }
                bfs(G, cand, seen, ++id, lv2);
                if (lv2.count() <= lv.count()) break;
                std::swap(lv, lv2);
            }
            const int64_t base = (int64_t)all.ord.size();
            for (int32_t v : lv.ord) done[v] = 1;
            all.ord.insert(all.ord.end(), lv.ord.begin(), lv.ord.end());
            for (size_t l = 1; l <= lv.count(); l++) all.lptr.push_back(base + lv.lptr[l]);
        }
        return all;
    }
    // subgraph of G on the ascending local vertices `keep`
    static SubGraph induce(const SubGraph& G, const std::vector<int32_t>& keep, std::vector<int32_t>& loc) {
        SubGraph H;
        const int64_t k = (int64_t)keep.size();
        for (int64_t i = 0; i < k; i++) loc[keep[i]] = (int32_t)i;
        H.gid.resize(k);
        H.xp.assign(k + 1, 0);
        for (int64_t i = 0; i < k; i++) {
            const int32_t x = keep[i];
            H.gid[i] = G.gid[x];
            for (int64_t e = G.xp[x]; e < G.xp[x + 1]; e++) {
                const int32_t y = loc[G.adj[e]];
                if (y >= 0) H.adj.push_back(y);
            }
            H.xp[i + 1] = (int64_t)H.adj.size();
        }
        for (int32_t x : keep) loc[x] = -1;
        return H;
    }
    // The nested-dissection subtree of column set G, nodes in preorder with
    // ids local to the subtree (its root is node 0, parent -1).  G is released
    // once its children's subgraphs exist, unless it is the root graph.  With
    // threads > 1 the two child subtrees are built concurrently: they share
    // nothing, and splicing them under the parent in preorder gives the same
    // tree whatever the timing.
    struct Tree {
        std::vector<NDNode> nodes;
        std::vector<std::vector<int64_t>> pts;
    };
    Tree build(SubGraph& G, int depth, int threads) {
        Tree T;
        T.nodes.emplace_back();
        T.pts.emplace_back();
        T.nodes[0].depth = depth;
        if (depth == L - 1) {
            T.pts[0] = G.gid;
            if (&G != &root) G = SubGraph();
            return T;
        }
        const int64_t m = G.size();
        std::vector<int32_t> S, Lf, Rt;
        if (m > 0) {
            Levels lv = level_structure(G);
            size_t l = 0;
            int64_t cum = 0;
            for (; l < lv.count(); l++) {
                cum += lv.lptr[l + 1] - lv.lptr[l];
                if (2 * cum >= m) break;
            }
            Lf.assign(lv.ord.begin(), lv.ord.begin() + lv.lptr[l]);
            Rt.assign(lv.ord.begin() + lv.lptr[l + 1], lv.ord.end());
            // thin the separator: a column with no right neighbour joins the left side
            std::vector<char> right(m, 0);
            for (int32_t y : Rt) right[y] = 1;
            for (int64_t i = lv.lptr[l]; i < lv.lptr[l + 1]; i++) {
                const int32_t x = lv.ord[i];
                bool r = false;
                for (int64_t e = G.xp[x]; e < G.xp[x + 1] && !r; e++) r = right[G.adj[e]];
                (r ? S : Lf).push_back(x);
            }
            std::sort(S.begin(), S.end());
            std::sort(Lf.begin(), Lf.end());
            std::sort(Rt.begin(), Rt.end());
        }
        std::vector<int32_t> loc(m, -1);
        SubGraph GL = induce(G, Lf, loc), GR = induce(G, Rt, loc);
        std::vector<int64_t> sep(S.size());
        for (size_t i = 0; i < S.size(); i++) sep[i] = G.gid[S[i]];
        if (&G != &root) G = SubGraph();
        { std::vector<int32_t>().swap(loc); std::vector<int32_t>().swap(Lf); std::vector<int32_t>().swap(Rt); }
        Tree A, B;
        std::thread th;
        std::exception_ptr err;
        if (threads > 1) {
            try {
                th = std::thread([&] {
                    try {
                        A = build(GL, depth + 1, threads / 2);
                    } catch (...) {
                        err = std::current_exception();
                    }
                });
            } catch (const std::system_error&) {
                threads = 1;   // no thread to be had: the same tree, serially
            }
        }
        if (threads > 1) {
            try {
                B = build(GR, depth + 1, threads - threads / 2);
            } catch (...) {
                th.join();
                throw;
            }
            th.join();
            if (err) std::rethrow_exception(err);
        } else {
            A = build(GL, depth + 1, 1);
            B = build(GR, depth + 1, 1);
        }
        const int na = (int)A.nodes.size(), nb = (int)B.nodes.size();
        auto splice = [&](Tree& X, int off) {
            for (NDNode nd : X.nodes) {
                nd.id += off;
                nd.parent = nd.parent < 0 ? 0 : nd.parent + off;
                if (nd.left >= 0) nd.left += off;
                if (nd.right >= 0) nd.right += off;
                T.nodes.push_back(nd);
            }
            for (auto& p : X.pts) T.pts.push_back(std::move(p));
        };
        T.nodes.reserve(1 + na + nb);
        T.pts.reserve(1 + na + nb);
        splice(A, 1);
        splice(B, 1 + na);
        T.nodes[0].left = 1;
        T.nodes[0].right = 1 + na;
        T.nodes[0].cut_dim = 0;
        T.nodes[0].size = 1 + na + nb;
        T.pts[0] = std::move(sep);
        return T;
    }
};

// rowcol[r] = the column row r is matched to; SINGULAR when no perfect
// matching exists.
int row_matching(const int64_t* rp, const int32_t* ci, const double* val, int64_t n, std::vector<int64_t>& rowcol) {
    const int64_t nnz = rp[n];
    // entries by decreasing |a_ij|, ties by row then column (entries equal in
    // all three are one (row, column) pair: their order does not matter)
    struct Entry {
        double mag;
        int64_t r;
        int32_t c;
    };
    std::vector<Entry> ent(nnz);
    for (int64_t r = 0; r < n; r++)
        for (int64_t e = rp[r]; e < rp[r + 1]; e++) ent[e] = Entry{val ? std::fabs(val[e]) : 1.0, r, ci[e]};
    std::sort(ent.begin(), ent.end(), [](const Entry& a, const Entry& b) {
        if (a.mag != b.mag) return a.mag > b.mag;
        if (a.r != b.r) return a.r < b.r;
        return a.c < b.c;
    });
    rowcol.assign(n, -1);
    std::vector<int64_t> colrow(n, -1);
    for (const Entry& x : ent) {
        if (rowcol[x.r] < 0 && colrow[x.c] < 0) {
            rowcol[x.r] = x.c;
            colrow[x.c] = x.r;
        }
    }
    std::vector<Entry>().swap(ent);
    // sorted distinct columns of every row, for the augmenting paths
    std::vector<int64_t> cp(n + 1, 0), cc;
    for (int64_t r = 0; r < n; r++) {
        std::vector<int64_t> t(ci + rp[r], ci + rp[r + 1]);
        std::sort(t.begin(), t.end());
        t.erase(std::unique(t.begin(), t.end()), t.end());
        cc.insert(cc.end(), t.begin(), t.end());
        cp[r + 1] = (int64_t)cc.size();
    }
    std::vector<int32_t> vis(n, 0);
    int32_t visid = 0;
    struct Frame { int64_t r, k, c; };
    std::vector<Frame> st;
    for (int64_t r0 = 0; r0 < n; r0++) {
        if (rowcol[r0] >= 0) continue;
        ++visid;
        st.assign(1, Frame{r0, cp[r0], -1});
        bool found = false;
        while (!st.empty() && !found) {
            const int64_t r = st.back().r;
            if (st.back().k >= cp[r + 1]) { st.pop_back(); continue; }
            const int64_t c = cc[st.back().k++];
            if (vis[c] == visid) continue;
            vis[c] = visid;
            st.back().c = c;
            if (colrow[c] < 0) {
                for (const Frame& f : st) {
                    rowcol[f.r] = f.c;
                    colrow[f.c] = f.r;
                }
                found = true;
            } else {
                st.push_back(Frame{colrow[c], cp[colrow[c]], -1});
            }
        }
        if (!found) { set_error("structurally singular matrix: no perfect row matching"); return SPAQR_ERR_SINGULAR; }
    }
    return SPAQR_OK;
}

// rowcol[r] = the column row r is matched to, maximising the product of the
// matched |a_ij| (the large-entries-on-the-diagonal matching Section 2.3 takes
// from MC64): a minimum-cost perfect matching on
// c_ij = log max_k |a_kj| - log |a_ij| over the nonzero entries (duplicates
// summed in storage order, explicit zeros dropped), by shortest augmenting
// paths with dual potentials u (rows) and v (columns):
//  * v = 0, u_i = min_j c_ij; every row (ascending) takes its first free
//    column (ascending) of zero reduced cost (c_ij - u_i) - v_j;
//  * every row left free (ascending) starts a Dijkstra search over columns
//    (ties to the smaller column) that crosses matched edges at no cost, up
//    to the first free column, at distance D; every column k settled on the
//    way gets v_k -= D - d_k and its matched row u += D - d_k, the start row
//    u += D; the path is flipped.
// SINGULAR when no perfect matching exists on the nonzero values.
int row_matching_max_product(const int64_t* rp, const int32_t* ci, const double* val, int64_t n,
                             std::vector<int64_t>& rowcol) {
    std::vector<int64_t> xp(n + 1, 0), ord;
    std::vector<int32_t> cc;
    std::vector<double> cv;
    for (int64_t r = 0; r < n; r++) {
        ord.clear();
        for (int64_t e = rp[r]; e < rp[r + 1]; e++) ord.push_back(e);
        std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return ci[a] < ci[b]; });
        size_t k = 0;
        while (k < ord.size()) {
            const int32_t c = ci[ord[k]];
            double x = val ? val[ord[k]] : 1.0;
            size_t m = k + 1;
            for (; m < ord.size() && ci[ord[m]] == c; m++) x = x + (val ? val[ord[m]] : 1.0);
            if (x != 0.0) {
                cc.push_back(c);
                cv.push_back(x);
            }
            k = m;
        }
        xp[r + 1] = (int64_t)cc.size();
    }
    std::vector<double> amax(n, 0.0);
    for (size_t e = 0; e < cc.size(); e++) amax[cc[e]] = std::max(amax[cc[e]], std::fabs(cv[e]));
    for (int64_t j = 0; j < n; j++)
        if (amax[j] == 0.0) { set_error("structurally singular matrix: an empty column"); return SPAQR_ERR_SINGULAR; }
    std::vector<double> w(cc.size());
    for (size_t e = 0; e < cc.size(); e++) w[e] = std::log(amax[cc[e]]) - std::log(std::fabs(cv[e]));
    std::vector<double> u(n, 0.0), v(n, 0.0);
    for (int64_t r = 0; r < n; r++)
        for (int64_t e = xp[r]; e < xp[r + 1]; e++)
            if (e == xp[r] || w[e] < u[r]) u[r] = w[e];
    rowcol.assign(n, -1);
    std::vector<int64_t> colrow(n, -1);
    for (int64_t r = 0; r < n; r++)
        for (int64_t e = xp[r]; e < xp[r + 1]; e++) {
            const int32_t c = cc[e];
            if (colrow[c] < 0 && (w[e] - u[r]) - v[c] == 0.0) {
                rowcol[r] = c;
                colrow[c] = r;
                break;
            }
        }
    std::vector<double> d(n, 0.0);
    std::vector<int64_t> pred(n, -1), touched, settled;
    std::vector<char> reached(n, 0), done(n, 0);
    using Entry = std::pair<double, int64_t>;   // (distance, column): ties to the smaller column
    std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> heap;
    auto relax = [&](int64_t c, double nd, int64_t i) {
        if (!reached[c] || nd < d[c]) {
            if (!reached[c]) { reached[c] = 1; touched.push_back(c); }
            d[c] = nd;
            pred[c] = i;
            heap.push(Entry(nd, c));
        }
    };
    for (int64_t r = 0; r < n; r++) {
        if (rowcol[r] >= 0) continue;
        for (int64_t e = xp[r]; e < xp[r + 1]; e++) relax(cc[e], (w[e] - u[r]) - v[cc[e]], r);
        int64_t end = -1;
        while (!heap.empty()) {
            const Entry top = heap.top();
            heap.pop();
            const double dj = top.first;
            const int64_t j = top.second;
            if (done[j]) continue;
            done[j] = 1;
            settled.push_back(j);
            if (colrow[j] < 0) { end = j; break; }
            const int64_t i = colrow[j];
            for (int64_t e = xp[i]; e < xp[i + 1]; e++) {
                const int32_t c = cc[e];
                if (done[c]) continue;
                relax(c, dj + ((w[e] - u[i]) - v[c]), i);
            }
        }
        if (end < 0) { set_error("structurally singular matrix: no perfect row matching"); return SPAQR_ERR_SINGULAR; }
        const double D = d[end];
        u[r] = u[r] + D;
        for (int64_t k : settled) {
            const double delta = D - d[k];
            v[k] = v[k] - delta;
            if (k != end) u[colrow[k]] = u[colrow[k]] + delta;
        }
        for (int64_t j = end;;) {
            const int64_t i = pred[j], prev = rowcol[i];
            rowcol[i] = j;
            colrow[j] = i;
            if (i == r) break;
            j = prev;
        }
        while (!heap.empty()) heap.pop();
        for (int64_t c : touched) reached[c] = done[c] = 0;
        touched.clear();
        settled.clear();
    }
    return SPAQR_OK;
}

// rowptr starts at 0, never decreases and ends at nnz (every host loop over a
// row's entries then stays inside colind)
int check_rowptr(const int64_t* rowptr, int64_t n, int64_t nnz) {
    if (rowptr[0] != 0 || rowptr[n] != nnz) { set_error("bad CSR rowptr (first entry not 0 or last not nnz)"); return SPAQR_ERR_INVALID_ARG; }
    for (int64_t r = 0; r < n; r++)
        if (rowptr[r + 1] < rowptr[r]) { set_error("bad CSR rowptr (decreasing at row " + std::to_string(r) + ")"); return SPAQR_ERR_INVALID_ARG; }
    return SPAQR_OK;
}

int check_grid(int dim, const int* dims, int64_t n, const int64_t* rowptr, int64_t nnz, int* dims3) {
    if (dim != 2 && dim != 3) { set_error("grid dim must be 2 or 3"); return SPAQR_ERR_INVALID_ARG; }
    int64_t N = 1;
    for (int k = 0; k < dim; k++) {
        if (dims[k] < 1) { set_error("grid sides must be >= 1"); return SPAQR_ERR_INVALID_ARG; }
        N *= dims[k];
    }
    if (N != n) { set_error("grid size does not match matrix size"); return SPAQR_ERR_INVALID_ARG; }
    if (check_rowptr(rowptr, n, nnz) != SPAQR_OK) return SPAQR_ERR_INVALID_ARG;
    for (int k = 0; k < 3; k++) dims3[k] = k < dim ? dims[k] : 1;
    return SPAQR_OK;
}

}  // namespace

int build_ordering(const int64_t* rowptr, const int32_t* colind, int64_t n, int64_t nnz, int dim,
                   const int* dims, int nlevels, Ordering& o) {
    int rc = check_grid(dim, dims, n, rowptr, nnz, o.dims);
    if (rc != SPAQR_OK) return rc;
    o.dim = dim;
    o.n = n;
    o.nnz = nnz;
    o.L = nlevels > 0 ? nlevels : num_levels(n);
    std::vector<std::vector<Atom>> node_atoms;
    rc = nd_grid(dim, o.dims, o.L, o.nodes, node_atoms);
    if (rc != SPAQR_OK) return rc;
    return plan_forest(o, rowptr, colind, node_atoms);
}

int build_ordering_general(const int64_t* rowptr, const int32_t* colind, const double* val, int64_t n,
                           int64_t nnz, int nlevels, int matching, Ordering& o) {
    if (matching != SPAQR_MATCH_GREEDY && matching != SPAQR_MATCH_MAX_PRODUCT) {
        set_error("unknown row matching");
        return SPAQR_ERR_INVALID_ARG;
    }
    if (check_rowptr(rowptr, n, nnz) != SPAQR_OK) return SPAQR_ERR_INVALID_ARG;
    for (int64_t e = 0; e < nnz; e++)
        if (colind[e] < 0 || colind[e] >= n) { set_error("column index out of range"); return SPAQR_ERR_INVALID_ARG; }
    // the matchings order entries by |a_ij|: a NaN has no place in that order
    if (val)
        for (int64_t e = 0; e < nnz; e++)
            if (!std::isfinite(val[e])) { set_error("non-finite matrix value"); return SPAQR_ERR_INVALID_ARG; }
    o.dim = 0;
    o.dims[0] = (int)std::min<int64_t>(n, 0x7fffffff);
    o.dims[1] = o.dims[2] = 1;
    o.n = n;
    o.nnz = nnz;
    o.L = nlevels > 0 ? nlevels : num_levels(n);
    // G(A^T A) holds up to sum_r nnz(row r)^2 entries: refuse patterns whose
    // dense rows would make it exceed 2^31 (a partitioner working on A's
    // hypergraph, Section 2.3, avoids forming it; not built here)
    {
        double pairs = 0.0;
        for (int64_t r = 0; r < n; r++) {
            const double k = (double)(rowptr[r + 1] - rowptr[r]);
            pairs += k * k;
        }
        if (pairs > 2147483648.0) {
            set_error("rows too dense for the G(A^T A) ordering (sum of squared row lengths above 2^31)");
            return SPAQR_ERR_UNSUPPORTED;
        }
    }
    int rc = matching == SPAQR_MATCH_GREEDY ? row_matching(rowptr, colind, val, n, o.rowcol)
                                            : row_matching_max_product(rowptr, colind, val, n, o.rowcol);
    if (rc != SPAQR_OK) return rc;
    GeneralND g;
    g.n = n;
    g.L = o.L;
    g.graph(rowptr, colind);
    {
        const unsigned hw = std::thread::hardware_concurrency();
        GeneralND::Tree T = g.build(g.root, 0, (int)std::max(1u, std::min(hw, 8u)));
        g.nodes = std::move(T.nodes);
        g.pts = std::move(T.pts);
    }
    const int nn = (int)g.nodes.size();
    std::vector<int> owner(n, -1);
    for (int id = 0; id < nn; id++)
        for (int64_t v : g.pts[id]) owner[v] = id;
    std::vector<std::vector<Atom>> node_atoms(nn);
    std::vector<std::array<char, 3>> mk(nn);
    std::vector<int32_t> mstamp(nn, -1);
    for (int id = 0; id < nn; id++) {
        const std::vector<int64_t>& S = g.pts[id];
        if (S.empty()) continue;
        if (g.nodes[id].depth == o.L - 1) {
            Atom a;
            a.pts = S;
            node_atoms[id].push_back(std::move(a));
            continue;
        }
        const int lo = id, hi = id + g.nodes[id].size;
        std::vector<std::vector<Key>> keys(S.size());
        for (size_t xi = 0; xi < S.size(); xi++) {
            const int64_t x = S[xi];
            std::vector<int> touched;
            for (int64_t e = g.root.xp[x]; e < g.root.xp[x + 1]; e++) {
                const int ow = owner[g.root.adj[e]];
                if (!(lo < ow && ow < hi)) continue;
                int child = -1;
                for (int D = ow; D != id; child = D, D = g.nodes[D].parent) {
                    if (g.nodes[D].depth >= o.L - 1) continue;
                    if (mstamp[D] != (int32_t)(xi + 1)) {
                        mstamp[D] = (int32_t)(xi + 1);
                        mk[D] = {0, 0, 0};
                        touched.push_back(D);
                    }
                    if (child < 0) mk[D][1] = 1;
                    else if (child == g.nodes[D].left) mk[D][0] = 1;
                    else mk[D][2] = 1;
                }
            }
            std::sort(touched.begin(), touched.end(), [&](int a, int b) {
                if (g.nodes[a].depth != g.nodes[b].depth) return g.nodes[a].depth < g.nodes[b].depth;
                return a < b;
            });
            for (int D : touched) {
                const int k = (mk[D][1] || (mk[D][0] && mk[D][2])) ? 1 : (mk[D][0] ? 0 : 2);
                keys[xi].push_back(Key{g.nodes[D].depth, D, k});
            }
            for (int D : touched) mstamp[D] = -1;
        }
        order_atoms(S, keys, node_atoms[id]);
    }
    o.nodes = std::move(g.nodes);
    rc = plan_forest(o, rowptr, colind, node_atoms);
    if (rc != SPAQR_OK) return rc;
    std::vector<int64_t> colrow(n);
    for (int64_t r = 0; r < n; r++) colrow[o.rowcol[r]] = r;
    o.rperm.resize(n);
    for (int64_t k = 0; k < n; k++) o.rperm[k] = colrow[o.perm[k]];
    return SPAQR_OK;
}

// Ordering of the block-diagonal matrix diag(A_0, ..., A_{count-1}): every
// grid gets its own tree with its own level count; the trees' depths are
// shifted so that all leaves sit at depth L - 1 (L = the largest count), so
// level k of the forest holds level k (from the leaves) of every matrix that
// has one.  Unknowns of matrix i keep their block: rows/columns base_i + r.
int build_ordering_batch(int count, const int64_t* const* rowptrs, const int32_t* const* colinds,
                         const int64_t* ns, const int64_t* nnzs, const int* dims_list, Ordering& o) {
    if (count < 1) { set_error("count must be >= 1"); return SPAQR_ERR_INVALID_ARG; }
    std::vector<std::vector<NDNode>> tnodes(count);
    std::vector<std::vector<std::vector<Atom>>> tatoms(count);
    std::vector<int> tl(count);
    int L = 1;
    int64_t n = 0, nnz = 0;
    for (int i = 0; i < count; i++) {
        const int* g = dims_list + 4 * i;   // dim, nx, ny, nz
        int dims3[3];
        int rc = check_grid(g[0], g + 1, ns[i], rowptrs[i], nnzs[i], dims3);
        if (rc != SPAQR_OK) return rc;
        tl[i] = num_levels(ns[i]);
        L = std::max(L, tl[i]);
        rc = nd_grid(g[0], dims3, tl[i], tnodes[i], tatoms[i]);
        if (rc != SPAQR_OK) return rc;
        n += ns[i];
        nnz += nnzs[i];
    }
    o.dim = 0;   // a forest of grids
    o.dims[0] = o.dims[1] = o.dims[2] = 1;
    o.n = n;
    o.nnz = nnz;
    o.L = L;
    o.nodes.clear();
    std::vector<std::vector<Atom>> node_atoms;
    std::vector<int64_t> rowptr(1, 0);
    std::vector<int32_t> colind;
    rowptr.reserve(n + 1);
    colind.reserve(nnz);
    int64_t base = 0;
    for (int i = 0; i < count; i++) {
        const int noff = (int)o.nodes.size();
        const int shift = L - tl[i];
        for (NDNode nd : tnodes[i]) {
            nd.id += noff;
            nd.depth += shift;
            if (nd.parent >= 0) nd.parent += noff;
            if (nd.left >= 0) nd.left += noff;
            if (nd.right >= 0) nd.right += noff;
            o.nodes.push_back(nd);
        }
        for (std::vector<Atom>& atoms : tatoms[i]) {
            for (Atom& a : atoms) {
                for (int64_t& p : a.pts) p += base;
                for (Key& kk : a.key) {
                    kk.depth += shift;
                    kk.node += noff;
                }
            }
            node_atoms.push_back(std::move(atoms));
        }
        const int64_t* rp = rowptrs[i];
        const int32_t* ci = colinds[i];
        const int64_t eb = (int64_t)colind.size();
        for (int64_t r = 0; r < ns[i]; r++) rowptr.push_back(eb + rp[r + 1]);
        for (int64_t e = 0; e < nnzs[i]; e++) {
            if (ci[e] < 0 || ci[e] >= ns[i]) { set_error("column index out of range"); return SPAQR_ERR_INVALID_ARG; }
            colind.push_back((int32_t)(ci[e] + base));
        }
        base += ns[i];
    }
    if (n > INT32_MAX) { set_error("batch too large for int32 column indices"); return SPAQR_ERR_INVALID_ARG; }
    return plan_forest(o, rowptr.data(), colind.data(), node_atoms);
}

}  // namespace spaqr

// ---------------------------------------------------------------------------
// C ABI: ordering
// ---------------------------------------------------------------------------

extern "C" int spaqr_ordering_info(const spaqr_ordering* ord, spaqr_ordering_info_t* info) {
    if (!ord || !info) { spaqr::set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    info->n = ord->o.n;
    info->nnz = ord->o.nnz;
    info->nlevels = ord->o.L;
    info->n_atoms = (int32_t)ord->o.atom_node.size();
    info->n_nodes = (int32_t)ord->o.nodes.size();
    info->plan_len = (int64_t)ord->o.plan_code.size();
    return SPAQR_OK;
}

extern "C" int spaqr_ordering_rows(const spaqr_ordering* ord, int64_t* rperm) {
    if (!ord || !rperm) { spaqr::set_error("null argument"); return SPAQR_ERR_INVALID_ARG; }
    const auto& o = ord->o;
    const std::vector<int64_t>& src = o.rperm.empty() ? o.perm : o.rperm;
    std::copy(src.begin(), src.end(), rperm);
    return SPAQR_OK;
}

extern "C" int spaqr_ordering_get(const spaqr_ordering* ord, int64_t* perm, int64_t* atom_ptr,
                                  int32_t* atom_node, int32_t* node_level, int32_t* plan) {
    if (!ord) { spaqr::set_error("null ordering"); return SPAQR_ERR_INVALID_ARG; }
    const spaqr::Ordering& o = ord->o;
    if (perm) std::memcpy(perm, o.perm.data(), sizeof(int64_t) * o.perm.size());
    if (atom_ptr) std::memcpy(atom_ptr, o.atom_ptr.data(), sizeof(int64_t) * o.atom_ptr.size());
    if (atom_node) std::memcpy(atom_node, o.atom_node.data(), sizeof(int32_t) * o.atom_node.size());
    if (node_level)
        for (size_t i = 0; i < o.nodes.size(); i++) node_level[i] = o.nodes[i].depth + 1;
    if (plan) std::memcpy(plan, o.plan_code.data(), sizeof(int32_t) * o.plan_code.size());
    return SPAQR_OK;
}

extern "C" void spaqr_ordering_destroy(spaqr_ordering* ord) { delete ord; }
