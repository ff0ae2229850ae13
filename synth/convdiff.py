"""Seeded convection-diffusion test matrices on regular 2D/3D grids.

This module builds INPUTS only: a sparse matrix A in CSR form, right-hand
sides, and the grid description.  It holds none of the factorisation's
arithmetic and is shared, unchanged, by the CPU oracle, the tests and the
benchmark.

Problem (the paper's benchmark family, Section 4): -div(a grad u) + v . grad u = f
on the unit square/cube with u = 0 on the boundary, n_k points in direction
k, h_k = 1/(n_k+1), lexicographic numbering with x fastest.

Discretisation (ours; the paper's own generator is not available):
  * diffusion: 5-/7-point stencil; the coefficient of the face between two
    cells is the harmonic mean of the cells' a; a boundary face uses the
    cell's own a;
  * convection: first-order upwind in advective form, per cell:
    v_d > 0 adds v_d/h_d to the diagonal and -v_d/h_d to the (c, c-e_d) entry,
    v_d < 0 adds |v_d|/h_d to the diagonal and -|v_d|/h_d to the (c, c+e_d) entry;
    entries that would couple to a boundary node are dropped.
The result is a non-singular M-matrix, weakly row diagonally dominant (strictly
on rows next to the boundary).

Random streams: numpy Generator(PCG64(seed)); draws in the order
coefficient field a, then the velocity angle field, then right-hand sides.
"""
import numpy as np

__all__ = ["Problem", "convdiff", "config_problem", "batch_problems", "rhs", "permuted", "random_local",
           "csr_from_coo"]


class Problem:
    """A CSR matrix plus the grid it lives on.

    rowptr: int64[n+1], colind: int32[nnz] (sorted within a row),
    val: float64[nnz], dims: tuple of grid sides (x fastest).
    """

    def __init__(self, dims, rowptr, colind, val, seed=None, name=""):
        # dims None: a general sparse matrix (no grid)
        self.dims = None if dims is None else tuple(int(d) for d in dims)
        self.rowptr = rowptr
        self.colind = colind
        self.val = val
        self.seed = seed
        self.name = name

    @property
    def n(self):
        return int(self.rowptr.shape[0] - 1)

    @property
    def nnz(self):
        return int(self.colind.shape[0])

    def to_dense(self):
        A = np.zeros((self.n, self.n))
        for r in range(self.n):
            for e in range(self.rowptr[r], self.rowptr[r + 1]):
                A[r, self.colind[e]] += self.val[e]
        return A

    def matvec(self, x):
        """y = A x for x of shape (n,) or (n, k) (float64)."""
        x = np.asarray(x, dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        prod = self.val[:, None] * x.reshape(self.n, -1)[self.colind]
        y = np.zeros((self.n, prod.shape[1]))
        np.add.at(y, rows, prod)
        return y.reshape(x.shape)


def convdiff(dims, a, v):
    """Assemble the upwinded convection-diffusion matrix.

    dims: (nx, ny) or (nx, ny, nz); a: cell diffusion, shape dims[::-1]
    flattened to (N,) in x-fastest order; v: velocity per cell, shape (N, d).
    """
    dims = tuple(int(d) for d in dims)
    d = len(dims)
    N = int(np.prod(dims))
    hs = [1.0 / (dims[k] + 1) for k in range(d)]   # the unit box, n_k points in direction k
    a = np.asarray(a, dtype=np.float64).reshape(N)
    v = np.asarray(v, dtype=np.float64).reshape(N, d)
    strides = [1]
    for k in range(1, d):
        strides.append(strides[-1] * dims[k - 1])
    idx = np.arange(N)
    coords = [(idx // strides[k]) % dims[k] for k in range(d)]
    diag = np.zeros(N)
    offd = {}  # (k, sign) -> coefficient array per row for neighbour c + sign*e_k
    for k in range(d):
        for sgn in (-1, 1):
            offd[(k, sgn)] = np.zeros(N)
    for k in range(d):
        for sgn in (-1, 1):
            inside = (coords[k] + sgn >= 0) & (coords[k] + sgn < dims[k])
            nb = np.where(inside, idx + sgn * strides[k], idx)
            an = a[nb]
            face = np.where(inside, 2.0 * a * an / (a + an), a)
            diag += face / (hs[k] * hs[k])
            offd[(k, sgn)] -= np.where(inside, face / (hs[k] * hs[k]), 0.0)
        vk = v[:, k]
        up = np.abs(vk) / hs[k]
        diag += up
        # v > 0: couple to c - e_k ; v < 0: couple to c + e_k
        has_m = (vk > 0) & (coords[k] - 1 >= 0)
        has_p = (vk < 0) & (coords[k] + 1 < dims[k])
        offd[(k, -1)] -= np.where(has_m, up, 0.0)
        offd[(k, 1)] -= np.where(has_p, up, 0.0)
    rows, cols, vals = [idx], [idx], [diag]
    for k in range(d):
        for sgn in (-1, 1):
            inside = (coords[k] + sgn >= 0) & (coords[k] + sgn < dims[k])
            rows.append(idx[inside])
            cols.append(idx[inside] + sgn * strides[k])
            vals.append(offd[(k, sgn)][inside])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(N + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int64)
    return rowptr, cols.astype(np.int32), vals.astype(np.float64)


def _uniform_a(rng, N):
    return rng.uniform(0.1, 10.0, size=N)


def gaussian_smooth(f, sigma=1.0, truncate=4.0):
    """Separable Gaussian convolution of a 2D array (standard deviation
    `sigma` grid cells, kernel cut at `truncate` sigma and normalised to sum
    1), mirrored at the edges (edge sample repeated)."""
    r = int(truncate * sigma + 0.5)
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / sigma) ** 2)
    k /= k.sum()
    out = np.asarray(f, dtype=np.float64)
    for ax in range(out.ndim):
        pad = [(0, 0)] * out.ndim
        pad[ax] = (r, r)
        g = np.pad(out, pad, mode="symmetric")
        acc = np.zeros_like(out)
        for i, w in enumerate(k):
            sl = [slice(None)] * out.ndim
            sl[ax] = slice(i, i + out.shape[ax])
            acc += w * g[tuple(sl)]
        out = acc
    return out


def high_contrast_field(rng, n, rho):
    """High-contrast coefficient of the paper's 2D experiments (Section 4):
    U[0,1] per grid point, smoothed with a unit-width Gaussian, then rho where
    the smoothed value is >= 0.5 and 1/rho elsewhere.  Returned in
    lexicographic order (x fastest)."""
    ahat = rng.uniform(0.0, 1.0, size=(n, n))          # [y, x]
    sm = gaussian_smooth(ahat, 1.0)
    return np.where(sm >= 0.5, float(rho), 1.0 / float(rho)).ravel()


def config_problem(kind, n=None, seed=None, rho=100.0):
    """Build one of the named synthetic workloads.

    kind:
      "2d_uniform_a"  : a ~ U[0.1,10] per cell, v = (10, 10)   (64x64 default)
      "2d_lognormal"  : a = exp(g), g ~ N(0,1); v = 50 (cos t, sin t),
                        t ~ U[0, 2 pi) per cell                 (256x256 default)
      "3d_uniform_a"  : a ~ U[0.1,10], v = 20 (1, 1, 1)         (32^3 default)
      "2d_high_contrast": a = rho / 1/rho from a thresholded smoothed
                        U[0,1] field (high_contrast_field), v = (1, 1)
                        (255x255 default; the draws do not depend on rho)
    """
    if kind == "2d_uniform_a":
        n = 64 if n is None else n
        seed = 1000 if seed is None else seed
        rng = np.random.Generator(np.random.PCG64(seed))
        N = n * n
        a = _uniform_a(rng, N)
        v = np.tile([10.0, 10.0], (N, 1))
        dims = (n, n)
    elif kind == "2d_lognormal":
        n = 256 if n is None else n
        seed = 2000 if seed is None else seed
        rng = np.random.Generator(np.random.PCG64(seed))
        N = n * n
        a = np.exp(rng.standard_normal(N))
        t = rng.uniform(0.0, 2.0 * np.pi, size=N)
        v = 50.0 * np.stack([np.cos(t), np.sin(t)], axis=1)
        dims = (n, n)
    elif kind == "3d_uniform_a":
        n = 32 if n is None else n
        seed = 3000 if seed is None else seed
        rng = np.random.Generator(np.random.PCG64(seed))
        N = n ** 3
        a = _uniform_a(rng, N)
        v = np.tile([20.0, 20.0, 20.0], (N, 1))
        dims = (n, n, n)
    elif kind == "2d_high_contrast":
        n = 255 if n is None else n
        seed = 6000 if seed is None else seed
        rng = np.random.Generator(np.random.PCG64(seed))
        N = n * n
        a = high_contrast_field(rng, n, rho)
        v = np.tile([1.0, 1.0], (N, 1))
        dims = (n, n)
    else:
        raise ValueError(kind)
    rowptr, colind, val = convdiff(dims, a, v)
    p = Problem(dims, rowptr, colind, val, seed=seed, name=f"{kind}_{n}")
    p.rng = rng
    return p


def batch_problems(count=64, seed=4000, sides=tuple(range(32, 129, 16))):
    """The batched workload: `count` independent 2D problems, matrix i seeded
    with seed + i: side drawn uniformly from `sides`, a ~ U[0.1,10] per cell,
    Pe ~ U[1,100] and v = Pe (1, 1).  Draw order per matrix: side, Pe, a."""
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(seed + i))
        n = int(sides[int(rng.integers(0, len(sides)))])
        pe = float(rng.uniform(1.0, 100.0))
        N = n * n
        a = _uniform_a(rng, N)
        v = np.tile([pe, pe], (N, 1))
        rowptr, colind, val = convdiff((n, n), a, v)
        p = Problem((n, n), rowptr, colind, val, seed=seed + i, name=f"batch{i}_{n}_pe{pe:.1f}")
        p.rng = rng
        p.pe = pe
        out.append(p)
    return out


def rhs(problem, nrhs=1, seed=None):
    """Right-hand sides, iid N(0,1), shape (n, nrhs) column-major in memory."""
    if seed is None:
        rng = problem.rng
    else:
        rng = np.random.Generator(np.random.PCG64(seed))
    b = rng.standard_normal((nrhs, problem.n))
    return np.asfortranarray(b.T)


def csr_from_coo(n, rows, cols, vals):
    """CSR (rowptr int64, colind int32 sorted in a row, val) of summed COO entries."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * n + cols
    uk, inv = np.unique(key, return_inverse=True)
    v = np.zeros(uk.shape[0])
    np.add.at(v, inv, vals)
    r, c = uk // n, uk % n
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    return np.cumsum(rowptr).astype(np.int64), c.astype(np.int32), v


def permuted(problem, seed, rows=True, cols=True):
    """P_r A P_c^T of a problem under random row / column permutations (a
    general sparse matrix: no grid).  Draws the row permutation, then the
    column one.  Row r of the result is row prow[r] of A; its entries move to
    the columns pinv_c[old column]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = problem.n
    prow = rng.permutation(n) if rows else np.arange(n)
    pcol = rng.permutation(n) if cols else np.arange(n)
    inv_c = np.empty(n, dtype=np.int64)
    inv_c[pcol] = np.arange(n)
    r_old = np.repeat(np.arange(n), np.diff(problem.rowptr))
    inv_r = np.empty(n, dtype=np.int64)
    inv_r[prow] = np.arange(n)
    rowptr, colind, val = csr_from_coo(n, inv_r[r_old], inv_c[problem.colind], problem.val)
    p = Problem(None, rowptr, colind, val, seed=seed, name=problem.name + "_perm")
    p.rng = rng
    p.prow, p.pcol = prow, pcol
    return p


def random_local(nside, k=4, radius=2.5, seed=7000, weak_diag=None):
    """A general unsymmetric sparse matrix: nside^2 points scattered in the
    unit square (one per grid cell, jittered); row i couples to k of the
    points within `radius` cell widths, chosen at random, with N(0,1)
    values; the diagonal is the row's absolute sum plus 1 (row diagonally
    dominant).  Unknowns are numbered in a random order.  Draws: jitter,
    numbering, then per row its neighbours and values.

    weak_diag = w > 0 instead draws the diagonal as w * N(0,1) right after
    the row's values (a matrix whose large entries are off the diagonal, so
    that the row matching matters); the other draws are unchanged."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = nside * nside
    base = np.stack(np.meshgrid(np.arange(nside), np.arange(nside), indexing="xy"), -1).reshape(-1, 2)
    pts = base + rng.uniform(-0.3, 0.3, size=(N, 2))
    label = rng.permutation(N)
    rows, cols, vals = [], [], []
    cell = {tuple(b): i for i, b in enumerate(base.tolist())}
    rr = int(np.ceil(radius))
    for i in range(N):
        bx, by = base[i]
        cand = []
        for dx in range(-rr, rr + 1):
            for dy in range(-rr, rr + 1):
                j = cell.get((bx + dx, by + dy))
                if j is not None and j != i and np.hypot(*(pts[j] - pts[i])) <= radius:
                    cand.append(j)
        cand = sorted(cand)
        pick = rng.choice(len(cand), size=min(k, len(cand)), replace=False) if cand else []
        off = rng.standard_normal(len(pick))
        for j, v in zip(pick, off):
            rows.append(label[i])
            cols.append(label[cand[j]])
            vals.append(v)
        rows.append(label[i])
        cols.append(label[i])
        vals.append(np.abs(off).sum() + 1.0 if weak_diag is None else weak_diag * rng.standard_normal())
    rowptr, colind, val = csr_from_coo(N, rows, cols, vals)
    name = f"random_local_{nside}" if weak_diag is None else f"random_local_weak_{nside}"
    p = Problem(None, rowptr, colind, val, seed=seed, name=name)
    p.rng = rng
    return p
