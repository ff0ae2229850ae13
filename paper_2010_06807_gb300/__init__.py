"""Python binding of libspaqr (GB300 spaQR): argument marshalling only.

Every call goes through the C ABI declared in include/spaqr.h; every numeric
step runs in the library's CUDA kernels.  Arrays may be numpy arrays (host) or
torch tensors (host or CUDA).  Dense right-hand sides are column-major
(n x nrhs with unit row stride), e.g. ``torch.empty(nrhs, n).T`` or
``np.asfortranarray``.

The library is loaded on first use; if it is missing this raises, there is no
fallback.

Typical use::

    o = spaqr_order(rowptr, colind, (nx, ny))         # grid: geometric ordering
    o = spaqr_order(rowptr, colind, None, val=val)    # general matrix: G(A^T A) ordering, matched rows
    o = spaqr_order(rowptr, colind, None, val=val, matching="max_product")
    F = spaqr_factor(o, rowptr, colind, val, eps=1e-2)          # scaled, FP64
    F = spaqr_factor(o, rowptr, colind, val, eps=1e-2, scaling=0, precision="fp32")
    X, iters, relres = spaqr_gmres(F, rowptr, colind, val, B, tol=1e-12)

Diagnostics per level: spaqr_factor_level, spaqr_factor_pivots,
spaqr_factor_ranks, spaqr_factor_sigmas (and the diagnostics module);
batches of independent grids: spaqr_order_batch + blockdiag_csr +
spaqr_gmres_batch; serving: the serve module.
"""
import ctypes
import os

import numpy as np

__all__ = [
    "SpaqrError", "load_library", "spaqr_order", "spaqr_order_batch", "blockdiag_csr",
    "spaqr_factor", "spaqr_solve", "spaqr_solve_noalloc",
    "spaqr_gmres", "spaqr_gmres_batch",
    "spaqr_factor_info", "spaqr_factor_ranks", "spaqr_factor_sigmas", "spaqr_factor_level",
    "spaqr_factor_pivots", "Ordering", "Factor", "num_levels",
    "spaqr_stats_reset", "spaqr_profile", "spaqr_stats", "spaqr_use_graphs", "spaqr_autotune",
    "spaqr_factor_tuning", "spaqr_test_fail_alloc",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspaqr.so")

SPAQR_OK = 0
_ERRNAMES = {
    -1: "INVALID_ARG", -2: "UNSUPPORTED", -3: "OOM", -4: "SINGULAR", -5: "NOT_CONVERGED",
    -6: "TIMEOUT", -7: "CUDA", -8: "NO_DEVICE",
}


class SpaqrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"spaqr error {code} ({_ERRNAMES.get(code, '?')}): {msg}")
        self.code = code
        self.name = _ERRNAMES.get(code, "?")


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("colind", ctypes.c_void_p), ("val", ctypes.c_void_p), ("on_device", ctypes.c_int)]


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class _Opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("nlevels", ctypes.c_int), ("skip", ctypes.c_int),
                ("scaling", ctypes.c_int), ("precision", ctypes.c_int), ("col_normalize", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class _OrdInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("nlevels", ctypes.c_int32),
                ("n_atoms", ctypes.c_int32), ("n_nodes", ctypes.c_int32), ("plan_len", ctypes.c_int64)]


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nlevels", ctypes.c_int32), ("skip", ctypes.c_int32),
                ("eps", ctypes.c_double), ("factor_bytes", ctypes.c_int64),
                ("solve_bytes", ctypes.c_int64), ("factor_flops", ctypes.c_double),
                ("solve_flops", ctypes.c_double), ("n_interfaces_sparsified", ctypes.c_int32),
                ("rank_sum", ctypes.c_int64), ("size_sum", ctypes.c_int64),
                ("phase_ms", ctypes.c_double * 4), ("top_size", ctypes.c_int32),
                ("peak_bytes", ctypes.c_int64), ("workspace_rows", ctypes.c_int64),
                ("precision", ctypes.c_int32), ("tc_levels", ctypes.c_int32)]


class _BlockInfo(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("kind", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("other", ctypes.c_int32), ("rows", ctypes.c_int32), ("cols", ctypes.c_int32)]


# kinds of stored factor blocks (spaqr_factor_block, include/spaqr.h)
BLOCK_KINDS = {0: "front", 1: "front_tau", 2: "rsj", 3: "scale", 4: "scale_tau", 5: "cpqr", 6: "cpqr_tau",
               7: "fine", 8: "fine_tau"}


class _LevelInfo(ctypes.Structure):
    _fields_ = [("n_fronts", ctypes.c_int32), ("max_front_rows", ctypes.c_int32),
                ("max_front_cols", ctypes.c_int32), ("n_interfaces", ctypes.c_int32),
                ("front_rows", ctypes.c_int64), ("front_cols", ctypes.c_int64),
                ("n_remaining", ctypes.c_int32), ("max_interface", ctypes.c_int32),
                ("remaining_size", ctypes.c_int64), ("interface_after", ctypes.c_int64),
                ("block_entries", ctypes.c_int64), ("factor_bytes", ctypes.c_int64),
                ("phase_ms", ctypes.c_double * 4)]


class _KStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double), ("idle_ms", ctypes.c_double)]


_lib = None

# every symbol include/spaqr.h declares
EXPORTS = [
    "spaqr_last_error", "spaqr_opts_default", "spaqr_order", "spaqr_order_general", "spaqr_order_batch",
    "spaqr_ordering_info",
    "spaqr_ordering_get", "spaqr_ordering_rows", "spaqr_ordering_destroy", "spaqr_factor", "spaqr_solve", "spaqr_solve_noalloc",
    "spaqr_gmres", "spaqr_gmres_history", "spaqr_gmres_batch",
    "spaqr_factor_info", "spaqr_factor_ranks", "spaqr_factor_sigmas", "spaqr_factor_level", "spaqr_factor_pivots",
    "spaqr_factor_destroy", "spaqr_stats_reset",
    "spaqr_profile", "spaqr_stats", "spaqr_use_graphs", "spaqr_autotune", "spaqr_factor_tuning",
    "spaqr_test_fail_alloc", "spaqr_factor_nblocks", "spaqr_factor_block", "spaqr_peak", "spaqr_op_cycles", "spaqr_tc_tile_check",
    "spaqr_tc_gemm", "spaqr_use_tensor_cores",
]


def load_library(path=None):
    """Load libspaqr.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libspaqr.so not built ({p}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(p)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.spaqr_last_error.restype = ctypes.c_char_p
    lib.spaqr_opts_default.argtypes = [ctypes.POINTER(_Opts)]
    lib.spaqr_opts_default.restype = None
    lib.spaqr_order.argtypes = [ctypes.POINTER(_CSR), ctypes.POINTER(_Grid), i32, ctypes.POINTER(vp)]
    lib.spaqr_order_general.argtypes = [ctypes.POINTER(_CSR), i32, i32, ctypes.POINTER(vp)]
    lib.spaqr_order_batch.argtypes = [i32, ctypes.POINTER(_CSR), ctypes.POINTER(_Grid), ctypes.POINTER(vp)]
    lib.spaqr_ordering_info.argtypes = [vp, ctypes.POINTER(_OrdInfo)]
    lib.spaqr_ordering_get.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.spaqr_ordering_rows.argtypes = [vp, vp]
    lib.spaqr_ordering_destroy.argtypes = [vp]
    lib.spaqr_ordering_destroy.restype = None
    if hasattr(lib, "spaqr_factor"):
        lib.spaqr_factor.argtypes = [vp, ctypes.POINTER(_CSR), ctypes.POINTER(_Opts), ctypes.POINTER(vp)]
        lib.spaqr_solve.argtypes = [vp, i32, vp, i64, vp, i64, vp]
        if hasattr(lib, "spaqr_solve_noalloc"):
            lib.spaqr_solve_noalloc.argtypes = [vp, i32, vp, i64, vp, i64, vp]
        lib.spaqr_gmres.argtypes = [vp, ctypes.POINTER(_CSR), i32, vp, i64, vp, i64, dbl, i32, vp, vp, vp]
        lib.spaqr_gmres_history.argtypes = [vp, ctypes.POINTER(_CSR), i32, vp, i64, vp, i64, dbl, i32, vp, vp, vp,
                                            vp]
        lib.spaqr_gmres_batch.argtypes = [vp, ctypes.POINTER(_CSR), i32, vp, i32, vp, i64, vp, i64, dbl, i32,
                                          vp, vp, vp]
        lib.spaqr_factor_info.argtypes = [vp, ctypes.POINTER(_Info)]
        lib.spaqr_factor_ranks.argtypes = [vp, i32, vp, vp, i32, ctypes.POINTER(ctypes.c_int)]
        lib.spaqr_factor_sigmas.argtypes = [vp, i32, vp, i32, ctypes.POINTER(ctypes.c_int)]
        lib.spaqr_factor_level.argtypes = [vp, i32, ctypes.POINTER(_LevelInfo)]
        lib.spaqr_factor_pivots.argtypes = [vp, i32, vp, i64, vp, i32, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int)]
        lib.spaqr_factor_nblocks.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        lib.spaqr_factor_block.argtypes = [vp, i64, ctypes.POINTER(_BlockInfo), vp]
        lib.spaqr_factor_destroy.argtypes = [vp]
        lib.spaqr_factor_destroy.restype = None
    if hasattr(lib, "spaqr_stats"):
        lib.spaqr_stats_reset.argtypes = []
        lib.spaqr_stats_reset.restype = None
        lib.spaqr_profile.argtypes = [i32]
        lib.spaqr_profile.restype = None
        lib.spaqr_use_graphs.argtypes = [i32]
        lib.spaqr_use_tensor_cores.argtypes = [i32]
        lib.spaqr_use_tensor_cores.restype = None
        lib.spaqr_test_fail_alloc.argtypes = [i64]
        lib.spaqr_test_fail_alloc.restype = None
        lib.spaqr_use_graphs.restype = None
        lib.spaqr_autotune.argtypes = [vp, i32, vp, vp, vp]
        lib.spaqr_factor_tuning.argtypes = [vp, i32, vp, i32, ctypes.POINTER(ctypes.c_int)]
        lib.spaqr_stats.argtypes = [ctypes.POINTER(_KStat), i32, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int64)]
    if hasattr(lib, "spaqr_peak"):
        lib.spaqr_peak.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.spaqr_op_cycles.argtypes = [i32, i32, i32, ctypes.POINTER(ctypes.c_double)]
        lib.spaqr_tc_tile_check.argtypes = [vp, vp, vp, i32, i32, vp]
        lib.spaqr_tc_gemm.argtypes = [i32, i32, i32, ctypes.c_float, vp, i64, i64, i32, vp, i64, i64,
                                      ctypes.c_float, vp, i64, i64, i32, vp]
    if path is None:
        _lib = lib
    return lib


def _check(rc):
    if rc != SPAQR_OK:
        raise SpaqrError(rc, _lib.spaqr_last_error().decode(errors="replace"))


def _check_gmres(rc, X, iters, relres):
    """As _check; a NOT_CONVERGED error carries the best iterate and the
    per-column counts (e.X, e.iters, e.relres)."""
    if rc != SPAQR_OK:
        e = SpaqrError(rc, _lib.spaqr_last_error().decode(errors="replace"))
        e.X, e.iters, e.relres = X, iters, relres
        raise e


def num_levels(n):
    """ceil(log2(N/64)), at least 1 (Section 4)."""
    import math
    if n <= 64:
        return 1
    return max(1, int(math.ceil(math.log2(n / 64.0) - 1e-12)))


# ---------------------------------------------------------------------------
# array marshalling
# ---------------------------------------------------------------------------

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, keepalive, on_device) for a numpy array or torch tensor of dtype."""
    if _is_torch(x):
        import torch
        tdt = {np.int64: torch.int64, np.int32: torch.int32, np.float64: torch.float64}[dtype]
        if x.dtype != tdt:
            raise TypeError(f"expected {tdt}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), x, bool(x.is_cuda)
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a, False


def _make_csr(rowptr, colind, val=None):
    rp, k1, d1 = _ptr(rowptr, np.int64)
    ci, k2, d2 = _ptr(colind, np.int32)
    keep = [k1, k2]
    vv, d3 = None, d1
    if val is not None:
        vv, k3, d3 = _ptr(val, np.float64)
        keep.append(k3)
    if not (d1 == d2 == d3):
        raise ValueError("CSR arrays must all be on the host or all on the device")
    n = int(rowptr.shape[0]) - 1
    nnz = int(colind.shape[0])
    c = _CSR(n, nnz, rp, ci, vv, 1 if d1 else 0)
    return c, keep


def _dense_colmajor(x, n, name):
    """(ptr, ld, nrhs, keepalive, on_device) for an n x nrhs column-major operand."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.float64:
            raise TypeError(f"{name} must be float64")
        if x.dim() == 1:
            if x.stride(0) != 1:
                raise ValueError(f"{name} must have unit stride")
            return x.data_ptr(), n, 1, x, bool(x.is_cuda)
        if x.shape[0] != n or x.stride(0) != 1:
            raise ValueError(f"{name} must be n x nrhs column-major (stride(0) == 1)")
        ld = x.stride(1) if x.shape[1] > 1 else n
        return x.data_ptr(), ld, int(x.shape[1]), x, bool(x.is_cuda)
    a = np.asarray(x)
    if a.dtype != np.float64:
        raise TypeError(f"{name} must be float64")
    if a.ndim == 1:
        a = a.reshape(n, 1)
    if a.shape[0] != n or not a.flags.f_contiguous:
        raise ValueError(f"{name} must be a Fortran-ordered n x nrhs float64 array")
    return a.ctypes.data, n, int(a.shape[1]), a, False


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ---------------------------------------------------------------------------
# ordering
# ---------------------------------------------------------------------------

class Ordering:
    """Owns a spaqr_ordering handle."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)
        info = _OrdInfo()
        _check(_lib.spaqr_ordering_info(self._h, ctypes.byref(info)))
        self.n = info.n
        self.nnz = info.nnz
        self.L = info.nlevels
        self.n_atoms = info.n_atoms
        self.n_nodes = info.n_nodes
        self.plan_len = info.plan_len

    def arrays(self):
        perm = np.zeros(self.n, dtype=np.int64)
        atom_ptr = np.zeros(self.n_atoms + 1, dtype=np.int64)
        atom_node = np.zeros(self.n_atoms, dtype=np.int32)
        node_level = np.zeros(self.n_nodes, dtype=np.int32)
        plan = np.zeros(self.plan_len, dtype=np.int32)
        _check(_lib.spaqr_ordering_get(self._h, perm.ctypes.data, atom_ptr.ctypes.data,
                                       atom_node.ctypes.data, node_level.ctypes.data, plan.ctypes.data))
        rperm = np.zeros(self.n, dtype=np.int64)
        _check(_lib.spaqr_ordering_rows(self._h, rperm.ctypes.data))
        return dict(perm=perm, atom_ptr=atom_ptr, atom_node=atom_node, node_level=node_level, plan=plan,
                    rperm=rperm)

    def plan(self):
        """Decode the symbolic plan: list of per-level dicts."""
        code = self.arrays()["plan"].tolist()
        out = []
        i = 0
        while i < len(code):
            lev = code[i]; ncl = code[i + 1]; i += 2
            cl = code[i:i + ncl]; i += ncl
            nf = code[i]; i += 1
            fronts = []
            for _ in range(nf):
                s, col, nr = code[i], code[i + 1], code[i + 2]; i += 3
                R = code[i:i + nr]; i += nr
                nc = code[i]; i += 1
                C = code[i:i + nc]; i += nc
                fronts.append(dict(id=s, colour=col, R=R, C=C))
            out.append(dict(level=lev, clusters=cl, fronts=fronts))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.spaqr_ordering_destroy(h)
            self._h = None


MATCHINGS = {"greedy": 0, "max_product": 1}


def spaqr_order(rowptr, colind, dims, nlevels=0, val=None, matching=None):
    """Modified nested dissection + symbolic plan (spaqr_order): geometric on
    the grid `dims`, or, with dims None, the general-matrix ordering on
    G(A^T A) with rows matched to columns (by |val| when given;
    spaqr_order_general): matching "max_product" (the default: the perfect
    matching maximising the product of the matched |a_ij|) or "greedy"
    (largest entries first, then augmenting paths)."""
    load_library()
    if dims is not None and matching is not None:
        raise ValueError("a row matching applies to the grid-free ordering (dims None); "
                         "grid orderings keep every row with its column")
    csr, keep = _make_csr(rowptr, colind, val if dims is None else None)
    h = ctypes.c_void_p()
    if dims is None:
        matching = "max_product" if matching is None else matching
        if matching not in MATCHINGS:
            raise ValueError(f"matching must be one of {sorted(MATCHINGS)}")
        _check(_lib.spaqr_order_general(ctypes.byref(csr), int(nlevels), MATCHINGS[matching], ctypes.byref(h)))
    else:
        dims = tuple(int(d) for d in dims)
        g = _Grid(len(dims), dims[0], dims[1], dims[2] if len(dims) > 2 else 1)
        _check(_lib.spaqr_order(ctypes.byref(csr), ctypes.byref(g), int(nlevels), ctypes.byref(h)))
    return Ordering(h.value)


def spaqr_order_batch(patterns, dims_list):
    """Ordering of the block-diagonal batch diag(A_0, ..., A_{k-1})
    (spaqr_order_batch).  patterns: [(rowptr, colind)] (all host or all
    device); dims_list: the grid sides of every matrix.  The returned
    Ordering has .part_ptr, the row offsets of the matrices."""
    load_library()
    k = len(patterns)
    if k < 1 or len(dims_list) != k:
        raise ValueError("one grid per matrix, at least one matrix")
    csrs = (_CSR * k)()
    grids = (_Grid * k)()
    keep = []
    part = [0]
    for i, ((rp, ci), dims) in enumerate(zip(patterns, dims_list)):
        c, kk = _make_csr(rp, ci)
        keep.append(kk)
        csrs[i] = c
        dims = tuple(int(d) for d in dims)
        grids[i] = _Grid(len(dims), dims[0], dims[1], dims[2] if len(dims) > 2 else 1)
        part.append(part[-1] + c.n)
    h = ctypes.c_void_p()
    _check(_lib.spaqr_order_batch(k, csrs, grids, ctypes.byref(h)))
    o = Ordering(h.value)
    o.part_ptr = np.asarray(part, dtype=np.int64)
    return o


def blockdiag_csr(mats):
    """Host CSR (rowptr int64, colind int32, val float64) of the block-diagonal
    matrix diag(A_0, ..., A_{k-1}) from [(rowptr, colind, val)] host arrays:
    the layout spaqr_order_batch orders."""
    rps, cis, vals = [], [], []
    e0 = 0
    base = 0
    for rp, ci, v in mats:
        rp = np.asarray(rp, dtype=np.int64)
        rps.append(rp[1:] + e0 if rps else rp + e0)
        cis.append(np.asarray(ci, dtype=np.int64) + base)
        vals.append(np.asarray(v, dtype=np.float64))
        e0 += int(rp[-1])
        base += rp.shape[0] - 1
    if base > np.iinfo(np.int32).max:
        raise ValueError("batch too large for int32 column indices")
    return (np.concatenate(rps), np.concatenate(cis).astype(np.int32), np.concatenate(vals))


# ---------------------------------------------------------------------------
# factor / solve / gmres
# ---------------------------------------------------------------------------

class Factor:
    """Owns a spaqr_factor_t handle."""

    def __init__(self, handle, n):
        self._h = ctypes.c_void_p(handle)
        self.n = n

    def close(self):
        """Free the factor's device memory now (waits for the device)."""
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.spaqr_factor_destroy(h)
        self._h = None

    def __del__(self):
        self.close()


SPAQR_FP64 = 0
SPAQR_FP32 = 1
SPAQR_TF32 = 2
# doubles of the fixed device scratch array of spaqr_solve_noalloc (include/spaqr.h)
SPAQR_NOALLOC_SCRATCH_DOUBLES = 2 * 1024 * 1024


def spaqr_factor(ordering, rowptr, colind, val, eps=1e-2, nlevels=0, skip=2, scaling=1,
                 col_normalize=1, precision="fp64", stream=None):
    """Numeric spaQR factorisation (Algorithm 2) on the current CUDA device.

    precision: "fp64" (plain form), "fp32" (mixed form: factor stored and
    applied in FP32, the contractions of large fronts on the tensor cores in
    three TF32 passes; rank decisions and GMRES stay FP64) or "tf32" (as
    "fp32" with one TF32 pass).
    """
    load_library()
    csr, keep = _make_csr(rowptr, colind, val)
    o = _Opts()
    _lib.spaqr_opts_default(ctypes.byref(o))
    o.precision = {"fp64": SPAQR_FP64, "fp32": SPAQR_FP32, "tf32": SPAQR_TF32}[precision]
    o.eps = float(eps)
    o.nlevels = int(nlevels)
    o.skip = int(skip)
    o.scaling = int(scaling)
    o.col_normalize = int(col_normalize)
    o.stream = _stream_ptr(stream)
    h = ctypes.c_void_p()
    _check(_lib.spaqr_factor(ordering._h, ctypes.byref(csr), ctypes.byref(o), ctypes.byref(h)))
    return Factor(h.value, csr.n)


def spaqr_solve(F, B, X=None, stream=None):
    """X = M^{-1} B (one application of the factor).  Returns X."""
    load_library()
    bp, ldb, nrhs, kb, bdev = _dense_colmajor(B, F.n, "B")
    if X is None:
        if bdev:
            import torch
            X = torch.empty(nrhs, F.n, dtype=torch.float64, device=B.device).T
            if B.dim() == 1:
                X = X[:, 0]
        else:
            X = np.zeros((F.n, nrhs), order="F")
            if np.asarray(B).ndim == 1:
                X = X[:, 0]
    xp, ldx, nrx, kx, xdev = _dense_colmajor(X, F.n, "X")
    if nrx != nrhs or xdev != bdev:
        raise ValueError("X must match B in shape and memory space")
    _check(_lib.spaqr_solve(F._h, nrhs, bp, ldb, xp, ldx, _stream_ptr(stream)))
    return X


def spaqr_solve_noalloc(F, B, X, stream=None):
    """X = M^{-1} B through spaqr_solve_noalloc: device tensors only, nothing
    allocated on the device (scratch is the library's fixed device array)."""
    load_library()
    bp, ldb, nrhs, kb, bdev = _dense_colmajor(B, F.n, "B")
    xp, ldx, nrx, kx, xdev = _dense_colmajor(X, F.n, "X")
    if nrx != nrhs:
        raise ValueError("X must match B in shape")
    _check(_lib.spaqr_solve_noalloc(F._h, nrhs, bp, ldb, xp, ldx, _stream_ptr(stream)))
    return X


def spaqr_gmres(F, rowptr, colind, val, B, X=None, tol=1e-12, maxit=300, stream=None, history=False):
    """Right-preconditioned GMRES; returns (X, iters[nrhs], relres[nrhs]), and
    with history=True also a list of per-column arrays: the Arnoldi estimate
    of the relative residual after each iteration (spaqr_gmres_history).

    Raises SpaqrError(NOT_CONVERGED) if a column misses tol; the error carries
    X, iters and relres (and .history with history=True).
    """
    load_library()
    csr, keep = _make_csr(rowptr, colind, val)
    bp, ldb, nrhs, kb, bdev = _dense_colmajor(B, F.n, "B")
    if X is None:
        if bdev:
            import torch
            X = torch.zeros(nrhs, F.n, dtype=torch.float64, device=B.device).T
            if B.dim() == 1:
                X = X[:, 0]
        else:
            X = np.zeros((F.n, nrhs), order="F")
            if np.asarray(B).ndim == 1:
                X = X[:, 0]
    xp, ldx, nrx, kx, xdev = _dense_colmajor(X, F.n, "X")
    iters = np.zeros(nrhs, dtype=np.int32)
    relres = np.zeros(nrhs, dtype=np.float64)
    if not history:
        _check_gmres(_lib.spaqr_gmres(F._h, ctypes.byref(csr), nrhs, bp, ldb, xp, ldx, float(tol), int(maxit),
                                      iters.ctypes.data, relres.ctypes.data, _stream_ptr(stream)), X, iters, relres)
        return X, iters, relres
    hist = np.zeros((max(nrhs, 1), int(maxit)), dtype=np.float64)
    rc = _lib.spaqr_gmres_history(F._h, ctypes.byref(csr), nrhs, bp, ldb, xp, ldx, float(tol), int(maxit),
                                  iters.ctypes.data, relres.ctypes.data, hist.ctypes.data, _stream_ptr(stream))
    per_col = [hist[c, :iters[c]].copy() for c in range(nrhs)]
    try:
        _check_gmres(rc, X, iters, relres)
    except SpaqrError as e:
        e.history = per_col
        raise
    return X, iters, relres, per_col


def spaqr_gmres_batch(F, rowptr, colind, val, part_ptr, B, X=None, tol=1e-12, maxit=300, stream=None):
    """GMRES on a block-diagonal batch (spaqr_gmres_batch): every matrix and
    column is its own Krylov process.  Returns (X, iters, relres) with iters /
    relres of shape (nrhs, count)."""
    load_library()
    csr, keep = _make_csr(rowptr, colind, val)
    part = np.ascontiguousarray(part_ptr, dtype=np.int64)
    count = part.shape[0] - 1
    bp, ldb, nrhs, kb, bdev = _dense_colmajor(B, F.n, "B")
    if X is None:
        if bdev:
            import torch
            X = torch.zeros(nrhs, F.n, dtype=torch.float64, device=B.device).T
            if B.dim() == 1:
                X = X[:, 0]
        else:
            X = np.zeros((F.n, nrhs), order="F")
            if np.asarray(B).ndim == 1:
                X = X[:, 0]
    xp, ldx, nrx, kx, xdev = _dense_colmajor(X, F.n, "X")
    iters = np.zeros(nrhs * count, dtype=np.int32)
    relres = np.zeros(nrhs * count, dtype=np.float64)
    _check_gmres(_lib.spaqr_gmres_batch(F._h, ctypes.byref(csr), count, part.ctypes.data, nrhs, bp, ldb, xp, ldx,
                                        float(tol), int(maxit), iters.ctypes.data, relres.ctypes.data,
                                        _stream_ptr(stream)),
                 X, iters.reshape(nrhs, count), relres.reshape(nrhs, count))
    return X, iters.reshape(nrhs, count), relres.reshape(nrhs, count)


def spaqr_factor_info(F):
    load_library()
    info = _Info()
    _check(_lib.spaqr_factor_info(F._h, ctypes.byref(info)))
    return {f: (list(getattr(info, f)) if f == "phase_ms" else getattr(info, f)) for f, _ in _Info._fields_}


def spaqr_factor_ranks(F, level):
    """[(size_before, rank)], margins [(|R_rr| first rejected or last kept, |R_11|)] of a level."""
    load_library()
    cnt = ctypes.c_int(0)
    _check(_lib.spaqr_factor_ranks(F._h, int(level), None, None, 0, ctypes.byref(cnt)))
    n = cnt.value
    pairs = np.zeros(2 * max(n, 1), dtype=np.int32)
    margins = np.zeros(2 * max(n, 1), dtype=np.float64)
    _check(_lib.spaqr_factor_ranks(F._h, int(level), pairs.ctypes.data, margins.ctypes.data, n,
                                   ctypes.byref(cnt)))
    return pairs[:2 * n].reshape(n, 2), margins[:2 * n].reshape(n, 2)


def spaqr_factor_level(F, level):
    """Per-level diagnostics (spaqr_level_info) of level k (0 = leaves) as a dict."""
    load_library()
    info = _LevelInfo()
    _check(_lib.spaqr_factor_level(F._h, int(level), ctypes.byref(info)))
    return {f: (list(getattr(info, f)) if f == "phase_ms" else getattr(info, f)) for f, _ in _LevelInfo._fields_}


def spaqr_factor_pivots(F, level):
    """CPQR pivot norms |R_kk| per interface sparsified at a level: a list of
    arrays (kept steps and the first rejected one), in spaqr_factor_ranks order."""
    load_library()
    nn, ni = ctypes.c_int64(0), ctypes.c_int(0)
    _check(_lib.spaqr_factor_pivots(F._h, int(level), None, 0, None, 0, ctypes.byref(nn), ctypes.byref(ni)))
    norms = np.zeros(max(nn.value, 1), dtype=np.float64)
    offs = np.zeros(ni.value + 1, dtype=np.int32)
    _check(_lib.spaqr_factor_pivots(F._h, int(level), norms.ctypes.data, nn.value, offs.ctypes.data, ni.value + 1,
                                    ctypes.byref(nn), ctypes.byref(ni)))
    return [norms[offs[i]:offs[i + 1]].copy() for i in range(ni.value)]


def spaqr_factor_blocks(F):
    """Every stored block of the factor (spaqr_factor_nblocks /
    spaqr_factor_block): a list of dicts with level, kind (a BLOCK_KINDS
    name), cluster, other (the column cluster of an R_sj block, else -1) and
    data (rows x cols float64 array, a copy)."""
    load_library()
    cnt = ctypes.c_int64(0)
    _check(_lib.spaqr_factor_nblocks(F._h, ctypes.byref(cnt)))
    out = []
    info = _BlockInfo()
    for i in range(cnt.value):
        _check(_lib.spaqr_factor_block(F._h, i, ctypes.byref(info), None))
        a = np.zeros((info.cols, info.rows), dtype=np.float64)   # column-major
        _check(_lib.spaqr_factor_block(F._h, i, ctypes.byref(info), a.ctypes.data if a.size else None))
        out.append({"level": info.level, "kind": BLOCK_KINDS[info.kind], "cluster": info.cluster,
                    "other": info.other, "data": a.T})
    return out


def spaqr_factor_sigmas(F, level):
    """sigma_p = 1 / sigma_min(A_p) per interface of a level (unscaled variant; 0 when scaled)."""
    load_library()
    cnt = ctypes.c_int(0)
    _check(_lib.spaqr_factor_sigmas(F._h, int(level), None, 0, ctypes.byref(cnt)))
    n = cnt.value
    out = np.zeros(max(n, 1), dtype=np.float64)
    _check(_lib.spaqr_factor_sigmas(F._h, int(level), out.ctypes.data, n, ctypes.byref(cnt)))
    return out[:n]


def spaqr_test_fail_alloc(after):
    """Fault injection: the device allocation after `after` more successful
    ones fails (once); -1 switches it off."""
    load_library()
    _lib.spaqr_test_fail_alloc(int(after))


def spaqr_stats_reset():
    """Zero the library's launch counters."""
    load_library()
    _lib.spaqr_stats_reset()


def spaqr_profile(on=True):
    """Bracket every library launch with CUDA events (for per-kernel timing)."""
    load_library()
    _lib.spaqr_profile(1 if on else 0)


def spaqr_use_tensor_cores(on=True):
    """Tensor-core application of large fronts in the FP32 / TF32 forms (default on)."""
    load_library()
    _lib.spaqr_use_tensor_cores(1 if on else 0)


def spaqr_autotune(F, nrhs, stream=None):
    """Time the launch forms of every unit of the application for nrhs
    columns and keep the fastest (spaqr_autotune).  Returns (ms_rule, ms_tuned)."""
    load_library()
    a = ctypes.c_double(0.0)
    b = ctypes.c_double(0.0)
    _check(_lib.spaqr_autotune(F._h, int(nrhs), _stream_ptr(stream), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def spaqr_factor_tuning(F, nrhs):
    """The launch forms spaqr_autotune kept for nrhs (empty: rules apply)."""
    load_library()
    cnt = ctypes.c_int(0)
    _check(_lib.spaqr_factor_tuning(F._h, int(nrhs), None, 0, ctypes.byref(cnt)))
    out = np.zeros(max(cnt.value, 1), dtype=np.int32)
    _check(_lib.spaqr_factor_tuning(F._h, int(nrhs), out.ctypes.data, cnt.value, ctypes.byref(cnt)))
    return out[:cnt.value]


def spaqr_use_graphs(on=True):
    """Replay the factor application inside GMRES as a CUDA graph (default on)."""
    load_library()
    _lib.spaqr_use_graphs(1 if on else 0)


def spaqr_stats():
    """(total launches, {kernel: dict(launches, total_ms, flops, bytes, idle_ms)}) since the last
    reset; idle_ms: time the stream stood idle before the kind's launches (profiling on)."""
    load_library()
    cnt = ctypes.c_int(0)
    tot = ctypes.c_int64(0)
    _check(_lib.spaqr_stats(None, 0, ctypes.byref(cnt), ctypes.byref(tot)))
    arr = (_KStat * cnt.value)()
    _check(_lib.spaqr_stats(arr, cnt.value, ctypes.byref(cnt), ctypes.byref(tot)))
    out = {}
    for k in arr:
        out[k.name.decode()] = dict(launches=int(k.launches), total_ms=float(k.total_ms),
                                    flops=float(k.flops), bytes=float(k.bytes), idle_ms=float(k.idle_ms))
    return int(tot.value), out


PEAKS = {"dfma": 0, "dmma": 1, "ffma": 2, "tf32": 3}


OPS = {"dfma": 0, "dadd": 1, "ddiv": 2, "dsqrt": 3, "ffma": 4, "f2f": 5, "dsel": 6}


def spaqr_op_cycles(op, warps=1, lanes=32):
    """Clock cycles per operation of a dependent chain of `op` (a key of OPS)
    in one CTA of `warps` warps, `lanes` active lanes each (slowest warp)."""
    load_library()
    c = ctypes.c_double(0.0)
    _check(_lib.spaqr_op_cycles(OPS[op], int(warps), int(lanes), ctypes.byref(c)))
    return c.value


def spaqr_peak(which, reps=10):
    """Arithmetic peak microbenchmark ("dfma", "dmma", "ffma" or "tf32"):
    returns (flops per launch, mean ms per launch); TFLOP/s = flops / ms / 1e9."""
    load_library()
    f, m = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(_lib.spaqr_peak(PEAKS[which], int(reps), ctypes.byref(f), ctypes.byref(m)))
    return f.value, m.value


def spaqr_tc_tile_check(A, B, stream=None):
    """D = A B^T (A 128 x K, B N x K, float32 CUDA tensors, row-major) through
    one tcgen05 TF32 tile; returns D (128 x N, float32)."""
    import torch
    load_library()
    if A.dim() != 2 or A.shape[0] != 128 or B.dim() != 2 or B.shape[1] != A.shape[1]:
        raise ValueError("A must be 128 x K and B N x K")
    A = A.contiguous()
    B = B.contiguous()
    D = torch.empty(A.shape[0], B.shape[0], dtype=torch.float32, device=A.device)
    _check(_lib.spaqr_tc_tile_check(A.data_ptr(), B.data_ptr(), D.data_ptr(), B.shape[0], A.shape[1],
                                    _stream_ptr(stream)))
    return D


def spaqr_tc_gemm(A, B, C, alpha=1.0, beta=0.0, reflectors=False, split3=False, stream=None):
    """C = alpha A B + beta C in place on the tensor cores (spaqr_tc_gemm):
    A (M x K), B (K x N), C (M x N) float32 CUDA tensors with any strides;
    reflectors: A read as its unit lower trapezoidal reflector matrix."""
    load_library()
    M, K = A.shape
    K2, N = B.shape
    if K2 != K or tuple(C.shape) != (M, N):
        raise ValueError("shapes do not match")
    _check(_lib.spaqr_tc_gemm(M, N, K, float(alpha), A.data_ptr(), A.stride(0), A.stride(1), int(bool(reflectors)),
                              B.data_ptr(), B.stride(0), B.stride(1), float(beta), C.data_ptr(), C.stride(0),
                              C.stride(1), int(bool(split3)), _stream_ptr(stream)))
    return C
