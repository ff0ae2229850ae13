"""Continuous-batching solve server over resident spaQR factorisations.

The server keeps factorisations resident in device memory and serves two
kinds of requests:
  * solve(mid, b): x = A_mid^{-1} b by GMRES with the spaQR factor as right
    preconditioner (Section 2.7), to a relative residual of `tol`;
  * factor(mid, problem): factor a new matrix (Algorithm 2), which then stays
    resident and takes solve requests.

Scheduling (continuous batching):
  * every resident matrix has a worker thread and a CUDA stream of its own;
  * a worker takes the solve requests waiting for its matrix, up to
    `max_slots` of them, and runs them as one multi-RHS GMRES call (every
    right-hand side keeps its own Krylov space, so a result does not depend on
    the batch it ran in, up to rounding);
  * requests that arrive meanwhile queue up and form the next batch of that
    matrix as soon as the running one returns;
  * batches of different matrices and factorisations run at the same time on
    their own streams, so their kernels overlap on the device;
  * one ledger of device bytes covers the resident factors and the workspace
    of every batch or factorisation in flight.  Work starts only when its
    bytes fit `hbm_budget`: a batch that does not fit is split or waits, a
    factor request evicts idle, non-pinned matrices (least recently used
    first) or waits, and work that can never fit fails with MemoryError.

Every numeric step runs in libspaqr's kernels; this module schedules only
(ctypes releases the GIL around each library call, so the worker threads
drive the device concurrently).
"""
import argparse
import json
import threading
import time

import numpy as np

__all__ = ["SolveServer", "Request", "DeviceOps", "run_workload", "run_plain"]


class Request:
    """A submitted request; `wait()` returns its result (x, or factor bytes)."""

    def __init__(self, kind, mid, payload, t_submit):
        self.kind = kind
        self.mid = mid
        self.payload = payload
        self.t_submit = t_submit
        self.t_start = None
        self.t_done = None
        self.result = None
        self.error = None
        self.iters = None
        self.relres = None
        self.batch = None
        self._ev = threading.Event()

    def _finish(self, result=None, error=None):
        self.result = result
        self.error = error
        self.t_done = time.perf_counter()
        self._ev.set()

    def done(self):
        return self._ev.is_set()

    def wait(self, timeout=None):
        if not self._ev.wait(timeout):
            raise TimeoutError("request not finished")
        if self.error is not None:
            raise self.error
        return self.result

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_submit


def _dim_key(problem):
    """Memory estimates are kept per grid dimension; general matrices (no
    grid) have their own key, 0."""
    return len(problem.dims) if problem.dims is not None else 0


class DeviceOps:
    """libspaqr + torch streams on one CUDA device: what the server runs."""

    def __init__(self, device=None, eps=1e-2, precision="fp32", tol=1e-12, maxit=300, matching="max_product"):
        """precision: of the resident factors, "fp32" by default (GMRES is
        FP64 and reaches tol either way; the FP32 factors serve 5x the
        requests of FP64 ones on the serving workload) or "fp64".
        matching: the row matching of general matrices (no grid),
        "max_product" (the default) or "greedy" (see spaqr_order)."""
        import torch

        from . import load_library
        load_library()
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda:0")
        self.eps = eps
        self.precision = precision
        self.tol = tol
        self.maxit = maxit
        from . import MATCHINGS
        if matching not in MATCHINGS:
            raise ValueError(f"matching must be one of {sorted(MATCHINGS)}")
        self.matching = matching
        self._per_unknown = {}

    def new_stream(self):
        return self.torch.cuda.Stream(device=self.device)

    def load(self, problem, stream):
        """Order and factor `problem` on `stream`; returns the resident handle."""
        from . import spaqr_factor, spaqr_order
        torch = self.torch
        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            csr = (torch.from_numpy(problem.rowptr).to(self.device),
                   torch.from_numpy(problem.colind).to(self.device),
                   torch.from_numpy(problem.val).to(self.device))
            # grids: geometric ordering; general matrices (dims None): the
            # G(A^T A) ordering with rows matched by |a_ij|
            general = problem.dims is None
            ordering = spaqr_order(problem.rowptr, problem.colind, problem.dims,
                                   val=problem.val if general else None,
                                   matching=self.matching if general else None)
            F = spaqr_factor(ordering, *csr, eps=self.eps, precision=self.precision, stream=stream)
        return {"F": F, "csr": csr, "ordering": ordering, "n": problem.n, "dim": _dim_key(problem)}

    def factor_bytes(self, h):
        from . import spaqr_factor_info
        info = spaqr_factor_info(h["F"])
        nbytes = int(info["factor_bytes"])
        per = self._per_unknown.get(h["dim"], 0.0)
        self._per_unknown[h["dim"]] = max(per, int(info["peak_bytes"]) / h["n"])
        return nbytes

    def batch_bytes(self, n, k):
        # device memory one k-RHS GMRES call takes: restarted Krylov bases V and
        # Z, the iterate, B, X and work vectors (a small over-estimate)
        cap = min(self.maxit, 48) + 1
        return 8 * n * k * (2 * cap + 8)

    def estimate_factor_bytes(self, problem):
        # the largest peak bytes per unknown (factor plus the factorisation's
        # temporaries) seen for factors of the same grid dimension, with a
        # quarter again for larger grids; 16 KB per unknown before any factor
        # of that dimension exists
        per = self._per_unknown.get(_dim_key(problem))
        return int(1.25 * per * problem.n) if per else 16384 * problem.n

    def solve(self, h, Bh, stream):
        """Bh: k x n host array (row i = right-hand side i).
        Returns (X k x n host array, iters[k], relres[k])."""
        from . import spaqr_gmres
        torch = self.torch
        k, n = Bh.shape
        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            B = torch.from_numpy(Bh).to(self.device).T
            X = torch.zeros(k, n, dtype=torch.float64, device=self.device).T
            X, it, rr = spaqr_gmres(h["F"], *h["csr"], B, X=X, tol=self.tol, maxit=self.maxit,
                                    stream=stream)
            Xh = X.T.cpu().numpy()
        return Xh, it, rr

    def release(self, h):
        h["F"].close()


class _Resident:
    def __init__(self, mid, n, handle, stream, nbytes, pinned):
        self.mid = mid
        self.n = n
        self.handle = handle
        self.stream = stream
        self.bytes = nbytes
        self.pinned = pinned
        self.queue = []
        self.cv = threading.Condition()
        self.busy = False
        self.stop = False
        self.last_used = time.perf_counter()
        self.batches = []
        self.thread = None


class SolveServer:
    """Resident factors, continuous batching of solves, factor requests
    admitted by device memory.

    ops: the device operations (DeviceOps on a GPU); max_slots: right-hand
    sides per batch; hbm_budget: bytes the ledger may hold (default: 90% of
    the device's free memory when the server starts, for DeviceOps).
    """

    def __init__(self, ops, max_slots=64, hbm_budget=None):
        self.ops = ops
        self.max_slots = int(max_slots)
        if hbm_budget is None:
            free, _ = ops.torch.cuda.mem_get_info(ops.device)
            hbm_budget = int(0.9 * free)
        self.hbm_budget = int(hbm_budget)
        self.mu = threading.Condition()
        self.res = {}
        self.held = 0          # bytes of resident factors
        self.reserved = 0      # bytes of work in flight
        self.peak = 0
        self.evicted = []
        self.closed = False
        self._factor_q = []
        self._factor_cv = threading.Condition()
        self._factor_thread = threading.Thread(target=self._factor_worker, daemon=True)
        self._factor_thread.start()

    # ---------------------------------------------------------------- ledger
    def _fits(self, need):
        return self.held + self.reserved + need <= self.hbm_budget

    def _note_peak(self):
        self.peak = max(self.peak, self.held + self.reserved)

    # ---------------------------------------------------------------- matrices
    def _install(self, mid, n, handle, stream, nbytes, pinned):
        r = _Resident(mid, n, handle, stream, nbytes, pinned)
        r.thread = threading.Thread(target=self._solve_worker, args=(r,), daemon=True)
        self.res[mid] = r
        self.held += nbytes
        self._note_peak()
        r.thread.start()
        return r

    def add_matrix(self, mid, problem, pinned=True):
        """Factor `problem` now (blocking) and keep it resident; pinned
        matrices are never evicted.  Returns the factor's device bytes."""
        req = self.submit_factor(mid, problem, pinned=pinned)
        return req.wait()

    def resident(self):
        with self.mu:
            return sorted(self.res)

    def held_bytes(self):
        with self.mu:
            return self.held

    def submit_solve(self, mid, b):
        """Queue one right-hand side (float64, length n) for matrix `mid`."""
        req = Request("solve", mid, np.asarray(b, dtype=np.float64), time.perf_counter())
        with self.mu:
            r = self.res.get(mid)
            if r is None or r.stop:
                raise KeyError(f"matrix {mid} is not resident")
            if req.payload.shape != (r.n,):
                raise ValueError(f"right-hand side must have length {r.n}")
            with r.cv:
                r.queue.append(req)
                r.cv.notify()
        return req

    def submit_factor(self, mid, problem, pinned=False):
        req = Request("factor", mid, (problem, pinned), time.perf_counter())
        with self._factor_cv:
            if self.closed:
                raise RuntimeError("server closed")
            self._factor_q.append(req)
            self._factor_cv.notify()
        return req

    # ---------------------------------------------------------------- workers
    def _evict_one(self):
        """Under self.mu: stop the least recently used idle non-pinned matrix.
        Returns its handle (to release outside the lock) or None."""
        idle = []
        for r in self.res.values():
            if r.pinned:
                continue
            with r.cv:
                if not r.busy and not r.queue:
                    idle.append(r)
        if not idle:
            return None
        v = min(idle, key=lambda r: r.last_used)
        with v.cv:
            v.stop = True
            v.cv.notify()
        del self.res[v.mid]
        self.held -= v.bytes
        self.evicted.append(v.mid)
        return v.handle

    def _factor_worker(self):
        while True:
            with self._factor_cv:
                while not self._factor_q and not self.closed:
                    self._factor_cv.wait()
                if not self._factor_q:
                    return
                req = self._factor_q.pop(0)
            problem, pinned = req.payload
            need = self.ops.estimate_factor_bytes(problem)
            to_release = []
            error = None
            with self.mu:
                while not self._fits(need):
                    h = self._evict_one()
                    if h is not None:
                        to_release.append(h)
                        continue
                    if self.reserved == 0:
                        error = MemoryError(f"factor of n={problem.n} needs ~{need} bytes; "
                                            f"{self.hbm_budget - self.held} of the budget are free")
                        break
                    self.mu.wait(0.02)
                if error is None:
                    if req.mid in self.res:
                        error = KeyError(f"matrix {req.mid} is already resident")
                    else:
                        self.reserved += need
                        self._note_peak()
            for h in to_release:
                self.ops.release(h)
            if error is not None:
                req._finish(error=error)
                continue
            req.t_start = time.perf_counter()
            try:
                stream = self.ops.new_stream()
                h = self.ops.load(problem, stream)
                nbytes = self.ops.factor_bytes(h)
            except Exception as e:  # surfaced to the caller
                with self.mu:
                    self.reserved -= need
                    self.mu.notify_all()
                req._finish(error=e)
                continue
            with self.mu:
                self.reserved -= need
                self._install(req.mid, problem.n, h, stream, nbytes, pinned)
                self.mu.notify_all()
            req._finish(result=nbytes)

    def _solve_worker(self, r):
        while True:
            with r.cv:
                while not r.queue and not r.stop:
                    r.cv.wait()
                if r.stop:
                    pending, r.queue = r.queue, []
                    for q in pending:
                        q._finish(error=KeyError(f"matrix {r.mid} was evicted"))
                    return
                batch = r.queue[:self.max_slots]
                del r.queue[:len(batch)]
                r.busy = True
            k = len(batch)
            need = self.ops.batch_bytes(r.n, k)
            fail = None
            with self.mu:
                while not self._fits(need):
                    if k > 1:
                        # split: the tail goes back to the front of the queue
                        k = (k + 1) // 2
                        with r.cv:
                            r.queue[0:0] = batch[k:]
                        batch = batch[:k]
                        need = self.ops.batch_bytes(r.n, k)
                        continue
                    if self.reserved == 0:
                        fail = MemoryError(f"one right-hand side of n={r.n} needs {need} bytes")
                        break
                    self.mu.wait(0.02)
                if fail is None:
                    self.reserved += need
                    self._note_peak()
            if fail is not None:
                for q in batch:
                    q._finish(error=fail)
                with r.cv:
                    r.busy = False
                continue
            t0 = time.perf_counter()
            for q in batch:
                q.t_start = t0
                q.batch = k
            try:
                Bh = np.stack([q.payload for q in batch])
                Xh, it, rr = self.ops.solve(r.handle, Bh, r.stream)
                for i, q in enumerate(batch):
                    q.iters = int(it[i])
                    q.relres = float(rr[i])
                    q._finish(result=np.array(Xh[i]))
            except Exception as e:
                for q in batch:
                    q._finish(error=e)
            with self.mu:
                self.reserved -= need
                self.mu.notify_all()
            with r.cv:
                r.batches.append(k)
                r.last_used = time.perf_counter()
                r.busy = False

    def close(self):
        """Finish queued work, stop the workers and free every factor."""
        with self._factor_cv:
            self.closed = True
            self._factor_cv.notify_all()
        self._factor_thread.join()
        with self.mu:
            rs = list(self.res.values())
        for r in rs:
            with r.cv:
                while r.queue or r.busy:
                    r.cv.wait(0.001)
                r.stop = True
                r.cv.notify()
        for r in rs:
            r.thread.join()
        with self.mu:
            for r in rs:
                self.res.pop(r.mid, None)
                self.held -= r.bytes
        for r in rs:
            self.ops.release(r.handle)

    def batch_sizes(self):
        with self.mu:
            return {mid: list(r.batches) for mid, r in self.res.items()}


def _pct(v, q):
    if len(v) == 0:
        return None
    return float(np.percentile(np.asarray(v, dtype=np.float64), q))


def _arrivals(probs, rate, duration, seed):
    """Poisson arrivals (time, matrix, N(0,1) right-hand side) over `duration`."""
    rng = np.random.Generator(np.random.PCG64(seed + 10 ** 6))
    out = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        mid = int(rng.integers(0, len(probs)))
        out.append((t, mid, rng.standard_normal(probs[mid].n)))
    return out


def run_plain(sides=(16, 24, 32, 40, 48, 48, 32, 24), requests=200, eps=1e-2, precision="fp64", seed=5000,
              device=None):
    """The same request stream served the plain way: resident factors, but
    every request solved alone (one-column GMRES), one after another on one
    stream, no batching and no overlap.  Returns its throughput."""
    import torch

    from synth.convdiff import config_problem
    ops = DeviceOps(device, eps=eps, precision=precision)
    probs = [config_problem("3d_uniform_a", n=s, seed=seed + i) for i, s in enumerate(sides)]
    st = ops.new_stream()
    handles = [ops.load(p, st) for p in probs]
    arr = _arrivals(probs, 2000.0, 1.0, seed)[:requests]
    torch.cuda.synchronize(ops.device)
    t0 = time.perf_counter()
    worst = 0.0
    for _, mid, b in arr:
        _, _, rr = ops.solve(handles[mid], b[None, :], st)
        worst = max(worst, float(rr[0]))
    dt = time.perf_counter() - t0
    for h in handles:
        ops.release(h)
    return {"precision": precision, "requests": len(arr), "solves_per_s": len(arr) / dt, "relres_max": worst,
            "note": "same arrivals, each request alone and in arrival order"}


def run_workload(sides=(16, 24, 32, 40, 48, 48, 32, 24), rate=2000.0, duration=2.0, factor_every=1.0,
                 factor_side=32, eps=1e-2, precision="fp32", seed=5000, max_slots=64, device=None):
    """The serving workload: resident factors of 3D 7-point convection-diffusion
    problems with the given sides (a ~ U[0.1,10], velocity 20(1,1,1)); an
    open-loop Poisson stream of single-RHS N(0,1) solve requests with mean
    `rate` per second to uniformly random resident matrices; one new factor
    request of side `factor_side` every `factor_every` seconds.  The
    right-hand sides are drawn before the clock starts.  Returns latency and
    throughput statistics."""
    from synth.convdiff import config_problem
    ops = DeviceOps(device, eps=eps, precision=precision)
    srv = SolveServer(ops, max_slots=max_slots)
    t0 = time.perf_counter()
    probs = [config_problem("3d_uniform_a", n=s, seed=seed + i) for i, s in enumerate(sides)]
    for i, p in enumerate(probs):
        srv.add_matrix(i, p)
    setup_s = time.perf_counter() - t0
    arrivals = _arrivals(probs, rate, duration, seed)
    fact_times = [factor_every * (j + 1) for j in range(int(duration / factor_every + 1e-9))]
    fact_probs = [config_problem("3d_uniform_a", n=factor_side, seed=seed + 100 + j) for j in range(len(fact_times))]
    reqs, freqs = [], []
    t_start = time.perf_counter()
    fi = 0
    for (ta, mid, b) in arrivals:
        while fi < len(fact_times) and fact_times[fi] <= ta:
            freqs.append(srv.submit_factor(100 + fi, fact_probs[fi]))
            fi += 1
        delay = t_start + ta - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        reqs.append(srv.submit_solve(mid, b))
    while fi < len(fact_times):
        freqs.append(srv.submit_factor(100 + fi, fact_probs[fi]))
        fi += 1
    for q in reqs + freqs:
        q.wait(timeout=900)
    t_end = time.perf_counter()
    lat = [q.latency * 1e3 for q in reqs]
    batches = [k for v in srv.batch_sizes().values() for k in v]
    out = {
        "precision": precision, "rate_per_s": rate, "duration_s": duration,
        "requests": len(reqs), "wall_s": t_end - t_start, "setup_s": setup_s,
        "solves_per_s": len(reqs) / (t_end - t_start),
        "latency_ms_p50": _pct(lat, 50), "latency_ms_p99": _pct(lat, 99),
        "relres_max": max(q.relres for q in reqs) if reqs else None,
        "batches": len(batches), "mean_batch": float(np.mean(batches)) if batches else None,
        "factor_requests": len(freqs),
        "factor_latency_ms_p50": _pct([q.latency * 1e3 for q in freqs], 50),
        "resident_gib": srv.held_bytes() / 2 ** 30, "peak_ledger_gib": srv.peak / 2 ** 30,
    }
    srv.close()
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser(description="spaQR serving workload (resident 3D factors, Poisson solves)")
    ap.add_argument("--duration", type=float, default=2.0)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--max-slots", type=int, default=64)
    a = ap.parse_args()
    print(json.dumps(run_workload(rate=a.rate, duration=a.duration, precision=a.precision,
                                  max_slots=a.max_slots)))
