"""Host logic of the continuous-batching server, on a fake device.

The fake device "solves" by scaling the right-hand side by the matrix id + 1
and sleeps to stand in for GPU time, so batching, overlap, the memory ledger
and eviction can be checked without a GPU.
"""
import threading
import time

import numpy as np
import pytest

from paper_2010_06807_gb300.serve import SolveServer


class _P:
    def __init__(self, n, dims=(8, 8)):
        self._n = n
        self.dims = dims

    @property
    def n(self):
        return self._n


class FakeOps:
    def __init__(self, solve_s=0.02, factor_s=0.01, per_unknown=100, rhs_bytes=8):
        self.solve_s = solve_s
        self.factor_s = factor_s
        self.per_unknown = per_unknown
        self.rhs_bytes = rhs_bytes
        self.intervals = []
        self.released = []
        self.lock = threading.Lock()
        self.live = 0
        self.max_live = 0

    def new_stream(self):
        return object()

    def load(self, problem, stream):
        time.sleep(self.factor_s)
        return {"n": problem.n, "mid": problem.mid}

    def factor_bytes(self, h):
        return self.per_unknown * h["n"]

    def estimate_factor_bytes(self, problem):
        return self.per_unknown * problem.n

    def batch_bytes(self, n, k):
        return self.rhs_bytes * n * k

    def solve(self, h, Bh, stream):
        with self.lock:
            self.live += 1
            self.max_live = max(self.max_live, self.live)
        t0 = time.perf_counter()
        time.sleep(self.solve_s)
        t1 = time.perf_counter()
        with self.lock:
            self.live -= 1
            self.intervals.append((h["mid"], Bh.shape[0], t0, t1))
        k = Bh.shape[0]
        return Bh * (h["mid"] + 1), np.full(k, 3), np.full(k, 1e-13)

    def release(self, h):
        self.released.append(h["mid"])


def _prob(mid, n):
    p = _P(n)
    p.mid = mid
    return p


def test_batches_form_while_busy_and_results_match():
    ops = FakeOps(solve_s=0.05)
    srv = SolveServer(ops, max_slots=8, hbm_budget=1 << 30)
    srv.add_matrix(0, _prob(0, 16))
    rng = np.random.default_rng(0)
    bs = [rng.standard_normal(16) for _ in range(20)]
    reqs = [srv.submit_solve(0, bs[0])]
    while reqs[0].t_start is None:       # the first batch is running
        time.sleep(0.001)
    reqs += [srv.submit_solve(0, b) for b in bs[1:]]
    for q, b in zip(reqs, bs):
        np.testing.assert_array_equal(q.wait(5), b)
        assert q.relres == 1e-13 and q.iters == 3
    sizes = [k for (_, k, _, _) in ops.intervals]
    assert sum(sizes) == 20
    assert max(sizes) <= 8
    assert max(sizes) > 1          # arrivals during a batch were batched
    # the first request did not wait for a full batch
    assert sizes[0] == 1
    srv.close()
    assert ops.released == [0]


def test_matrices_run_concurrently():
    ops = FakeOps(solve_s=0.1)
    srv = SolveServer(ops, max_slots=4, hbm_budget=1 << 30)
    for m in range(3):
        srv.add_matrix(m, _prob(m, 8))
    reqs = [srv.submit_solve(m, np.ones(8)) for m in range(3)]
    for m, q in enumerate(reqs):
        np.testing.assert_array_equal(q.wait(5), np.full(8, m + 1.0))
    assert ops.max_live == 3
    srv.close()


def test_factor_admission_evicts_lru_idle_unpinned():
    ops = FakeOps()
    # room for the pinned matrix (100*10) plus one 100*20 matrix, not two
    srv = SolveServer(ops, max_slots=4, hbm_budget=100 * 10 + 100 * 20 + 500)
    srv.add_matrix(0, _prob(0, 10), pinned=True)
    assert srv.submit_factor(1, _prob(1, 20)).wait(5) == 2000
    srv.submit_solve(1, np.ones(20)).wait(5)
    assert srv.submit_factor(2, _prob(2, 20)).wait(5) == 2000
    assert srv.resident() == [0, 2]
    assert srv.evicted == [1]
    assert ops.released == [1]
    with pytest.raises(KeyError):
        srv.submit_solve(1, np.ones(20))
    np.testing.assert_array_equal(srv.submit_solve(2, np.ones(20)).wait(5), np.full(20, 3.0))
    assert srv.held_bytes() == 1000 + 2000
    assert srv.peak <= srv.hbm_budget
    srv.close()


def test_factor_that_can_never_fit_fails():
    ops = FakeOps()
    srv = SolveServer(ops, max_slots=4, hbm_budget=5000)
    srv.add_matrix(0, _prob(0, 40), pinned=True)
    with pytest.raises(MemoryError):
        srv.submit_factor(1, _prob(1, 20)).wait(5)
    with pytest.raises(KeyError):
        srv.submit_factor(0, _prob(0, 5)).wait(5)
    srv.close()


def test_factor_waits_for_busy_matrix_then_evicts():
    ops = FakeOps(solve_s=0.2)
    srv = SolveServer(ops, max_slots=4, hbm_budget=100 * 20 + 100 * 20 + 8 * 20 * 4)
    srv.add_matrix(1, _prob(1, 20), pinned=False)
    q = srv.submit_solve(1, np.ones(20))
    time.sleep(0.05)                      # matrix 1 is busy now
    f = srv.submit_factor(2, _prob(2, 30))
    np.testing.assert_array_equal(q.wait(5), np.full(20, 2.0))
    assert f.wait(5) == 3000
    assert srv.evicted == [1]
    # the factor started only after the batch on matrix 1 returned
    assert f.t_start >= q.t_done
    srv.close()


def test_batch_split_to_fit_memory():
    ops = FakeOps(solve_s=0.05, rhs_bytes=8)
    # resident 100*10 bytes; room for 2 right-hand sides of n=10 in flight
    srv = SolveServer(ops, max_slots=16, hbm_budget=1000 + 8 * 10 * 2)
    srv.add_matrix(0, _prob(0, 10))
    reqs = [srv.submit_solve(0, np.full(10, float(i))) for i in range(9)]
    for i, q in enumerate(reqs):
        np.testing.assert_array_equal(q.wait(5), np.full(10, float(i)))
    sizes = [k for (_, k, _, _) in ops.intervals]
    assert sum(sizes) == 9 and max(sizes) <= 2
    assert srv.peak <= srv.hbm_budget
    srv.close()


def test_bad_requests():
    ops = FakeOps()
    srv = SolveServer(ops, max_slots=4, hbm_budget=1 << 20)
    srv.add_matrix(0, _prob(0, 10))
    with pytest.raises(KeyError):
        srv.submit_solve(7, np.ones(10))
    with pytest.raises(ValueError):
        srv.submit_solve(0, np.ones(11))
    srv.close()
    with pytest.raises(RuntimeError):
        srv.submit_factor(3, _prob(3, 10))


def test_device_ops_memory_estimates(monkeypatch, spaqr_lib):
    """DeviceOps keeps the largest peak bytes per unknown of each grid
    dimension (general matrices under their own key) and estimates a new
    factor from it; resident bytes are the factor's own."""
    import paper_2010_06807_gb300 as sq
    from paper_2010_06807_gb300.serve import DeviceOps
    infos = iter([{"factor_bytes": 1000, "peak_bytes": 4000}, {"factor_bytes": 50, "peak_bytes": 90}])
    monkeypatch.setattr(sq, "spaqr_factor_info", lambda F: next(infos))
    ops = DeviceOps("cuda:0")
    p3 = _P(100, dims=(5, 5, 4))
    assert ops.estimate_factor_bytes(p3) == 16384 * 100       # nothing seen yet
    assert ops.factor_bytes({"F": None, "n": 100, "dim": 3}) == 1000
    assert ops.estimate_factor_bytes(_P(200, dims=(5, 5, 8))) == int(1.25 * 40 * 200)
    g = _P(10, dims=None)
    g.dims = None
    assert ops.estimate_factor_bytes(g) == 16384 * 10          # general matrices: own key
    assert ops.factor_bytes({"F": None, "n": 10, "dim": 0}) == 50
    assert ops.estimate_factor_bytes(g) == int(1.25 * 9 * 10)


def test_device_ops_matching_option():
    """The served ordering of general matrices takes the row matching given
    to DeviceOps; an unknown one is refused when the server is set up."""
    import pytest as _pt
    from paper_2010_06807_gb300.serve import DeviceOps
    assert DeviceOps("cuda:0").matching == "max_product"
    assert DeviceOps("cuda:0", matching="greedy").matching == "greedy"
    with _pt.raises(ValueError):
        DeviceOps("cuda:0", matching="mc64")
