"""Continuous-batching server on the GPU: every solve result is the same alone
and in the mix.

Requests to three resident factors arrive from several threads while other
batches run, and a factor request lands in the middle; afterwards each
right-hand side is solved again alone (one-column GMRES on the same resident
factor).  Both runs must reach the 1e-12 relative residual and agree to 1e-10
relative, and the host-side residual of each result is checked too.
"""
import threading

import numpy as np
import pytest

from synth.convdiff import config_problem

pytestmark = pytest.mark.gpu

TOL_SAME = 1e-10


def _run_mix(precision, seed):
    import torch

    from paper_2010_06807_gb300.serve import DeviceOps, SolveServer
    ops = DeviceOps(torch.device("cuda:0"), eps=1e-2, precision=precision)
    srv = SolveServer(ops, max_slots=8)
    probs = {0: config_problem("3d_uniform_a", n=12, seed=seed),
             1: config_problem("3d_uniform_a", n=16, seed=seed + 1),
             2: config_problem("2d_lognormal", n=64, seed=seed + 2)}
    for mid, p in probs.items():
        srv.add_matrix(mid, p)
    late = config_problem("3d_uniform_a", n=20, seed=seed + 3)
    rng = np.random.default_rng(seed)
    plan = [int(rng.integers(0, 3)) for _ in range(60)]
    reqs = [None] * len(plan)
    fac = {}

    def client(lo, step):
        for i in range(lo, len(plan), step):
            mid = plan[i]
            b = np.random.default_rng(seed * 1000 + i).standard_normal(probs[mid].n)
            reqs[i] = (mid, b, srv.submit_solve(mid, b))
            if i == 20:
                fac["req"] = srv.submit_factor(3, late)

    threads = [threading.Thread(target=client, args=(t, 3)) for t in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert fac["req"].wait(600) > 0
    probs[3] = late
    late_reqs = []
    for i in range(6):
        b = np.random.default_rng(seed * 7 + i).standard_normal(late.n)
        late_reqs.append((3, b, srv.submit_solve(3, b)))
    mixed = []
    for mid, b, q in reqs + late_reqs:
        x = q.wait(600)
        mixed.append((mid, b, x, q.relres, q.batch))
    return srv, ops, probs, mixed


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_same_alone_and_in_mix(spaqr_lib, precision):
    srv, ops, probs, mixed = _run_mix(precision, 4242)
    try:
        batch_sizes = [k for _, _, _, _, k in mixed]
        assert max(batch_sizes) > 1, "no request was batched with another"
        worst = 0.0
        for mid, b, x, relres, _ in mixed:
            assert relres <= 1e-12
            r = srv.res[mid]
            xa, it, rr = ops.solve(r.handle, b[None, :], r.stream)
            assert rr[0] <= 1e-12
            d = np.linalg.norm(xa[0] - x) / np.linalg.norm(xa[0])
            worst = max(worst, d)
            assert d <= TOL_SAME, (mid, d)
            res = np.linalg.norm(b - probs[mid].matvec(x)) / np.linalg.norm(b)
            assert res <= 1e-11, (mid, res)
        print(f"{precision}: {len(mixed)} requests, batches up to {max(batch_sizes)}, "
              f"max relative difference alone vs mix {worst:.2e}")
    finally:
        srv.close()


def test_batches_overlap_on_device(spaqr_lib):
    """Batches of different matrices are in flight at the same time."""
    import torch

    from paper_2010_06807_gb300.serve import DeviceOps, SolveServer
    ops = DeviceOps(torch.device("cuda:0"), eps=1e-2)
    srv = SolveServer(ops, max_slots=16)
    try:
        probs = [config_problem("3d_uniform_a", n=24, seed=77 + m) for m in range(3)]
        for m, p in enumerate(probs):
            srv.add_matrix(m, p)
        reqs = []
        for rep in range(4):
            for m, p in enumerate(probs):
                for j in range(4):
                    reqs.append(srv.submit_solve(m, np.random.default_rng(rep * 100 + m * 10 + j).standard_normal(p.n)))
        for q in reqs:
            q.wait(600)
        spans = sorted({(q.mid, q.t_start, q.t_done) for q in reqs}, key=lambda s: s[1])
        overlap = any(a[0] != b[0] and b[1] < a[2] for i, a in enumerate(spans) for b in spans[i + 1:])
        assert overlap
    finally:
        srv.close()


def test_admission_evicts_on_device(spaqr_lib):
    """A factor request that does not fit next to an idle non-pinned factor
    evicts it; the device memory of the evicted factor is returned."""
    import torch

    from paper_2010_06807_gb300.serve import DeviceOps, SolveServer
    ops = DeviceOps(torch.device("cuda:0"), eps=1e-2)
    p0 = config_problem("3d_uniform_a", n=16, seed=11)
    p1 = config_problem("3d_uniform_a", n=16, seed=12)
    srv = SolveServer(ops, max_slots=4, hbm_budget=1 << 40)
    b0 = srv.add_matrix(0, p0, pinned=False)
    srv.close()
    est = ops.estimate_factor_bytes(p1)       # from p0's peak bytes per unknown
    assert est >= b0
    # budget: room for the factorisation of p1 alone, not next to p0
    srv = SolveServer(ops, max_slots=4, hbm_budget=int(est + 0.5 * b0))
    try:
        srv.add_matrix(0, p0, pinned=False)
        x0 = srv.submit_solve(0, np.ones(p0.n)).wait(600)
        assert srv.submit_factor(1, p1).wait(600) > 0
        assert srv.evicted == [0] and srv.resident() == [1]
        x1 = srv.submit_solve(1, np.ones(p1.n)).wait(600)
        assert np.linalg.norm(np.ones(p0.n) - p0.matvec(x0)) / np.sqrt(p0.n) <= 1e-11
        assert np.linalg.norm(np.ones(p1.n) - p1.matvec(x1)) / np.sqrt(p1.n) <= 1e-11
    finally:
        srv.close()
