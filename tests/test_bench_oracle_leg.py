"""The bench's oracle legs on the CPU (no GPU): one oracle process factors a
small headline-type matrix, times one right-hand side's GMRES on one core,
then brings all 16 right-hand sides to 1e-12 in forked worker processes (the
multi-core CPU baseline).  Every column converges with the iteration count
the single-core run reports."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_leg_single_and_parallel():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.run_oracle(1, parallel=2, nside=24)
    assert r["factor_s"] > 0 and len(r["gmres_s"]) == 1
    assert r["relres_max"] <= bench.TOL
    assert "parallel_error" not in r, r.get("parallel_error")
    assert r["parallel_cores"] == 2 and len(r["parallel_iters"]) == bench.NRHS
    assert r["parallel_relres_max"] <= bench.TOL
    # column 0 in a worker is the same computation as the single-core run
    assert r["parallel_iters"][0] == r["iters"][0]
    assert bench.host_cores() >= 1


def test_reference_steps_side_by_side():
    """The reference arm's steps (one right-hand side's oracle GMRES each)
    run in forked workers: the warm-up steps first, then the timed ones,
    whose times, iteration counts and wall clock come back."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.run_oracle(5, mode="reference", parallel=2, nside=24, warm=2)
    assert r["cores"] == 2 and r["wall_s"] > 0
    assert len(r["gmres_s"]) == 3 and len(r["iters"]) == 3
    assert r["relres_max"] <= bench.TOL
    serial = bench.run_oracle(3, mode="reference", parallel=1, nside=24)
    assert "wall_s" not in serial and len(serial["gmres_s"]) == 3
    # steps 2..4 use right-hand sides 2..4 side by side, 0..2 one after the other
    assert r["iters"][0] == serial["iters"][2]
