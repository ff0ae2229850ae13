"""Per-level diagnostics (spaqr_factor_level, spaqr_factor_pivots) against
the oracle's own record of the same factorisation: fronts and their sizes,
the interfaces left after them and their sizes before and after
sparsification, and every CPQR pivot norm |R_kk| (the quantities of the
paper's profiling figures, Section 4)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2010_06807_gb300 as sq
from oracle import spaqr as osq
from paper_2010_06807_gb300 import diagnostics
from synth.convdiff import config_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev(spaqr_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("kind,n,eps,skip,scaling", [("2d_uniform_a", 32, 1e-2, 0, 1), ("3d_uniform_a", 10, 1e-2, 1, 1),
                                                     ("2d_lognormal", 40, 1e-3, 2, 0)])
def test_levels_match_oracle(dev, kind, n, eps, skip, scaling):
    p = config_problem(kind, n=n)
    o, F, _, ms = diagnostics.factor_problem(p, eps, scaling=scaling, skip=skip, device=dev)
    Fo = osq.factor(p.n, p.rowptr, p.colind, p.val, p.dims, eps, nlevels=o.L, skip=skip, scaling=bool(scaling))
    info = sq.spaqr_factor_info(F)
    total = np.zeros(4)
    last_bytes = 0
    for k, st in enumerate(Fo.steps):
        d = sq.spaqr_factor_level(F, k)
        sizes, fronts = st["sizes"], st["fronts"]
        assert d["n_fronts"] == len(fronts)
        assert d["front_cols"] == sum(sizes[s] for s in fronts)
        assert d["front_rows"] == sum(sizes[i] for s in fronts for i in st["R"][s])
        rest = [c for c in sizes if c not in fronts]
        assert d["n_remaining"] == len(rest) and d["remaining_size"] == sum(sizes[c] for c in rest)
        R = Fo.ranks[k]
        after = sum(R[c][1] if c in R else sizes[c] for c in rest)
        assert d["interface_after"] == after
        assert d["n_interfaces"] == sum(1 for c in R if R[c][0] > 0)
        piv = sq.spaqr_factor_pivots(F, k)
        ref = [Fo.rdiag[k][c] for c in sorted(R) if R[c][0] > 0]
        assert len(piv) == len(ref)
        for g, r in zip(piv, ref):
            assert g.shape == r.shape
            np.testing.assert_allclose(g, r, rtol=1e-10, atol=1e-14 * max(r.max(), 1e-300))
        assert d["factor_bytes"] >= last_bytes
        last_bytes = d["factor_bytes"]
        total += d["phase_ms"]
    assert last_bytes <= info["factor_bytes"]
    # the per-level phase times add up to the factor's (the gather before
    # level 0 is counted in the factor's merge phase only)
    assert np.all(total <= np.array(info["phase_ms"]) + 1e-6)
    assert total.sum() >= 0.5 * sum(info["phase_ms"])
    rep = diagnostics.level_report(F)
    assert len(rep) == o.L and all(set(r["pivot_decay"]) <= set(diagnostics.DECAY_AT) for r in rep)


def test_scaling_study_runs(dev):
    st = diagnostics.scaling_study("3d_uniform_a", [8, 12], 1e-2, device=dev)
    assert [r["N"] for r in st] == [512, 1728]
    assert all(r["gmres_relres"] <= 1e-12 for r in st)
    assert all(len(r["gmres_history"]) == r["gmres_iters"] and r["gmres_history"][-1] <= 1e-12 for r in st)
    md = diagnostics.markdown(st, "t")
    assert "| 12 | 1728 |" in md and "GMRES residual estimates" in md
