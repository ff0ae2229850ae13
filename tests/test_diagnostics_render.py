"""The diagnostics tables render from a study record, also after a JSON
round trip (integer keys of the pivot decay become strings), and the pivot
decay is the median over interfaces of |R_kk| / |R_11|."""
import json

import numpy as np

from paper_2010_06807_gb300 import diagnostics


def _study():
    piv = [np.array([2.0, 1.0, 0.5]), np.array([4.0, 1.0]), np.array([1.0])]
    dec = diagnostics.pivot_decay(piv)
    lev = {"level": 0, "n_fronts": 3, "max_front_rows": 40, "max_front_cols": 20, "n_interfaces": 3,
           "max_interface": 12, "remaining_size": 30, "interface_after": 18, "phase_ms": [1.0, 0.5, 0.25, 0.125],
           "pivot_decay": dec}
    return [{"n_side": 8, "N": 64, "levels": 1, "factor_ms": 1.5, "factor_bytes": 2 ** 20, "bytes_per_unknown": 16384,
             "top_separator": 5, "rank_sum": 18, "size_sum": 30, "gmres_iters": 4, "levels_detail": [lev]}], dec


def test_pivot_decay_medians():
    _, dec = _study()
    assert dec[1] == 1.0
    assert dec[2] == 0.375          # median of 1/2 and 1/4
    assert dec[4] is None


def test_markdown_survives_json_round_trip():
    st, _ = _study()
    a = diagnostics.markdown(st, "t")
    b = diagnostics.markdown(json.loads(json.dumps(st)), "t")
    assert a == b
    assert "| 8 | 64 | 1 | 1.5 | 1 | 16384 | 5 | 18 / 30 | 4 |" in a
    assert "1.0e+00 3.8e-01 -" in a


def test_plan_report_invariants():
    """The host-only plan report (no GPU): without sparsification every
    unknown is a front column exactly once, and each level's interfaces are
    the next level's fronts and interfaces; level 0 holds every atom."""
    import paper_2010_06807_gb300 as sq
    from paper_2010_06807_gb300.diagnostics import plan_markdown, plan_report
    from synth.convdiff import config_problem, permuted, random_local
    g = config_problem("2d_lognormal", n=48)
    q = permuted(g, 3)
    r = random_local(20, seed=7050)
    c = config_problem("3d_uniform_a", n=9)
    cases = [sq.spaqr_order(g.rowptr, g.colind, g.dims),
             sq.spaqr_order(q.rowptr, q.colind, None, val=q.val),
             sq.spaqr_order(r.rowptr, r.colind, None, val=r.val, matching="max_product"),
             sq.spaqr_order(c.rowptr, c.colind, c.dims)]
    for o in cases:
        rep = plan_report(o)
        lv = rep["per_level"]
        assert len(lv) == o.L and lv[0]["clusters"] == rep["atoms"]
        assert sum(x["front_cols"] for x in lv) == o.n
        assert lv[0]["front_cols"] + lv[0]["interface_cols"] == o.n
        for a, b in zip(lv, lv[1:]):
            assert a["interface_cols"] == b["front_cols"] + b["interface_cols"]
            assert a["n_interfaces"] >= b["clusters"]          # interfaces only merge
        assert lv[-1]["n_interfaces"] == 0 and lv[-1]["n_fronts"] == 1
        assert plan_markdown(rep, "t").count("\n|") == o.L + 2   # header, rule, one row per level


def test_markdown_residual_history():
    """A study row with its GMRES residual estimates renders them in order,
    also after a JSON round trip."""
    st, _ = _study()
    st[0]["gmres_history"] = [0.5, 2.5e-3, 7.0e-13]
    a = diagnostics.markdown(st, "t")
    assert "- side 8: 5.0e-01 2.5e-03 7.0e-13" in a
    assert diagnostics.markdown(json.loads(json.dumps(st)), "t") == a
