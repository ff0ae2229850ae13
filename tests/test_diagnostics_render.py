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
