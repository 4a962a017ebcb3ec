"""The stored oracle spread (tests/golden/oracle_spread.json, written by
tests/golden/make_oracle_spread.py) is current: one realization of a case
re-run now gives the stored values exactly, and every case holds eight
realizations."""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _maker():
    spec = importlib.util.spec_from_file_location("make_oracle_spread",
                                                  os.path.join(HERE, "golden", "make_oracle_spread.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_spread_cases_complete():
    from parity_util import oracle_spread
    for case in ("small_slab_500", "kvac_history", "partial_early", "subdomain_64x64"):
        g = oracle_spread(case)
        assert g["keys"] == list(range(1, 9))
        for name, d in g["diagnostics"].items():
            v = np.array(d["values"])
            assert v.size == 8
            assert abs(v.mean() - d["mean"]) <= 1e-12 * max(abs(d["mean"]), 1.0), (case, name)


def test_stored_realization_reproduces(tables):
    m = _maker()
    m.TABLES = tables
    from parity_util import oracle_spread
    g = oracle_spread("kvac_history")
    _, vals = m.case_kvac_history(1)
    for name, v in vals.items():
        assert v == g["diagnostics"][name]["values"][0], name
