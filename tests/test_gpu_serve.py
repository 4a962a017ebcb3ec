"""Continuous batching of served slab requests: every request's result is
the same as when it runs alone, whatever it shared the GPU with."""
import numpy as np
import pytest

import pic_inputs as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1704_01202_gb300 as pkg  # noqa: E402
from paper_1704_01202_gb300 import serve  # noqa: E402


def _trace():
    # small slabs, fast arrivals, a few steps each; uneven horizons so that
    # slabs leave and enter between steps
    tr = P.request_trace(n=10, rate_hz=2000.0, seed=5, horizon_fs=0.2, cells=(8, 96), ppc=(16, 80))
    for k, r in enumerate(tr):
        r.nsteps = 6 + 3 * (k % 4)
    return tr


def _by_id(d):
    o = np.argsort(d["id"], kind="stable")
    return {k: v[o] for k, v in d.items()}


def test_served_results_equal_alone():
    pkg.build()
    tab = P.standin_tables()
    tr = _trace()
    fp = np.array([serve.footprint(r.cfg) for r in tr])
    # three slots and room for about half the trace: requests queue, slots
    # and space are reused
    cap_e, cap_i = (max(int(fp[:, q].sum() // 2), int(fp[:, q].max())) for q in (0, 1))
    init = lambda r: P.init_particles(r.cfg)  # noqa: E731
    out = serve.serve_batched(tr, tab, init, max_slabs=3, slot_cells=96,
                              cap_e=cap_e, cap_i=cap_i, tick_steps=4, keep=lambda rid: True)
    ref = serve.serve_one_at_a_time(tr, tab, init, keep=lambda rid: True)
    assert sorted(out["results"]) == [r.rid for r in tr]
    for r in tr:
        a, b = out["results"][r.rid], ref["results"][r.rid]
        assert a["counts"] == b["counts"], r.rid
        assert a["n_e"] == b["n_e"] and a["n_i"] == b["n_i"], r.rid
        assert a["t_fs"] == pytest.approx(r.nsteps * r.cfg.dt_fs)
        for k in ("ke_e", "ke_i", "e_ion", "e_phot", "e_trans"):
            assert a[k] == pytest.approx(b[k], rel=1e-9, abs=1e-12), (r.rid, k)
        (ge, gi), (re_, ri) = out["finals"][r.rid], ref["finals"][r.rid]
        ge, re_, gi, ri = _by_id(ge), _by_id(re_), _by_id(gi), _by_id(ri)
        for k in re_:
            assert np.array_equal(ge[k], re_[k]), (r.rid, "e", k)
        for k in ri:
            assert np.array_equal(gi[k], ri[k]), (r.rid, "i", k)
    for o in (out, ref):
        assert o["slabs"] == len(tr) and o["ttr_p99_s"] >= o["ttr_p50_s"] > 0
