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


def _equal_runs(a, b, fa, fb, rid):
    assert a["counts"] == b["counts"], rid
    assert a["n_e"] == b["n_e"] and a["n_i"] == b["n_i"], rid
    for k in ("ke_e", "ke_i", "e_ion", "e_phot", "e_trans"):
        assert a[k] == pytest.approx(b[k], rel=1e-9, abs=1e-12), (rid, k)
    (ge, gi), (re_, ri) = fa, fb
    ge, re_, gi, ri = _by_id(ge), _by_id(re_), _by_id(gi), _by_id(ri)
    for k in re_:
        assert np.array_equal(ge[k], re_[k]), (rid, "e", k)
    for k in ri:
        assert np.array_equal(gi[k], ri[k]), (rid, "i", k)


def test_budget_failure_stays_with_its_slab():
    """A slab given an electron budget it outgrows (hot electrons ionizing
    by impact) fails alone: its slot reports FAILED, the slab beside it
    runs on bit for bit as alone, and a slab admitted into the freed slot
    runs as alone too (nothing of the failed one is left in its cells)."""
    pkg.build()
    tab = P.standin_tables()
    hot = P.cfg_small_1d(nx=16, ppc_e=64, ppc_i=16, T_e_eV=300.0, seed=3,
                         flags=P.F_COLL_EE | P.F_COLL_EI | P.F_IONIZE)
    tr = _trace()
    y, z = tr[1], tr[2]
    bt = pkg.Batch(tab, 2, 96, 40000, 10000)
    try:
        sx = bt.admit(hot, P.init_particles(hot))
        sy = bt.admit(y.cfg, P.init_particles(y.cfg), y.pulse)
        bt.set_budget(sx, hot.ncell * hot.ppc_e + 5)
        bt.set_budget(sy, serve.footprint(y.cfg, y.pulse)[0])
        bt.step(y.nsteps)
        assert bt.slot(sx)[0] == pkg.SLOT_FAILED and bt.failed() == [sx]
        assert bt.slot(sx)[1] < y.nsteps                      # stopped at the failing step
        with pytest.raises(pkg.PicError, match="STATE"):
            bt.diagnostics(sx)
        dy, fy = bt.diagnostics(sy), (bt.electrons(sy), bt.ions(sy))
        bt.retire(sx)
        bt.step(1)                                            # drops the failed slab's particles
        bt.retire(sy)
        sz = bt.admit(z.cfg, P.init_particles(z.cfg), z.pulse)
        bt.set_budget(sz, serve.footprint(z.cfg, z.pulse)[0])
        bt.step(z.nsteps)
        dz, fz = bt.diagnostics(sz), (bt.electrons(sz), bt.ions(sz))
    finally:
        bt.close()
    ref = serve.serve_one_at_a_time([y, z], tab, lambda r: P.init_particles(r.cfg), keep=lambda rid: True)
    _equal_runs(dy, ref["results"][y.rid], fy, ref["finals"][y.rid], y.rid)
    _equal_runs(dz, ref["results"][z.rid], fz, ref["finals"][z.rid], z.rid)


def test_scarce_photon_request_outgrows_its_footprint_and_completes():
    """A thin slab of one ion per cell under a photon flux just below one
    ion weight per cell and bin: nearly every absorption is partial (a
    fractional-weight electron, the ion's charge advanced by the fraction),
    so its electrons outgrow the footprint reservation.  Served with a
    capacity sized by the footprints, it is stopped by its budget,
    preempted and re-run with a larger reservation until it completes; the
    request beside it is not disturbed, and both results equal their runs
    alone."""
    pkg.build()
    tab = P.standin_tables()
    tab["sigma_photo"] = tab["sigma_photo"] * 200.0
    a_cfg = P.cfg_small_1d(nx=8, ppc_e=2, ppc_i=1, rad_every=1, seed=41,
                           flags=P.F_PHOTO | P.F_PUSH | P.F_FIELD | P.F_DECAY)
    a = P.Request(rid=0, t_arrive=0.0, cfg=a_cfg, nsteps=600,
                  pulse=P.Pulse(I_peak_Wcm2=1e17, fwhm_fs=200.0, t_peak_fs=3.0, hv_eV=1700.0))
    b_cfg = P.cfg_small_1d(nx=48, ppc_e=32, ppc_i=8, seed=42, flags=P.F_ALL)
    b = P.Request(rid=1, t_arrive=0.0, cfg=b_cfg, nsteps=300,
                  pulse=P.Pulse(I_peak_Wcm2=1e16, fwhm_fs=20.0, t_peak_fs=3.0, hv_eV=1650.0))
    tr = [a, b]
    fp = [serve.footprint(r.cfg, r.pulse) for r in tr]
    cap_e, cap_i = fp[0][0] + fp[1][0], fp[0][1] + fp[1][1]
    init = lambda r: P.init_particles(r.cfg)  # noqa: E731
    out = serve.serve_batched(tr, tab, init, max_slabs=2, slot_cells=48, cap_e=cap_e, cap_i=cap_i,
                              tick_steps=25, keep=lambda rid: True)
    ref = serve.serve_one_at_a_time(tr, tab, init, keep=lambda rid: True)
    assert not out["failed"] and sorted(out["results"]) == [0, 1]
    assert out["preempted"] >= 1
    # it did outgrow the footprint the batch reserved at first
    assert ref["results"][0]["n_e"] > fp[0][0]
    assert ref["results"][0]["counts"]["PART"] > 0
    for r in tr:
        _equal_runs(out["results"][r.rid], ref["results"][r.rid], out["finals"][r.rid], ref["finals"][r.rid],
                    r.rid)
