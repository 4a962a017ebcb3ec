"""The oracle's decision trace and the flip classifier of the parity tests
(CPU only): the trace changes nothing in the step, counts every decision
and records exactly those within the relative distance asked for; the
classifier finds no difference between two identical runs and reports a
difference planted in one of them as unexplained."""
import numpy as np

import oracle
import pic_inputs as P
from parity_util import classify


def _busy(cfg, seed=5):
    st = P.init_particles(cfg)
    st = P.perturb_ions(st, seed, frac_hollow=0.4, z_spread=3, zfrac_share=0.25)
    return P.neutralize(st, cfg)


def _setup(tables):
    cfg = P.cfg_small_1d(nx=24, ppc_e=64, ppc_i=16, T_e_eV=25.0, flags=P.F_ALL & ~P.F_PUSH & ~P.F_FIELD,
                         rad_every=1)
    pl = P.Pulse(I_peak_Wcm2=3e17, fwhm_fs=30.0, t_peak_fs=0.0, hv_eV=1700.0, n_bins=3, bandwidth_eV=400.0)
    tab = dict(tables)
    tab["sigma_photo"] = tables["sigma_photo"] * 50.0
    st = _busy(cfg)
    ph = P.photons_uniform(cfg, pl, 1.0)
    ph[:, cfg.nx // 2:, :] = 0.3 * cfg.w_ion
    return cfg, pl, tab, st, ph


def _run(cfg, tab, pl, st, ph, rel):
    o = oracle.OracleSlab(cfg, tab, pl)
    o.load(st)
    o.set_photons(ph)
    if rel is not None:
        o.trace(rel)
    o.step(1)
    return o


def test_trace_changes_nothing_and_counts_every_decision(tables):
    cfg, pl, tab, st, ph = _setup(tables)
    a = _run(cfg, tab, pl, st, ph, None)
    b = _run(cfg, tab, pl, st, ph, oracle.FLIP_REL)
    ea, eb = a.electrons(), b.electrons()
    assert np.array_equal(ea["id"], eb["id"]) and np.array_equal(ea["u"], eb["u"])
    assert np.array_equal(a.ions()["Z"], b.ions()["Z"])
    near, n_draw, n_dec = b.near()
    assert n_draw > 1000 and n_dec > 1000
    d = np.abs(near["x"] - near["thr"])
    assert (d <= oracle.FLIP_REL * np.abs(near["thr"])).all()
    # an unbounded relative distance: every decision with a nonzero threshold is recorded
    c = _run(cfg, tab, pl, st, ph, 1e30)
    near1, n_draw1, n_dec1 = c.near()
    assert (n_draw1, n_dec1) == (n_draw, n_dec)
    assert len(near1) > 0.9 * (n_draw + n_dec)
    assert set(np.unique(near1["kind"])) >= {2, 4, 6, 7, 8, 11, 12}


def test_classifier_clean_on_identical_runs_and_flags_a_planted_difference(tables):
    cfg, pl, tab, st, ph = _setup(tables)
    a = _run(cfg, tab, pl, st, ph, oracle.FLIP_REL)
    b = _run(cfg, tab, pl, st, ph, None)
    near, n_draw, n_dec = a.near()
    cls = classify(cfg, st, b.electrons(), a.electrons(), b.ions(), a.ions(), near, n_draw, n_dec)
    assert cls["unexplained"] == [] and cls["flips"] == 0
    # plant: one electron's momentum, one ion's charge, one electron dropped
    e, i = b.electrons(), b.ions()
    e["u"][3] *= 1.001
    i["Z"][5] += 1
    keep = np.ones(e["id"].size, bool)
    keep[7] = False
    e = {k: v[keep] for k, v in e.items()}
    cls = classify(cfg, st, e, a.electrons(), i, a.ions(), near[:0], n_draw, n_dec)
    assert len(cls["unexplained"]) == 3, cls["unexplained"]
    # the same differences inside cells that hold a near-threshold decision
    # count as flips
    fake = np.zeros(cfg.nx, dtype=oracle.NEAR_DTYPE)
    fake["cell"] = np.arange(cfg.nx)
    cls = classify(cfg, st, e, a.electrons(), i, a.ions(), fake, n_draw, n_dec)
    assert cls["unexplained"] == [] and cls["flips"] >= 1
