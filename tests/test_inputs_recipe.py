"""The seeded synthetic inputs are what the design states they are (no GPU):
the initial solid-Al state (per-cell counts, positions inside their cells,
neutral weights, the Maxwellian and the 1.5 keV beam share, every value
exact in FP32), the batched ensemble (cells and particles per cell
log-uniform, electrons : ions = 4 : 1, peak intensity log-uniform, photon
energy uniform) and the served trace (Poisson arrivals at 200/s, foil
thickness uniform in 0.2-2 um, cells at least 1 nm wide, 150 fs horizon)."""
import math

import numpy as np

import pic_inputs as P


def _exact_f32(a):
    a = np.asarray(a, dtype=np.float64)
    return np.array_equal(a, a.astype(np.float32).astype(np.float64))


def test_initial_state():
    cfg = P.cfg_foil_2d(nx=64, ny=16)
    st = P.init_particles(cfg)
    assert st.n_e == cfg.ncell * cfg.ppc_e and st.n_i == cfg.ncell * cfg.ppc_i
    for X, Y, per in ((st.eX, st.eY, cfg.ppc_e), (st.iX, st.iY, cfg.ppc_i)):
        assert X.min() >= 0 and X.max() < cfg.nx and Y.min() >= 0 and Y.max() < cfg.ny
        cell = np.floor(Y).astype(np.int64) * cfg.nx + np.floor(X).astype(np.int64)
        assert np.all(np.bincount(cell, minlength=cfg.ncell) == per)
        assert _exact_f32(X - np.floor(X)) and _exact_f32(Y - np.floor(Y))
    assert _exact_f32(st.eu) and _exact_f32(st.iu) and _exact_f32(st.ew)
    # neutral: electron weight = ion charge, slab-wide and per cell
    q = (st.iZ + st.izf).astype(np.float64) * cfg.w_ion
    assert abs(st.ew.sum() - q.sum()) <= 1e-6 * q.sum()
    assert np.all(st.iZ == cfg.Z_init) and np.all(st.inK == 0)
    assert len(np.unique(st.eid)) == st.n_e and len(np.unique(st.iid)) == st.n_i
    # beam share at 1.5 keV, the rest a 10 eV Maxwellian
    u2 = (st.eu ** 2).sum(axis=1)
    ke = 510998.95 * u2 / (np.sqrt(1 + u2) + 1)
    beam = np.abs(ke - cfg.beam_E_eV) < 1e-3 * cfg.beam_E_eV
    share = beam.mean()
    assert abs(share - cfg.beam_frac) < 4 * math.sqrt(cfg.beam_frac * (1 - cfg.beam_frac) / st.n_e)
    assert abs(ke[~beam].mean() / (1.5 * cfg.T_e_eV) - 1) < 0.02     # <KE> = 3/2 T
    ke_i = 0.5 * cfg.m_ion_me * 510998.95 * (st.iu ** 2).sum(axis=1)
    assert abs(ke_i.mean() / (1.5 * cfg.T_i_eV) - 1) < 0.05


def test_batched_ensemble():
    ens = P.batched_ensemble(256)
    nx = np.array([c.nx for c, _ in ens])
    ppc = np.array([c.ppc_e + c.ppc_i for c, _ in ens])
    ratio = np.array([c.ppc_e / c.ppc_i for c, _ in ens])
    I = np.array([p.I_peak_Wcm2 for _, p in ens])
    hv = np.array([p.hv_eV for _, p in ens])
    assert nx.min() >= 64 and nx.max() <= 4096 and ppc.min() >= 32 and ppc.max() <= 512
    assert np.all((ratio > 3.3) & (ratio < 4.8))
    assert I.min() >= 1e15 and I.max() <= 1e18 and hv.min() >= 1580 and hv.max() <= 1900
    # log-uniform: the logs' mean in the middle of the range (sd of the mean ~ width / sqrt(12 n))
    n = len(ens)
    for v, lo, hi in ((nx, 64, 4096), (ppc, 32, 512), (I, 1e15, 1e18)):
        mid, sd = 0.5 * (math.log(lo) + math.log(hi)), (math.log(hi) - math.log(lo)) / math.sqrt(12 * n)
        assert abs(np.log(v).mean() - mid) < 4 * sd
    assert abs(hv.mean() - 1740.0) < 4 * 320.0 / math.sqrt(12 * n)
    assert len({c.seed for c, _ in ens}) == n
    assert all(c.flags == P.F_ALL and c.ny == 1 and c.dx_nm == 2.0 for c, _ in ens)


def test_served_trace():
    tr = P.request_trace(2000)
    t = np.array([r.t_arrive for r in tr])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() / (1 / 200.0) - 1) < 4 / math.sqrt(len(tr))     # Poisson at 200/s
    assert abs(np.std(gaps) / np.mean(gaps) - 1) < 0.1                      # exponential gaps
    thick = np.array([r.cfg.nx * r.cfg.dx_nm for r in tr])
    assert thick.min() >= 200 - 1e-6 and thick.max() <= 2000 + 1e-6
    assert all(r.cfg.dx_nm >= 1.0 - 1e-12 or r.cfg.nx == 2 for r in tr)
    assert all(r.nsteps == 7500 for r in tr)                                  # 150 fs at 0.02 fs
    assert sorted(r.rid for r in tr) == list(range(len(tr)))
