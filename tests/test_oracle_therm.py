"""Pins of the oracle's forced-thermalization variant (Sec. VI C): on a rad
step the cell's free electrons are redrawn from a Maxwellian at
kT = (2/3) E_ave with the cell's total momentum and kinetic energy kept
exactly."""
import math

import numpy as np
from scipy import stats

import oracle
import pic_inputs as P

MC2 = 510998.95


def _kin(u):
    u2 = (u * u).sum(axis=1)
    return MC2 * u2 / (np.sqrt(1.0 + u2) + 1.0)


def _one_cell(ppc_e=6000, beam=0.25, seed=3, drift=0.0):
    cfg = P.cfg_small_1d(nx=2, ppc_e=ppc_e, ppc_i=ppc_e // 4, beam_frac=beam, seed=seed, rad_every=1,
                         flags=P.F_THERM)
    st = P.init_particles(cfg)
    st.eu[:, 0] += drift
    return cfg, st


def _run(cfg, st, tables, n=1):
    o = oracle.OracleSlab(cfg, tables)
    o.load(st)
    o.step(n)
    return o.electrons()


def test_thermalization_conserves_momentum_and_energy(tables):
    """A beam-heated, drifting electron population: the cell's weighted
    momentum and kinetic energy after the redraw equal those before (the
    step has no other process)."""
    cfg, st = _one_cell(drift=0.01)
    e = _run(cfg, st, tables)
    cell0 = np.floor(st.eX).astype(int)
    cell1 = np.floor(e["X"]).astype(int)
    for c in range(cfg.nx):
        m0, m1 = cell0 == c, cell1 == c
        p0 = (st.ew[m0, None] * st.eu[m0]).sum(axis=0)
        p1 = (e["w"][m1, None] * e["u"][m1]).sum(axis=0)
        assert np.allclose(p1, p0, rtol=1e-12, atol=1e-13 * np.abs(p0).max())
        k0 = (st.ew[m0] * _kin(st.eu[m0])).sum()
        k1 = (e["w"][m1] * _kin(e["u"][m1])).sum()
        assert abs(k1 / k0 - 1) < 1e-12
        assert not np.allclose(e["u"][m1][:10], st.eu[m0][:10])


def test_thermalized_distribution_is_maxwellian(tables):
    """Momentum components relative to the mean are normal with variance
    kT / m c^2, kT = (2/3) E_ave of the cell before the redraw (the beam
    holds a large share of the energy, so the redraw changes the shape)."""
    cfg, st = _one_cell(ppc_e=20000, beam=0.1)
    e = _run(cfg, st, tables)
    c0 = np.floor(st.eX).astype(int) == 0
    c1 = np.floor(e["X"]).astype(int) == 0
    T = (2.0 / 3.0) * (st.ew[c0] * _kin(st.eu[c0])).sum() / st.ew[c0].sum()
    u = e["u"][c1]
    d = (u - u.mean(axis=0)) / math.sqrt(T / MC2)
    for comp in range(3):
        assert stats.kstest(d[:, comp], "norm").pvalue > 1e-3
    # before: far from Maxwellian (the hot beam)
    u0 = st.eu[c0]
    d0 = (u0 - u0.mean(axis=0)) / math.sqrt(T / MC2)
    assert stats.kstest(d0[:, 0], "norm").pvalue < 1e-6


def test_thermalization_independent_of_order(tables):
    """Draws are keyed by electron id: loading the electrons in another
    order gives the same momenta per id."""
    cfg, st = _one_cell(ppc_e=500)
    a = _run(cfg, st, tables)
    perm = np.random.default_rng(1).permutation(st.n_e)
    st2 = P.ParticleState(eX=st.eX[perm], eY=st.eY[perm], eu=st.eu[perm], ew=st.ew[perm], eid=st.eid[perm],
                          iX=st.iX, iY=st.iY, iu=st.iu, izf=st.izf, iZ=st.iZ, inK=st.inK, iid=st.iid)
    b = _run(cfg, st2, tables)
    oa, ob = np.argsort(a["id"]), np.argsort(b["id"])
    assert np.allclose(a["u"][oa], b["u"][ob], rtol=1e-12, atol=1e-15)


def test_thermalization_only_on_rad_steps(tables):
    cfg, st = _one_cell(ppc_e=500)
    cfg.rad_every = 2
    o = oracle.OracleSlab(cfg, tables)
    o.load(st)
    o.step(2)           # step 0 is a rad step, step 1 is not
    e2 = o.electrons()
    e1 = _run(cfg, st, tables, 1)
    oa, ob = np.argsort(e1["id"]), np.argsort(e2["id"])
    assert np.array_equal(e1["u"][oa], e2["u"][ob])
