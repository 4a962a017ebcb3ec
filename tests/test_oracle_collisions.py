"""Pins of the oracle's binary collisions, push and relaxation physics.

Sec. IV of the paper takes its binary e-e / e-i Monte-Carlo collisions from
its references; the oracle reads them as Takizuka-Abe pairing and angle
with a relativistic centre-of-momentum rotation.  Pinned here by:
exact per-collision conservation, Spitzer/NRL e-i temperature relaxation,
Maxwellian stationarity under e-e collisions, the Boris rotation angle and
the E x B drift.
"""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.integrate import solve_ivp

import oracle
import pic_inputs as P

MC2 = 510998.95


def _energy(u, m):
    """kinetic energy in m_e c^2, as m u^2 / (gamma + 1)"""
    u2 = float(np.dot(u, u))
    return m * u2 / (math.sqrt(1.0 + u2) + 1.0)


@pytest.mark.parametrize("ma,mb,qb", [(1.0, 1.0, -1.0), (1.0, P.M_AL_ME, 3.0), (1.0, 100.0, 7.5)])
def test_collision_conserves_momentum_energy(ma, mb, qb):
    rng = np.random.default_rng(3)
    worst_p = worst_e = 0.0
    for _ in range(300):
        ua = rng.standard_normal(3) * 0.05
        ub = rng.standard_normal(3) * 0.05 * math.sqrt(ma / mb)
        r = rng.random(4)
        a, b, did = oracle.collide(ua, ub, ma, mb, -1.0, qb, 1.0, 1.0, 1e23, 3.0, 0.05, r)
        assert did
        p0 = ma * ua + mb * ub
        p1 = ma * a + mb * b
        e0 = _energy(ua, ma) + _energy(ub, mb)
        e1 = _energy(a, ma) + _energy(b, mb)
        scale = np.linalg.norm(ma * ua) + np.linalg.norm(mb * ub)
        worst_p = max(worst_p, np.linalg.norm(p1 - p0) / scale)
        worst_e = max(worst_e, abs(e1 - e0) / e0)
    assert worst_p < 1e-12
    assert worst_e < 1e-12


def test_collision_frame_near_the_pole():
    """Centre-of-momentum directions within a few degrees of the z axis
    (the azimuth frame then switches to the x axis): momentum and energy
    conserved to 1e-12 and the scattering angle between the old and new
    relative momentum is 2 atan(delta) on both sides of the switch."""
    rng = np.random.default_rng(8)
    for k in range(200):
        th = rng.uniform(0.0, 0.4) if k % 2 else rng.uniform(0.45, 0.6)   # |n_xy| below / above 1/2
        ph = rng.uniform(0, 2 * math.pi)
        d = 0.02 * np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        ua, ub = d, -d                                     # equal masses: COM at rest, n along d
        r = rng.random(4)
        a, b, did = oracle.collide(ua, ub, 1.0, 1.0, -1.0, -1.0, 1.0, 1.0, 1e23, 3.0, 0.05, r)
        assert did
        assert np.linalg.norm(a + b) < 1e-15
        assert abs(np.linalg.norm(a) - np.linalg.norm(ua)) < 1e-15
        cos_t = float(np.dot(a, ua) / np.dot(ua, ua))
        var = 2 * math.pi * 2.8179403262e-13 ** 2 * 2.99792458e-5 * 1e23 * 3.0 * 0.05 / \
            (0.25 * (2 * 0.02 / math.sqrt(1 + 0.02 ** 2)) ** 3)
        delta = math.sqrt(var) * math.sqrt(-2 * math.log(r[0])) * math.cos(2 * math.pi * r[1])
        assert abs(cos_t - (1 - delta * delta) / (1 + delta * delta)) < 1e-12


def test_collision_weighted_acceptance():
    """Unequal weights: the lighter particle always moves, the heavier one
    with probability w_light / w_heavy (Nanbu-Yonemura)."""
    rng = np.random.default_rng(5)
    moved_heavy = 0
    n = 4000
    for _ in range(n):
        ua = rng.standard_normal(3) * 0.01
        ub = rng.standard_normal(3) * 0.01
        r = rng.random(4)
        a, b, _ = oracle.collide(ua, ub, 1.0, 1.0, -1.0, -1.0, 1.0, 4.0, 1e23, 3.0, 0.05, r)
        assert not np.allclose(a, ua)
        moved_heavy += not np.allclose(b, ub)
    p = moved_heavy / n
    assert abs(p - 0.25) < 4 * math.sqrt(0.25 * 0.75 / n)


def test_spitzer_nrl_relaxation():
    """e-i temperature relaxation against the Spitzer rate (NRL formulary
    form with its exact coefficient 8 sqrt(2 pi) e^4 / 3), within 3 %.
    Ions of mass 100 m_e make the exchange measurable in a short run;
    dt is small enough for the small-angle limit."""
    mi = 100.0
    cfg = P.cfg_small_1d(flags=P.F_COLL_EI | P.F_COLL_EE, nx=192, ppc_e=128, ppc_i=128, Z_init=1,
                         T_e_eV=200.0, T_i_eV=20.0, beam_frac=0.0, m_ion_me=mi, coulomb_log=5.0,
                         n_ref_cm3=5.4e22, dt_fs=0.002)
    st = P.init_particles(cfg)
    o = oracle.OracleSlab(cfg, P.standin_tables())
    o.load(st)

    def temps():
        e, i = o.electrons(), o.ions()
        ke = lambda u, m: m * MC2 * ((u ** 2).sum(1) / (np.sqrt(1 + (u ** 2).sum(1)) + 1))
        return (2 / 3) * np.average(ke(e["u"], 1.0), weights=e["w"]), (2 / 3) * ke(i["u"], mi).mean()

    T0 = temps()
    T_phys = 1.0
    o.step(int(round(T_phys / cfg.dt_fs)))
    T1 = temps()
    e_esu, erg, me_g = 4.80320471e-10, 1.602176634e-12, 9.1093837015e-28
    coef = 8 * math.sqrt(2 * math.pi) * e_esu ** 4 / 3 / erg ** 1.5
    ni = cfg.n_ref_cm3
    ne = ni * cfg.Z_init

    def rhs(t, y):
        Te, Ti = y
        nu = coef * math.sqrt(me_g * mi * me_g) * cfg.Z_init ** 2 * ni * 5.0 \
            / (me_g * Ti + mi * me_g * Te) ** 1.5 * 1e-15
        return [-nu * (Te - Ti), nu * (ne / ni) * (Te - Ti)]

    sol = solve_ivp(rhs, (0, T_phys), T0, rtol=1e-10)
    th = sol.y[1, -1] - T0[1]
    got = T1[1] - T0[1]
    assert abs(got / th - 1.0) < 0.03


def test_maxwellian_stationary_under_ee():
    """e-e collisions keep a Maxwellian a Maxwellian (KS on each momentum
    component) and conserve energy exactly (equal weights)."""
    cfg = P.cfg_small_1d(flags=P.F_COLL_EE, nx=64, ppc_e=256, ppc_i=64, T_e_eV=50.0,
                         beam_frac=0.0, dt_fs=0.02)
    st = P.init_particles(cfg)
    o = oracle.OracleSlab(cfg, P.standin_tables())
    o.load(st)
    t0, _ = o.tallies()
    o.step(100)
    t1, c = o.tallies()
    assert c["EE"] > 0
    assert abs(t1["KE_E"] - t0["KE_E"]) / t0["KE_E"] < 1e-12
    u = o.electrons()["u"]
    s = math.sqrt(50.0 / MC2)
    for k in range(3):
        assert stats.kstest(u[:, k] / s, "norm").pvalue > 1e-3


def test_two_temperature_relaxes_to_maxwellian():
    """An anisotropic electron population (T_x != T_y = T_z) isotropizes
    under e-e collisions while the energy stays fixed."""
    cfg = P.cfg_small_1d(flags=P.F_COLL_EE, nx=32, ppc_e=256, T_e_eV=50.0, beam_frac=0.0)
    st = P.init_particles(cfg)
    st.eu[:, 0] *= 2.0
    o = oracle.OracleSlab(cfg, P.standin_tables())
    o.load(st)
    o.step(400)
    u = o.electrons()["u"]
    tx, ty, tz = (u ** 2).mean(0)
    assert abs(tx / ty - 1) < 0.05 and abs(tx / tz - 1) < 0.05


def test_boris_gyration_closed_form():
    """Uniform B, no E: |u| is conserved to rounding and the momentum turns
    by 2 atan(Omega dt / (2 gamma)) per step."""
    u0 = np.array([0.03, 0.0, 0.01])
    b = np.array([0.0, 0.0, 0.7])
    qm, dt = -1.0, 0.01
    g = math.sqrt(1 + u0 @ u0)
    u = u0.copy()
    n = 500
    for _ in range(n):
        u = oracle.boris(u, [0, 0, 0], b, qm, dt)
    assert abs(np.linalg.norm(u) - np.linalg.norm(u0)) < 1e-14
    theta = 2 * math.atan(abs(qm) * 0.7 * dt / (2 * g))
    ang = n * theta
    # electrons (q<0) gyrate counter-clockwise about +z
    exp = np.array([u0[0] * math.cos(ang) - u0[1] * math.sin(ang),
                    u0[0] * math.sin(ang) + u0[1] * math.cos(ang), u0[2]])
    assert np.allclose(u, exp, atol=1e-12)


def test_boris_exb_drift():
    """Crossed E and B: the gyro-averaged velocity is E x B / B^2."""
    e = np.array([0.0, 1e-4, 0.0])
    b = np.array([0.0, 0.0, 0.5])
    u = np.zeros(3)
    qm, dt = -1.0, 0.005
    period = 2 * math.pi / (0.5)
    n = int(round(20 * period / dt))
    vs = []
    for _ in range(n):
        u = oracle.boris(u, e, b, qm, dt)
        vs.append(u / math.sqrt(1 + u @ u))
    v = np.mean(vs, axis=0)
    drift = np.cross(e, b) / (b @ b)
    assert abs(v[0] / drift[0] - 1) < 2e-3
    assert abs(v[1]) < 1e-3 * abs(drift[0])
