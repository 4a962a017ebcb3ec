"""Pins of the oracle's radiation transport (Sec. II, Eqs. 1a and 1b; CPU
only): the CIP advection is exact for integer Courant numbers and for cubic
profiles at any Courant number (its Hermite interpolant reproduces cubics),
the linear split conserves content exactly, the ordinate quadrature
integrates the low moments of an isotropic field exactly, a collimated beam
through a frozen absorber follows the Beer-Lambert law, the single-ordinate,
full-resolution, linear-split transport is the ballistic march, K-alpha
emission enters the diffuse ordinates in proportion to their solid angle,
and a whole step with every atomic process conserves energy to 1e-12 with
the transport tallies (absorbed beyond the Monte-Carlo events: to the bulk
electrons; the scheme's own numerical gain: tallied)."""
import math

import numpy as np
import pytest

import oracle
import pic_inputs as P

C_NM_FS = 299.792458


def test_cip_exact_shift_at_integer_courant():
    rng = np.random.default_rng(1)
    n = 40
    f, g = rng.random(n), rng.standard_normal(n)
    for nu in (1, 2, 3, -1, -2):
        f1, g1, _, _, _ = oracle.rt_line(f, g, float(nu))
        inner = range(4, n - 4)
        assert all(f1[i] == f[i - nu] and g1[i] == g[i - nu] for i in inner), nu


@pytest.mark.parametrize("nu", [0.37, -0.81, 1.63, -2.25])
def test_cip_exact_for_cubic_profiles(nu):
    """f = a + b x + c x^2 + d x^3 with g = f' at the nodes: the advected
    values are the cubic at the departure points, f(x_i - nu), f'(x_i - nu)."""
    a, b, c, d = 0.3, -0.02, 0.004, -1e-4
    x = np.arange(30, dtype=np.float64)
    f = a + b * x + c * x ** 2 + d * x ** 3
    g = b + 2 * c * x + 3 * d * x ** 2
    f1, g1, _, _, _ = oracle.rt_line(f, g, nu)
    xd = x - nu
    for i in range(5, 25):
        assert abs(f1[i] - (a + b * xd[i] + c * xd[i] ** 2 + d * xd[i] ** 3)) < 1e-13
        assert abs(g1[i] - (b + 2 * c * xd[i] + 3 * d * xd[i] ** 2)) < 1e-13


def test_linear_split_conserves_content():
    rng = np.random.default_rng(2)
    n = 50
    f = rng.random(n)
    fin = rng.random(8)
    for nu in (0.3, 1.7, 3.2, -0.6, -2.4):
        f1, _, _, i, o = oracle.rt_line(f, np.zeros(n), nu, scheme=1, fin=fin, gin=np.zeros(8))
        assert abs(f1.sum() - (f.sum() + i - o)) < 1e-12 * f.sum(), nu
    f1, _, _, i, o = oracle.rt_line(f, np.zeros(n), 2.7, scheme=1, periodic=True)
    assert abs(f1.sum() - f.sum()) < 1e-12 and i == 0.0 and o == 0.0


def _rt_slab(ny=1, n_polar=4, n_az=3):
    cfg = P.cfg_small_1d(nx=40, ny=ny, dx_nm=2.0, dy_nm=2.0, ppc_e=4, ppc_i=4, flags=P.F_PHOTO)
    o = oracle.OracleSlab(cfg, P.standin_tables(), P.Pulse(I_peak_Wcm2=0.0, n_bins=2))
    o.set_rt(coarsen=4, n_polar=n_polar, n_azimuth=n_az)
    return o


@pytest.mark.parametrize("ny", [1, 8])
def test_ordinate_quadrature(ny):
    """Diffuse ordinates: weights sum to 1 and the isotropic moments of the
    in-plane direction cosines are exact: <mu> = 0, <mu^2> = 1/3, and in
    2D <n_y> = 0, <n_y^2> = 1/3; the beam ordinate is +x with no share."""
    o = _rt_slab(ny=ny)
    mu, vy, w = o.ordinates
    assert mu[0] == 1.0 and vy[0] == 0.0 and w[0] == 0.0
    assert abs(w.sum() - 1.0) < 1e-14
    assert abs((w * mu).sum()) < 1e-14 and abs((w * mu ** 2).sum() - 1.0 / 3.0) < 1e-14
    if ny > 1:
        assert abs((w * vy).sum()) < 1e-14 and abs((w * vy ** 2).sum() - 1.0 / 3.0) < 1e-14


def test_single_beam_linear_transport_is_the_march(tables):
    """The beam ordinate alone, rad cells the size of PIC cells, the linear
    split, nothing absorbing: the photon numbers of every cell after 30 rad
    steps are those of the ballistic march, bit for bit, and the incident
    and transmitted energies agree."""
    tab = dict(tables)
    tab["sigma_photo"] = tables["sigma_photo"] * 0.0
    cfg = P.cfg_small_1d(nx=48, ppc_e=4, ppc_i=4, flags=P.F_PHOTO, beam_frac=0.0)
    pl = P.Pulse(I_peak_Wcm2=1e17, fwhm_fs=3.0, t_peak_fs=4.0, hv_eV=1600.0, n_bins=2)
    st = P.init_particles(cfg)
    a, b = oracle.OracleSlab(cfg, tab, pl), oracle.OracleSlab(cfg, tab, pl)
    a.load(st)
    b.load(st)
    b.set_rt(coarsen=1, n_polar=0, scheme=1)
    a.step(150)
    b.step(150)
    assert np.array_equal(a.photons(), b.photons())
    ta, tb = a.tallies()[0], b.tallies()[0]
    assert ta["INC"] > 0 and ta["TRANS"] > 0
    for k in ("INC", "TRANS", "PHOT"):
        assert abs(ta[k] - tb[k]) <= 1e-12 * ta["INC"], k
    assert abs(tb["RT_NUM"]) <= 1e-12 * ta["INC"] and tb["BACK"] == 0.0


def test_beer_lambert_through_a_frozen_absorber(tables):
    """A flat-top beam through Al3+ with rad cells exactly c dt_rad wide
    (Courant number 1: the CIP transport is an exact shift) and a pulse too
    weak to change the ions noticeably: the transmitted fraction is
    exp(-mu L), mu = n_i sum_s N_s sigma_s (the same cross sections as
    photoionization, Eq. 2), within 0.2 %."""
    R = 5
    dx = C_NM_FS * 5 * 0.02 / R
    nx = 60
    cfg = P.cfg_small_1d(nx=nx, dx_nm=dx, dy_nm=dx, ppc_e=2, ppc_i=64, flags=P.F_PHOTO, beam_frac=0.0,
                         ipd_model=P.IPD_NONE, rad_every=5)
    hv = 1700.0
    tab = dict(tables)
    tab["sigma_photo"] = tables["sigma_photo"] * 3.0
    w = cfg.w_ion
    n_ph = 0.02 * w
    I = n_ph * cfg.n_ref_cm3 * 2.99792458e10 * hv * 1.602176634e-19
    pl = P.Pulse(shape=1, I_peak_Wcm2=I, fwhm_fs=200.0, t_peak_fs=100.0, hv_eV=hv, bandwidth_eV=0.0, n_bins=1)
    o = oracle.OracleSlab(cfg, tab, pl)
    o.load(P.init_particles(cfg))
    o.set_rt(coarsen=R, n_polar=0, scheme=0)
    L = nx * dx
    o.step(int(math.ceil(L / C_NM_FS / 0.1) + 3) * 5)
    t0, _ = o.tallies()
    o.step(40 * 5)
    t1, _ = o.tallies()
    trans = (t1["TRANS"] - t0["TRANS"]) / (t1["INC"] - t0["INC"])
    occ = oracle.occ(10, 0)
    hv_tab, sig = tab["hv_tab"], tab["sigma_photo"]
    mu = sum(cfg.n_ref_cm3 * occ[s] * math.exp(np.interp(math.log(hv), np.log(hv_tab), np.log(sig[s])))
             for s in range(5) if occ[s] and hv > tab["E_bind"][3, s])
    expect = math.exp(-mu * L * 1e-7)
    assert 0.2 < expect < 0.8
    assert abs(trans / expect - 1) < 2e-3, (trans, expect)


@pytest.mark.parametrize("ny", [1, 8])
def test_kalpha_emission_is_isotropic_over_the_diffuse_ordinates(tables, ny):
    """Photons that the cells add to their bins between two transport steps
    (K-alpha photons of the decays) enter the diffuse ordinates of their rad
    cell in proportion to each ordinate's solid angle at the next transport
    step, energy exact (a time step short enough that the transport moves
    them by 1e-4 of a rad cell)."""
    cfg = P.cfg_small_1d(nx=40, ny=ny, dx_nm=2.0, dy_nm=2.0, dt_fs=1e-6, ppc_e=2, ppc_i=2, flags=0,
                         beam_frac=0.0, rad_every=1)
    pl = P.Pulse(I_peak_Wcm2=0.0, n_bins=2, hv_eV=1500.0, bandwidth_eV=40.0)
    o = oracle.OracleSlab(cfg, tables, pl)
    o.load(P.init_particles(cfg))
    o.set_rt(coarsen=4, n_polar=3, n_azimuth=2, scheme=0)
    o.step(1)
    X = np.random.default_rng(3).random((cfg.ny, cfg.nx, 2)) * 1e-3
    o.set_photons(X)
    hv = np.array([1490.0, 1510.0])
    e_in = float((X * hv).sum())
    assert abs(o.tallies()[0]["PHOT"] - e_in) < 1e-12 * e_in
    o.step(1)
    F, _, _ = o.rt_field()
    t, _ = o.tallies()
    mu, vy, w = o.ordinates
    per_ord = F.sum(axis=(1, 2, 3))
    assert per_ord[0] == 0.0
    share = per_ord[1:] / per_ord[1:].sum()
    assert np.allclose(share, w[1:], rtol=1e-4, atol=0)
    lost = t["TRANS"] + t["BACK"] - t["RT_NUM"]
    assert abs(t["PHOT"] + lost - e_in) < 1e-12 * e_in
    assert abs(lost) < 1e-3 * e_in


def test_rt_step_conserves_energy(tables):
    """Collisions, impact ionization, recombination, photoionization and
    K decay with the transport on (no push: the field solver's own energy is
    not the subject here), a 2D slab under a pulse: kinetic + ionization +
    photon (field and pending K-alpha) + escaped K-alpha + transmitted +
    back-escaped - incident - transport gain + energy on its way to the
    electrons stays constant to 1e-12 relative, step by step."""
    cfg = P.cfg_small_1d(nx=20, ny=10, dx_nm=4.0, dy_nm=4.0, ppc_e=32, ppc_i=8, T_e_eV=30.0,
                         flags=P.F_COLL_EE | P.F_COLL_EI | P.F_IONIZE | P.F_RECOMB | P.F_PHOTO | P.F_DECAY,
                         rad_every=1)
    tab = dict(tables)
    tab["sigma_photo"] = tables["sigma_photo"] * 30.0
    pl = P.Pulse(I_peak_Wcm2=5e17, fwhm_fs=5.0, t_peak_fs=0.5, hv_eV=1700.0, n_bins=3, bandwidth_eV=300.0)
    st = P.perturb_ions(P.init_particles(cfg), 3, frac_hollow=0.3, z_spread=2, zfrac_share=0.1)
    st = P.neutralize(st, cfg)
    o = oracle.OracleSlab(cfg, tab, pl)
    o.load(st)
    o.set_rt(coarsen=5, n_polar=3, n_azimuth=2, scheme=0)

    def total(t):
        return (t["KE_E"] + t["KE_I"] + t["ION"] + t["PHOT"] + t["KA_ESC"] + t["TRANS"] + t["BACK"] - t["INC"]
                - t["RT_NUM"] + t["RT_PEND"])

    t0, _ = o.tallies()
    e0 = total(t0)
    seen = {"A": False, "pend": False}
    for k in range(12):
        o.step(1)
        t, c = o.tallies()
        scale = max(abs(e0), t["INC"])
        assert abs(total(t) - e0) < 1e-12 * scale, (k, total(t) - e0, scale)
        seen["pend"] |= t["RT_PEND"] != 0.0
    assert t["INC"] > 0 and c["PH0"] > 0 and c["KA"] + c["AUG"] > 0 and seen["pend"]
    cells = o.rt_cells()
    assert cells["chi"].max() > 0 and cells["w"].min() > 0
