"""Radiation transport mode (Sec. II, Eqs. 1a and 1b) on the device against
the oracle, through the C ABI: one rad step with every atomic process in
1D and 2D (particles by the flip classification, the rad field and what the
cells recorded for it), the first rad steps of a pulse (field and energy
bookkeeping), the ballistic march as the single-ordinate, full-resolution,
linear-split special case (to 1e-12 against the device's own march), and
the device's energy bookkeeping over many steps."""
import numpy as np
import pytest

import pic_inputs as P
from parity_util import assert_flip_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1704_01202_gb300 as pkg  # noqa: E402

RT_FLAGS = P.F_COLL_EE | P.F_COLL_EI | P.F_IONIZE | P.F_RECOMB | P.F_PHOTO | P.F_DECAY


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    oracle.build()


def _setup(tables, ny, flags=RT_FLAGS, seed=4):
    cfg = P.cfg_small_1d(nx=40, ny=ny, dx_nm=3.0, dy_nm=3.0, ppc_e=48, ppc_i=12, T_e_eV=30.0, flags=flags,
                         rad_every=1)
    tab = dict(tables)
    tab["sigma_photo"] = tables["sigma_photo"] * 40.0
    pl = P.Pulse(I_peak_Wcm2=4e17, fwhm_fs=4.0, t_peak_fs=0.3, hv_eV=1700.0, n_bins=3, bandwidth_eV=300.0)
    st = P.perturb_ions(P.init_particles(cfg), seed, frac_hollow=0.3, z_spread=2, zfrac_share=0.1)
    return cfg, tab, pl, P.neutralize(st, cfg)


def _both(cfg, tab, pl, st, rt):
    g = pkg.Slab(cfg, tab, pl)
    g.load(st)
    g.set_rt(**rt)
    o = oracle.OracleSlab(cfg, tab, pl)
    o.load(st)
    o.set_rt(**rt)
    return g, o


def _field_close(g, o, rtol=1e-5):
    Fg, Gxg, Gyg = g.rt_field()
    Fo, Gxo, Gyo = o.rt_field()
    for a, b, name in ((Fg, Fo, "F"), (Gxg, Gxo, "Gx"), (Gyg, Gyo, "Gy")):
        scale = np.abs(b).max() + 1e-300
        assert np.abs(a - b).max() <= rtol * scale, (name, np.abs(a - b).max(), scale)
    return Fo


@pytest.mark.parametrize("ny", [1, 10])
def test_rad_step_every_process(tables, ny):
    """Step 0 (a rad step): the transport publishes the pulse's inflow, the
    cells ionize with it; then a second rad step absorbs with the opacity
    the cells recorded, books the energy beyond the events for the bulk
    electrons, emits their K-alpha photons and advects: particles equal up
    to threshold flips, the field, the cells' records and the tallies to
    FP32 accuracy."""
    cfg, tab, pl, st = _setup(tables, ny)
    g, o = _both(cfg, tab, pl, st, dict(coarsen=5, n_polar=3, n_azimuth=2, scheme=0))
    o.trace()
    g.step(1)
    o.step(1)
    _, co = o.tallies()
    assert_flip_parity(cfg, st, g.electrons(), g.ions(), o, g.diagnostics()["counts"], co,
                       ("ION", "REC", "PH0", "PH1", "PH2", "PART", "AUG", "KA"))
    assert co["PH0"] > 0
    Fo = _field_close(g, o)
    assert Fo[0].max() > 0
    cg, cor = g.rt_cells(), o.rt_cells()
    assert np.abs(cg["chi"] - cor["chi"]).max() <= 1e-5 * cor["chi"].max()
    assert cor["emc"].max() > 0
    assert np.abs(cg["emc"] - cor["emc"]).max() <= 1e-5 * cor["emc"].max()
    assert np.abs(cg["w"] - cor["w"]).max() <= 1e-5 * cor["w"].max()
    # second rad step from the same state on both sides (teacher forcing of
    # the particles; the field and the cells' records as each side has them)
    e, i = g.electrons(), g.ions()
    st2 = P.ParticleState(eX=e["X"], eY=e["Y"], eu=e["u"], ew=e["w"], eid=e["id"], iX=i["X"], iY=i["Y"],
                          iu=i["u"], izf=i["zf"].astype(np.float64), iZ=i["Z"], inK=i["nK"], iid=i["id"])
    o.load(st2)
    o.trace()
    g.step(1)
    o.step(1)
    _field_close(g, o)
    cg, cor = g.rt_cells(), o.rt_cells()
    # energy still due to the cells' electrons: what the FP32 scaling left
    # of the share given at this rad step, against the events' energy scale
    assert np.abs(cg["dE"] - cor["dE"]).max() <= 1e-5 * cor["emc"].max()
    dg = g.diagnostics()
    to, _ = o.tallies()
    for k, ko in (("e_inc", "INC"), ("e_trans", "TRANS"), ("e_back", "BACK"), ("e_rt_num", "RT_NUM"),
                  ("e_rt_pend", "RT_PEND"), ("e_phot", "PHOT")):
        assert abs(dg[k] - to[ko]) <= 1e-5 * max(to["INC"], 1e-300), (k, dg[k], to[ko])


def test_single_beam_linear_transport_is_the_march(tables):
    """The beam ordinate alone, rad cells the size of PIC cells, the linear
    split, nothing absorbing: the device's photon numbers after 30 rad
    steps are those of its ballistic march (the same arithmetic; the march
    keeps its photon numbers as float pairs, ~48 bits, between steps, the
    transport in double: 1e-12), and the oracle's."""
    tab = dict(tables)
    tab["sigma_photo"] = tables["sigma_photo"] * 0.0
    cfg = P.cfg_small_1d(nx=48, ny=4, dx_nm=2.0, dy_nm=2.0, ppc_e=4, ppc_i=4, flags=P.F_PHOTO, beam_frac=0.0)
    pl = P.Pulse(I_peak_Wcm2=1e17, fwhm_fs=3.0, t_peak_fs=4.0, hv_eV=1600.0, n_bins=2, spot_sigma_nm=3.0)
    st = P.init_particles(cfg)
    a = pkg.Slab(cfg, tab, pl)
    a.load(st)
    b = pkg.Slab(cfg, tab, pl)
    b.load(st)
    b.set_rt(coarsen=1, n_polar=0, scheme=1)
    a.step(150)
    b.step(150)
    pa, pb = a.photons(), b.photons()
    assert pa.max() > 0 and np.abs(pa - pb).max() <= 1e-12 * pa.max()
    da, db = a.diagnostics(), b.diagnostics()
    for k in ("e_inc", "e_trans", "e_phot"):
        assert abs(da[k] - db[k]) <= 1e-12 * da["e_inc"], k
    o = oracle.OracleSlab(cfg, tab, pl)
    o.load(st)
    o.set_rt(coarsen=1, n_polar=0, scheme=1)
    o.step(150)
    assert np.abs(pb - o.photons()).max() <= 1e-6 * o.photons().max()


def test_device_energy_bookkeeping_with_transport(tables):
    """Collisions, ionization, recombination, photoionization and K decay
    with the transport on (no push), 200 steps through a pulse: the device's
    kinetic + ionization + photon + escaped + transmitted + back-escaped -
    incident - transport gain + owed energy stays constant to 2e-6 of the
    incident energy."""
    cfg, tab, pl, st = _setup(tables, 10)
    cfg.rad_every = 5
    g = pkg.Slab(cfg, tab, pl)
    g.load(st)
    g.set_rt(coarsen=5, n_polar=3, n_azimuth=2, scheme=0)

    def total(d):
        return (d["ke_e"] + d["ke_i"] + d["e_ion"] + d["e_phot"] + d["e_ka_esc"] + d["e_trans"] + d["e_back"]
                - d["e_inc"] - d["e_rt_num"] + d["e_rt_pend"])

    e0 = total(g.diagnostics())
    for _ in range(4):
        g.step(50)
        d = g.diagnostics()
        assert abs(total(d) - e0) <= 2e-6 * max(d["e_inc"], abs(e0)), (total(d) - e0, d["e_inc"])
    assert d["counts"]["PH0"] > 0 and d["e_inc"] > 0


def test_transport_refused_where_it_does_not_apply(tables):
    cfg = P.cfg_small_1d(nx=40, flags=P.F_PHOTO)
    g = pkg.Slab(cfg, tables)
    with pytest.raises(pkg.PicError, match="STATE"):
        g.set_rt(coarsen=5)                      # no pulse yet
    g.set_pulse(P.Pulse(I_peak_Wcm2=1e16))
    with pytest.raises(pkg.PicError, match="ARG"):
        g.set_rt(coarsen=7)                      # 40 cells are not whole rad cells of 7
    g.set_rt(coarsen=5, n_polar=2)
    with pytest.raises(pkg.PicError, match="STATE"):
        g.set_rt(coarsen=5)                      # already on
    g.close()


def test_transport_mode_is_bit_reproducible(tables):
    """Two runs of the same seeded slab in transport mode agree particle for
    particle after 40 rad steps with every process: the rad cells' heating
    share comes from electron weights summed in canonical order (the order
    of a cell's slots is the scatter's and differs between runs)."""
    cfg, tab, pl, st = _setup(tables, 1)
    runs = []
    for _ in range(2):
        g = pkg.Slab(cfg, tab, pl)
        g.load(st)
        g.set_rt(coarsen=5, n_polar=3, n_azimuth=2, scheme=0)
        g.step(40)
        e = g.electrons()
        o = np.argsort(e["id"], kind="stable")
        runs.append({k: v[o] for k, v in e.items()})
        g.close()
    for k in runs[0]:
        assert np.array_equal(runs[0][k], runs[1][k]), k
