"""The FP64 build of the device kernels (the same sources compiled with
real = double) against the FP64 oracle.

With single-precision rounding out of the way, the device logic must
reproduce the oracle's arithmetic: the same events, and momenta, weights,
positions, fields and currents that differ only by the rounding of two
double-precision evaluations of the same formulas (summation order,
reciprocals, cospi against cos of 2 pi r).  That pins the device code to
the method independently of the FP32 tolerance the production build is
held to.  Trajectories still decorrelate over many steps (collisions
amplify rounding differences), so multi-step runs keep their events
identical while their momenta drift apart slowly.
"""
import numpy as np
import pytest

import pic_inputs as P
from parity_util import match

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1704_01202_gb300 as pkg  # noqa: E402

# relative floor of the momentum comparison (u = gamma v / c)
U_FLOOR = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    oracle.build()


def _run_both64(cfg, tables, st, nsteps, pulse=None, photons=None, fields=None):
    g = pkg.Slab(cfg, tables, pulse, fp64=True)
    g.load(st)
    o = oracle.OracleSlab(cfg, tables, pulse)
    o.load(st)
    if photons is not None:
        g.set_photons(photons)
        o.set_photons(photons)
    if fields is not None:
        g.set_fields(fields)
        o.set_fields(fields)
    g.step(nsteps)
    g.sync()
    o.step(nsteps)
    return g, o


def _compare64(g, o):
    """Largest relative momentum and weight differences, largest position
    difference (cells), and mismatching integer states, particles matched
    by id."""
    ge, oe = g.electrons(full=True), o.electrons()
    gi, oi = g.ions(full=True), o.ions()
    out = {}
    ia, ib, same = match(ge["id"], oe["id"])
    ja, jb, same_i = match(gi["id"], oi["id"])
    out["same_ids"] = bool(same and same_i)
    if not out["same_ids"]:
        out["n"] = (len(ge["id"]), len(oe["id"]), len(gi["id"]), len(oi["id"]))
        return out
    du = np.linalg.norm(ge["u"][ia] - oe["u"][ib], axis=1) / (np.linalg.norm(oe["u"][ib], axis=1) + U_FLOOR)
    out["u_max"] = float(du.max()) if du.size else 0.0
    out["u_p99"] = float(np.quantile(du, 0.99)) if du.size else 0.0
    out["u_p999"] = float(np.quantile(du, 0.999)) if du.size else 0.0
    out["w_max"] = float((np.abs(ge["w"][ia] - oe["w"][ib]) / np.maximum(oe["w"][ib], 1e-300)).max())
    out["x_max"] = float(max(np.abs(ge["X"][ia] - oe["X"][ib]).max(), np.abs(ge["Y"][ia] - oe["Y"][ib]).max()))
    dui = np.linalg.norm(gi["u"][ja] - oi["u"][jb], axis=1) / (np.linalg.norm(oi["u"][jb], axis=1) + 1e-9)
    out["ui_max"] = float(dui.max()) if dui.size else 0.0
    out["Z_mismatch"] = int((gi["Z"][ja] != oi["Z"][jb]).sum())
    out["nK_mismatch"] = int((gi["nK"][ja] != oi["nK"][jb]).sum())
    out["zf_max"] = float(np.abs(gi["zf"][ja] - oi["zf"][jb]).max())
    return out


def _busy(cfg, seed=5):
    st = P.init_particles(cfg)
    st = P.perturb_ions(st, seed, frac_hollow=0.4, z_spread=3, zfrac_share=0.25)
    return P.neutralize(st, cfg)


def test_fp64_build_reports_its_type():
    assert pkg.lib(True).pic_real_bytes() == 8 and pkg.lib().pic_real_bytes() == 4


@pytest.mark.parametrize("ny", [1, 6])
def test_fp64_single_step_every_process(tables, ny):
    """A rad step with dense and scarce photons, hollow ions, fractional
    charges and random fields (every branch of the step): the same events
    as the oracle and every particle, field and current value within 1e-12
    relative."""
    cfg = P.cfg_small_1d(nx=40, ny=ny, dx_nm=2.0, dy_nm=2.0, ppc_e=64, ppc_i=16, T_e_eV=25.0,
                         flags=P.F_ALL, rad_every=1)
    pl = P.Pulse(I_peak_Wcm2=3e17, fwhm_fs=30.0, t_peak_fs=0.0, hv_eV=1700.0, n_bins=3, bandwidth_eV=400.0)
    tab = dict(tables)
    tab["sigma_photo"] = tables["sigma_photo"] * 50.0
    st = _busy(cfg)
    ph = P.photons_uniform(cfg, pl, 1.0)
    ph[:, cfg.nx // 2:, :] = 0.3 * cfg.w_ion
    f = P.random_fields(cfg, 3, e_amp=2e-3, b_amp=2e-3)
    g, o = _run_both64(cfg, tab, st, 1, pulse=pl, photons=ph, fields=f)
    res = _compare64(g, o)
    assert res["same_ids"], res
    assert res["Z_mismatch"] == 0 and res["nK_mismatch"] == 0, res
    assert res["u_max"] < 1e-12 and res["ui_max"] < 1e-12 and res["w_max"] < 1e-12, res
    assert res["x_max"] < 1e-12 and res["zf_max"] < 1e-12, res
    cg = g.diagnostics()["counts"]
    _, co = o.tallies()
    assert cg == co
    assert co["ION"] > 0 and co["REC"] > 0 and co["PH0"] > 0 and co["AUG"] > 0 and co["PART"] > 0
    pg, po = g.photons(), o.photons()
    assert np.allclose(pg, po, rtol=1e-12, atol=1e-14 * po.max())
    jg, jo = g.current(), o.current()
    for c in range(3):
        scale = np.abs(jo[c]).max() + 1e-300
        # the device sums the current in 2^-48 fixed point, half a unit per
        # contribution and up to a few hundred contributions per node
        assert np.abs(jg[c] - jo[c]).max() < 1e-12 * scale + 2.0 ** -49 * 512, c


def test_fp64_multi_step_error_growth(tables):
    """Twenty steps of the small 1D slab with every process but photons: the
    events stay identical step by step.  Momenta leave the rounding level
    after the first step: a collision of two particles of nearly equal
    velocity (electrons created at rest by ionization, for one) turns a
    rounding difference of the relative velocity into a much larger one of
    the deflection, so the largest difference jumps while the bulk (99th
    percentile) grows slowly."""
    cfg = P.cfg_small_1d(nx=32)
    st = P.init_particles(cfg)
    g = pkg.Slab(cfg, tables, fp64=True)
    g.load(st)
    o = oracle.OracleSlab(cfg, tables)
    o.load(st)
    rows = []
    for n in range(20):
        g.step(1)
        o.step(1)
        res = _compare64(g, o)
        assert res["same_ids"] and res["Z_mismatch"] == 0, (n, res)
        rows.append((res["u_p99"], res["u_max"]))
    print("\nper step, 99th percentile / largest relative momentum difference:")
    print(" ".join(f"{a:.1e}/{b:.1e}" for a, b in rows))
    assert rows[0][1] < 1e-12 and rows[-1][0] < 1e-9, rows
    cg = g.diagnostics()["counts"]
    _, co = o.tallies()
    assert cg == co
