"""Edge cases of the CUDA path through the C ABI: empty and one-species
slabs, single particles, the smallest grids, capacity exhaustion reported as
an error, and invalid arguments refused on the host."""
import ctypes as C

import numpy as np
import pytest

import pic_inputs as P
from parity_util import assert_flip_parity, compare_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_1704_01202_gb300 as pkg  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    oracle.build()


def _subset(st, e_mask, i_mask):
    return P.ParticleState(eX=st.eX[e_mask], eY=st.eY[e_mask], eu=st.eu[e_mask], ew=st.ew[e_mask],
                           eid=st.eid[e_mask], iX=st.iX[i_mask], iY=st.iY[i_mask], iu=st.iu[i_mask],
                           izf=st.izf[i_mask], iZ=st.iZ[i_mask], inK=st.inK[i_mask], iid=st.iid[i_mask])


@pytest.mark.parametrize("which", ["empty", "electrons only", "ions only", "one each"])
def test_sparse_slabs(tables, which):
    cfg = P.cfg_small_1d(nx=8, ppc_e=16, ppc_i=4, flags=P.F_ALL, rad_every=1)
    pl = P.Pulse(I_peak_Wcm2=3e17, fwhm_fs=5.0, t_peak_fs=0.0, hv_eV=1700.0)
    st = P.init_particles(cfg)
    e = np.zeros(st.n_e, bool)
    i = np.zeros(st.n_i, bool)
    if which == "electrons only":
        e[:] = True
    elif which == "ions only":
        i[:] = True
    elif which == "one each":
        e[0] = True
        i[0] = True
    sub = _subset(st, e, i)
    g = pkg.Slab(cfg, tables, pl, cap_e=4096, cap_i=1024)
    g.load(sub)
    g.step(4)
    g.sync()
    d = g.diagnostics()
    o = oracle.OracleSlab(cfg, tables, pl)
    o.load(sub)
    o.step(4)
    assert (d["n_e"], d["n_i"]) == (len(o.electrons()["id"]), len(o.ions()["id"]))
    if which == "one each":
        res = compare_state(g.electrons(), o.electrons(), g.ions(), o.ions(), cfg.nx, cfg.ny)
        assert res["e_same_ids"] and res["i_same_ids"] and res["Z_mismatch"] == 0, res
    g.close()


def test_smallest_grids(tables):
    """Two cells in 1D and a 2 x 1 ... 3 x 2 2D slab step like the oracle."""
    for nx, ny in ((2, 1), (3, 2)):
        cfg = P.cfg_small_1d(nx=nx, ny=ny, ppc_e=32, ppc_i=8, flags=P.F_ALL & ~P.F_PHOTO)
        st = P.init_particles(cfg)
        g = pkg.Slab(cfg, tables)
        g.load(st)
        g.step(1)
        o = oracle.OracleSlab(cfg, tables)
        o.load(st)
        o.trace()
        o.step(1)
        assert_flip_parity(cfg, st, g.electrons(), g.ions(), o)
        g.close()


def test_capacity_exhaustion_is_reported(tables):
    """An electron capacity with no room for the electrons that ionization
    creates: the step completes, the device error word reports the capacity
    and the context stays usable for reading."""
    cfg = P.cfg_small_1d(nx=16, ppc_e=64, ppc_i=16, T_e_eV=300.0, flags=P.F_COLL_EE | P.F_IONIZE)
    st = P.init_particles(cfg)
    g = pkg.Slab(cfg, tables, cap_e=st.n_e + 2, cap_i=st.n_i)
    g.load(st)
    g.step(3)
    with pytest.raises(pkg.PicError, match="CAPACITY"):
        g.sync()
    g.close()


def test_invalid_arguments_refused(tables):
    L = pkg.lib()
    h = C.c_void_p()
    t, keep = pkg._tables(tables)
    for nx, ny, dt in ((0, 1, 0.02), (8, 0, 0.02), (8, 1, 0.0), (9000, 1, 0.02)):
        g = pkg.Grid(nx=nx, ny=ny, dx_nm=2.0, dy_nm=2.0, dt_fs=dt, rad_every=5, seed=0, cfl=0.95)
        s = pkg.Species(n_ref_cm3=6e22, w_ion=1.0, m_ion_me=49184.0, E_bulk_eV=0.0, ipd_model=1,
                        coulomb_log=0.0, flags=255, cap_e=100, cap_i=100)
        st = L.pic_init(C.byref(h), C.byref(g), C.byref(s), C.byref(t), None, 0, None)
        assert pkg.STATUS[st] == "PIC_ERR_ARG", (nx, ny, dt)
    assert pkg.STATUS[L.pic_step(None, 1)] == "PIC_ERR_ARG"
    assert pkg.STATUS[L.pic_batch_init(C.byref(h), 0, 64, 10, 10, C.byref(t), None, 0, None)] == "PIC_ERR_ARG"
