"""Checkpoint and restore of a slab (pic_checkpoint / pic_restore): a
context restored from a host image continues as the original does, particle
for particle (the random streams are keyed by id and step, so no generator
state is saved), with every process on and the march, and in transport
mode; images of another slab or truncated ones are refused."""
import numpy as np
import pytest

import pic_inputs as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1704_01202_gb300 as pkg  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _by_id(d):
    o = np.argsort(d["id"], kind="stable")
    return {k: v[o] for k, v in d.items()}


def _same_state(a, b, photons=True):
    for get in ("electrons", "ions"):
        x, y = _by_id(getattr(a, get)()), _by_id(getattr(b, get)())
        for k in x:
            assert np.array_equal(x[k], y[k]), (get, k)
    if photons:
        assert np.array_equal(a.photons(), b.photons())
    da, db = a.diagnostics(), b.diagnostics()
    assert da["counts"] == db["counts"] and da["t_fs"] == db["t_fs"]
    for k in ("ke_e", "ke_i", "e_ion", "e_phot", "e_inc", "e_trans", "e_field"):
        assert da[k] == pytest.approx(db[k], rel=1e-9, abs=1e-12), k


def _make(cfg, tables, pl, rt=None):
    g = pkg.Slab(cfg, tables, pl)
    if rt:
        g.set_rt(**rt)
    return g


@pytest.mark.parametrize("case", ["2d_march", "1d_transport"])
def test_restored_slab_continues_as_the_original(tables, case):
    if case == "2d_march":
        cfg = P.cfg_foil_2d(nx=48, ny=8, ppc_e=32, ppc_i=8)
        pl = P.pulse_foil_2d(t_peak_fs=1.0, fwhm_fs=4.0, I_peak_Wcm2=3e17)
        rt = None
    else:
        cfg = P.cfg_small_1d(nx=40, ppc_e=48, ppc_i=12, rad_every=1, flags=P.F_ALL)
        pl = P.Pulse(I_peak_Wcm2=4e17, fwhm_fs=4.0, t_peak_fs=0.3, hv_eV=1700.0, n_bins=3, bandwidth_eV=300.0)
        rt = dict(coarsen=5, n_polar=3, n_azimuth=2, scheme=0)
    a = _make(cfg, tables, pl, rt)
    a.load(P.init_particles(cfg))
    a.step(40)
    image = a.checkpoint()
    a.step(40)
    b = _make(cfg, tables, pl, rt)
    b.restore(image)
    b.step(40)
    _same_state(a, b)
    assert a.diagnostics()["counts"]["PH0"] > 0
    a.close()
    b.close()


def test_restore_refuses_other_slabs_and_truncated_images(tables):
    cfg = P.cfg_small_1d(nx=16, ppc_e=16, ppc_i=4)
    a = pkg.Slab(cfg, tables)
    a.load(P.init_particles(cfg))
    a.step(3)
    image = a.checkpoint()
    other = pkg.Slab(P.cfg_small_1d(nx=20, ppc_e=16, ppc_i=4), tables)
    with pytest.raises(pkg.PicError, match="ARG"):
        other.restore(image)
    b = pkg.Slab(cfg, tables)
    with pytest.raises(pkg.PicError, match="ARG"):
        b.restore(image[:-8])
    bad = bytearray(image)
    bad[0:8] = b"NOTACKPT"
    with pytest.raises(pkg.PicError, match="ARG"):
        b.restore(bytes(bad))
    b.restore(image)
    a.step(5)
    b.step(5)
    _same_state(a, b, photons=False)
    for g in (a, other, b):
        g.close()
