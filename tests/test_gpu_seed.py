"""The initial plasma seeded on the device (pic_seed, the solid-density
start of Sec. II): layout (cells, ids, charge states, weights, neutrality),
the distributions it draws from (uniform positions, Maxwellian momenta at
T_e and T_i, the beam share at its energy with isotropic directions) within
4 standard errors, determinism, and a seeded slab stepping like the same
state loaded from the host."""
import numpy as np
import pytest

import pic_inputs as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1704_01202_gb300 as pkg  # noqa: E402

MC2 = 510998.95


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _ke(u, mass=1.0):
    u2 = (np.asarray(u, dtype=np.float64) ** 2).sum(axis=1)
    return mass * MC2 * u2 / (np.sqrt(1.0 + u2) + 1.0)


def _by_id(d):
    o = np.argsort(d["id"], kind="stable")
    return {k: v[o] for k, v in d.items()}


def _seeded(cfg, tables, seed=None):
    g = pkg.Slab(cfg, tables)
    g.seed(seed)
    return g


@pytest.mark.parametrize("ny", [1, 4])
def test_seeded_layout(tables, ny):
    cfg = P.cfg_small_1d(nx=48, ny=ny, ppc_e=120, ppc_i=30, Z_init=3)
    g = _seeded(cfg, tables)
    e, i = g.electrons(), g.ions()
    g.close()
    ne, ni = cfg.ncell * cfg.ppc_e, cfg.ncell * cfg.ppc_i
    assert len(e["id"]) == ne and len(i["id"]) == ni
    assert np.array_equal(np.sort(e["id"]), np.arange(ne)) and np.array_equal(np.sort(i["id"]), np.arange(ni))
    for d, ppc in ((e, cfg.ppc_e), (i, cfg.ppc_i)):
        cell = np.floor(d["X"]).astype(int) + cfg.nx * (np.floor(d["Y"]).astype(int) if ny > 1 else 0)
        assert np.all(np.bincount(cell, minlength=cfg.ncell) == ppc)
        # cell-major ids: particle id sits in cell id // ppc
        assert np.array_equal(cell, (d["id"] // ppc).astype(int))
        if ny == 1:
            assert np.all(d["Y"] == 0.5)
    assert np.all(i["Z"] == 3) and np.all(i["nK"] == 0) and np.all(i["zf"] == 0)
    w_e = np.float32(cfg.Z_init * cfg.ppc_i * cfg.w_ion / cfg.ppc_e)
    assert np.all(e["w"] == w_e)
    # neutral: electron weight = Z_init x ion weight, to the weight's rounding
    assert abs(e["w"].astype(np.float64).sum() / (cfg.Z_init * ni * cfg.w_ion) - 1) < 1e-6


def test_seeded_distributions(tables):
    cfg = P.cfg_small_1d(nx=128, ny=2, ppc_e=256, ppc_i=64, T_e_eV=10.0, T_i_eV=4.0, beam_frac=0.05,
                         beam_E_eV=1500.0)
    g = _seeded(cfg, tables)
    e, i = g.electrons(), g.ions()
    g.close()
    n = len(e["id"])
    ke = _ke(e["u"])
    beam = np.abs(ke - cfg.beam_E_eV) < 1e-3 * cfg.beam_E_eV
    nb = int(beam.sum())
    f = cfg.beam_frac
    assert abs(nb / n - f) <= 4.0 * np.sqrt(f * (1 - f) / n)
    # beam: its energy to FP32, isotropic directions
    assert np.allclose(ke[beam], cfg.beam_E_eV, rtol=1e-5)
    ub = e["u"][beam].astype(np.float64)
    cos = ub / np.linalg.norm(ub, axis=1)[:, None]
    assert np.all(np.abs(cos.mean(axis=0)) <= 4.0 / np.sqrt(3.0 * nb))
    assert np.all(np.abs((cos ** 2).mean(axis=0) - 1.0 / 3.0) <= 4.0 * np.sqrt(4.0 / 45.0 / nb))
    # bulk: Gaussian momentum components of variance T / mc^2, mean kinetic
    # energy 3/2 T (the relativistic correction is 1e-4 of it here)
    for d, sel, T, m in ((e, ~beam, cfg.T_e_eV, 1.0), (i, slice(None), cfg.T_i_eV, cfg.m_ion_me)):
        u = d["u"][sel].astype(np.float64)
        k = len(u)
        var = T / (m * MC2)
        assert np.all(np.abs(u.mean(axis=0)) <= 4.0 * np.sqrt(var / k))
        assert np.all(np.abs(u.var(axis=0) / var - 1.0) <= 4.0 * np.sqrt(2.0 / k))
        kk = _ke(u, m)
        assert abs(kk.mean() / (1.5 * T) - 1.0) <= 4.0 * np.sqrt(1.5) / 1.5 / np.sqrt(k) + 1e-3
    # positions uniform in their cells (both directions in 2D)
    for d in (e, i):
        for ax in ("X", "Y"):
            xi = d[ax] - np.floor(d[ax])
            assert np.all((xi >= 0) & (xi < 1))
            assert abs(xi.mean() - 0.5) <= 4.0 * np.sqrt(1.0 / 12.0 / len(xi))
            h = np.histogram(xi, bins=10, range=(0, 1))[0] / len(xi)
            assert np.all(np.abs(h - 0.1) <= 4.0 * np.sqrt(0.09 / len(xi)))


def test_seed_is_deterministic_and_steps_like_a_loaded_state(tables):
    cfg = P.cfg_small_1d(nx=40, ppc_e=64, ppc_i=16, seed=5)
    a = _seeded(cfg, tables)
    b = _seeded(cfg, tables)
    c = _seeded(cfg, tables, seed=6)
    # the order within a cell's storage is the scatter's; compare by id
    ea, eb, ec = (_by_id(s.electrons()) for s in (a, b, c))
    for k in ea:
        assert np.array_equal(ea[k], eb[k]), k
    assert not np.array_equal(ea["u"], ec["u"])
    # the seeded state as host arrays, loaded into a fresh slab: the same steps
    ia = a.ions()
    st = P.ParticleState(eX=ea["X"], eY=ea["Y"], eu=ea["u"], ew=ea["w"], eid=ea["id"], iX=ia["X"], iY=ia["Y"],
                         iu=ia["u"], izf=ia["zf"].astype(np.float64), iZ=ia["Z"], inK=ia["nK"], iid=ia["id"])
    d = pkg.Slab(cfg, tables)
    d.load(st)
    a.step(30)
    d.step(30)
    da, dd = a.diagnostics(), d.diagnostics()
    assert da["counts"] == dd["counts"] and da["n_e"] == dd["n_e"]
    assert da["ke_e"] == pytest.approx(dd["ke_e"], rel=1e-12)
    for g in (a, b, c, d):
        g.close()


def test_seed_refusals(tables):
    cfg = P.cfg_small_1d(nx=8, ppc_e=4, ppc_i=1)
    g = pkg.Slab(cfg, tables, cap_e=16, cap_i=8)
    with pytest.raises(pkg.PicError, match="CAPACITY"):
        g.seed()                                    # 32 electrons > 16
    g.cfg = P.cfg_small_1d(nx=8, ppc_e=1, ppc_i=1, Z_init=13)
    with pytest.raises(pkg.PicError, match="ARG"):
        g.seed()
    g.close()
