"""Batched slabs through the C ABI (pic_batch_*).

A slab's random streams are keyed by its own seed, particle ids and step
count, and every sum across particles is fixed-point or taken in a
canonical order, so a slab stepped inside a batch must be bit-identical to
the same slab stepped alone, whatever its neighbours, when they were
admitted or retired.  One batch slot is also checked against the oracle.
"""
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

SLOT = 64


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    oracle.build()


def _slabs():
    """Three 1D slabs of different sizes, seeds, weights and cell widths
    (so different field speeds); A has every process on and a pulse."""
    a = P.cfg_small_1d(nx=48, seed=11, ppc_e=96, ppc_i=24, rad_every=1, flags=P.F_ALL)
    b = P.cfg_small_1d(nx=64, seed=12, ppc_e=128, ppc_i=32)
    c = P.cfg_small_1d(nx=30, seed=13, ppc_e=64, ppc_i=16, dx_nm=2.5, Z_init=4)
    pa = P.pulse_foil_2d(I_peak_Wcm2=3e17, fwhm_fs=10.0, t_peak_fs=0.0)
    return (a, P.init_particles(a), pa), (b, P.init_particles(b), None), (c, P.init_particles(c), None)


def _caps(specs):
    ce = ci = 0
    for cfg, st, _ in specs:
        e, i = pkg.default_capacity(st.n_e, st.n_i, cfg.Z_init)
        ce, ci = ce + e, ci + i
    return ce, ci


def _alone(cfg, st, pulse, n):
    s = pkg.Slab(cfg, P.standin_tables(), pulse)
    s.load(st)
    s.step(n)
    s.sync()
    out = s.electrons(), s.ions(), s.diagnostics()
    s.close()
    return out


def _by_id(d):
    o = np.argsort(d["id"], kind="stable")
    return {k: v[o] for k, v in d.items()}


def _assert_identical(got, ref):
    ge, gi, gd = got
    re, ri, rd = ref
    ge, re, gi, ri = _by_id(ge), _by_id(re), _by_id(gi), _by_id(ri)
    for k in re:
        assert np.array_equal(ge[k], re[k]), ("electrons", k)
    for k in ri:
        assert np.array_equal(gi[k], ri[k]), ("ions", k)
    assert gd["counts"] == rd["counts"]
    assert gd["n_e"] == rd["n_e"] and gd["n_i"] == rd["n_i"]
    assert gd["t_fs"] == rd["t_fs"]
    for k in ("ke_e", "ke_i", "e_ion", "e_phot", "e_inc", "e_trans", "e_field", "Zbar"):
        assert gd[k] == pytest.approx(rd[k], rel=1e-9, abs=1e-12), k
    assert np.allclose(gd["csd"], rd["csd"], rtol=1e-6, atol=1e-9)


def test_batch_slot_identical_to_alone():
    specs = _slabs()
    (a, sa, pa), (b, sb, pb), (c, sc, pc) = specs
    ce, ci = _caps(specs)
    bt = pkg.Batch(P.standin_tables(), 4, SLOT, ce, ci)
    kb = bt.admit(b, sb, pb)
    ka = bt.admit(a, sa, pa)
    kc = bt.admit(c, sc, pc)
    assert (kb, ka, kc) == (0, 1, 2)
    bt.step(6)
    bt.sync()
    for k, (cfg, st, pl) in ((ka, specs[0]), (kb, specs[1]), (kc, specs[2])):
        got = bt.electrons(k), bt.ions(k), bt.diagnostics(k)
        _assert_identical(got, _alone(cfg, st, pl, 6))
        assert bt.slot(k) == (1, 6)
    bt.close()


def test_admit_and_retire_between_steps():
    specs = _slabs()
    (a, sa, pa), (b, sb, pb), (c, sc, pc) = specs
    ce, ci = _caps(specs)
    bt = pkg.Batch(P.standin_tables(), 3, SLOT, ce, ci)
    kb = bt.admit(b, sb, pb)
    bt.step(3)
    ka = bt.admit(a, sa, pa)
    bt.step(2)
    bt.retire(kb)
    assert bt.slot(kb)[0] == 2
    kc = bt.admit(c, sc, pc)               # a free slot, not the retired one
    assert kc not in (ka, kb)
    bt.step(4)
    assert bt.slot(kb)[0] == 0
    assert bt.counts(kb) == (0, 0)
    assert bt.slot(ka) == (1, 6) and bt.slot(kc) == (1, 4)
    _assert_identical((bt.electrons(ka), bt.ions(ka), bt.diagnostics(ka)), _alone(a, sa, pa, 6))
    _assert_identical((bt.electrons(kc), bt.ions(kc), bt.diagnostics(kc)), _alone(c, sc, pc, 4))
    # the freed slot takes a new slab that starts at step 0
    kb2 = bt.admit(b, sb, pb)
    assert kb2 == kb
    bt.step(2)
    _assert_identical((bt.electrons(kb2), bt.ions(kb2), bt.diagnostics(kb2)), _alone(b, sb, pb, 2))
    bt.close()


def test_batch_limits():
    specs = _slabs()
    (a, sa, pa), (b, sb, _), _ = specs
    ce, ci = _caps(specs)
    bt = pkg.Batch(P.standin_tables(), 1, SLOT, ce, ci)
    bt.admit(a, sa, pa)
    with pytest.raises(pkg.PicError, match="CAPACITY"):
        bt.admit(b, sb)
    big = P.cfg_small_1d(nx=SLOT + 1)
    with pytest.raises(pkg.PicError, match="ARG"):
        bt.admit(big, P.init_particles(big))
    two_d = P.cfg_small_1d(nx=8, ny=2, ppc_e=8, ppc_i=2)
    with pytest.raises(pkg.PicError, match="ARG"):
        bt.admit(two_d, P.init_particles(two_d))
    # single-slab calls refuse a batch context
    assert pkg.STATUS[bt.L.pic_counts(bt.h, None, None)] == "PIC_ERR_STATE"
    with pytest.raises(pkg.PicError, match="STATE"):
        bt.retire(0)
        bt.retire(0)
    bt.close()


def test_batch_slot_against_oracle():
    """One step of slab A in slot 1 of a batch, against the FP64 oracle."""
    specs = _slabs()
    (a, sa, pa), (b, sb, pb), _ = specs
    ce, ci = _caps(specs)
    bt = pkg.Batch(P.standin_tables(), 2, SLOT, ce, ci)
    bt.admit(b, sb, pb)
    k = bt.admit(a, sa, pa)
    bt.step(1)
    o = oracle.OracleSlab(a, P.standin_tables(), pa)
    o.load(sa)
    o.trace()
    o.step(1)
    _, co = o.tallies()
    assert_flip_parity(a, sa, bt.electrons(k), bt.ions(k), o, bt.diagnostics(k)["counts"], co,
                       ("ION", "ION_REJ", "REC", "PH0", "PART", "AUG", "KA", "EE", "EI"))
    bt.close()
