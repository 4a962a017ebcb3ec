"""Steps replayed through CUDA graphs give the same state as steps launched
one by one (single slab and batch, odd and even step counts)."""
import numpy as np
import pytest

import pic_inputs as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1704_01202_gb300 as pkg  # noqa: E402


def _by_id(d):
    o = np.argsort(d["id"], kind="stable")
    return {k: v[o] for k, v in d.items()}


def _same(a, b):
    a, b = _by_id(a), _by_id(b)
    return all(np.array_equal(a[k], b[k]) for k in a)


@pytest.mark.parametrize("dims", ["1d", "2d"])
def test_graph_steps_identical(dims):
    pkg.build()
    if dims == "1d":
        cfg = P.cfg_small_1d(nx=40, ppc_e=96, ppc_i=24, rad_every=1, flags=P.F_ALL)
    else:
        cfg = P.cfg_foil_2d(nx=24, ny=12, rad_every=2)
    pl = P.pulse_foil_2d(I_peak_Wcm2=3e17, fwhm_fs=10.0, t_peak_fs=0.0)
    st = P.init_particles(cfg)
    runs = []
    for graphs in (False, True):
        s = pkg.Slab(cfg, P.standin_tables(), pl)
        s.use_graphs(graphs)
        s.load(st)
        for n in (3, 4, 1, 2):          # odd counts leave the buffers swapped
            s.step(n)
        s.sync()
        runs.append((s.electrons(), s.ions(), s.fields(), s.diagnostics()))
        s.close()
    (e0, i0, f0, d0), (e1, i1, f1, d1) = runs
    assert _same(e0, e1) and _same(i0, i1)
    for k in f0:
        assert np.array_equal(f0[k], f1[k]), k
    assert d0["counts"] == d1["counts"]


def test_graph_batch_identical():
    pkg.build()
    ens = P.batched_ensemble(n=5, seed=3, cells=(16, 64), ppc=(16, 64))
    states = [P.init_particles(c) for c, _ in ens]
    cap_e = sum(pkg.default_capacity(s.n_e, s.n_i, c.Z_init)[0] for (c, _), s in zip(ens, states))
    cap_i = sum(pkg.default_capacity(s.n_e, s.n_i, c.Z_init)[1] for (c, _), s in zip(ens, states))
    out = []
    for graphs in (False, True):
        bt = pkg.Batch(P.standin_tables(), 5, 64, cap_e, cap_i)
        bt.use_graphs(graphs)
        slots = [bt.admit(c, s, pl) for (c, pl), s in zip(ens, states)]
        bt.step(4)
        bt.retire(slots[1])
        bt.step(5)
        out.append([(bt.electrons(k), bt.ions(k)) for k in slots if k != slots[1]])
        bt.close()
    for (ea, ia), (eb, ib) in zip(*out):
        assert _same(ea, eb) and _same(ia, ib)


def test_autotune_keeps_results():
    """The autotuner times real steps with other launch shapes; the state
    must not change."""
    pkg.build()
    cfg = P.cfg_foil_2d(nx=32, ny=16, rad_every=2)
    pl = P.pulse_foil_2d(I_peak_Wcm2=3e17, fwhm_fs=10.0, t_peak_fs=0.0)
    st = P.init_particles(cfg)
    runs = []
    for tune in (False, True):
        s = pkg.Slab(cfg, P.standin_tables(), pl)
        s.autotune(tune)
        s.load(st)
        s.step(5)           # tuning goes on across calls
        s.step(7)
        s.sync()
        w, ms = s.autotune()
        runs.append((s.electrons(), s.ions()))
        s.close()
        if tune:
            assert w in (1, 2, 4, 8) and (ms > 0).sum() >= 1
            assert ms[[1, 2, 4, 8].index(w)] == ms[ms > 0].min()
    (e0, i0), (e1, i1) = runs
    assert _same(e0, e1) and _same(i0, i1)
