"""Host helpers of the drivers, without a GPU: the hot-electron shares the
10 keV and thermalization legs report (Sec. VI C quotes the number and the
energy share of electrons above a threshold), the layout of the K-edge
sweep's batch (one slab per photon energy and continuum-lowering model),
the served loop's time-to-result summary and the default capacity of a
slab (every ion stripped, plus headroom)."""
import numpy as np
import pytest

import pic_inputs as P
from paper_1704_01202_gb300 import default_capacity, kedge, serve, thermal

MC2 = 510998.95


def _u_for(ke_eV):
    """Momentum (units of m c) along x of an electron of kinetic energy ke."""
    g = 1.0 + ke_eV / MC2
    return np.sqrt(g * g - 1.0)


def test_tail_share_by_hand():
    ke = np.array([10.0, 100.0, 1000.0, 8000.0])
    w = np.array([4.0, 3.0, 2.0, 1.0])
    u = np.zeros((4, 3))
    u[:, 0] = _u_for(ke)
    share_w, share_k = thermal.tail_share({"u": u.astype(np.float32), "w": w.astype(np.float32)}, 700.0)
    assert share_w == pytest.approx(3.0 / 10.0)
    K = (w * ke).sum()
    assert share_k == pytest.approx((2.0 * 1000.0 + 8000.0) / K, rel=1e-6)
    # nobody above the threshold, and no electrons at all
    assert thermal.tail_share({"u": u[:1], "w": w[:1]}, 700.0) == (0.0, 0.0)
    assert thermal.tail_share({"u": np.zeros((0, 3)), "w": np.zeros(0)}, 700.0) == (0.0, 0.0)


def test_kedge_sweep_layout():
    hv = [1540.0, 1560.0, 1600.0]
    pts = kedge.scan_slabs(P, hv, models=(1, 2), nx=50)
    assert len(pts) == 6
    assert [p[3] for p in pts] == [1, 1, 1, 2, 2, 2]
    assert [p[2] for p in pts] == hv + hv
    seeds = [p[0].seed for p in pts]
    assert len(set(seeds)) == len(seeds)
    for cfg, pl, h, ipd in pts:
        assert cfg.ny == 1 and cfg.nx == 50 and cfg.ipd_model == ipd and cfg.flags == P.F_ALL
        assert cfg.rad_every == 1 and pl.hv_eV == h
    assert len({p[0].name for p in pts}) == len(pts)


def test_served_summary_percentiles():
    ttr = {k: float(k + 1) for k in range(100)}          # 1 .. 100 s
    s = serve._summary(ttr, 10.0, 60.0, 100)
    assert s["slabs"] == 100 and s["wall_s"] == 50.0 and s["slabs_per_s"] == 2.0
    assert s["ttr_p50_s"] == pytest.approx(50.5) and s["ttr_p99_s"] == pytest.approx(99.01)
    assert s["ttr_mean_s"] == pytest.approx(50.5)


def test_default_capacity_strips_every_ion():
    ce, ci = default_capacity(800, 200, 3, headroom=1.0)
    assert (ce, ci) == (800 + 200 * 10 + 1024, 200 + 1024)
    ce13, _ = default_capacity(800, 200, 13, headroom=1.0)
    assert ce13 == 800 + 1024
    assert default_capacity(800, 200, 3)[0] == int((800 + 2000) * 1.3) + 1024
