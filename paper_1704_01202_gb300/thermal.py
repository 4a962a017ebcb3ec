"""Non-thermal against force-thermalized electrons (Sec. VI C).

Two copies of the same slab, one with the forced-thermalization variant
(PIC_F_THERM: on every rad step each cell's free electrons are redrawn from
a Maxwellian at (2/3) E_ave, momentum and energy kept), run side by side in
one batch; the mean charge, its rate and the electron temperature are read
every `every_fs`.  The paper finds the two ionization histories nearly
identical for 1.7 keV photons (its Fig. 5c).

    python -m paper_1704_01202_gb300.thermal --horizon-fs 100
"""
from __future__ import annotations

import argparse
import json
import time

from . import Batch, default_capacity


def tail_share(e: dict, threshold_eV: float) -> tuple[float, float]:
    """Weight fraction of the electrons above threshold_eV and the fraction
    of the free-electron kinetic energy they carry."""
    import numpy as np
    u = e["u"].astype(np.float64)
    u2 = (u * u).sum(axis=1)
    ke = 510998.95 * u2 / (np.sqrt(1.0 + u2) + 1.0)
    w = e["w"].astype(np.float64)
    hot = ke > threshold_eV
    W, K = w.sum(), (w * ke).sum()
    return (float(w[hot].sum() / W) if W > 0 else 0.0, float((w * ke)[hot].sum() / K) if K > 0 else 0.0)


def compare(tables, cfg, pulse, init_state, horizon_fs: float, every_fs: float = 5.0, therm_flag: int = 256,
            tail_eV: float = 0.0) -> dict:
    import copy
    import torch
    cfg_t = copy.deepcopy(cfg)
    cfg_t.flags = cfg.flags | therm_flag
    st = init_state(cfg)
    ce, ci = default_capacity(st.n_e, st.n_i, cfg.Z_init)
    bt = Batch(tables, 2, cfg.nx, 2 * ce, 2 * ci)
    try:
        k_plain = bt.admit(cfg, st, pulse)
        k_therm = bt.admit(cfg_t, st, pulse)
        per = max(1, int(round(every_fs / cfg.dt_fs)))
        nsteps = int(round(horizon_fs / cfg.dt_fs))
        out = {"t_fs": [], "Zbar": [], "Zbar_therm": [], "T_e_eV": [], "T_e_eV_therm": []}
        if tail_eV > 0:
            out["tail_number_share"], out["tail_energy_share"] = [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = 0
        while done < nsteps:
            n = min(per, nsteps - done)
            bt.step(n)
            done += n
            a, b = bt.diagnostics(k_plain), bt.diagnostics(k_therm)
            out["t_fs"].append(a["t_fs"])
            out["Zbar"].append(a["Zbar"])
            out["Zbar_therm"].append(b["Zbar"])
            out["T_e_eV"].append(a["T_e_eV"])
            out["T_e_eV_therm"].append(b["T_e_eV"])
            if tail_eV > 0:     # of the non-thermal run (outside the timing would be fairer; it is small)
                ns, es = tail_share(bt.electrons(k_plain), tail_eV)
                out["tail_number_share"].append(ns)
                out["tail_energy_share"].append(es)
        wall = time.perf_counter() - t0
    finally:
        bt.close()
    out.update(steps=nsteps, wall_s=wall, particle_steps_per_s=2 * (st.n_e + st.n_i) * nsteps / wall)
    return out


def main():
    import pic_inputs as P
    ap = argparse.ArgumentParser()
    ap.add_argument("--horizon-fs", type=float, default=100.0)
    ap.add_argument("--every-fs", type=float, default=5.0)
    args = ap.parse_args()
    cfg = P.cfg_small_1d(nx=128, flags=P.F_ALL)
    pulse = P.Pulse(I_peak_Wcm2=1.36e17, fwhm_fs=80.0, t_peak_fs=80.0, hv_eV=1700.0)
    print(json.dumps(compare(P.standin_tables(), cfg, pulse, P.init_particles, args.horizon_fs, args.every_fs,
                             P.F_THERM)))


if __name__ == "__main__":
    main()
