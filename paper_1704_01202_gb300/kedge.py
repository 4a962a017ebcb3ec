"""K-edge transmission scan: a photon-energy sweep through the cold Al K edge
for two continuum-lowering models, run as one batch.

Sec. VI compares transmissions through a foil heated by the pulse itself
for photon energies around the K edge (~1560 eV cold), and Sec. V shows
that where the edge sits depends on the continuum-lowering model (Ecker-
Kroell, Eq. 4, against Stewart-Pyatt, Eq. 5).  Every (photon energy, model)
point is one 1D slab of a batch context, so the whole sweep is one launch of
each kernel per step.  Inputs are the stand-in atomic tables, so the curve
is a workload of the method, not the paper's measurement.

    python -m paper_1704_01202_gb300.kedge --points 12 --horizon-fs 40
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import Batch, default_capacity


def scan_slabs(P, hv_eV, models=(1, 2), nx: int = 250, dx_nm: float = 2.0, ppc=(64, 16),
               I_Wcm2: float = 1e17, fwhm_fs: float = 10.0, t_peak_fs: float = 10.0, seed: int = 500):
    """(config, pulse, photon energy, model) of every point of the sweep; P is
    the input-generator module (pic_inputs)."""
    out = []
    k = 0
    for ipd in models:
        for hv in hv_eV:
            cfg = P.SlabConfig(name=f"al_1d_{nx}x{dx_nm:g}nm_hv{hv:.0f}_ipd{ipd}", nx=nx, ny=1, dx_nm=dx_nm,
                               dy_nm=dx_nm, ppc_e=ppc[0], ppc_i=ppc[1], seed=seed + k, flags=P.F_ALL,
                               ipd_model=ipd, rad_every=1)
            pl = P.Pulse(I_peak_Wcm2=I_Wcm2, fwhm_fs=fwhm_fs, t_peak_fs=t_peak_fs, hv_eV=float(hv),
                         bandwidth_eV=3.0, n_bins=2)
            out.append((cfg, pl, float(hv), ipd))
            k += 1
    return out


def run_scan(tables, slabs, init_state, nsteps: int) -> dict:
    """Admit every point into one batch, step nsteps, read the diagnostics."""
    import torch
    states = [init_state(c) for c, _, _, _ in slabs]
    cap_e = sum(default_capacity(s.n_e, s.n_i, c.Z_init)[0] for (c, _, _, _), s in zip(slabs, states))
    cap_i = sum(default_capacity(s.n_e, s.n_i, c.Z_init)[1] for (c, _, _, _), s in zip(slabs, states))
    bt = Batch(tables, len(slabs), max(c.nx for c, _, _, _ in slabs), cap_e, cap_i)
    try:
        slots = [bt.admit(c, s, pl) for (c, pl, _, _), s in zip(slabs, states)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bt.step(nsteps)
        bt.sync()
        wall = time.perf_counter() - t0
        rows = []
        for k, (c, pl, hv, ipd) in zip(slots, slabs):
            d = bt.diagnostics(k)
            rows.append({"hv_eV": hv, "ipd": ipd, "transmission": d["transmission"], "Zbar": d["Zbar"],
                         "T_e_eV": d["T_e_eV"], "photoionizations": int(sum(d["counts"][f"PH{q}"] for q in range(5))),
                         "auger": d["counts"]["AUG"], "kalpha": d["counts"]["KA"]})
        n_part = sum(s.n_e + s.n_i for s in states)
    finally:
        bt.close()
    return {"points": rows, "steps": nsteps, "wall_s": wall, "slabs": len(slabs),
            "particle_steps_per_s": n_part * nsteps / wall}


def main():
    import pic_inputs as P
    ap = argparse.ArgumentParser()
    ap.add_argument("--points", type=int, default=12)
    ap.add_argument("--hv-min", type=float, default=1540.0)
    ap.add_argument("--hv-max", type=float, default=1870.0)
    ap.add_argument("--horizon-fs", type=float, default=40.0)
    args = ap.parse_args()
    hv = np.linspace(args.hv_min, args.hv_max, args.points)
    slabs = scan_slabs(P, hv)
    res = run_scan(P.standin_tables(), slabs, P.init_particles, int(round(args.horizon_fs / slabs[0][0].dt_fs)))
    print(json.dumps(res))


if __name__ == "__main__":
    main()
