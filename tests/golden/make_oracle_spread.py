"""Writes tests/golden/oracle_spread.json: the statistical spread of the
oracle itself on the multi-step workloads that the GPU tests compare.

A multi-step run is one realization of a Monte-Carlo method whose single
trajectories decorrelate (the collisions are chaotic), so the FP32 device
run and the FP64 oracle run of the same seeded input agree only as two
realizations do.  This script runs the oracle from the same initial state
(the input generator's seed 0, the state the device starts from) with the
Philox key of the step's random streams set to 1 .. 8: eight independent
realizations of each workload.  It records, per diagnostic, every
realization's value with their mean and standard deviation; a device run
(key 0) then has to lie within 3 sd * sqrt(1 + 1/8) of the mean, plus a
stated floor.

Only the oracle and the seeded input generators are used.

    python tests/golden/make_oracle_spread.py            # every case
    python tests/golden/make_oracle_spread.py small_slab_500
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import pic_inputs as P  # noqa: E402

MC2 = 510998.95
KEYS = list(range(1, 9))
OUT = os.path.join(HERE, "oracle_spread.json")


def _energy_total(t):
    return sum(t[k] for k in ("KE_E", "KE_I", "ION", "PHOT", "FIELD", "ESC", "TRANS", "KA_ESC")) - t["INC"]


def _final(o):
    t, c = o.tallies()
    csd, _ = o.diag()
    e = o.electrons()
    u2 = (e["u"] ** 2).sum(axis=1)
    ke = MC2 * u2 / (np.sqrt(1.0 + u2) + 1.0)
    i = o.ions()
    return t, c, csd, {"Zbar": float((np.arange(len(csd)) * csd).sum()),
                       "T_e_eV": float((2.0 / 3.0) * (e["w"] * ke).sum() / e["w"].sum()),
                       "n_e": float(len(e["id"])), "n_hollow": float((i["nK"] > 0).sum())}


def case_small_slab_500(key):
    """The plain 1D slab at full size and length (128 x 2 nm, 256 e + 64 i
    per cell, collisions, Lotz, recombination, push, fields; 500 steps),
    with the total energy every 100 steps."""
    cfg = P.cfg_small_1d()
    st = P.init_particles(cfg, seed=0)
    cfg.seed = key
    o = oracle.OracleSlab(cfg, TABLES)
    o.load(st)
    e0 = _energy_total(o.tallies()[0])
    vals = {}
    for k in range(5):
        o.step(100)
        vals[f"drift_{100 * (k + 1)}"] = (_energy_total(o.tallies()[0]) - e0) / e0
    t, c, csd, f = _final(o)
    vals.update({k: f[k] for k in ("Zbar", "T_e_eV", "n_e")})
    for k in ("ION", "REC", "EE", "EI"):
        vals["count_" + k] = float(c[k])
    for z in range(len(csd)):
        vals[f"csd_{z}"] = float(csd[z])
    return {"workload": cfg.name, "steps": 500}, vals


def _foil_slice(key, t_peak, nsteps):
    cfg = P.cfg_foil_2d(nx=64, ny=2)
    st = P.init_particles(cfg, seed=0)
    cfg.seed = key
    o = oracle.OracleSlab(cfg, TABLES, P.pulse_foil_2d(t_peak_fs=t_peak))
    o.load(st)
    o.step(nsteps)
    t, c, csd, f = _final(o)
    vals = {"count_" + k: float(c[k]) for k in ("PH0", "AUG", "PART", "KA", "ION", "REC")}
    vals["n_hollow"] = f["n_hollow"]
    vals["transmission"] = t["TRANS"] / t["INC"] if t["INC"] > 0 else 0.0
    return {"workload": cfg.name + f", 64 x 2 slice, pulse peak at {t_peak:g} fs", "steps": nsteps}, vals


def case_kvac_history(key):
    """A 64 x 2 slice of the 2D foil through 200 steps of the 1.6 keV pulse
    peaking at 5 fs: K vacancies, KLL Auger and K-alpha over many rad steps."""
    return _foil_slice(key, 5.0, 200)


def case_partial_early(key):
    """The same slice early in the pulse (peak at 80 fs, 250 steps): every
    absorption a partial event."""
    return _foil_slice(key, 80.0, 250)


def case_subdomain_64x64(key):
    """64 x 64 cells of the large 2D study (80 e + 20 i per cell) through 150
    steps of its pulse moved to peak at 1.5 fs, every process on."""
    cfg = P.cfg_large_2d(nx=64, ny=64)
    st = P.init_particles(cfg, seed=0)
    cfg.seed = key
    o = oracle.OracleSlab(cfg, TABLES, P.pulse_large_2d(t_peak_fs=1.5))
    o.load(st)
    o.step(150)
    t, c, csd, f = _final(o)
    _, eedf = o.diag()
    vals = {k: f[k] for k in ("Zbar", "T_e_eV", "n_e")}
    vals["transmission"] = t["TRANS"] / t["INC"]
    vals["ke_e"] = t["KE_E"]
    vals["e_ion"] = t["ION"]
    for k in ("ION", "REC", "PH0", "AUG"):
        vals["count_" + k] = float(c[k])
    for z in range(len(csd)):
        vals[f"csd_{z}"] = float(csd[z])
    for b in range(len(eedf)):
        vals[f"eedf_{b}"] = float(eedf[b])
    return {"workload": cfg.name + ", 64 x 64 subdomain, pulse peak at 1.5 fs", "steps": 150}, vals


CASES = {"small_slab_500": case_small_slab_500, "kvac_history": case_kvac_history,
         "partial_early": case_partial_early, "subdomain_64x64": case_subdomain_64x64}


def main(names):
    global TABLES
    TABLES = P.standin_tables()
    out = json.load(open(OUT)) if os.path.exists(OUT) else {}
    out["_about"] = ("Oracle realizations of multi-step workloads: same initial state (input seed 0), "
                     f"Philox keys {KEYS}; per diagnostic the values, their mean and sample standard "
                     "deviation. Written by tests/golden/make_oracle_spread.py (oracle only).")
    for name in names:
        t0 = time.time()
        rows, meta = [], None
        for key in KEYS:
            meta, vals = CASES[name](key)
            rows.append(vals)
        diag = {}
        for k in rows[0]:
            v = np.array([r[k] for r in rows], dtype=np.float64)
            diag[k] = {"values": v.tolist(), "mean": float(v.mean()), "sd": float(v.std(ddof=1))}
        out[name] = {**meta, "keys": KEYS, "diagnostics": diag}
        print(f"{name}: {time.time() - t0:.1f} s", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
