"""Helpers for comparing the CUDA path with the oracle particle by particle."""
import numpy as np

# tolerance of per-particle momenta (relative, FP32 state vs FP64 oracle)
U_RTOL = 1e-5
# floor of the momentum scale (u = gamma v / c) for particles at rest
U_FLOOR = 1e-6


def match(a_ids, b_ids):
    """Indices that put both id lists in the same order; asserts equal sets."""
    ia, ib = np.argsort(a_ids, kind="stable"), np.argsort(b_ids, kind="stable")
    return ia, ib, np.array_equal(a_ids[ia], b_ids[ib])


def momentum_errors(u_gpu, u_ref):
    du = np.linalg.norm(u_gpu.astype(np.float64) - u_ref, axis=1)
    return du / (np.linalg.norm(u_ref, axis=1) + U_FLOOR)


def compare_state(g_e, o_e, g_i, o_i, nx, ny):
    """Per-particle comparison; returns a dict of measures."""
    out = {}
    ia, ib, same = match(g_e["id"], o_e["id"])
    out["e_same_ids"] = same
    out["n_e"] = (g_e["id"].size, o_e["id"].size)
    if same:
        err = momentum_errors(g_e["u"][ia], o_e["u"][ib])
        out["e_bad"] = int((err > U_RTOL).sum())
        out["e_err_max"] = float(err.max()) if err.size else 0.0
        out["e_err_p999"] = float(np.quantile(err, 0.999)) if err.size else 0.0
        wg, wo = g_e["w"][ia].astype(np.float64), o_e["w"][ib]
        out["w_err"] = float((np.abs(wg - wo) / np.maximum(wo, 1e-30)).max()) if wg.size else 0.0
        dx = np.abs(g_e["X"][ia] - o_e["X"][ib])
        out["x_err"] = float(dx.max()) if dx.size else 0.0
    ja, jb, same_i = match(g_i["id"], o_i["id"])
    out["i_same_ids"] = same_i
    if same_i:
        out["Z_mismatch"] = int((g_i["Z"][ja] != o_i["Z"][jb]).sum())
        out["nK_mismatch"] = int((g_i["nK"][ja] != o_i["nK"][jb]).sum())
        out["zf_err"] = float(np.abs(g_i["zf"][ja] - o_i["zf"][jb]).max()) if ja.size else 0.0
        erri = momentum_errors(g_i["u"][ja], o_i["u"][jb])
        out["i_bad"] = int((erri > U_RTOL).sum())
        out["i_err_max"] = float(erri.max()) if erri.size else 0.0
    return out


def _cells_of(cfg, X, Y):
    return np.floor(Y).astype(np.int64) * cfg.nx + np.floor(X).astype(np.int64)


def sampled_cell_state(cfg, st, cells):
    """The particles of `cells` (sorted cell indices of a large slab) as a
    len(cells) x 1 slab of their own, cell k of the list becoming cell k,
    with the in-cell offsets, momenta, weights and ids kept."""
    import pic_inputs as P
    rank = np.full(cfg.ncell, -1, dtype=np.int64)
    rank[cells] = np.arange(len(cells))
    ce, ci = _cells_of(cfg, st.eX, st.eY), _cells_of(cfg, st.iX, st.iY)
    me, mi = rank[ce] >= 0, rank[ci] >= 0
    sub_cfg = P.SlabConfig(**{**cfg.to_dict(), "nx": len(cells), "ny": 1})
    sub = P.ParticleState(
        eX=rank[ce[me]] + (st.eX[me] - np.floor(st.eX[me])), eY=np.full(me.sum(), 0.5),
        eu=st.eu[me], ew=st.ew[me], eid=st.eid[me],
        iX=rank[ci[mi]] + (st.iX[mi] - np.floor(st.iX[mi])), iY=np.full(mi.sum(), 0.5),
        iu=st.iu[mi], izf=st.izf[mi], iZ=st.iZ[mi], inK=st.inK[mi], iid=st.iid[mi])
    return sub_cfg, sub


def select_cells(cfg, e, i, cells):
    """The electrons and ions of a device read-back that sit in `cells`."""
    keep = np.zeros(cfg.ncell, dtype=bool)
    keep[cells] = True
    se = keep[_cells_of(cfg, e["X"], e["Y"])]
    si = keep[_cells_of(cfg, i["X"], i["Y"])]
    return {k: v[se] for k, v in e.items()}, {k: v[si] for k, v in i.items()}


# ---- classification of mismatches as threshold flips ----

REC_TAKE = 13      # oracle decision kind: recombination weight reaching an electron's whole weight

def _cell_of_ids(cfg, X, Y):
    return (np.floor(Y).astype(np.int64) * cfg.nx + np.floor(X).astype(np.int64)) if cfg.ny > 1 \
        else np.floor(X).astype(np.int64)


def classify(cfg, st, g_e, o_e, g_i, o_i, near, n_draw, n_dec):
    """Every difference between the device's state after one step and the
    oracle's, classified against the oracle's decision trace of that step.

    Momenta: an electron's error is taken relative to the momentum scale of
    the binary collisions that produced it (the oracle's cscale: the larger
    |u| of itself and each e-e partner, before the collision), since an FP32
    evaluation of a collision rounds both outgoing momenta at the pair's
    scale; the error of a slow electron scattered by a fast one is relative
    to the fast one.

    A decision that lies within 2^-20 of its threshold (|x - thr| <= 2^-20
    |thr|: the definition of a threshold flip used here) may go the other
    way in FP32; its consequences stay inside its cell but spread there (the
    impact-ionization payment and the collision energy restore scale every
    electron of the cell, an extra or missing ionization moves the
    recombination count, photons taken from a bin change what later ions
    see).  So a difference is explained when the cell its particle sat in at
    the start of the step holds a near-threshold decision, and the flips
    counted are the near decisions of the cells that differ.  st is the
    state both sides started from (positions name the cells).
    Returns a dict: draws, decisions, near, flip_cells, flips, unexplained
    (a list of descriptions; empty when every difference is a flip)."""
    ecell = dict(zip(st.eid.tolist(), _cell_of_ids(cfg, st.eX, st.eY).tolist()))
    icell = dict(zip(st.iid.astype(np.uint64).tolist(), _cell_of_ids(cfg, st.iX, st.iY).tolist()))

    def cell_of_e(eid):
        eid = int(eid)
        if eid in ecell:
            return ecell[eid]
        return icell.get(eid & 0xffffffff, -1)         # created: at its parent ion

    near_cells = {}
    for r in near:
        near_cells.setdefault(int(r["cell"]), []).append(r)
    unexplained, diff_cells = [], set()

    def note(what, cell):
        if cell in near_cells:
            diff_cells.add(cell)
        else:
            unexplained.append(f"{what} (cell {cell})")

    ge_ids, oe_ids = set(g_e["id"].tolist()), set(o_e["id"].tolist())
    for eid in ge_ids ^ oe_ids:
        note(f"electron {eid} on one side only", cell_of_e(eid))
    gi_ids, oi_ids = set(g_i["id"].tolist()), set(o_i["id"].tolist())
    for iid in gi_ids ^ oi_ids:
        note(f"ion {iid} on one side only", icell.get(int(iid), -1))
    # common electrons: momentum and weight
    ce = np.array(sorted(ge_ids & oe_ids), dtype=np.uint64)
    if ce.size:
        ga, oa = np.argsort(g_e["id"]), np.argsort(o_e["id"])
        gk = ga[np.searchsorted(g_e["id"][ga], ce)]
        ok = oa[np.searchsorted(o_e["id"][oa], ce)]
        du = np.linalg.norm(g_e["u"][gk].astype(np.float64) - o_e["u"][ok], axis=1)
        scale = np.linalg.norm(o_e["u"][ok], axis=1)
        if "cscale" in o_e:
            scale = np.maximum(scale, o_e["cscale"][ok])
        err = du / (scale + U_FLOOR)
        wg, wo = g_e["w"][gk].astype(np.float64), o_e["w"][ok]
        werr = np.abs(wg - wo) / np.maximum(np.abs(wo), 1e-30)
        for k in np.nonzero((err > U_RTOL) | (werr > U_RTOL))[0]:
            uo = o_e["u"][ok[k]]
            note(f"electron {int(ce[k])} momentum {err[k]:.2e} |u| {np.linalg.norm(uo):.3e} weight {werr[k]:.2e}",
                 cell_of_e(ce[k]))
    ci = np.array(sorted(gi_ids & oi_ids), dtype=np.uint64)
    if ci.size:
        ga, oa = np.argsort(g_i["id"]), np.argsort(o_i["id"])
        gk = ga[np.searchsorted(g_i["id"][ga].astype(np.uint64), ci)]
        ok = oa[np.searchsorted(o_i["id"][oa].astype(np.uint64), ci)]
        err = momentum_errors(g_i["u"][gk], o_i["u"][ok])
        bad = (g_i["Z"][gk] != o_i["Z"][ok]) | (g_i["nK"][gk] != o_i["nK"][ok]) | \
              (np.abs(g_i["zf"][gk].astype(np.float64) - o_i["zf"][ok]) > U_RTOL) | (err > U_RTOL)
        for k in np.nonzero(bad)[0]:
            note(f"ion {int(ci[k])} Z {g_i['Z'][gk[k]]}/{o_i['Z'][ok[k]]} nK {g_i['nK'][gk[k]]}/{o_i['nK'][ok[k]]} "
                 f"momentum {err[k]:.2e}", icell.get(int(ci[k]), -1))
    # a recombination that takes an electron's whole weight on one side and
    # leaves a rounding-size remainder on the other changes no charge state
    # and no event count: counted apart from the event flips
    flips = sum(1 for c in diff_cells for r in near_cells[c] if int(r["kind"]) != REC_TAKE)
    remainders = sum(1 for c in diff_cells for r in near_cells[c] if int(r["kind"]) == REC_TAKE)
    import oracle
    kinds = [(oracle.NEAR_KINDS.get(int(r["kind"]), int(r["kind"])), int(r["cell"]), float(r["x"]), float(r["thr"]))
             for c in sorted(diff_cells) for r in near_cells[c]]
    return {"draws": n_draw, "decisions": n_dec, "near": len(near), "flip_cells": sorted(diff_cells),
            "flips": flips, "remainders": remainders, "flip_kinds": kinds, "unexplained": unexplained}


def flip_summary(cls):
    kinds = cls.get("flip_kinds", [])
    return (f"flips: {cls['flips']} of {cls['draws']} draws ({cls['decisions']} other decisions), "
            f"{cls.get('remainders', 0)} recombination remainders, "
            f"{cls['near']} near-threshold decisions, cells with differences {cls['flip_cells'][:8]} {kinds[:8]}")


# the bound on threshold flips: fewer than 1e-5 of the draws
FLIP_SHARE = 1e-5


def assert_flip_parity(cfg, st, g_e, g_i, o, counts=None, o_counts=None, keys=()):
    """One step of both sides from the same state `st`, the oracle run with
    its decision trace on (OracleSlab.trace before the step): every
    difference must be a threshold flip, and flips must stay below 1e-5 of
    the step's Monte-Carlo draws.  With the device's and the oracle's event
    counters given, the counts of `keys` must be equal, or differ by no more
    than the ions of the cells that flipped.  Returns the classification."""
    near, n_draw, n_dec = o.near()
    o_e, o_i = o.electrons(), o.ions()
    cls = classify(cfg, st, g_e, o_e, g_i, o_i, near, n_draw, n_dec)
    print("\n" + flip_summary(cls))
    assert not cls["unexplained"], (flip_summary(cls), cls["unexplained"][:20])
    assert cls["flips"] <= FLIP_SHARE * cls["draws"], flip_summary(cls)
    if counts is not None:
        ci = _cell_of_ids(cfg, st.iX, st.iY)
        slack = int(np.isin(ci, np.array(cls["flip_cells"], dtype=np.int64)).sum())
        for k in keys:
            assert abs(int(counts[k]) - int(o_counts[k])) <= slack, (k, counts[k], o_counts[k], flip_summary(cls))
    return cls


# ---- multi-step runs against the oracle's own spread ----

# |device - mean| <= SPREAD_K sd sqrt(1 + 1/n) + floor, with mean and sd of n
# oracle realizations: 4.0 is about the 99.5 % two-sided quantile of
# Student's t with 7 degrees of freedom (n = 8), so a device run that is one
# more realization of the method fails a given diagnostic by chance about
# once in 200
SPREAD_K = 4.0


def oracle_spread(case):
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_spread.json")
    return json.load(open(path))[case]


def spread_violations(case, values, floors=None, default_floor=0.0):
    """Diagnostics of a device run (dict name -> value) outside the spread
    of the oracle's realizations of `case` (tests/golden/oracle_spread.json);
    floors: absolute floor per name (default_floor otherwise).  Returns
    {name: (value, mean, bound)} of the violations and prints the table."""
    g = oracle_spread(case)["diagnostics"]
    floors = floors or {}
    bad = {}
    print(f"\n{case}: diagnostic, device, oracle mean, oracle sd, |z|")
    for name, v in values.items():
        d = g[name]
        n = len(d["values"])
        scale = d["sd"] * (1.0 + 1.0 / n) ** 0.5
        bound = SPREAD_K * scale + floors.get(name, default_floor)
        z = abs(v - d["mean"]) / scale if scale > 0 else float("inf") if v != d["mean"] else 0.0
        print(f"  {name:14s} {v:14.6g} {d['mean']:14.6g} {d['sd']:11.3g} {z:7.2f}")
        if abs(v - d["mean"]) > bound:
            bad[name] = (v, d["mean"], bound)
    return bad


def spread_hist_l1(case, prefix, hist):
    """L1 distance of a device histogram (csd_* or eedf_* bins of `case`)
    from the mean of the oracle's realizations, and the bound it must stay
    within: 1.5 times the largest distance of one realization from the mean
    of the other seven (the realizations' own scatter).  Returns (d, bound)."""
    g = oracle_spread(case)["diagnostics"]
    names = sorted((k for k in g if k.startswith(prefix + "_")), key=lambda k: int(k.split("_")[1]))
    V = np.array([g[k]["values"] for k in names])          # bins x realizations
    mean = V.mean(axis=1)
    n = V.shape[1]
    loo = [np.abs(V[:, j] - (V.sum(axis=1) - V[:, j]) / (n - 1)).sum() for j in range(n)]
    d = float(np.abs(np.asarray(hist, dtype=np.float64)[:len(names)] - mean).sum())
    print(f"  {prefix} L1 from the oracle mean {d:.3e}; realizations' own {min(loo):.3e} .. {max(loo):.3e}")
    return d, 1.5 * max(loo)


def welch_violations(case, dev_rows, floors=None, default_floor=0.0):
    """Eight device realizations (dev_rows: one dict of diagnostics per
    Philox key 1..8) against the oracle's eight of `case`: for every
    diagnostic |mean_dev - mean_oracle| <= SPREAD_K * s + floor with
    s = sqrt(sd_dev^2 / n_dev + sd_oracle^2 / n_oracle) (Welch's standard
    error of the difference of two means; a systematic difference between
    the two implementations shows here at a fraction of one realization's
    scatter).  Returns {name: (mean_dev, mean_oracle, bound)} of the
    violations and prints the table."""
    g = oracle_spread(case)["diagnostics"]
    floors = floors or {}
    bad = {}
    print(f"\n{case}: diagnostic, device mean, oracle mean, standard error, |t|")
    for name in dev_rows[0]:
        v = np.array([r[name] for r in dev_rows], dtype=np.float64)
        o = g[name]
        se = float(np.sqrt(v.var(ddof=1) / v.size + o["sd"] ** 2 / len(o["values"])))
        diff = abs(v.mean() - o["mean"])
        t = diff / se if se > 0 else (0.0 if diff == 0 else float("inf"))
        print(f"  {name:14s} {v.mean():14.6g} {o['mean']:14.6g} {se:11.3g} {t:7.2f}")
        if diff > SPREAD_K * se + floors.get(name, default_floor):
            bad[name] = (float(v.mean()), o["mean"], SPREAD_K * se + floors.get(name, default_floor))
    return bad


def welch_hist_l1(case, prefix, dev_hists):
    """L1 distance between the mean histogram (csd_* or eedf_* bins) of
    eight device realizations and the oracle's eight, and its bound: 1.5
    times the largest distance of one oracle realization from the mean of
    the other seven, scaled to a difference of two eight-run means
    (sqrt(2 / 8) / sqrt(1 + 1/7)).  Returns (d, bound)."""
    g = oracle_spread(case)["diagnostics"]
    names = sorted((k for k in g if k.startswith(prefix + "_")), key=lambda k: int(k.split("_")[1]))
    V = np.array([g[k]["values"] for k in names])
    n = V.shape[1]
    loo = [np.abs(V[:, j] - (V.sum(axis=1) - V[:, j]) / (n - 1)).sum() for j in range(n)]
    dm = np.mean(np.asarray(dev_hists, dtype=np.float64)[:, :len(names)], axis=0)
    d = float(np.abs(dm - V.mean(axis=1)).sum())
    bound = 1.5 * max(loo) * np.sqrt(2.0 / n) / np.sqrt(1.0 + 1.0 / (n - 1))
    print(f"  {prefix} L1 between the mean histograms {d:.3e} (bound {bound:.3e})")
    return d, bound


def key_realizations(run, keys=range(1, 9)):
    """run(key) -> dict of diagnostics, for the Philox keys of the oracle's
    spread (the same initial state, seed 0 of the input generator)."""
    return [run(k) for k in keys]
