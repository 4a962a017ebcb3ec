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
