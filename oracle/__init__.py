"""FP64 CPU oracle (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this package.  The product path (paper_1704_01202_gb300) never
does.  The C source is oracle/oracle.c; it is compiled here with gcc into
oracle/_build/liboracle.so.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NS, NZ = 5, 14
T_NAMES = ["KE_E", "KE_I", "ION", "PHOT", "INC", "TRANS", "KA_ESC", "ESC", "FIELD", "BACK", "RT_NUM", "RT_PEND"]
C_NAMES = ["ION", "ION_REJ", "REC", "PH0", "PH1", "PH2", "PH3", "PH4", "PART",
           "AUG", "KA", "PGT1", "ESC_E", "ESC_I", "EE", "EI"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over cells)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src),
                                                os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
           "-Wno-unused-function", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dt", C.c_double), ("rad_every", C.c_int), ("seed", C.c_uint64),
                ("cfl", C.c_double), ("n_ref", C.c_double), ("w_ion", C.c_double),
                ("m_ion", C.c_double), ("E_bulk", C.c_double), ("ipd_model", C.c_int),
                ("coulomb_log", C.c_double), ("flags", C.c_uint)]


class Tables(C.Structure):
    _fields_ = [("lotz_a", C.c_double * NS), ("lotz_b", C.c_double * NS), ("lotz_c", C.c_double * NS),
                ("E_bind", (C.c_double * NS) * NZ), ("tauK", (C.c_double * 2) * NZ),
                ("omegaK", (C.c_double * 2) * NZ), ("E_Ka", C.c_double * NZ),
                ("n_hv", C.c_int), ("hv_tab", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
                ("n_T", C.c_int), ("n_n", C.c_int), ("eos_T", C.POINTER(C.c_double)),
                ("eos_n", C.POINTER(C.c_double)), ("eos_Z", C.POINTER(C.c_double))]


class RT(C.Structure):
    _fields_ = [("coarsen", C.c_int), ("n_polar", C.c_int), ("n_azimuth", C.c_int), ("scheme", C.c_int)]


class Pulse(C.Structure):
    _fields_ = [("shape", C.c_int), ("I_peak", C.c_double), ("fwhm", C.c_double),
                ("t_peak", C.c_double), ("hv", C.c_double), ("bandwidth", C.c_double),
                ("n_bins", C.c_int), ("spot_sigma", C.c_double)]


_D = C.POINTER(C.c_double)
_U64 = C.POINTER(C.c_uint64)
_U32 = C.POINTER(C.c_uint32)
_I32 = C.POINTER(C.c_int32)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.POINTER(Params), C.POINTER(Tables)]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_set_pulse.argtypes = [C.c_void_p, C.POINTER(Pulse)]
            L.orc_set_step.argtypes = [C.c_void_p, C.c_uint32]
            L.orc_get_step.restype = C.c_uint32
            L.orc_get_step.argtypes = [C.c_void_p]
            L.orc_load_electrons.argtypes = [C.c_void_p, C.c_int, _D, _D, _D, _D, _U64]
            L.orc_load_ions.argtypes = [C.c_void_p, C.c_int, _D, _D, _D, _D, _I32, _I32, _U32]
            L.orc_n_electrons.restype = C.c_int
            L.orc_n_electrons.argtypes = [C.c_void_p]
            L.orc_n_ions.restype = C.c_int
            L.orc_n_ions.argtypes = [C.c_void_p]
            L.orc_get_electrons.argtypes = [C.c_void_p, _D, _D, _D, _D, _U64]
            L.orc_get_electron_scales.argtypes = [C.c_void_p, _D]
            L.orc_get_ions.argtypes = [C.c_void_p, _D, _D, _D, _D, _I32, _I32, _U32]
            for fn in ("orc_set_fields", "orc_get_fields", "orc_get_current",
                       "orc_set_photons", "orc_get_photons"):
                getattr(L, fn).argtypes = [C.c_void_p, _D]
            L.orc_step.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.orc_tallies.argtypes = [C.c_void_p, _D, _U64]
            L.orc_diag.argtypes = [C.c_void_p, _D, C.c_int, C.c_double, _D]
            L.orc_philox.argtypes = [_U32, _U32, _U32]
            L.orc_u01.restype = C.c_double
            L.orc_u01.argtypes = [C.c_uint32]
            L.orc_occ.restype = C.c_int
            L.orc_occ.argtypes = [C.c_int, C.c_int, _I]
            L.orc_ipd.restype = C.c_double
            L.orc_ipd.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
            L.orc_lotz.restype = C.c_double
            L.orc_lotz.argtypes = [C.POINTER(Tables), C.c_int, C.c_double, C.c_double]
            L.orc_coulomb_log.restype = C.c_double
            L.orc_coulomb_log.argtypes = [C.c_double, C.c_double, C.c_double]
            L.orc_field_speed.restype = C.c_double
            L.orc_field_speed.argtypes = [C.c_void_p]
            L.orc_collide.restype = C.c_int
            L.orc_collide.argtypes = [_D, _D] + [C.c_double] * 9 + [_D, C.c_void_p]
            L.orc_boris.argtypes = [_D, _D, _D, C.c_double, C.c_double]
            L.orc_pair_order.argtypes = [C.c_int, _U64, C.c_uint32, C.c_uint32, C.c_uint64, _I]
            L.orc_ee_pairs.restype = C.c_int
            L.orc_ee_pairs.argtypes = [C.c_int, _I, _I, _D]
            L.orc_deposit.argtypes = [C.c_int, C.c_int] + [C.c_double] * 10 + [_D]
            L.orc_rho.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, _D]
            L.orc_eos.restype = C.c_double
            L.orc_eos.argtypes = [C.POINTER(Tables), C.c_double, C.c_double]
            L.orc_trace.argtypes = [C.c_void_p, C.c_double]
            L.orc_set_rt.restype = C.c_int
            L.orc_set_rt.argtypes = [C.c_void_p, C.POINTER(RT)]
            L.orc_rt_ordinates.restype = C.c_int
            L.orc_rt_ordinates.argtypes = [C.c_void_p, _D, _D, _D]
            L.orc_rt_get.argtypes = [C.c_void_p, _D, _D, _D]
            L.orc_rt_set.argtypes = [C.c_void_p, _D, _D, _D]
            L.orc_rt_cells.argtypes = [C.c_void_p, _D, _D, _D, _D]
            L.orc_rt_line.argtypes = [_D, _D, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int,
                                      C.c_void_p, C.c_void_p, C.c_int, _D, _D]
            L.orc_trace_count.restype = C.c_int
            L.orc_trace_count.argtypes = [C.c_void_p]
            L.orc_trace_decisions.argtypes = [C.c_void_p, _U64]
            L.orc_trace_get.argtypes = [C.c_void_p, C.c_void_p]
            _lib = L
    return _lib


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def make_tables(tab: dict):
    """ctypes Tables from pic_inputs.standin_tables(); returns (struct, keepalive)."""
    t = Tables()
    for s in range(NS):
        t.lotz_a[s] = float(tab["lotz_a"][s])
        t.lotz_b[s] = float(tab["lotz_b"][s])
        t.lotz_c[s] = float(tab["lotz_c"][s])
    for z in range(NZ):
        for s in range(NS):
            t.E_bind[z][s] = float(tab["E_bind"][z, s])
        for k in range(2):
            t.tauK[z][k] = float(tab["tauK"][z, k])
            t.omegaK[z][k] = float(tab["omegaK"][z, k])
        t.E_Ka[z] = float(tab["E_Kalpha"][z])
    keep = [np.ascontiguousarray(tab["hv_tab"], dtype=np.float64),
            np.ascontiguousarray(tab["sigma_photo"], dtype=np.float64),
            np.ascontiguousarray(tab["eos_T"], dtype=np.float64),
            np.ascontiguousarray(tab["eos_n"], dtype=np.float64),
            np.ascontiguousarray(tab["eos_Zbar"], dtype=np.float64)]
    t.n_hv = keep[0].size
    t.hv_tab, t.sigma = _p(keep[0]), _p(keep[1])
    t.n_T, t.n_n = keep[2].size, keep[3].size
    t.eos_T, t.eos_n, t.eos_Z = _p(keep[2]), _p(keep[3]), _p(keep[4])
    return t, keep


M_AL_ME = 26.9815385 * 1822.888486

# one record of the decision trace (orc_near)
NEAR_DTYPE = np.dtype([("step", np.uint32), ("cell", np.int32), ("kind", np.int32), ("species", np.int32),
                       ("id", np.uint64), ("x", np.float64), ("thr", np.float64)])
NEAR_KINDS = {1: "COLL_ACC", 2: "ION_DRAW", 3: "ION_PAY", 4: "REC_K", 5: "REC_CAP", 6: "PH_EDGE",
              7: "PH_DRAW", 8: "PH_BIN", 9: "PH_PART", 10: "PH_ZF", 11: "DECAY", 12: "BRANCH",
              13: "REC_TAKE", 14: "EBULK", 15: "BASIS"}
# relative distance from a threshold within which an FP32 evaluation of a
# decision may differ from the FP64 one (a threshold flip)
FLIP_REL = 2.0 ** -20


class OracleSlab:
    """One slab simulated by the oracle."""

    def __init__(self, cfg, tables: dict, pulse=None):
        self.L = lib()
        self.cfg = cfg
        p = Params(nx=cfg.nx, ny=cfg.ny, dx=cfg.dx_nm, dy=cfg.dy_nm, dt=cfg.dt_fs,
                   rad_every=cfg.rad_every, seed=cfg.seed, cfl=cfg.cfl, n_ref=cfg.n_ref_cm3,
                   w_ion=cfg.w_ion, m_ion=cfg.m_ion_me, E_bulk=cfg.E_bulk_eV, ipd_model=cfg.ipd_model,
                   coulomb_log=cfg.coulomb_log, flags=cfg.flags)
        self._t, self._keep = make_tables(tables)
        self.h = self.L.orc_create(C.byref(p), C.byref(self._t))
        self.n_bins = 0
        if pulse is not None:
            self.set_pulse(pulse)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.L.orc_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def set_pulse(self, pl):
        P = Pulse(shape=pl.shape, I_peak=pl.I_peak_Wcm2, fwhm=pl.fwhm_fs, t_peak=pl.t_peak_fs,
                  hv=pl.hv_eV, bandwidth=pl.bandwidth_eV, n_bins=pl.n_bins, spot_sigma=pl.spot_sigma_nm)
        self.L.orc_set_pulse(self.h, C.byref(P))
        self.n_bins = pl.n_bins

    def load(self, st):
        eu = np.ascontiguousarray(st.eu, dtype=np.float64)
        ex = np.ascontiguousarray(st.eX, dtype=np.float64)
        ey = np.ascontiguousarray(st.eY, dtype=np.float64)
        ew = np.ascontiguousarray(st.ew, dtype=np.float64)
        eid = np.ascontiguousarray(st.eid, dtype=np.uint64)
        self.L.orc_load_electrons(self.h, ex.size, _p(ex), _p(ey), _p(eu), _p(ew), _p(eid, C.c_uint64))
        iu = np.ascontiguousarray(st.iu, dtype=np.float64)
        ix = np.ascontiguousarray(st.iX, dtype=np.float64)
        iy = np.ascontiguousarray(st.iY, dtype=np.float64)
        zf = np.ascontiguousarray(st.izf, dtype=np.float64)
        Z = np.ascontiguousarray(st.iZ, dtype=np.int32)
        nK = np.ascontiguousarray(st.inK, dtype=np.int32)
        iid = np.ascontiguousarray(st.iid, dtype=np.uint32)
        self.L.orc_load_ions(self.h, ix.size, _p(ix), _p(iy), _p(iu), _p(zf), _p(Z, C.c_int32),
                             _p(nK, C.c_int32), _p(iid, C.c_uint32))

    def set_step(self, n):
        self.L.orc_set_step(self.h, n)

    @property
    def step_index(self):
        return self.L.orc_get_step(self.h)

    def step(self, n=1, threads=0):
        self.L.orc_step(self.h, n, threads)

    def electrons(self):
        n = self.L.orc_n_electrons(self.h)
        X, Y, w = np.zeros(n), np.zeros(n), np.zeros(n)
        u = np.zeros((n, 3))
        i = np.zeros(n, dtype=np.uint64)
        cs = np.zeros(n)
        if n:
            self.L.orc_get_electrons(self.h, _p(X), _p(Y), _p(u), _p(w), _p(i, C.c_uint64))
            self.L.orc_get_electron_scales(self.h, _p(cs))
        return dict(X=X, Y=Y, u=u, w=w, id=i, cscale=cs)

    def ions(self):
        n = self.L.orc_n_ions(self.h)
        X, Y, zf = np.zeros(n), np.zeros(n), np.zeros(n)
        u = np.zeros((n, 3))
        Z = np.zeros(n, dtype=np.int32)
        nK = np.zeros(n, dtype=np.int32)
        i = np.zeros(n, dtype=np.uint32)
        if n:
            self.L.orc_get_ions(self.h, _p(X), _p(Y), _p(u), _p(zf), _p(Z, C.c_int32),
                                _p(nK, C.c_int32), _p(i, C.c_uint32))
        return dict(X=X, Y=Y, u=u, zf=zf, Z=Z, nK=nK, id=i)

    def _grid(self):
        return self.cfg.ny, self.cfg.nx + 1

    def set_fields(self, f: dict):
        a = np.ascontiguousarray(np.stack([f[k] for k in ("ex", "ey", "ez", "bx", "by", "bz")]),
                                 dtype=np.float64)
        self.L.orc_set_fields(self.h, _p(a))

    def fields(self):
        a = np.zeros((6,) + self._grid())
        self.L.orc_get_fields(self.h, _p(a))
        return dict(zip(("ex", "ey", "ez", "bx", "by", "bz"), a))

    def current(self):
        a = np.zeros((3,) + self._grid())
        self.L.orc_get_current(self.h, _p(a))
        return a

    def set_photons(self, ph):
        a = np.ascontiguousarray(ph, dtype=np.float64)
        self.L.orc_set_photons(self.h, _p(a))

    def photons(self):
        a = np.zeros((self.cfg.ny, self.cfg.nx, max(self.n_bins, 1)))
        if self.n_bins:
            self.L.orc_get_photons(self.h, _p(a))
        return a

    def tallies(self):
        t = np.zeros(len(T_NAMES))
        c = np.zeros(len(C_NAMES), dtype=np.uint64)
        self.L.orc_tallies(self.h, _p(t), _p(c, C.c_uint64))
        return dict(zip(T_NAMES, t)), dict(zip(C_NAMES, (int(x) for x in c)))

    def set_rt(self, coarsen=5, n_polar=4, n_azimuth=2, scheme=0):
        """Switch on radiation transport (see orc_set_rt in oracle.h)."""
        if self.n_bins == 0:
            raise ValueError("radiation transport needs a pulse")
        r = RT(coarsen=coarsen, n_polar=n_polar, n_azimuth=n_azimuth, scheme=scheme)
        if self.L.orc_set_rt(self.h, C.byref(r)) != 0:
            raise ValueError("invalid radiation transport setting")
        self.rt = r
        self.nrx = self.cfg.nx // coarsen
        self.nry = self.cfg.ny // coarsen if self.cfg.ny > 1 else 1
        mu, vy, w = np.zeros(1 + 16 * 16), np.zeros(1 + 16 * 16), np.zeros(1 + 16 * 16)
        self.nord = self.L.orc_rt_ordinates(self.h, _p(mu), _p(vy), _p(w))
        self.ordinates = (mu[:self.nord], vy[:self.nord], w[:self.nord])

    def rt_field(self):
        shp = (self.nord, self.n_bins, self.nry, self.nrx)
        F, Gx, Gy = np.zeros(shp), np.zeros(shp), np.zeros(shp)
        self.L.orc_rt_get(self.h, _p(F), _p(Gx), _p(Gy))
        return F, Gx, Gy

    def set_rt_field(self, F, Gx=None, Gy=None):
        F = np.ascontiguousarray(F, dtype=np.float64)
        Gx = np.zeros_like(F) if Gx is None else np.ascontiguousarray(Gx, dtype=np.float64)
        Gy = np.zeros_like(F) if Gy is None else np.ascontiguousarray(Gy, dtype=np.float64)
        self.L.orc_rt_set(self.h, _p(F), _p(Gx), _p(Gy))

    def rt_cells(self):
        nc = self.cfg.nx * self.cfg.ny
        chi, emc, w, dE = np.zeros((nc, self.n_bins)), np.zeros(nc), np.zeros(nc), np.zeros(nc)
        self.L.orc_rt_cells(self.h, _p(chi), _p(emc), _p(w), _p(dE))
        return dict(chi=chi, emc=emc, w=w, dE=dE)

    def trace(self, rel=FLIP_REL):
        """Start the decision trace (rel <= 0 stops it): every threshold
        decision of the following steps is counted, and recorded when it
        lies within rel (relative) of its threshold."""
        self.L.orc_trace(self.h, rel)

    def near(self):
        """Recorded near-threshold decisions (NEAR_DTYPE records) and the
        counts of Monte-Carlo draws and of other decisions."""
        n = self.L.orc_trace_count(self.h)
        out = np.zeros(n, dtype=NEAR_DTYPE)
        if n:
            self.L.orc_trace_get(self.h, out.ctypes.data_as(C.c_void_p))
        d = np.zeros(2, dtype=np.uint64)
        self.L.orc_trace_decisions(self.h, _p(d, C.c_uint64))
        return out, int(d[0]), int(d[1])

    def diag(self, n_E=64, E_max=1e4):
        csd = np.zeros(NZ)
        eedf = np.zeros(n_E)
        self.L.orc_diag(self.h, _p(csd), n_E, E_max, _p(eedf))
        return csd, eedf


# ---- thin wrappers of the building blocks (for pins) ----

def philox(ctr, key):
    L = lib()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    L.orc_philox(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(o, C.c_uint32))
    return o


def occ(nb, nk):
    o = np.zeros(NS, dtype=np.int32)
    ok = lib().orc_occ(nb, nk, _p(o, C.c_int))
    return o if ok else None


def ipd(model, z, n_e, n_i, T_e, zbar):
    return lib().orc_ipd(model, z, n_e, n_i, T_e, zbar)


def coulomb_log(n_e, T_e, zbar):
    return lib().orc_coulomb_log(n_e, T_e, zbar)


def field_speed(cfg):
    """Speed (nm/fs) of the oracle's Yee update for a slab configuration."""
    p = Params(nx=cfg.nx, ny=cfg.ny, dx=cfg.dx_nm, dy=cfg.dy_nm, dt=cfg.dt_fs, rad_every=cfg.rad_every,
               seed=cfg.seed, cfl=cfg.cfl, n_ref=cfg.n_ref_cm3, w_ion=cfg.w_ion, m_ion=cfg.m_ion_me,
               E_bulk=cfg.E_bulk_eV, ipd_model=cfg.ipd_model, coulomb_log=cfg.coulomb_log, flags=cfg.flags)
    return lib().orc_field_speed(C.byref(p))


class TableHandle:
    def __init__(self, tab):
        self.t, self.keep = make_tables(tab)


def lotz(th: TableHandle, z, dE, E):
    return lib().orc_lotz(C.byref(th.t), z, dE, E)


def eos(th: TableHandle, n_i, T_e):
    return lib().orc_eos(C.byref(th.t), n_i, T_e)


def collide(ua, ub, ma, mb, qa, qb, wa, wb, n_l, lnL, dtc, r):
    a = np.array(ua, dtype=np.float64)
    b = np.array(ub, dtype=np.float64)
    rr = np.array(r, dtype=np.float64)
    did = lib().orc_collide(_p(a), _p(b), ma, mb, qa, qb, wa, wb, n_l, lnL, dtc, _p(rr), None)
    return a, b, did


def boris(u, e, b, qm, dt):
    uu = np.array(u, dtype=np.float64)
    ee = np.array(e, dtype=np.float64)
    bb = np.array(b, dtype=np.float64)
    lib().orc_boris(_p(uu), _p(ee), _p(bb), qm, dt)
    return uu


def pair_order(ids, step, purpose, seed):
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    perm = np.zeros(ids.size, dtype=np.int32)
    lib().orc_pair_order(ids.size, _p(ids, C.c_uint64), step, purpose, seed, _p(perm, C.c_int))
    return perm


def ee_pairs(n):
    pa = np.zeros(n + 3, dtype=np.int32)
    pb = np.zeros(n + 3, dtype=np.int32)
    fr = np.zeros(n + 3)
    m = lib().orc_ee_pairs(n, _p(pa, C.c_int), _p(pb, C.c_int), _p(fr))
    return pa[:m], pb[:m], fr[:m]


def rt_line(f, g, nu, scheme=0, periodic=False, fin=None, gin=None, gt=None):
    """One advection of a line (orc_rt_line): returns (f, g, gt, inflow, outflow)."""
    f = np.array(f, dtype=np.float64)
    g = np.array(g, dtype=np.float64)
    gt = None if gt is None else np.array(gt, dtype=np.float64)
    fin = None if fin is None else np.ascontiguousarray(fin, dtype=np.float64)
    gin = None if gin is None else np.ascontiguousarray(gin, dtype=np.float64)
    i, o = np.zeros(1), np.zeros(1)
    lib().orc_rt_line(_p(f), _p(g), None if gt is None else gt.ctypes.data_as(C.c_void_p), f.size, nu, scheme,
                      1 if periodic else 0, None if fin is None else fin.ctypes.data_as(C.c_void_p),
                      None if gin is None else gin.ctypes.data_as(C.c_void_p), 0 if fin is None else fin.size,
                      _p(i), _p(o))
    return f, g, gt, float(i[0]), float(o[0])


def deposit(nx, ny, dx, dy, dt, X0, Y0, X1, Y1, vz, vy, qw, j3=None):
    if j3 is None:
        j3 = np.zeros((3, ny, nx + 1))
    lib().orc_deposit(nx, ny, dx, dy, dt, X0, Y0, X1, Y1, vz, vy, qw, _p(j3))
    return j3


def rho(nx, ny, X, Y, qw, out=None):
    if out is None:
        out = np.zeros((ny, nx + 1))
    lib().orc_rho(nx, ny, X, Y, qw, _p(out))
    return out
