"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This module holds no arithmetic of the simulation method itself.  It makes:

* the stand-in atomic tables (the paper's LANL cross sections, Lotz constants,
  binding energies, K-vacancy lifetimes and SCFLY equation of state are not
  available; every table here is synthetic and labelled as such),
* slab configurations with the shapes of the paper's workloads,
* seeded initial particle states (Maxwellian electrons with a hot beam,
  Al3+ ions), rounded to values that FP32 stores exactly so that an FP32
  and an FP64 implementation start from bit-identical inputs,
* pulse descriptions.

Units: lengths nm, times fs, energies eV, momenta u = gamma*v/c, particle
weights in units of n_ref * V_cell (n_ref = the initial ion density).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

Z_AL = 13
N_SUB = 5                      # 1s, 2s, 2p, 3s, 3p
SUB_CAP = (2, 2, 6, 2, 6)
SUB_N = (1, 2, 2, 3, 3)
ME_C2_EV = 510998.95
M_AL_ME = 26.9815385 * 1822.888486   # Al mass in electron masses
RYD_EV = 13.605693

# --------------------------------------------------------------------------
# stand-in atomic tables
# --------------------------------------------------------------------------


def _config(nb: int, nk: int = 0):
    """Occupation of (1s,2s,2p,3s,3p) for nb bound electrons with nk extra
    K vacancies (lowest-energy filling otherwise)."""
    occ = [0] * N_SUB
    k = min(nb, 2) - nk
    if k < 0:
        return None
    occ[0] = k
    rest = nb - k
    for s in range(1, N_SUB):
        take = min(rest, SUB_CAP[s])
        occ[s] = take
        rest -= take
    if rest:
        return None
    return occ


def _slater_energy(occ, z=Z_AL):
    """Total electronic energy (eV, negative) of a configuration from Slater's
    1930 screening rules (s and p of one shell grouped)."""
    shells = {1: occ[0], 2: occ[1] + occ[2], 3: occ[3] + occ[4]}
    e = 0.0
    for n, cnt in shells.items():
        if cnt == 0:
            continue
        same = cnt - 1
        if n == 1:
            sigma = 0.30 * same
        else:
            sigma = 0.35 * same + 0.85 * shells.get(n - 1, 0) \
                + 1.0 * sum(shells.get(m, 0) for m in range(1, n - 1))
        zeff = z - sigma
        e -= cnt * RYD_EV * zeff * zeff / (n * n)
    return e


def standin_tables() -> dict:
    """Synthetic stand-ins for the paper's atomic data (NOT the paper's data).

    * E_bind[z][s]: binding of subshell s in charge state z (lowest-energy
      configuration), as the Slater total-energy difference between the
      configuration and the one with that electron removed.  K binding is
      scaled by (1 - 0.04 (N_b - 1)/12) so that cold Al sits at ~1560 eV
      (the cold K edge the paper quotes) while the H-like value is kept.
    * Lotz a=4.5e-14 cm^2 eV^2, b=0 (1s) / 0.3, c=0.5 (n>=2).
    * sigma_photo[s][hv]: Kramers-like power laws, per electron, cm^2.
    * tauK[N_b][nK-1], omegaK: K-vacancy lifetime (fs) and fluorescence
      yield from rates proportional to L-electron pair/2p counts, scaled to
      ~1.2 fs and omega=0.04 at a full L shell; for N_b >= 10 linearly
      interpolated between N_b=10 and the neutral value (the paper's rule
      for building the table).  tau <= 0 means no decay channel.
    * E_Kalpha[z] = E_bind[z][1s] - E_bind[z][2p] (or 1s only if no 2p).
    * EOS Zbar(n, T) = 3 + 10 x^1.5/(1+x^1.5), x = T/T0(n), T0 = 131 eV at
      solid density (gives Zbar~7 at 100 eV), Zbar = 3 (pressure-ionized
      baseline) at T=0.
    """
    nz = Z_AL + 1
    e_bind = np.zeros((nz, N_SUB))
    for z in range(Z_AL):
        nb = Z_AL - z
        occ = _config(nb)
        e0 = _slater_energy(occ)
        for s in range(N_SUB):
            if occ[s] == 0:
                continue
            o2 = list(occ)
            o2[s] -= 1
            eb = _slater_energy(o2) - e0
            if s == 0:
                eb *= 1.0 - 0.04 * (nb - 1) / 12.0
            e_bind[z, s] = eb
    # binding energies for empty subshells of a charge state are still needed
    # by photoionization of hollow ions and by the Auger rule: fill them with
    # the value of the nearest charge state that occupies the subshell.
    for s in range(N_SUB):
        for z in range(Z_AL):
            if e_bind[z, s] == 0.0:
                cands = [zz for zz in range(Z_AL) if e_bind[zz, s] > 0]
                if cands:
                    zz = min(cands, key=lambda q: abs(q - z))
                    e_bind[z, s] = e_bind[zz, s]

    lotz_a = np.full(N_SUB, 4.5e-14)
    lotz_b = np.array([0.0, 0.3, 0.3, 0.3, 0.3])
    lotz_c = np.array([0.0, 0.5, 0.5, 0.5, 0.5])

    hv_tab = np.geomspace(800.0, 20000.0, 96)
    ref = 1560.0
    sig0 = np.array([8.0e-20, 5.0e-21, 2.0e-21, 4.0e-22, 3.0e-22])
    expo = np.array([2.75, 2.6, 3.0, 2.6, 3.0])
    sigma_photo = np.array([sig0[s] * (ref / hv_tab) ** expo[s] for s in range(N_SUB)])

    tau0, om0 = 1.2, 0.04
    ga0 = (1.0 - om0) / tau0
    gx0 = om0 / tau0
    tauK = np.zeros((nz, 2))
    omegaK = np.ones((nz, 2))
    for nk in (1, 2):
        for nb in range(0, nz):
            occ = _config(nb, nk)
            if occ is None:
                continue
            nl = occ[1] + occ[2]
            ga = ga0 * nl * (nl - 1) / 56.0 * nk
            gx = gx0 * occ[2] / 6.0 * nk
            if ga + gx > 0:
                tauK[nb, nk - 1] = 1.0 / (ga + gx)
                omegaK[nb, nk - 1] = gx / (ga + gx)
        # N_b >= 10: linear between N_b = 10 and the neutral value
        t10, t13 = tauK[10, nk - 1], tauK[13, nk - 1]
        o10, o13 = omegaK[10, nk - 1], omegaK[13, nk - 1]
        for nb in (11, 12):
            f = (nb - 10) / 3.0
            tauK[nb, nk - 1] = t10 + f * (t13 - t10)
            omegaK[nb, nk - 1] = o10 + f * (o13 - o10)

    e_ka = np.zeros(nz)
    for z in range(Z_AL):
        e_ka[z] = e_bind[z, 0] - e_bind[z, 2]

    eos_n = np.geomspace(1.0e22, 1.0e24, 5)
    eos_T = np.linspace(0.0, 3000.0, 301)
    zb = np.zeros((eos_n.size, eos_T.size))
    for a, n in enumerate(eos_n):
        t0 = 131.0 * (n / 6.0e22) ** 0.2
        x = eos_T / t0
        zb[a] = 3.0 + 10.0 * x ** 1.5 / (1.0 + x ** 1.5)
    return dict(
        n_sub=N_SUB,
        lotz_a=lotz_a, lotz_b=lotz_b, lotz_c=lotz_c,
        E_bind=e_bind,
        hv_tab=hv_tab, sigma_photo=sigma_photo,
        tauK=tauK, omegaK=omegaK, E_Kalpha=e_ka,
        eos_n=eos_n, eos_T=eos_T, eos_Zbar=zb,
    )


# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------

# process switches (bit flags; both implementations use the same meaning)
F_COLL_EE = 1
F_COLL_EI = 2
F_IONIZE = 4
F_RECOMB = 8
F_PHOTO = 16
F_DECAY = 32
F_PUSH = 64
F_FIELD = 128
F_ALL = 255
F_THERM = 256      # forced-thermalization variant (Sec. VI C), off in F_ALL

IPD_NONE, IPD_EK, IPD_SP = 0, 1, 2


@dataclass
class SlabConfig:
    """One slab simulation: grid, species, switches (all inputs)."""
    name: str = "slab"
    nx: int = 128
    ny: int = 1
    dx_nm: float = 2.0
    dy_nm: float = 2.0
    dt_fs: float = 0.02
    rad_every: int = 5
    seed: int = 0
    cfl: float = 0.5                # Courant number of the field update (see the field reading)
    n_ref_cm3: float = 6.0e22       # ion density; weight unit is n_ref*V_cell
    Z_init: int = 3
    T_e_eV: float = 10.0
    T_i_eV: float = 10.0
    ppc_e: int = 256
    ppc_i: int = 64
    beam_frac: float = 0.05
    beam_E_eV: float = 1500.0
    E_bulk_eV: float = 0.0          # <= 0: every free electron is "bulk"
    ipd_model: int = IPD_EK
    coulomb_log: float = 0.0        # <= 0: computed per cell
    m_ion_me: float = M_AL_ME       # ion mass in electron masses
    flags: int = F_COLL_EE | F_COLL_EI | F_IONIZE | F_RECOMB | F_PUSH | F_FIELD

    @property
    def ncell(self) -> int:
        return self.nx * self.ny

    @property
    def w_ion(self) -> float:
        # rounded to FP32 so that both precisions see the same ion weight
        return float(np.float32(1.0 / self.ppc_i))

    @property
    def w_e(self) -> float:
        return self.Z_init * self.ppc_i * self.w_ion / self.ppc_e

    def to_dict(self):
        return asdict(self)


@dataclass
class Pulse:
    """XFEL pulse entering at x = 0 travelling along +x."""
    shape: int = 0                   # 0 Gaussian, 1 flat-top
    I_peak_Wcm2: float = 1.0e17
    fwhm_fs: float = 80.0
    t_peak_fs: float = 80.0
    hv_eV: float = 1600.0
    bandwidth_eV: float = 3.0
    n_bins: int = 2
    spot_sigma_nm: float = 0.0       # <= 0: uniform in y


def cfg_small_1d(**kw) -> SlabConfig:
    """Plain 1D slab of solid Al: 128 cells x 2 nm, 256 e + 64 Al3+ per cell,
    10 eV Maxwellian plus a 5 % 1.5 keV beam, dt 0.02 fs, collisions + Lotz +
    recombination, seed 0."""
    c = SlabConfig(name="al_1d_128x2nm_256e64i", **kw)
    return c


def cfg_foil_2d(**kw) -> SlabConfig:
    """2D XFEL-driven Al foil: 2048 x 256 cells of 5 nm, 64 e + 16 Al3+ per
    cell, every process on (pulse 1.6 keV, 80 fs FWHM, 1e17 W/cm^2)."""
    base = dict(name="al_2d_2048x256x5nm_64e16i", nx=2048, ny=256, dx_nm=5.0,
                dy_nm=5.0, ppc_e=64, ppc_i=16, flags=F_ALL)
    base.update(kw)
    return SlabConfig(**base)


def pulse_foil_2d(**kw) -> Pulse:
    p = Pulse(I_peak_Wcm2=1.0e17, fwhm_fs=80.0, t_peak_fs=80.0, hv_eV=1600.0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def cfg_large_2d(**kw) -> SlabConfig:
    """Large 2D precision study: 8192 x 1024 cells of 5 nm (40.96 x 5.12 um),
    80 e + 20 Al3+ per cell (0.84e9 particles), every process on."""
    base = dict(name="al_2d_8192x1024x5nm_80e20i", nx=8192, ny=1024, dx_nm=5.0,
                dy_nm=5.0, ppc_e=80, ppc_i=20, flags=F_ALL)
    base.update(kw)
    return SlabConfig(**base)


def pulse_large_2d(**kw) -> Pulse:
    """1.8 keV, 5e17 W/cm^2, 80 fs FWHM, peaking at 40 fs (two thirds into
    the study's 3000 steps of 0.02 fs)."""
    p = Pulse(I_peak_Wcm2=5.0e17, fwhm_fs=80.0, t_peak_fs=40.0, hv_eV=1800.0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# --------------------------------------------------------------------------
# initial particle state
# --------------------------------------------------------------------------


@dataclass
class ParticleState:
    """Particle arrays of one slab.  Positions are absolute in cell units
    (X in [0,nx), Y in [0,ny)), built as cell + an FP32 offset so both
    precisions see identical values."""
    eX: np.ndarray
    eY: np.ndarray
    eu: np.ndarray          # [n,3]
    ew: np.ndarray
    eid: np.ndarray         # uint64
    iX: np.ndarray
    iY: np.ndarray
    iu: np.ndarray          # [n,3]
    izf: np.ndarray         # fractional extra charge
    iZ: np.ndarray          # int32 charge state
    inK: np.ndarray         # int32 K vacancies
    iid: np.ndarray         # uint32

    @property
    def n_e(self):
        return self.eX.size

    @property
    def n_i(self):
        return self.iX.size


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _positions(rng, ncell_x, ncell_y, per_cell):
    cx = np.repeat(np.arange(ncell_x * ncell_y) % ncell_x, per_cell)
    cy = np.repeat(np.arange(ncell_x * ncell_y) // ncell_x, per_cell)
    ox = _f32(rng.random(cx.size))
    oy = _f32(rng.random(cx.size)) if ncell_y > 1 else np.full(cx.size, 0.5)
    # an FP32 offset that rounded up to 1.0 would leave the cell
    ox = np.where(ox >= 1.0, np.float64(np.nextafter(np.float32(1.0), np.float32(0.0))), ox)
    oy = np.where(oy >= 1.0, np.float64(np.nextafter(np.float32(1.0), np.float32(0.0))), oy)
    return cx + ox, cy + oy


def _maxwell_u(rng, n, T_eV, mass_me):
    s = math.sqrt(T_eV / (mass_me * ME_C2_EV))
    return rng.standard_normal((n, 3)) * s


def _iso(rng, n):
    c = 2.0 * rng.random(n) - 1.0
    ph = 2.0 * math.pi * rng.random(n)
    s = np.sqrt(1.0 - c * c)
    return np.stack([s * np.cos(ph), s * np.sin(ph), c], axis=1)


def init_particles(cfg: SlabConfig, seed: int | None = None) -> ParticleState:
    """Seeded initial state: cfg.ppc_e electrons and cfg.ppc_i ions per cell,
    uniform positions, Maxwellian momenta at T_e / T_i, a cfg.beam_frac share
    of electrons at cfg.beam_E_eV with isotropic directions, ions at Z_init."""
    rng = np.random.default_rng(cfg.seed if seed is None else seed)
    ex, ey = _positions(rng, cfg.nx, cfg.ny, cfg.ppc_e)
    ne = ex.size
    eu = _maxwell_u(rng, ne, cfg.T_e_eV, 1.0)
    beam = rng.random(ne) < cfg.beam_frac
    nb = int(beam.sum())
    if nb:
        g = 1.0 + cfg.beam_E_eV / ME_C2_EV
        umag = math.sqrt(g * g - 1.0)
        eu[beam] = _iso(rng, nb) * umag
    eu = _f32(eu)
    ew = np.full(ne, _f32(cfg.w_e))
    eid = np.arange(ne, dtype=np.uint64)

    ix, iy = _positions(rng, cfg.nx, cfg.ny, cfg.ppc_i)
    ni = ix.size
    iu = _f32(_maxwell_u(rng, ni, cfg.T_i_eV, cfg.m_ion_me))
    return ParticleState(
        eX=ex, eY=ey, eu=eu, ew=ew, eid=eid,
        iX=ix, iY=iy, iu=iu, izf=np.zeros(ni),
        iZ=np.full(ni, cfg.Z_init, dtype=np.int32),
        inK=np.zeros(ni, dtype=np.int32),
        iid=np.arange(ni, dtype=np.uint32),
    )


def perturb_ions(st: ParticleState, rng_seed: int, frac_hollow=0.3, z_spread=2,
                 zfrac_share=0.2) -> ParticleState:
    """Give a share of the ions K vacancies, higher charge states and
    fractional charges so that one step exercises every branch (decay,
    recombination, partial charges).  Charge neutrality is restored by
    adjusting electron weights is NOT done here; callers that need it
    rebuild electron weights with `neutralize`."""
    rng = np.random.default_rng(rng_seed)
    n = st.n_i
    dz = rng.integers(0, z_spread + 1, n).astype(np.int32)
    st.iZ = np.minimum(st.iZ + dz, Z_AL - 1).astype(np.int32)
    hol = rng.random(n) < frac_hollow
    nb = Z_AL - st.iZ
    nk = np.where(hol, rng.integers(1, 3, n), 0)
    nk = np.where(nb >= 3, nk, 0).astype(np.int32)
    st.inK = nk
    zf = np.where(rng.random(n) < zfrac_share, _f32(rng.random(n) * 0.9), 0.0)
    st.izf = zf
    return st


def neutralize(st: ParticleState, cfg: SlabConfig) -> ParticleState:
    """Scale electron weights cell by cell so each cell is neutral."""
    cell_e = (np.floor(st.eY).astype(np.int64) * cfg.nx + np.floor(st.eX).astype(np.int64))
    cell_i = (np.floor(st.iY).astype(np.int64) * cfg.nx + np.floor(st.iX).astype(np.int64))
    q = np.bincount(cell_i, weights=(st.iZ + st.izf) * cfg.w_ion, minlength=cfg.ncell)
    cnt = np.bincount(cell_e, minlength=cfg.ncell)
    w = q[cell_e] / np.maximum(cnt[cell_e], 1)
    st.ew = _f32(w)
    return st


def photons_uniform(cfg: SlabConfig, pulse: Pulse, density_nref: float) -> np.ndarray:
    """Photon number per cell and bin (units of n_ref*V_cell), [ny, nx, nb]."""
    return np.full((cfg.ny, cfg.nx, pulse.n_bins), density_nref / pulse.n_bins)


def random_fields(cfg: SlabConfig, rng_seed: int, e_amp=1e-4, b_amp=1e-4) -> dict:
    """Small random fields (normalized units) on the (nx+1) x ny node grid."""
    rng = np.random.default_rng(rng_seed)
    shp = (cfg.ny, cfg.nx + 1)
    out = {}
    for k in ("ex", "ey", "ez"):
        out[k] = _f32(rng.standard_normal(shp) * e_amp)
    for k in ("bx", "by", "bz"):
        out[k] = _f32(rng.standard_normal(shp) * b_amp)
    return out


# --------------------------------------------------------------------------
# batched ensembles and served request traces
# --------------------------------------------------------------------------


def _log_uniform(rng, lo, hi, n=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n))


def ensemble_slab(rng, k: int, seed0: int = 1000, cells=(64, 4096), ppc=(32, 512),
                  I_Wcm2=(1e15, 1e18), hv_eV=(1580.0, 1900.0), dx_nm: float = 2.0) -> tuple:
    """One member of the batched ensemble: a 1D Al slab with log-uniform cell
    count and particles per cell (electrons : ions = 4 : 1), log-uniform
    peak intensity and uniform photon energy; every process on."""
    nx = int(round(_log_uniform(rng, *cells)))
    p = int(round(_log_uniform(rng, *ppc)))
    ppc_i = max(1, int(round(p / 5)))
    ppc_e = max(1, p - ppc_i)
    cfg = SlabConfig(name=f"al_1d_{nx}x{dx_nm:g}nm_{ppc_e}e{ppc_i}i", nx=nx, ny=1, dx_nm=dx_nm, dy_nm=dx_nm,
                     ppc_e=ppc_e, ppc_i=ppc_i, seed=seed0 + k, flags=F_ALL)
    pl = Pulse(I_peak_Wcm2=float(_log_uniform(rng, *I_Wcm2)), hv_eV=float(rng.uniform(*hv_eV)))
    return cfg, pl


def batched_ensemble(n: int = 256, seed: int = 7, **kw) -> list:
    """n independent slabs drawn as in ensemble_slab (dx = 2 nm)."""
    rng = np.random.default_rng(seed)
    return [ensemble_slab(rng, k, **kw) for k in range(n)]


@dataclass
class Request:
    """A served slab simulation: arrival time (s), the slab, its pulse and
    the number of steps to run (horizon / dt)."""
    rid: int
    t_arrive: float
    cfg: SlabConfig
    pulse: Pulse
    nsteps: int


def request_trace(n: int = 2000, rate_hz: float = 200.0, seed: int = 11, horizon_fs: float = 150.0,
                  thickness_um=(0.2, 2.0), min_dx_nm: float = 1.0, **kw) -> list:
    """Poisson arrivals of slab requests.  Each request is an ensemble draw
    plus a foil thickness ~ U(0.2, 2) um; the cell size is thickness / cells,
    with the cell count capped so that cells stay at least min_dx_nm wide
    (finer cells would only lower the field speed the step resolves and
    multiply the cells)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    out = []
    for k in range(n):
        cfg, pl = ensemble_slab(rng, k, seed0=20000, **kw)
        thick_nm = 1e3 * float(rng.uniform(*thickness_um))
        nx = max(2, min(cfg.nx, int(thick_nm / min_dx_nm)))
        cfg.nx = nx
        cfg.dx_nm = cfg.dy_nm = thick_nm / nx
        cfg.name = f"al_1d_{nx}x{cfg.dx_nm:.3g}nm_{cfg.ppc_e}e{cfg.ppc_i}i"
        out.append(Request(rid=k, t_arrive=float(t[k]), cfg=cfg, pulse=pl,
                           nsteps=max(1, int(round(horizon_fs / cfg.dt_fs)))))
    return out
