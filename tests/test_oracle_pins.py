"""Pins of five oracle functions by values the mathematics fixes (CPU only).

* the EOS interpolation Zbar_EOS(n_i, T_e) that drives the recombination
  clamp (Sec. IV): exact on tables of a bilinear function, node and
  mid-cell values of a non-bilinear one, both clamps, and the number of
  recombinations of a whole step against the clamp evaluated by hand;
* the Lotz cross section (Sec. IV, Eq. 3) with its b exp(-c (E/P - 1))
  factor switched on: hand values at chosen energies and the Monte-Carlo
  ionization count of a step on a Maxwellian against an independent
  quadrature of sigma v f_M;
* the photon-bin choice of subshell photoionization (Sec. III, Eq. 2):
  with three or four bins of unequal n_b sigma_b, the share of events each
  bin takes is its n_b sigma_b / sum within binomial error, and every
  photoelectron carries exactly hv_b - E_b;
* the diagnostics (Sec. VI): charge-state histogram with fractional charges
  split between Z and Z + 1, and the logarithmic electron energy
  histogram, on hand-built states;
* the per-electron collision momentum scale the parity tolerance uses
  (test bookkeeping): the larger initial |u| of a fixed pair.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
import pic_inputs as P

MC2 = 510998.95
C_CM_FS = 2.99792458e-5


# ---------------------------------------------------------------- EOS ----

def _eos_tables(tables, n_grid, T_grid, f):
    t = dict(tables)
    t["eos_n"] = np.asarray(n_grid, dtype=np.float64)
    t["eos_T"] = np.asarray(T_grid, dtype=np.float64)
    t["eos_Zbar"] = np.array([[f(n, T) for T in T_grid] for n in n_grid])
    return t


N_GRID = [1e22, 4e22, 2e23, 1e24]          # 4 densities (cm^-3), uneven
T_GRID = [0.0, 5.0, 40.0, 300.0, 3000.0]   # 5 temperatures (eV), uneven


def _bilinear(n, T):
    # a + b n + c T + d n T: bilinear in (n, T), so bilinear interpolation
    # on any grid reproduces it exactly
    return 2.0 + 3.0e-24 * n + 0.004 * T + 1.0e-27 * n * T


def test_eos_exact_on_bilinear_function(tables):
    th = oracle.TableHandle(_eos_tables(tables, N_GRID, T_GRID, _bilinear))
    rng = np.random.default_rng(3)
    for _ in range(200):
        n = math.exp(rng.uniform(math.log(1e22), math.log(1e24)))
        T = rng.uniform(0.0, 3000.0)
        assert abs(oracle.eos(th, n, T) - _bilinear(n, T)) < 1e-12 * _bilinear(n, T), (n, T)


def test_eos_clamps_at_both_ends_of_both_axes(tables):
    th = oracle.TableHandle(_eos_tables(tables, N_GRID, T_GRID, _bilinear))
    for n_in, n_cl in ((1e20, 1e22), (5e25, 1e24), (7e22, 7e22)):
        for T_in, T_cl in ((-5.0, 0.0), (1e5, 3000.0), (77.0, 77.0)):
            want = _bilinear(n_cl, T_cl)
            assert abs(oracle.eos(th, n_in, T_in) - want) < 1e-12 * want, (n_in, T_in)


def test_eos_nodes_and_mid_cells_of_a_curved_table(tables):
    """A table that is not bilinear: the nodes come back exactly, a
    mid-cell point is the mean of its four corners, a point halfway along
    one edge the mean of that edge's two nodes."""
    def f(n, T):
        return 3.0 + math.sin(n / 1e23) + (T / 100.0) ** 2
    t = _eos_tables(tables, N_GRID, T_GRID, f)
    th = oracle.TableHandle(t)
    Z = t["eos_Zbar"]
    for a, n in enumerate(N_GRID):
        for b, T in enumerate(T_GRID):
            assert oracle.eos(th, n, T) == pytest.approx(Z[a, b], rel=1e-14)
    for a in range(len(N_GRID) - 1):
        for b in range(len(T_GRID) - 1):
            nm = 0.5 * (N_GRID[a] + N_GRID[a + 1])
            Tm = 0.5 * (T_GRID[b] + T_GRID[b + 1])
            mid = 0.25 * (Z[a, b] + Z[a + 1, b] + Z[a, b + 1] + Z[a + 1, b + 1])
            assert oracle.eos(th, nm, Tm) == pytest.approx(mid, rel=1e-13)
            edge_T = 0.5 * (Z[a, b] + Z[a, b + 1])
            assert oracle.eos(th, N_GRID[a], Tm) == pytest.approx(edge_T, rel=1e-13)
            edge_n = 0.5 * (Z[a, b] + Z[a + 1, b])
            assert oracle.eos(th, nm, T_GRID[b]) == pytest.approx(edge_n, rel=1e-13)


def test_recombination_count_follows_the_clamp_by_hand(tables):
    """A recombination-only step on cells of Al7+ against an EOS table of a
    bilinear function: each cell recombines round((Zbar - Zbar_EOS(n_i,
    T_e)) N_i) times, with T_e = (2/3) of the weighted mean kinetic energy
    of the cell's electrons and n_i its ion density, all evaluated here
    from the loaded state."""
    def f(n, T):
        return 4.0 + 1.5e-23 * n + 0.05 * T + 2e-25 * n * T
    t = _eos_tables(tables, N_GRID, T_GRID, f)
    cfg = P.cfg_small_1d(flags=P.F_RECOMB, nx=24, ppc_e=64, ppc_i=32, T_e_eV=20.0, beam_frac=0.0)
    st = P.init_particles(cfg)
    st.iZ[:] = 7
    st = P.neutralize(st, cfg)
    o = oracle.OracleSlab(cfg, t)
    o.load(st)
    o.step(1)
    _, c = o.tallies()
    ce = np.floor(st.eX).astype(int)
    ci = np.floor(st.iX).astype(int)
    u2 = (st.eu ** 2).sum(1)
    ke = MC2 * (np.sqrt(1.0 + u2) - 1.0)
    expect = 0
    for cell in range(cfg.nx):
        me, mi = ce == cell, ci == cell
        ni = int(mi.sum())
        Te = (2.0 / 3.0) * (st.ew[me] * ke[me]).sum() / st.ew[me].sum()
        n_i = ni * cfg.w_ion * cfg.n_ref_cm3
        zb = st.iZ[mi].mean()
        zeos = f(n_i, Te)
        assert 4.5 < zeos < 6.5          # well inside the caps (charge, electron weight)
        expect += int(math.floor((zb - zeos) * ni + 0.5))
    assert c["REC"] == expect > 0


# --------------------------------------------------------------- Lotz ----

def _lotz_tables(tables):
    t = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in tables.items()}
    t["E_bind"][11, 0] = 2000.0            # Al11+: 1s^2 only, P = 2000 eV
    t["lotz_a"][0], t["lotz_b"][0], t["lotz_c"][0] = 4.5e-14, 0.3, 0.5
    return t


def test_lotz_hand_values_with_the_b_c_factor(tables):
    """sigma = a N ln(E/P) / (E P) (1 - b exp(-c (E/P - 1))) for Al11+
    (N = 2 electrons in 1s, P = 2000 eV, a = 4.5e-14 cm^2 eV^2, b = 0.3,
    c = 0.5), evaluated by hand:
      E = 4000:    9e-14 / 8e6 * ln 2 = 7.79791e-21; 1 - 0.3 e^-0.5 = 0.818041
      E = 2000 e:  9e-14 / (2000 e * 2000) = 8.27730e-21; 1 - 0.3 e^-(e-1)/2 = 0.872941
      E = 20000:   9e-14 / 4e7 * ln 10 = 5.18082e-21; 1 - 0.3 e^-4.5 = 0.996667
      E = 2100:    9e-14 / 4.2e6 * ln 1.05 = 1.045504e-21; 1 - 0.3 e^-0.025 = 0.707407
    and zero at and below threshold."""
    th = oracle.TableHandle(_lotz_tables(tables))
    for E, want in ((4000.0, 6.379005099926842e-21), (2000.0 * math.e, 7.22559406455009e-21),
                    (20000.0, 5.163550357603325e-21), (2100.0, 7.395965346910939e-22)):
        assert oracle.lotz(th, 11, 0.0, E) == pytest.approx(want, rel=1e-12), E
    assert oracle.lotz(th, 11, 0.0, 2000.0) == 0.0
    assert oracle.lotz(th, 11, 0.0, 1999.0) == 0.0
    # a lowering dE moves the threshold: P = 2000 - 100
    assert oracle.lotz(th, 11, 100.0, 1950.0) > 0.0


def test_lotz_maxwellian_rate_with_b_c_against_quadrature(tables):
    """Monte-Carlo impact ionizations of one step on Al3+ with the stand-in
    L-shell constants b = 0.3, c = 0.5 (the tables the product runs with)
    against N_i dt n_e <sigma v>, the average taken by numerical quadrature
    of sigma(E) v(E) over the Maxwellian energy distribution
    2 sqrt(E / pi) T^-3/2 exp(-E / T): within 2 %."""
    T = 100.0
    tab = tables
    assert tab["lotz_b"][2] == 0.3 and tab["lotz_c"][2] == 0.5
    cfg = P.cfg_small_1d(flags=P.F_IONIZE, nx=4096, ppc_e=512, ppc_i=256, T_e_eV=T,
                         beam_frac=0.0, ipd_model=P.IPD_NONE)
    st = P.init_particles(cfg)
    o = oracle.OracleSlab(cfg, tab)
    o.load(st)
    o.step(1)
    _, c = o.tallies()
    occ = oracle.occ(10, 0)

    def sigma(E, with_bc=True):
        s = 0.0
        for q in range(5):
            Pq = tab["E_bind"][3, q]
            if occ[q] and E > Pq:
                x = E / Pq
                f = 1.0 - tab["lotz_b"][q] * math.exp(-tab["lotz_c"][q] * (x - 1.0)) if with_bc else 1.0
                s += tab["lotz_a"][q] * occ[q] * math.log(x) / (E * Pq) * f
        return s

    def rate(with_bc):
        def integrand(E):
            v = math.sqrt(2.0 * E / MC2) * 2.99792458e10            # cm/s
            return sigma(E, with_bc) * v * 2.0 * math.sqrt(E / math.pi) * T ** -1.5 * math.exp(-E / T)
        pts = sorted({tab["E_bind"][3, q] for q in range(5) if occ[q]})
        return integrate.quad(integrand, 0.0, 60.0 * T, points=pts, limit=400, epsabs=0.0, epsrel=1e-10)[0]

    sv = rate(True)
    n_e = cfg.Z_init * cfg.n_ref_cm3
    expect = st.n_i * cfg.dt_fs * 1e-15 * n_e * sv
    assert expect > 10000
    assert abs(c["ION"] / expect - 1) < 0.02, (c["ION"], expect)
    # the b, c factor matters at this temperature: without it the expected
    # count would be more than 10 % higher, far outside the tolerance
    assert rate(False) / sv - 1 > 0.1


# ------------------------------------------------- photon-bin choice ----

BIN_HV = [1550.0, 1650.0, 1750.0, 1850.0]        # pulse bins (hv 1700, 400 eV wide, 4 bins)
# per-electron cross sections (cm^2) on the nodes 800, 1550, 1650, 1750, 1850, 20000 eV
SIG = {0: [1e-19, 3.0e-19, 2.0e-19, 0.6e-19, 1.0e-19, 1e-21],   # 1s (edge of Al3+ at 1610.69 eV)
       1: [1e-20, 1.0e-20, 0.5e-20, 2.0e-20, 0.8e-20, 1e-22],   # 2s
       2: [1e-20, 0.4e-20, 1.2e-20, 0.6e-20, 0.9e-20, 1e-22],   # 2p
       3: [1e-22] * 6, 4: [1e-22] * 6}
PH_W = [50.0, 20.0, 120.0, 60.0]                 # photons per cell and bin, in ion weights


def test_photon_bin_choice_follows_n_sigma_and_photoelectron_energy_is_exact(tables):
    """One rad step with photoionization only, four photon bins of unequal
    n_b sigma_b (Sec. III, Eq. 2) and the 2s and 2p bindings of Al3+ set
    apart (140 and 110 eV) so that each photoelectron's energy names its
    subshell and bin: every photoelectron has exactly hv_b - E_b; per
    subshell, the share of events in bin b is n_b sigma_sb / sum_b' n_b'
    sigma_sb' over the bins above that subshell's edge, within binomial
    error (the K edge of Al3+ lies between the first two bins)."""
    t = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in tables.items()}
    t["hv_tab"] = np.array([800.0] + BIN_HV + [20000.0])
    t["sigma_photo"] = np.array([[v * 2.0 for v in SIG[s]] for s in range(5)])
    t["E_bind"][3, 1], t["E_bind"][3, 2] = 140.0, 110.0
    edges = t["E_bind"][3, :3]
    cfg = P.cfg_small_1d(flags=P.F_PHOTO, nx=512, ppc_e=2, ppc_i=256, beam_frac=0.0,
                         ipd_model=P.IPD_NONE, rad_every=5)
    pl = P.Pulse(I_peak_Wcm2=0.0, n_bins=4, hv_eV=1700.0, bandwidth_eV=400.0)
    st = P.init_particles(cfg)
    o = oracle.OracleSlab(cfg, t, pl)
    o.load(st)
    ph = np.zeros((1, cfg.nx, 4))
    ph[..., :] = np.array(PH_W) * cfg.w_ion
    o.set_photons(ph)
    o.step(1)
    e = o.electrons()
    new = (e["id"] >> np.uint64(32)) == np.uint64((1 << 2) | 2)      # photoelectrons of step 0
    u2 = (e["u"][new] ** 2).sum(1)
    ke = MC2 * u2 / (np.sqrt(1.0 + u2) + 1.0)
    cand = np.array([[hv - edges[s] if hv > edges[s] else np.nan for hv in BIN_HV] for s in range(3)])
    counts = np.zeros((3, 4), dtype=int)
    for k in ke:
        d = np.abs(cand - k)
        s, b = np.unravel_index(np.nanargmin(d), d.shape)
        assert d[s, b] < 1e-9 * k, k
        counts[s, b] += 1
    assert (e["w"][new] == cfg.w_ion).all()          # dense photons: no partial event
    _, c = o.tallies()
    assert [c["PH0"], c["PH1"], c["PH2"]] == list(counts.sum(1))
    assert counts[0, 0] == 0                          # 1550 eV is below the K edge
    for s in range(3):
        ns = np.array(PH_W) * np.array(SIG[s][1:5]) * (np.array(BIN_HV) > edges[s])
        share = ns / ns.sum()
        N = counts[s].sum()
        assert N > 800, (s, N)
        for b in range(4):
            sd = math.sqrt(N * share[b] * (1 - share[b])) + 1e-9
            assert abs(counts[s, b] - N * share[b]) < 4 * sd + 1, (s, b, counts[s], share)


# --------------------------------------------------------- diagnostics ----

def test_diagnostics_on_a_hand_built_state(tables):
    """Five ions (3, 3.25, 5.5, 13, 12.75) and six electrons of 0.05, 0.5,
    5, 50, 500 and 5000 eV with weights 1..6; 4 log bins on 0.1..1000 eV
    (edges 0.1, 1, 10, 100, 1000, the ends clamped into the first and last
    bin).  By hand: CSD = 0.35 at Z = 3, 0.05 at 4, 0.1 at 5 and 6, 0.05
    at 12, 0.35 at 13 (a fractional charge f puts 1 - f of the ion at Z
    and f at Z + 1), mean charge 7.5; EEDF = (1 + 2, 3, 4, 5 + 6) / 21."""
    cfg = P.cfg_small_1d(nx=2, ppc_e=1, ppc_i=1, flags=0)
    o = oracle.OracleSlab(cfg, tables)
    ke = np.array([0.05, 0.5, 5.0, 50.0, 500.0, 5000.0])
    x = ke / MC2
    um = np.sqrt(x * (2.0 + x))
    st = P.ParticleState(
        eX=np.full(6, 0.5), eY=np.full(6, 0.5), eu=np.stack([um, 0 * um, 0 * um], 1),
        ew=np.arange(1.0, 7.0), eid=np.arange(6, dtype=np.uint64),
        iX=np.array([0.5, 0.5, 1.5, 1.5, 1.5]), iY=np.full(5, 0.5), iu=np.zeros((5, 3)),
        izf=np.array([0.0, 0.25, 0.5, 0.0, 0.75]), iZ=np.array([3, 3, 5, 13, 12], dtype=np.int32),
        inK=np.zeros(5, dtype=np.int32), iid=np.arange(5, dtype=np.uint32))
    o.load(st)
    csd, eedf = o.diag(n_E=4, E_max=1000.0)
    want = np.zeros(14)
    want[[3, 4, 5, 6, 12, 13]] = [0.35, 0.05, 0.1, 0.1, 0.05, 0.35]
    assert np.allclose(csd, want, rtol=0, atol=1e-15)
    assert (np.arange(14) * csd).sum() == pytest.approx(7.5, rel=1e-14)
    assert np.allclose(eedf, np.array([3.0, 3.0, 4.0, 11.0]) / 21.0, rtol=0, atol=1e-15)
    # more bins: each decade split in two (edges 0.1, 0.316, 1, 3.16, ...)
    _, e8 = o.diag(n_E=8, E_max=1000.0)
    assert np.allclose(e8, np.array([1, 2, 0, 3, 0, 4, 0, 11]) / 21.0, atol=1e-15)


# ------------------------------------------- collision momentum scale ----

def test_collision_scale_is_the_larger_pair_momentum(tables):
    """The oracle's per-electron collision momentum scale (test
    bookkeeping: the scale of the momentum tolerance of parity, no part of
    the method): the larger |u| of the electron and its e-e partner before
    their collision.  Two electrons per cell, so the pairing is fixed:
    both get the larger initial |u| of their cell; with collisions off,
    zero."""
    for flags, on in ((P.F_COLL_EE, True), (P.F_IONIZE, False)):
        cfg = P.cfg_small_1d(nx=3, ppc_e=2, ppc_i=1, T_e_eV=50.0, flags=flags)
        st = P.init_particles(cfg)
        o = oracle.OracleSlab(cfg, tables)
        o.load(st)
        o.step(1)
        e = o.electrons()
        cell = np.floor(st.eX).astype(int)
        mag = np.sqrt((np.asarray(st.eu, dtype=np.float64) ** 2).sum(axis=1))
        want = np.array([mag[cell == c].max() for c in cell]) if on else np.zeros(len(mag))
        order = np.argsort(e["id"])
        got = e["cscale"][order]
        assert np.allclose(got, want[np.argsort(st.eid)], rtol=0, atol=0), (got, want)
