// The per-cell collision and atomic-process kernel k_cell: one warp per
// cell, phase-synchronous rounds (see pic_cell.cuh for the building blocks;
// the push and deposit follow in pic_push.cuh).
#pragma once
#include <type_traits>
#include "pic_cell.cuh"

namespace pic {

// event counts and energy tallies of one warp, lane-uniform, flushed to the
// slab's tally when the warp moves to another slab and at the end
struct WarpTally {
    int slab;
    dd ion, ka, esc;
    dd rt;          // energy the electrons took from the radiation field (transport mode)
    int cnt[NCOUNT];
};

__device__ __forceinline__ void tally_flush(const CellArgs &a, WarpTally &w, int lane)
{
    if (w.slab >= 0 && lane == 0) {
        SlabTally *tl = a.tally + w.slab;
        if (dd_f(w.ion) != RF(0.0)) atomicAdd(&tl->ion, (double)w.ion.hi + (double)w.ion.lo);
        if (dd_f(w.ka) != RF(0.0)) atomicAdd(&tl->ka_esc, (double)w.ka.hi + (double)w.ka.lo);
        if (dd_f(w.esc) != RF(0.0)) atomicAdd(&tl->esc, (double)w.esc.hi + (double)w.esc.lo);
        if (dd_f(w.rt) != RF(0.0)) atomicAdd(&tl->rt_pend, -((double)w.rt.hi + (double)w.rt.lo));
        for (int q = 0; q < NCOUNT; ++q)
            if (w.cnt[q]) atomicAdd(tl->cnt + q, (unsigned long long)w.cnt[q]);
    }
    w.ion = w.ka = w.esc = w.rt = dd_zero();
    for (int q = 0; q < NCOUNT; ++q) w.cnt[q] = 0;
}

// per-cell scalars shared by the stages of one cell
struct CellCtx {
    int s, lc, cx, cy, e0, ne, i0, ni;
    unsigned step, flags;
    unsigned long long seed;
    real wi, mi, n_e, n_i, nref;
    bool rad;
    // sums the recombination stage needs, when the earlier stages already
    // hold them (every electron bulk, impact ionization run): kinetic
    // energy of the electrons after the ionization payment, their weight,
    // and the ion charge after ionization
    bool have_sums;
    dd K_after;
    real W_e, Q_after;
};

// ---- forced-thermalization variant (Sec. VI C), rad steps ----
// The cell's free electrons, those created in this step included, are
// redrawn from a Maxwellian at kT = (2/3) E_ave (components normal with
// standard deviation sqrt(kT / m c^2), Box-Muller on the electron's Philox
// draw); the mean momentum is shifted back to the cell's and the momenta
// about it scaled by one factor (Newton) so that the cell's kinetic energy
// is kept.  Sums are double-float (double-double in the FP64 build).
struct ThermSums { dd W, K, Px, Py, Pz; int n; };

__device__ __forceinline__ void therm_add(ThermSums &t, real4 u)
{
    t.W = dd_addf(t.W, u.w);
    t.K = dd_addf(t.K, u.w * (real)kMeC2 * gm1(u.x, u.y, u.z));
    t.Px = dd_addf(t.Px, u.w * u.x); t.Py = dd_addf(t.Py, u.w * u.y); t.Pz = dd_addf(t.Pz, u.w * u.z);
    t.n += 1;
}

__device__ __noinline__ void stage_therm(const CellArgs &a, const WarpMem &m, const CellCtx &c, int lane, int nnew)
{
    const int ne = c.ne;
    const real MC2 = (real)kMeC2;
    ThermSums t0{dd_zero(), dd_zero(), dd_zero(), dd_zero(), dd_zero(), 0};
    for (int k = lane; k < ne; k += 32) { real4 u = m.eu[m.eperm[k]]; if (u.w > RF(0.0)) therm_add(t0, u); }
    for (int k = lane; k < nnew; k += 32) {
        NewE q = m.nw[k];
        if (q.w > RF(0.0)) therm_add(t0, make_real4(q.ux, q.uy, q.uz, q.w));
    }
    const dd W = wsum_dd(t0.W), K = wsum_dd(t0.K);
    const real P[3] = {dd_f(wsum_dd(t0.Px)), dd_f(wsum_dd(t0.Py)), dd_f(wsum_dd(t0.Pz))};
    const int n = wsum_i(t0.n);
    const real Wf = dd_f(W), Kf = dd_f(K);
    if (n < 2 || !(Wf > RF(0.0)) || !(Kf > RF(0.0))) return;
    const real sig = r_sqrt((RF(2.0) / RF(3.0)) * Kf / Wf / MC2);
    // redraw; the new momenta replace the old ones in shared memory
    auto redraw = [&](unsigned long long id) {
        U4 r = draw(c.seed, id, c.step, PU_THERM);
        const real a0 = r_sqrt(-RF(2.0) * r_log(u01(r.x))), a1 = r_sqrt(-RF(2.0) * r_log(u01(r.z)));
        real sn, cs;
        r_sincos(RF(2.0) * kPiR * u01(r.y), &sn, &cs);
        return make_real3(sig * a0 * cs, sig * a0 * sn, sig * a1 * r_cos(RF(2.0) * kPiR * u01(r.w)));
    };
    dd Qx = dd_zero(), Qy = dd_zero(), Qz = dd_zero();
    for (int k = lane; k < ne; k += 32) {
        const int sl = m.eperm[k];
        real4 u = m.eu[sl];
        if (!(u.w > RF(0.0))) continue;
        real3 v = redraw(m.eid[k]);
        m.eu[sl] = make_real4(v.x, v.y, v.z, u.w);
        Qx = dd_addf(Qx, u.w * v.x); Qy = dd_addf(Qy, u.w * v.y); Qz = dd_addf(Qz, u.w * v.z);
    }
    for (int k = lane; k < nnew; k += 32) {
        NewE q = m.nw[k];
        if (!(q.w > RF(0.0))) continue;
        const int islot = q.meta & 0xffff, kind = q.meta >> 16;
        const unsigned ion_id = rec_iid(a.i1[c.i0 + islot]);
        const unsigned long long id = ((unsigned long long)(((c.step + 1u) << 2) | (unsigned)kind) << 32) | ion_id;
        real3 v = redraw(id);
        q.ux = v.x; q.uy = v.y; q.uz = v.z;
        m.nw[k] = q;
        Qx = dd_addf(Qx, q.w * v.x); Qy = dd_addf(Qy, q.w * v.y); Qz = dd_addf(Qz, q.w * v.z);
    }
    __syncwarp();
    const real iW = RF(1.0) / Wf;
    const real V[3] = {P[0] * iW, P[1] * iW, P[2] * iW};
    const real M[3] = {dd_f(wsum_dd(Qx)) * iW, dd_f(wsum_dd(Qy)) * iW, dd_f(wsum_dd(Qz)) * iW};
    // kinetic energy of the cell with the peculiar momenta d = u - M scaled by s
    auto energy = [&](real s, real &slope) {
        dd e = dd_zero(), de = dd_zero();
        auto one = [&](real4 u) {
            real dx = u.x - M[0], dy = u.y - M[1], dz = u.z - M[2];
            real ux = V[0] + s * dx, uy = V[1] + s * dy, uz = V[2] + s * dz;
            e = dd_addf(e, u.w * MC2 * gm1(ux, uy, uz));
            de = dd_addf(de, u.w * MC2 * (ux * dx + uy * dy + uz * dz) * r_rsqrt(RF(1.0) + ux * ux + uy * uy + uz * uz));
        };
        for (int k = lane; k < ne; k += 32) { real4 u = m.eu[m.eperm[k]]; if (u.w > RF(0.0)) one(u); }
        for (int k = lane; k < nnew; k += 32) {
            NewE q = m.nw[k];
            if (q.w > RF(0.0)) one(make_real4(q.ux, q.uy, q.uz, q.w));
        }
        slope = dd_f(wsum_dd(de));
        return wsum_dd(e);
    };
    real s = RF(1.0);
    for (int it = 0; it < 8; ++it) {
        real slope;
        const dd e = energy(s, slope);
        if (!(slope > RF(0.0))) break;
        const real ds = dd_f(dd_sub(e, K)) / slope;
        s = r_fmax(s - ds, RF(0.0));
        if (r_fabs(ds) <= RF(1e-7) * s) break;
    }
    for (int k = lane; k < ne; k += 32) {
        const int sl = m.eperm[k];
        real4 u = m.eu[sl];
        if (!(u.w > RF(0.0))) continue;
        m.eu[sl] = make_real4(V[0] + s * (u.x - M[0]), V[1] + s * (u.y - M[1]), V[2] + s * (u.z - M[2]), u.w);
    }
    for (int k = lane; k < nnew; k += 32) {
        NewE q = m.nw[k];
        if (!(q.w > RF(0.0))) continue;
        q.ux = V[0] + s * (q.ux - M[0]); q.uy = V[1] + s * (q.uy - M[1]); q.uz = V[2] + s * (q.uz - M[2]);
        m.nw[k] = q;
    }
    __syncwarp();
}

// ---- EOS-clamped three-body recombination (Sec. IV) ----
__device__ __noinline__ void stage_recombine(const CellArgs &a, const WarpMem &m, const Tables &T, const SlabDev &S,
                                             const CellCtx &c, int lane, real Wnew_imp, WarpTally &wt)
{
    const int ne = c.ne, ni = c.ni;
    const real wi = c.wi, MC2 = (real)kMeC2;
    real zb, Wb2, Kb2, Wex;
    if (c.have_sums) {
        // every electron is bulk: the sums of the moments and ionization
        // stages, which the ionization payment changed by a known amount
        zb = c.Q_after / ni;
        Wb2 = c.W_e + Wnew_imp;
        Kb2 = dd_f(c.K_after);
        Wex = c.W_e;
    } else {
        real pq = RF(0.0);
        for (int k = lane; k < ni; k += 32) { int sl = m.iperm[k]; pq += (real)(m.ist[sl] & 0xff) + m.iu[sl].w; }
        zb = wsum_f(pq) / ni;
        dd pkb = dd_zero();
        real pwb = RF(0.0), pwx = RF(0.0);
        for (int k = lane; k < ne; k += 32) {
            real4 u = m.eu[m.eperm[k]];
            real ke = MC2 * gm1(u.x, u.y, u.z);
            pwx += u.w;
            if (S.E_bulk <= RF(0.0) || ke < S.E_bulk) { pwb += u.w; pkb = dd_addf(pkb, u.w * ke); }
        }
        Wb2 = wsum_f(pwb) + Wnew_imp;
        Kb2 = dd_f(wsum_dd(pkb));
        Wex = wsum_f(pwx);
    }
    const real Te2 = Wb2 > RF(0.0) ? (RF(2.0) / RF(3.0)) * Kb2 / Wb2 : RF(0.0);
    const real zeos = eos_lookup(*a.eos, c.n_i, Te2);
    int Kev = zb > zeos ? (int)r_floor((zb - zeos) * ni + RF(0.5)) : 0;
    int pel = 0;
    for (int k = lane; k < ni; k += 32) pel += m.ist[k] & 0xff;
    const int elig = wsum_i(pel);
    Kev = min(Kev, elig);
    Kev = min(Kev, (int)r_floor(Wex / wi * (RF(1.0) + RF(1e-6))));
    if (Kev <= 0) return;
    int *nrec = (int *)m.ikey;            // sort keys are no longer needed
    real *take = (real *)m.ekey;
    for (int k = lane; k < ni; k += 32) nrec[k] = 0;
    __syncwarp();
    int left = Kev;
    for (int round = 0; left > 0; ++round) {
        if (round > ZNUC * 2) {          // cannot happen when Kev <= sum Z
            if (lane == 0) atomicOr(a.err, ERR_NUMERIC);
            break;
        }
        for (int b0 = 0; b0 < ni && left > 0; b0 += 32) {
            int t = b0 + lane;
            bool e = false;
            if (t < ni) e = (m.ist[m.iperm[t]] & 0xff) - nrec[t] >= 1;
            unsigned bal = __ballot_sync(FULL, e);
            int rank = __popc(bal & ((1u << lane) - 1u));
            if (e && rank < left) nrec[t] += 1;
            left -= min(left, __popc(bal));
            __syncwarp();
        }
    }
    const dd Wrem = dd{(real)Kev * wi, RF(0.0)};
    dd carry = dd_zero(), remKE = dd_zero();
    for (int b0 = 0; b0 < ne; b0 += 32) {
        int t = b0 + lane;
        real w = RF(0.0), ke = RF(0.0);
        if (t < ne) { real4 u = m.eu[m.eperm[t]]; w = u.w; ke = MC2 * gm1(u.x, u.y, u.z); }
        dd incl = dd_add(carry, wscan_dd(dd{w, RF(0.0)}, lane));
        dd before = dd_sub(incl, dd{w, RF(0.0)});
        real tk = r_fmin(r_fmax(dd_f(dd_sub(Wrem, before)), RF(0.0)), w);
        if (t < ne) take[t] = tk;
        remKE = dd_addf(remKE, tk * ke);
        carry = wbcast_dd(incl, 31);
    }
    __syncwarp();
    remKE = wsum_dd(remKE);
    dd pb = dd_zero();
    for (int k = lane; k < ni; k += 32) {
        int st = m.ist[m.iperm[k]];
        int Z = st & 0xff, nK = (st >> 8) & 0xff;
        for (int r = 1; r <= nrec[k]; ++r) pb = dd_addf(pb, wi * removal_energy(T, Z - r, nK, m.dE[Z - r]));
    }
    const dd bind = wsum_dd(pb);
    dd pkr = dd_zero();
    for (int k = lane; k < ne; k += 32) {
        real4 u = m.eu[m.eperm[k]];
        real ke = MC2 * gm1(u.x, u.y, u.z);
        if (S.E_bulk <= RF(0.0) || ke < S.E_bulk) pkr = dd_addf(pkr, (u.w - take[k]) * ke);
    }
    const real Krem = dd_f(wsum_dd(pkr));
    if (Krem > RF(0.0)) {
        real delta = -dd_f(dd_add(remKE, bind)) / Krem;
        for (int k = lane; k < ne; k += 32) {
            int sl = m.eperm[k];
            real4 u = m.eu[sl];
            real ke = MC2 * gm1(u.x, u.y, u.z);
            bool bulk = S.E_bulk <= RF(0.0) || ke < S.E_bulk;
            real tk = take[k];
            real wn = u.w - tk;
            bool dead = tk > RF(0.0) && wn <= RF(0.0);
            u.w = dead ? RF(0.0) : wn;
            if (bulk && !dead) scale_kinetic(u.x, u.y, u.z, delta);
            m.eu[sl] = u;
        }
        for (int k = lane; k < ni; k += 32) {
            int sl = m.iperm[k];
            m.ist[sl] = m.ist[sl] - nrec[k];
        }
        wt.ion = dd_sub(wt.ion, bind);
        if (lane == 0) wt.cnt[C_REC] += Kev;
    }
    __syncwarp();
}

// ---- rad step: subshell photoionization (Eq. 2) ----
__device__ __noinline__ void stage_photo(const CellArgs &a, const WarpMem &m, const Tables &T, const SlabDev &S,
                                         const CellCtx &c, int lane, int &nnew, WarpTally &wt)
{
    const int ni = c.ni, nb = S.nb;
    const real wi = c.wi;
    const real dtr = S.rad_every * S.dt;
    ph2 *ph = a.photons + S.ph_off + (size_t)c.lc * nb;
    dd *n0 = m.ph, *used = m.ph + MAXB;
    int *carry = m.phc;
    if (lane < nb) { ph2 v = ph[lane]; n0[lane] = dd{v.hi, v.lo}; used[lane] = dd_zero(); carry[lane] = 0; }
    __syncwarp();
    const real cph = (real)kCcmPerFs * dtr * c.nref;
    int c_part = 0, c_ph[NS] = {0, 0, 0, 0, 0};
    // transport mode: the ions' opacity per bin (sum over occupied subshells
    // of N_s sigma_s above the lowered edge) and the photon energy the
    // events take; the field is not depleted here (its opacity does that)
    const bool rtm = S.rt != 0;
    real chi_l[MAXB];
    for (int b = 0; b < MAXB; ++b) chi_l[b] = RF(0.0);
    dd emc = dd_zero();
    for (int b0 = 0; b0 < ni; b0 += 32) {
        int t = b0 + lane;
        int sub = -1, bin = -1, sl = 0, Z = 0, nK = 0;
        real edge = RF(0.), rc = RF(0.), rp = RF(0.);
        if (t < ni) {
            sl = m.iperm[t];
            int st = m.ist[sl];
            Z = st & 0xff; nK = (st >> 8) & 0xff;
            int occ[NS];
            if (Z < ZNUC && occupancy(ZNUC - Z, nK, occ)) {
                if (rtm)
                    for (int q = 0; q < NS; ++q) {
                        if (!occ[q]) continue;
                        const real ed = lowered_binding(T, Z, q, m.dE[Z]);
                        for (int b = 0; b < nb; ++b)
                            if (S.hv_b[b] > ed) chi_l[b] += (real)occ[q] * S.sig_b[q][b];
                    }
                U4 ra = draw(c.seed, (unsigned long long)m.iid[t], c.step, PU_PHOTO_A);
                U4 rb = draw(c.seed, (unsigned long long)m.iid[t], c.step, PU_PHOTO_B);
                real rs[NS] = {u01(ra.x), u01(ra.y), u01(ra.z), u01(ra.w), u01(rb.x)};
                real Ps = RF(0.);
                for (int q = 0; q < NS; ++q) {
                    if (!occ[q]) continue;
                    real ed = lowered_binding(T, Z, q, m.dE[Z]);
                    real acc = RF(0.);
                    for (int b = 0; b < nb; ++b)
                        if (S.hv_b[b] > ed) acc += dd_f(n0[b]) * S.sig_b[q][b];
                    real P = cph * occ[q] * acc;
                    if (rs[q] < P) { sub = q; Ps = P; edge = ed; break; }
                }
                if (sub >= 0) {
                    real target = u01(rb.y) * Ps, cum = RF(0.);
                    int lastpos = -1;
                    for (int b = 0; b < nb; ++b) {
                        real cb = S.hv_b[b] > edge ? cph * occ[sub] * dd_f(n0[b]) * S.sig_b[sub][b] : RF(0.);
                        if (cb > RF(0.)) lastpos = b;
                        cum += cb;
                        if (cum > target) { bin = b; break; }
                    }
                    if (bin < 0) bin = lastpos;
                    rc = u01(rb.z); rp = u01(rb.w);
                }
            }
        }
        // the k-th event of a bin gets min(w, max(0, n_bin - k w)) photons
        real g = RF(0.0);
        bool full = false;
        for (int b = 0; b < nb; ++b) {
            bool eb = bin == b && sub >= 0;
            unsigned bal = __ballot_sync(FULL, eb);
            if (eb) {
                int rank = carry[b] + __popc(bal & ((1u << lane) - 1u));
                dd rest = dd_addf(n0[b], -(real)rank * wi);
                if (dd_le(dd{wi, RF(0.0)}, rest)) { g = wi; full = true; }
                else g = r_fmax(dd_f(rest), RF(0.0));
            }
            __syncwarp();
            if (lane == 0) carry[b] += __popc(bal);
            __syncwarp();
        }
        bool ev = sub >= 0 && bin >= 0 && g > RF(0.0);
        if (ev) {
            if (full) {
                lose_electron(Z, nK, sub);
            } else {
                real zf = m.iu[sl].w + g / wi;
                if (zf >= RF(1.0)) {
                    zf -= RF(1.0);
                    int so = outer_shell(ZNUC - Z, nK);
                    if (so >= 0) lose_electron(Z, nK, so);
                }
                m.iu[sl].w = zf;
                c_part++;
            }
            m.ist[sl] = Z | (nK << 8);
            c_ph[sub]++;
        }
        for (int b = 0; b < nb; ++b) {
            dd ub = wsum_dd(dd{ev && bin == b ? g : RF(0.0), RF(0.0)});
            if (lane == 0) used[b] = dd_add(used[b], ub);
        }
        wt.ion = dd_add(wt.ion, wsum_dd(dd{ev ? g * edge : RF(0.0), RF(0.0)}));
        if (rtm) emc = dd_add(emc, wsum_dd(dd{ev ? g * S.hv_b[bin] : RF(0.0), RF(0.0)}));
        unsigned bal = __ballot_sync(FULL, ev);
        if (ev) {
            int pos = nnew + __popc(bal & ((1u << lane) - 1u));
            if (pos < a.cap_new) {
                real3 u = iso_momentum(S.hv_b[bin] - edge, rc, rp);
                NewE q; q.ux = u.x; q.uy = u.y; q.uz = u.z; q.w = g;
                q.meta = sl | (KIND_PHOTO << 16);
                m.nw[pos] = q;
            } else {
                atomicOr(a.err, ERR_NEW_OVERFLOW);
            }
        }
        nnew = min(nnew + __popc(bal), a.cap_new);
        __syncwarp();
    }
    if (rtm) {
        // opacity (cm^-1) and the events' photon energy, owed to the field
        // until its opacity takes it at the next transport step
        for (int b = 0; b < nb; ++b) {
            const real v = wsum_f(chi_l[b]);
            if (lane == 0) S.rt_chi[(size_t)c.lc * nb + b] = (float)(v * c.nref * c.wi);
        }
        if (lane == 0) S.rt_emc[c.lc] = (double)emc.hi + (double)emc.lo;
        wt.rt = dd_add(wt.rt, emc);
    } else if (lane < nb) {
        dd r = dd_sub(n0[lane], used[lane]);
        ph[lane] = ph2{r.hi, r.lo};
    }
    wt.cnt[C_PART] += wsum_i(c_part);
    for (int q = 0; q < NS; ++q) wt.cnt[C_PH0 + q] += wsum_i(c_ph[q]);
    __syncwarp();
}

// ---- rad step: K-vacancy decay with KLL Auger / K-alpha branching ----
__device__ __noinline__ void stage_decay(const CellArgs &a, const WarpMem &m, const Tables &T, const SlabDev &S,
                                         const CellCtx &c, int lane, int &nnew, WarpTally &wt)
{
    const int ni = c.ni, nb = S.nb;
    const real wi = c.wi;
    const real dtr = S.rad_every * S.dt;
    dd *addph = m.ph;
    if (lane < MAXB) addph[lane] = dd_zero();
    __syncwarp();
    int c_aug = 0, c_ka = 0;
    for (int b0 = 0; b0 < ni; b0 += 32) {
        int t = b0 + lane;
        int kind = 0, sl = 0, Z = 0;
        real EA = RF(0.), rc = RF(0.), rp = RF(0.), Eka = RF(0.);
        if (t < ni) {
            sl = m.iperm[t];
            int st = m.ist[sl];
            Z = st & 0xff;
            int nK = (st >> 8) & 0xff;
            int nbd = ZNUC - Z, occ[NS];
            if (nK > 0 && occupancy(nbd, nK, occ)) {
                real tau = T.tauK[nbd][nK - 1];
                if (tau > RF(0.)) {
                    U4 r = draw(c.seed, (unsigned long long)m.iid[t], c.step, PU_DECAY);
                    if (u01(r.x) < dtr / tau) {
                        real om = T.omegaK[nbd][nK - 1];
                        int nl = occ[1] + occ[2];
                        if (u01(r.y) < RF(1.0) - om) {
                            if (nl >= 2) {
                                real e2s = lowered_binding(T, Z, 1, m.dE[Z]);
                                real e2p = lowered_binding(T, Z, 2, m.dE[Z]);
                                EA = r_fmax(T.E_Ka[Z] - (occ[1] * e2s + occ[2] * e2p) / nl, RF(0.0));
                                int kocc = occ[0] + 1, nb2 = nbd - 1;
                                int Zn = Z + 1, nKn = (nb2 < 2 ? nb2 : 2) - kocc;
                                m.ist[sl] = Zn | (nKn << 8);
                                kind = 1;
                                rc = u01(r.z); rp = u01(r.w);
                            }
                        } else if (occ[2] >= 1) {
                            Eka = T.E_Ka[Z];
                            m.ist[sl] = Z | ((nK - 1) << 8);
                            kind = 2;
                        }
                    }
                }
            }
        }
        unsigned bal = __ballot_sync(FULL, kind == 1);
        if (kind == 1) {
            int pos = nnew + __popc(bal & ((1u << lane) - 1u));
            if (pos < a.cap_new) {
                real3 u = iso_momentum(EA, rc, rp);
                NewE q; q.ux = u.x; q.uy = u.y; q.uz = u.z; q.w = wi; q.meta = sl | (KIND_AUGER << 16);
                m.nw[pos] = q;
            } else {
                atomicOr(a.err, ERR_NEW_OVERFLOW);
            }
            c_aug++;
        }
        nnew = min(nnew + __popc(bal), a.cap_new);
        int hit = -1;
        if (kind == 2) {
            c_ka++;
            for (int b = 0; b < nb; ++b)
                if (Eka >= S.hv_b[b] - S.bin_hw && Eka < S.hv_b[b] + S.bin_hw) { hit = b; break; }
        }
        for (int b = 0; b < nb; ++b) {
            dd v = wsum_dd(dd{hit == b ? wi * Eka / S.hv_b[b] : RF(0.0), RF(0.0)});
            if (lane == 0) addph[b] = dd_add(addph[b], v);
        }
        wt.ka = dd_add(wt.ka, wsum_dd(dd{kind == 2 && hit < 0 ? wi * Eka : RF(0.0), RF(0.0)}));
        wt.ion = dd_sub(wt.ion, wsum_dd(dd{kind == 1 ? wi * EA : (kind == 2 ? wi * Eka : RF(0.0)), RF(0.0)}));
        __syncwarp();
    }
    if (nb && lane < nb) {
        ph2 *ph = a.photons + S.ph_off + (size_t)c.lc * nb;
        ph2 v = ph[lane];
        dd r = dd_add(dd{v.hi, v.lo}, addph[lane]);
        ph[lane] = ph2{r.hi, r.lo};
    }
    wt.cnt[C_AUG] += wsum_i(c_aug);
    wt.cnt[C_KA] += wsum_i(c_ka);
    __syncwarp();
}

// One round: every warp of the block takes at most one cell; the stages
// are separated by block barriers so the warps of an SM fetch the same code
// at the same time (the stages are long and the instruction cache small).
template <int RMAX>
__device__ void process_round(const CellArgs &a, const WarpMem &m, const Tables &T, int g, int lane, WarpTally &wt)
{
    bool on = g >= 0;
    int s = 0;
    const SlabDev *Sp = a.slabs;
    unsigned step = 0, flags = 0;
    unsigned long long seed = 0;
    int lc = 0, cx = 0, cy = 0, e0 = 0, ne = 0, i0 = 0, ni = 0;
    if (on) {
        s = __ldg(a.cell_slab + g);
        if (s != wt.slab) { tally_flush(a, wt, lane); wt.slab = s; }
        Sp = a.slabs + s;
        step = a.steps[s];
        seed = Sp->seed;
        flags = Sp->flags;
        lc = g - Sp->cell0;
        cx = lc % Sp->nx; cy = lc / Sp->nx;
        e0 = a.cs_e[g]; ne = a.cs_e[g + 1] - e0;
        i0 = a.cs_i[g]; ni = a.cs_i[g + 1] - i0;
        on = (ne > 0 || ni > 0) && Sp->active;
    }
    const SlabDev &S = *Sp;
    const real wi = S.w_ion;
    const real mi = S.m_ion;
    const bool rad = S.rad_every > 0 && (step % (unsigned)S.rad_every) == 0;
    const real MC2 = (real)kMeC2;
    const real nref = S.nref_f;
    int c_ee = 0, c_ei = 0, c_ion = 0, c_rej = 0;
    real n_e = RF(0.), n_i = RF(0.), Te = RF(0.), zbar = RF(0.), lnL = RF(2.);
    const bool coll = (flags & 3u) != 0;
    const bool all_bulk = S.E_bulk <= RF(0.0);
    dd Kpre = dd_zero();
    int nnew = 0;
    real Wnew_imp = RF(0.0);
    // sums carried from stage to stage (see CellCtx)
    dd Qcell = dd_zero(), Kall = dd_zero(), Kt = dd_zero(), paid_cell = dd_zero();
    real We_cell = RF(0.0);
    int n_imp = 0;
    bool ew_ready = false, ionized = false;

    if (on) {
    // ---- stage in shared memory; Philox sort keys ----
    for (int k = lane; k < ne; k += 32) {
        real4 P0 = a.e0[e0 + k], P1 = a.e1[e0 + k];
        m.eu[k] = make_real4(P0.z, P0.w, P1.x, P1.y);
        m.epos[k] = make_real2(P0.x, P0.y);
        unsigned long long id = rec_eid(P1);
        U4 r = draw(seed, id, step, PU_PAIR_E);
        m.ekey[k] = ((unsigned long long)r.x << 32) | r.y;
        m.eid[k] = id;
        m.eperm[k] = (unsigned short)k;
    }
    for (int k = lane; k < ni; k += 32) {
        real4 P0 = a.i0[i0 + k], P1 = a.i1[i0 + k];
        m.iu[k] = make_real4(P0.z, P0.w, P1.x, P1.y);
        m.ipos[k] = make_real2(P0.x, P0.y);
        m.ist[k] = rec_ist(P1);
        unsigned id = rec_iid(P1);
        U4 r = draw(seed, (unsigned long long)id, step, PU_PAIR_I);
        m.ikey[k] = ((unsigned long long)r.x << 32) | r.y;
        m.iid[k] = id;
        m.iperm[k] = (unsigned short)k;
    }
    __syncwarp();
    // the sorted keys are not needed after the sort: they serve as scratch
    warp_sort<unsigned long long, RMAX>(m.ekey, m.eid, m.eperm, m.ekey, m.rbuf, m.rhist, ne, lane);
    warp_sort<unsigned int, RMAX>(m.ikey, m.iid, m.iperm, m.ikey, m.rbuf, m.rhist, ni, lane);

    }
    __syncthreads();

    if (on && rad && S.rt) {
    // ---- transport mode: the energy the radiation field gave up to (or
    //      took from) this cell goes to its bulk electrons by one factor on
    //      their kinetic energy (Sec. II), at most 90 % of it taken; the rest
    //      waits for the next rad step ----
    if (lane < S.nb) S.rt_chi[(size_t)lc * S.nb + lane] = 0.0f;
    if (lane == 0) S.rt_emc[lc] = 0.0;
    const double dEc = S.rt_dE[lc];
    if (dEc != 0.0) {
        dd pk = dd_zero();
        for (int k = lane; k < ne; k += 32) {
            const real4 u = m.eu[m.eperm[k]];
            const real ke = MC2 * gm1(u.x, u.y, u.z);
            if (S.E_bulk <= RF(0.0) || ke < S.E_bulk) pk = dd_addf(pk, u.w * ke);
        }
        const real K = dd_f(wsum_dd(pk));
        if (K > RF(0.0)) {
            const real dEa = (real)dEc < -RF(0.9) * K ? -RF(0.9) * K : (real)dEc;
            const real delta = -dEa / K;
            for (int k = lane; k < ne; k += 32) {
                const int sl = m.eperm[k];
                real4 u = m.eu[sl];
                const real ke = MC2 * gm1(u.x, u.y, u.z);
                if (S.E_bulk <= RF(0.0) || ke < S.E_bulk) { scale_kinetic(u.x, u.y, u.z, delta); m.eu[sl] = u; }
            }
            if (lane == 0) S.rt_dE[lc] = dEc - (double)dEa;
            wt.rt = dd_addf(wt.rt, dEa);
        }
    }
    __syncwarp();
    }

    if (on) {
    // ---- cell moments (Sec. II: T_e = 2/3 E_ave over bulk electrons) ----
    dd We = dd_zero(), Wb = dd_zero(), Kb = dd_zero(), Q = dd_zero(), Ka = dd_zero();
    for (int k = lane; k < ne; k += 32) {
        real4 u = m.eu[m.eperm[k]];
        const real g1 = gm1(u.x, u.y, u.z);
        const real ke = MC2 * g1;
        // w * MC2 * g1: the same rounding as the kernel's other kinetic-energy
        // sums, so that the collision energy restore does not see a bias
        // between two formulas of the same energy
        const real wk = u.w * MC2 * g1;
        We = dd_addf(We, u.w);
        if (all_bulk || ke < S.E_bulk) { Wb = dd_addf(Wb, u.w); Kb = dd_addf(Kb, wk); }
        if (!all_bulk) Ka = dd_addf(Ka, wk);
    }
    for (int k = lane; k < ni; k += 32) {
        int sl = m.iperm[k];
        Q = dd_addf(Q, (real)(m.ist[sl] & 0xff) + m.iu[sl].w);
    }
    We = wsum_dd(We); Wb = wsum_dd(Wb); Kb = wsum_dd(Kb); Q = wsum_dd(Q);
    Kall = all_bulk ? Kb : wsum_dd(Ka);
    Qcell = Q;
    We_cell = dd_f(We);
    n_e = dd_f(We) * nref; n_i = (real)ni * wi * nref;
    Te = dd_f(Wb) > RF(0.0) ? (RF(2.0) / RF(3.0)) * dd_f(Kb) / dd_f(Wb) : RF(0.0);
    zbar = ni > 0 ? dd_f(Q) / ni : RF(0.0);
    if (lane < NZ) m.dE[lane] = ipd_shift(S.ipd, lane, n_e, n_i, Te, zbar);
    lnL = S.coulomb_log > RF(0.0) ? S.coulomb_log : coulomb_log(n_e, Te, zbar);
    __syncwarp();

    // ---- binary collisions (Sec. IV): e-e, then e-i; exact energy restore ----
    if (coll) {
        // electron part from the moments above; the ions' own pass
        dd pki = dd_zero();
        for (int k = lane; k < ni; k += 32) { real4 u = m.iu[m.iperm[k]]; pki = dd_addf(pki, wi * MC2 * mi * gm1(u.x, u.y, u.z)); }
        Kpre = dd_add(Kall, wsum_dd(pki));
    }
    if ((flags & 1u) && ne >= 2) {
        const int start = (ne & 1) ? 3 : 0;
        auto ee = [&](int pa, int pb, real dtc) {
            int sa = m.eperm[pa], sb = m.eperm[pb];
            real4 A = m.eu[sa], B = m.eu[sb];
            real3 ua = make_real3(A.x, A.y, A.z), ub = make_real3(B.x, B.y, B.z);
            U4 r = draw(seed, m.eid[pa], step, PU_COLL_EE);
            if (binary_collision(ua, ub, RF(1.0), RF(1.0), -RF(1.0), -RF(1.0), A.w, B.w, n_e, lnL, dtc,
                                 u01(r.x), u01(r.y), u01(r.z), u01(r.w))) c_ee++;
            m.eu[sa] = make_real4(ua.x, ua.y, ua.z, A.w);
            m.eu[sb] = make_real4(ub.x, ub.y, ub.z, B.w);
        };
        if ((ne & 1) && lane == 0) {
            ee(0, 1, RF(0.5) * S.dt);
            ee(1, 2, RF(0.5) * S.dt);
            ee(2, 0, RF(0.5) * S.dt);
        }
        const int npairs = (ne - start) >> 1;
        for (int p = lane; p < npairs; p += 32) ee(start + 2 * p, start + 2 * p + 1, S.dt);
        __syncwarp();
    }

    }
    __syncthreads();     // the e-i code next: warps in step, as elsewhere

    if (on) {
    if ((flags & 2u) && ne >= 1 && ni >= 1) {
        const bool e_long = ne >= ni;
        const int nlong = e_long ? ne : ni, nshort = e_long ? ni : ne;
        for (int base = 0; base < nlong; base += nshort) {
            int cnt = min(nshort, nlong - base);
            for (int t = lane; t < cnt; t += 32) {
                int pe = e_long ? base + t : t;
                int pi = e_long ? t : base + t;
                int se = m.eperm[pe], si = m.iperm[pi];
                real4 A = m.eu[se], B = m.iu[si];
                real q = (real)(m.ist[si] & 0xff) + B.w;
                real npair = e_long ? n_i * r_fmax(A.w, wi) / wi : n_e * r_fmax(A.w, wi) / A.w;
                U4 r = e_long ? draw(seed, m.eid[pe], step, PU_COLL_EI)
                              : draw(seed, (unsigned long long)m.iid[pi], step, PU_COLL_IE);
                real3 ua = make_real3(A.x, A.y, A.z), ub = make_real3(B.x, B.y, B.z);
                if (binary_collision(ua, ub, RF(1.0), mi, -RF(1.0), q, A.w, wi, npair, lnL, S.dt,
                                     u01(r.x), u01(r.y), u01(r.z), u01(r.w))) c_ei++;
                m.eu[se] = make_real4(ua.x, ua.y, ua.z, A.w);
                m.iu[si] = make_real4(ub.x, ub.y, ub.z, B.w);
            }
            __syncwarp();
        }
    }
    if (coll && ne >= 1) {
        dd pk = dd_zero(), pki = dd_zero();
        for (int k = lane; k < ne; k += 32) { real4 u = m.eu[m.eperm[k]]; pk = dd_addf(pk, u.w * MC2 * gm1(u.x, u.y, u.z)); }
        for (int k = lane; k < ni; k += 32) { real4 u = m.iu[m.iperm[k]]; pki = dd_addf(pki, wi * MC2 * mi * gm1(u.x, u.y, u.z)); }
        dd Ke = wsum_dd(pk), Ki = wsum_dd(pki);
        real ke = dd_f(Ke);
        real delta = RF(0.0);
        if (ke > RF(0.0)) {
            delta = -dd_f(dd_sub(dd_sub(Kpre, Ke), Ki)) / ke;     // f = 1 - delta
            if (!(delta < RF(1.0))) delta = RF(0.0);
        }
        if ((flags & 4u) && ni >= 1) {
            // the restore and the ionization stage's per-electron inputs in
            // one pass: kinetic energy and w * beta after the restore, in
            // the sort-key storage (free until recombination), and their sum
            real2 *ew = reinterpret_cast<real2 *>(m.ekey);
            dd pt = dd_zero();
            for (int k = lane; k < ne; k += 32) {
                const int sl = m.eperm[k];
                real4 u = m.eu[sl];
                scale_kinetic(u.x, u.y, u.z, delta);
                m.eu[sl] = u;
                real u2 = u.x * u.x + u.y * u.y + u.z * u.z;
                real g1 = u2 / (r_sqrt(RF(1.0) + u2) + RF(1.0));
                pt = dd_addf(pt, u.w * MC2 * g1);
                ew[k] = make_real2(MC2 * g1, u.w * (r_sqrt(u2) / (RF(1.0) + g1)));
            }
            Kt = wsum_dd(pt);
            ew_ready = true;
        } else if (delta != RF(0.0)) {
            for (int k = lane; k < ne; k += 32) {
                real4 u = m.eu[k];
                scale_kinetic(u.x, u.y, u.z, delta);
                m.eu[k] = u;
            }
        }
        __syncwarp();
    }

    }
    __syncthreads();

    if (on) {
    // ---- Lotz impact ionization, cell-average probability (Eq. 3) ----
    if ((flags & 4u) && ne >= 1 && ni >= 1) {
        unsigned pmask = 0;
        for (int k = lane; k < ni; k += 32) { int Z = m.ist[k] & 0xff; if (Z < ZNUC) pmask |= 1u << Z; }
        for (int o = 16; o > 0; o >>= 1) pmask |= __shfl_xor_sync(FULL, pmask, o);
        // kinetic energy and w * beta of each electron (canonical order), kept
        // in the sort-key storage, which is free until recombination
        real2 *ew = reinterpret_cast<real2 *>(m.ekey);
        int nhot;
        if (!ew_ready) {
            dd pk = dd_zero();
            for (int k = lane; k < ne; k += 32) {
                real4 u = m.eu[m.eperm[k]];
                real u2 = u.x * u.x + u.y * u.y + u.z * u.z;
                real g1 = u2 / (r_sqrt(RF(1.0) + u2) + RF(1.0));
                pk = dd_addf(pk, u.w * MC2 * g1);
                ew[k] = make_real2(MC2 * g1, u.w * (r_sqrt(u2) / (RF(1.0) + g1)));
            }
            Kt = wsum_dd(pk);
        }
        __syncwarp();
        // Electrons at or below the lowest lowered binding of every charge
        // state present ionize nothing and add nothing to the sums: the
        // others (a hot tail, typically a few per cent) are gathered in
        // canonical order to the front of the storage, so that a warp's
        // lanes do not idle beside the one lane with a hot electron.
        nhot = ne;
        {
            real Pall = RF(3.0e38);
            for (int z = 0; z < ZNUC; ++z) {
                if (!(pmask & (1u << z))) continue;
                if (lane < NS && subshell_occ(ZNUC - z, lane) > 0)
                    Pall = r_fmin(Pall, lowered_binding(T, z, lane, m.dE[z]));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) Pall = r_fmin(Pall, __shfl_xor_sync(FULL, Pall, o));
            int nh = 0;
            for (int b0 = 0; b0 < ne; b0 += 32) {
                const int k = b0 + lane;
                const real2 q = k < ne ? ew[k] : make_real2(RF(0.0), RF(0.0));
                const bool hot = k < ne && q.x > Pall;
                const unsigned bal = __ballot_sync(FULL, hot);
                __syncwarp();
                if (hot) ew[nh + __popc(bal & ((1u << lane) - 1u))] = q;
                nh += __popc(bal);
                __syncwarp();
            }
            nhot = nh;
        }
        const real cfac = (real)(kCcmPerFs) * S.dt * nref;
        for (int z = 0; z < ZNUC; ++z) {
            if (!(pmask & (1u << z))) continue;
            // Lotz constants of charge state z (lowest-energy configuration):
            // lowered binding P, 1/P, ln P, a * occupation (0: empty subshell)
            if (lane < NS) {
                const int o = subshell_occ(ZNUC - z, lane);
                real4 v = make_real4(RF(0.0), RF(0.0), RF(0.0), RF(0.0));
                if (o > 0) {
                    const real P = lowered_binding(T, z, lane, m.dE[z]);
                    v = make_real4(P, RF(1.0) / P, r_log(P), T.lotz_a[lane] * (real)o);
                }
                m.lz[lane] = v;
            }
            __syncwarp();
            // the lowest lowered binding of the charge state: electrons at
            // or below it ionize no subshell and add nothing to the sum
            real Pmin = RF(3.0e38);
#pragma unroll
            for (int sh = 0; sh < NS; ++sh)
                if (m.lz[sh].w > RF(0.0)) Pmin = r_fmin(Pmin, m.lz[sh].x);
            // fast log / exp: a few ulp on a probability; only a decision
            // within that of its threshold could flip
            dd pr = dd_zero();
            for (int k = lane; k < nhot; k += 32) {
                const real2 q = ew[k];
                if (!(q.x > Pmin)) continue;
                const real E = q.x, lnE = r_flog(E), invE = RF(1.0) / E;
                real sig = RF(0.0);
#pragma unroll
                for (int sh = 0; sh < NS; ++sh) {
                    const real4 L = m.lz[sh];
                    if (L.w > RF(0.0) && E > L.x) {
                        const real x = E * L.y;
                        sig += L.w * (lnE - L.z) * (invE * L.y) *
                               (RF(1.0) - T.lotz_b[sh] * r_fexp(-T.lotz_c[sh] * (x - RF(1.0))));
                    }
                }
                pr = dd_addf(pr, q.y * sig);
            }
            real P = cfac * dd_f(wsum_dd(pr));
            if (lane == 0) m.Pz[z] = P;
            if (P > RF(1.0) && lane == 0) wt.cnt[C_PGT1]++;
            __syncwarp();
        }
        __syncwarp();
        dd carry = dd_zero(), paid = dd_zero();
        for (int b0 = 0; b0 < ni; b0 += 32) {
            int t = b0 + lane;
            bool cand = false;
            real cost = RF(0.0);
            int sl = 0, Z = 0, nK = 0;
            if (t < ni) {
                sl = m.iperm[t];
                int st = m.ist[sl];
                Z = st & 0xff; nK = (st >> 8) & 0xff;
                if (Z < ZNUC) {
                    U4 r = draw(seed, (unsigned long long)m.iid[t], step, PU_ION);
                    if (u01(r.x) < m.Pz[Z]) {
                        cand = true;
                        cost = wi * removal_energy(T, Z, nK, m.dE[Z]);
                    }
                }
            }
            dd incl = dd_add(carry, wscan_dd(dd{cost, RF(0.0)}, lane));
            bool acc = cand && dd_le(incl, Kt);
            if (cand && !acc) c_rej++;
            unsigned bal = __ballot_sync(FULL, acc);
            if (acc) {
                int so = outer_shell(ZNUC - Z, nK);
                lose_electron(Z, nK, so);
                m.ist[sl] = Z | (nK << 8);
                int pos = nnew + __popc(bal & ((1u << lane) - 1u));
                if (pos < a.cap_new) {
                    NewE q; q.ux = q.uy = q.uz = RF(0.0); q.w = wi; q.meta = sl | (KIND_IMPACT << 16);
                    m.nw[pos] = q;
                } else {
                    atomicOr(a.err, ERR_NEW_OVERFLOW);
                }
                c_ion++;
            }
            paid = dd_add(paid, wsum_dd(dd{acc ? cost : RF(0.0), RF(0.0)}));
            nnew += __popc(bal);
            n_imp += __popc(bal);
            carry = wbcast_dd(incl, 31);
        }
        nnew = min(nnew, a.cap_new);
        Wnew_imp = nnew * wi;
        paid_cell = paid;
        ionized = true;
        real pf = dd_f(paid);
        if (pf > RF(0.0)) {
            real delta = pf / dd_f(Kt);
            for (int k = lane; k < ne; k += 32) {
                real4 u = m.eu[k];
                scale_kinetic(u.x, u.y, u.z, delta);
                m.eu[k] = u;
            }
            wt.ion = dd_add(wt.ion, paid);
        }
        __syncwarp();
    }

    }
    __syncthreads();

    if (on) {
    CellCtx cc;
    cc.s = s; cc.lc = lc; cc.cx = cx; cc.cy = cy; cc.e0 = e0; cc.ne = ne; cc.i0 = i0; cc.ni = ni;
    cc.step = step; cc.flags = flags; cc.seed = seed; cc.wi = wi; cc.mi = mi; cc.n_e = n_e; cc.n_i = n_i;
    cc.nref = nref; cc.rad = rad;
    cc.have_sums = all_bulk && ionized;
    cc.K_after = dd_sub(Kt, paid_cell);
    cc.W_e = We_cell;
    cc.Q_after = dd_f(Qcell) + (real)n_imp;
    if ((flags & 8u) && ni >= 1) stage_recombine(a, m, T, S, cc, lane, Wnew_imp, wt);
    if (rad && (flags & 16u) && S.nb && ni >= 1) stage_photo(a, m, T, S, cc, lane, nnew, wt);
    if (rad && (flags & 32u) && ni >= 1) stage_decay(a, m, T, S, cc, lane, nnew, wt);
    if (rad && (flags & 256u)) stage_therm(a, m, cc, lane, nnew);

    // ---- write the collided state back, each cell's records in its
    //      canonical order (the order the push kernel follows) ----
    for (int k = lane; k < ne; k += 32) {
        const int sl = m.eperm[k];
        const real4 u = m.eu[sl];
        const real2 x = m.epos[sl];
        a.e0[e0 + k] = make_real4(x.x, x.y, u.x, u.y);
        a.e1[e0 + k] = rec_e1(u.z, u.w, m.eid[k]);
    }
    if (rad && S.rt) {
        // transport mode: the cell's electron weight after the step, created
        // electrons included: its share of the next heating of its rad cell
        // (summed in canonical order: the slots' order is the scatter's)
        real wsum = RF(0.0);
        for (int k = lane; k < ne; k += 32) {
            const real w = m.eu[m.eperm[k]].w;
            wsum += w > RF(0.0) ? w : RF(0.0);
        }
        for (int k = lane; k < nnew; k += 32) wsum += m.nw[k].w;
        wsum = wsum_f(wsum);
        if (lane == 0) S.rt_w[lc] = (float)wsum;
    }
    // ---- created electrons: after the sorted range, at their ion, with their cell as key ----
    if (nnew > 0) {
        // a slab with a budget of its own keeps its electrons within it: a
        // cell that would take it beyond drops what it created and fails
        // the slab alone (it is stopped at the end of the step); the others
        // never see the shared capacity run out when the budgets fit in it
        int base = 0, fits = 1;
        if (lane == 0) {
            if (S.budget_e > 0) {
                const int held = a.cs_e[S.cell0 + S.ncell] - a.cs_e[S.cell0];
                if (held + atomicAdd(a.slab_app + s, nnew) + nnew > S.budget_e) {
                    atomicOr(a.slab_err + s, ERR_CAPACITY);
                    fits = 0;
                }
            }
            if (fits) base = atomicAdd(a.append, nnew);
        }
        fits = __shfl_sync(FULL, fits, 0);
        base = __shfl_sync(FULL, base, 0);
        const int sorted = a.cs_e[a.ncell];
        int n_ok = fits ? nnew : 0;
        if (fits && sorted + base + nnew > a.cap_e) {
            if (lane == 0) atomicOr(a.err, ERR_CAPACITY);
            for (int k = sorted + base + lane; k < min(a.cap_e, sorted + base + nnew); k += 32) a.ekey[k] = -1;
            n_ok = 0;
        }
        for (int k = lane; k < n_ok; k += 32) {
            NewE q = m.nw[k];
            int islot = q.meta & 0xffff, kind = q.meta >> 16;
            real4 I0 = a.i0[i0 + islot];
            real4 I1 = a.i1[i0 + islot];
            unsigned idhi = ((step + 1u) << 2) | (unsigned)kind;
            a.e0[sorted + base + k] = make_real4(I0.x, I0.y, q.ux, q.uy);
            a.e1[sorted + base + k] = rec_e1(q.uz, q.w, ((unsigned long long)idhi << 32) | rec_iid(I1));
            a.ekey[sorted + base + k] = g;
        }
    }
    __syncwarp();
    // ions last: the created electrons above read their parent ions' records
    // at the ions' slots
    for (int k = lane; k < ni; k += 32) {
        const int sl = m.iperm[k];
        const real4 u = m.iu[sl];
        const real2 x = m.ipos[sl];
        a.i0[i0 + k] = make_real4(x.x, x.y, u.x, u.y);
        a.i1[i0 + k] = rec_i1(u.z, u.w, m.iid[k], m.ist[sl]);
    }

    // ---- tallies (lane-uniform) ----
    wt.cnt[C_EE] += wsum_i(c_ee);
    wt.cnt[C_EI] += wsum_i(c_ei);
    wt.cnt[C_ION] += wsum_i(c_ion);
    wt.cnt[C_ION_REJ] += wsum_i(c_rej);
    __syncwarp();
    }
    __syncthreads();
}

// Each round the block takes one cell per warp from a shared counter.
// Cells whose population exceeds this launch's shared-memory capacity go to
// a list for the large-cell launch.
// RMAX: the largest cell sorted in registers (128: launches whose staging
// holds at most 128 entries per species; 512: up to 512; 1024: the launches
// for larger cells, with up to 255 registers a thread for the 32-entry
// register sort, radix-sorting cells above 1024).
template <int RMAX>
__global__ void __launch_bounds__(RMAX > 512 ? 128 : 256, RMAX > 512 ? 1 : 2) k_cell(CellArgs a)
{
    extern __shared__ __align__(kSmAlign) char smem[];
    __shared__ Tables T;
    __shared__ int round_base;
    for (int k = threadIdx.x; k < (int)(sizeof(Tables) / sizeof(real)); k += blockDim.x)
        ((real *)&T)[k] = ((const real *)a.tab)[k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const size_t gwarp = (size_t)blockIdx.x * nwarp + warp;
    WarpMem m = carve(smem + (size_t)warp * warp_mem_bytes(a.cap_ce, a.cap_ci), a.cap_ce, a.cap_ci,
                      a.nw + gwarp * a.cap_new, a.gw + gwarp * warp_gmem_words(a.cap_ce, a.cap_ci));
    const int total = a.list ? *a.n_list : a.ncell;
    WarpTally wt;
    wt.slab = -1;
    wt.ion = wt.ka = wt.esc = wt.rt = dd_zero();
    for (int q = 0; q < NCOUNT; ++q) wt.cnt[q] = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) round_base = atomicAdd(a.work, nwarp);
        __syncthreads();
        const int base = round_base;
        if (base >= total) break;
        int g = -1;
        if (base + warp < total) {
            g = a.list ? a.list[base + warp] : base + warp;
            int ne = a.cs_e[g + 1] - a.cs_e[g], ni = a.cs_i[g + 1] - a.cs_i[g];
            if (ne > a.cap_ce || ni > a.cap_ci || 3 * ni > a.cap_new) {
                if (a.ovf_list) {
                    if (lane == 0) a.ovf_list[atomicAdd(a.ovf_count, 1)] = g;
                } else {
                    // no larger pass left: report, and drop the cell's particles so
                    // that the next sort stays consistent
                    if (lane == 0) atomicOr(a.err, ERR_CELL_OVERFLOW);
                    for (int k = a.cs_e[g] + lane; k < a.cs_e[g + 1]; k += 32)
                        reinterpret_cast<real *>(a.e1 + k)[1] = RF(0.0);
                    for (int k = a.cs_i[g] + lane; k < a.cs_i[g + 1]; k += 32) a.i1[k].w = bits_real(0xffu);
                }
                g = -1;
            }
        }
        process_round<RMAX>(a, m, T, g, lane, wt);
    }
    tally_flush(a, wt, lane);
}

}  // namespace pic
