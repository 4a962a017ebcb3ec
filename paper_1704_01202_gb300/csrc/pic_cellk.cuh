// The fused per-cell kernel (see pic_cell.cuh for the building blocks).
#pragma once
#include <type_traits>
#include "pic_cell.cuh"

namespace pic {

struct LaneTally {        // per-lane event counts, reduced once per cell
    int coll_ee, coll_ei, ion, ion_rej, rec, ph[NS], part, aug, ka, pgt1, esc_e, esc_i;
};

template <int DIM>
__device__ void cell_push_deposit(const CellArgs &a, const SlabDev &S, const WarpMem &m, int g, int cx, int cy,
                                  int e0, int ne, int i0, int ni, int nnew, int lane, double &esc_e_energy,
                                  LaneTally &lt)
{
    const unsigned flags = S.flags;
    const bool do_push = flags & 64u, do_dep = (flags & 128u) != 0;
    SlabGrid grid;
    grid.nx = S.nx; grid.ny = S.ny; grid.W = S.nx + 1;
    grid.fe = a.fldE + S.fld_off; grid.fb = a.fldB + S.fld_off; grid.npts = a.npts; grid.fo = S.fld_off;
    typename std::conditional<DIM == 2, JAcc2, JAcc1>::type A = {};
    const int cell0 = S.cell0;
    const float wi = S.w_ion;

    // electrons present at the start of the step, canonical order
    for (int k = lane; k < ne; k += 32) {
        int slot = m.eperm[k];
        float4 uw = m.eu[slot];
        float4 P0 = a.e0[e0 + slot];
        float4 P1 = a.e1[e0 + slot];
        int key;
        if (uw.w <= 0.0f) {
            key = -1;
        } else {
            float xi = P0.x, eta = P0.y, ux = uw.x, uy = uw.y, uz = uw.z;
            float ke = (float)kMeC2 * gm1(ux, uy, uz);
            int nc = push_one<DIM>(S, grid, a.J, a.npts, cx, cy, xi, eta, ux, uy, uz, -1.0f, -uw.w, do_push, do_dep, A);
            if (nc == -2) { key = -1; atomicOr(a.err, ERR_NUMERIC); }
            else if (nc < 0) { key = -1; esc_e_energy += (double)uw.w * ke; lt.esc_e++; }
            else key = cell0 + nc;
            P0 = make_float4(xi, eta, ux, uy);
            P1.x = uz; P1.y = uw.w;
        }
        a.e0[e0 + slot] = P0;
        a.e1[e0 + slot] = P1;
        a.ekey[e0 + slot] = key;
        if (key >= 0) atomicAdd(a.cnt_e + key, 1);
    }

    // electrons created in this cell this step
    int base = 0;
    if (nnew > 0) {
        if (lane == 0) base = atomicAdd(a.append, nnew);
        base = __shfl_sync(FULL, base, 0);
        const int sorted = a.cs_e[a.ncell];
        if (sorted + base + nnew > a.cap_e) {
            if (lane == 0) atomicOr(a.err, ERR_CAPACITY);
            for (int k = sorted + base + lane; k < min(a.cap_e, sorted + base + nnew); k += 32) a.ekey[k] = -1;
            nnew = 0;
        }
        base += sorted;
    }
    for (int k = lane; k < nnew; k += 32) {
        NewE q = m.nw[k];
        int islot = q.meta & 0xffff, kind = q.meta >> 16;
        float4 I0 = a.i0[i0 + islot];
        float4 I1 = a.i1[i0 + islot];
        float xi = I0.x, eta = I0.y, ux = q.ux, uy = q.uy, uz = q.uz;
        float ke = (float)kMeC2 * gm1(ux, uy, uz);
        int nc = push_one<DIM>(S, grid, a.J, a.npts, cx, cy, xi, eta, ux, uy, uz, -1.0f, -q.w, do_push, do_dep, A);
        int key;
        if (nc == -2) { key = -1; atomicOr(a.err, ERR_NUMERIC); }
        else if (nc < 0) { key = -1; esc_e_energy += (double)q.w * ke; lt.esc_e++; }
        else key = cell0 + nc;
        unsigned idhi = ((a.steps[a.cell_slab[g]] + 1u) << 2) | (unsigned)kind;
        unsigned idlo = __float_as_uint(I1.z);
        a.e0[base + k] = make_float4(xi, eta, ux, uy);
        a.e1[base + k] = make_float4(uz, q.w, __uint_as_float(idlo), __uint_as_float(idhi));
        a.ekey[base + k] = key;
        if (key >= 0) atomicAdd(a.cnt_e + key, 1);
    }

    // ions, canonical order
    for (int k = lane; k < ni; k += 32) {
        int slot = m.iperm[k];
        float4 iu = m.iu[slot];
        int st = m.ist[slot];
        float4 P0 = a.i0[i0 + slot];
        float4 P1 = a.i1[i0 + slot];
        float q = (float)(st & 0xff) + iu.w;
        float xi = P0.x, eta = P0.y, ux = iu.x, uy = iu.y, uz = iu.z;
        float ke = (float)kMeC2 * S.m_ion * gm1(ux, uy, uz);
        int nc = push_one<DIM>(S, grid, a.J, a.npts, cx, cy, xi, eta, ux, uy, uz, q / S.m_ion, q * wi, do_push, do_dep, A);
        int key;
        if (nc == -2) { key = -1; atomicOr(a.err, ERR_NUMERIC); }
        else if (nc < 0) { key = -1; esc_e_energy += (double)wi * ke; lt.esc_i++; }
        else key = cell0 + nc;
        a.i0[i0 + slot] = make_float4(xi, eta, ux, uy);
        a.i1[i0 + slot] = make_float4(uz, iu.w, P1.z, __int_as_float(st));
        a.ikey[i0 + slot] = key;
        if (key >= 0) atomicAdd(a.cnt_i + key, 1);
    }

    // the cell's current stencil: fixed reduction tree, then fixed point
    if (do_dep) {
        const int fo = S.fld_off, W = S.nx + 1;
        if constexpr (DIM == 2) {
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float v = A.x[p][q];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
                    A.x[p][q] = v;
                    float y = A.y[q][p];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(FULL, y, o);
                    A.y[q][p] = y;
                }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float v = A.z[p][q];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
                    A.z[p][q] = v;
                }
            if (lane == 0) {
                for (int p = 0; p < 4; ++p) {
                    int i = cx - 1 + p;
                    for (int q = 0; q < 4; ++q) {
                        int j = (cy - 1 + q) % S.ny; if (j < 0) j += S.ny;
                        size_t o = (size_t)fo + (size_t)j * W + i;
                        if (p < 3 && i >= 0 && i < S.nx) jatomic(a.J + o, A.x[p][q]);
                        if (q < 3 && i >= 0 && i <= S.nx) jatomic(a.J + a.npts + o, A.y[p][q]);
                        if (i >= 0 && i <= S.nx) jatomic(a.J + 2 * (size_t)a.npts + o, A.z[p][q]);
                    }
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                float x = p < 3 ? A.x[p < 3 ? p : 0] : 0.0f;
                float y = A.y[p], z = A.z[p];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    x += __shfl_down_sync(FULL, x, o);
                    y += __shfl_down_sync(FULL, y, o);
                    z += __shfl_down_sync(FULL, z, o);
                }
                if (p < 3) A.x[p] = x;
                A.y[p] = y; A.z[p] = z;
            }
            if (lane == 0) {
                for (int p = 0; p < 4; ++p) {
                    int i = cx - 1 + p;
                    if (p < 3 && i >= 0 && i < S.nx) jatomic(a.J + fo + i, A.x[p]);
                    if (i >= 0 && i <= S.nx) {
                        jatomic(a.J + a.npts + fo + i, A.y[p]);
                        jatomic(a.J + 2 * (size_t)a.npts + fo + i, A.z[p]);
                    }
                }
            }
        }
    }
}

__device__ void process_cell(const CellArgs &a, const WarpMem &m, const Tables &T, int g, int lane)
{
    const int s = __ldg(a.cell_slab + g);
    const SlabDev &S = a.slabs[s];
    const unsigned step = a.steps[s];
    const unsigned long long seed = S.seed;
    const unsigned flags = S.flags;
    const int lc = g - S.cell0;
    const int cx = lc % S.nx, cy = lc / S.nx;
    const int e0 = a.cs_e[g], ne = a.cs_e[g + 1] - e0;
    const int i0 = a.cs_i[g], ni = a.cs_i[g + 1] - i0;
    if (ne == 0 && ni == 0) return;
    const float wi = S.w_ion;
    const float mi = S.m_ion;
    const bool rad = S.rad_every > 0 && (step % (unsigned)S.rad_every) == 0;
    const float MC2 = (float)kMeC2;
    LaneTally lt = {};
    double tal_ion = 0.0, tal_ka = 0.0, tal_esc = 0.0;

    // ---- stage in shared memory; Philox sort keys ----
    for (int k = lane; k < ne; k += 32) {
        float4 P0 = a.e0[e0 + k], P1 = a.e1[e0 + k];
        m.eu[k] = make_float4(P0.z, P0.w, P1.x, P1.y);
        unsigned long long id = ((unsigned long long)__float_as_uint(P1.w) << 32) | __float_as_uint(P1.z);
        U4 r = draw(seed, id, step, PU_PAIR_E);
        m.ekey[k] = ((unsigned long long)r.x << 32) | r.y;
        m.eid[k] = id;
        m.eperm[k] = (unsigned short)k;
    }
    for (int k = lane; k < ni; k += 32) {
        float4 P0 = a.i0[i0 + k], P1 = a.i1[i0 + k];
        m.iu[k] = make_float4(P0.z, P0.w, P1.x, P1.y);
        m.ist[k] = __float_as_int(P1.w);
        unsigned id = __float_as_uint(P1.z);
        U4 r = draw(seed, (unsigned long long)id, step, PU_PAIR_I);
        m.ikey[k] = ((unsigned long long)r.x << 32) | r.y;
        m.iid[k] = id;
        m.iperm[k] = (unsigned short)k;
    }
    __syncwarp();
    warp_bitonic<unsigned long long>(m.ekey, m.eid, m.eperm, ne, lane);
    warp_bitonic<unsigned int>(m.ikey, m.iid, m.iperm, ni, lane);

    // ---- FP64 cell moments (Sec. II: T_e = 2/3 E_ave over bulk electrons) ----
    double We, Wb, Kb, Q;
    {
        float pw = 0.f, pwb = 0.f, pkb = 0.f, pq = 0.f;
        for (int k = lane; k < ne; k += 32) {
            float4 u = m.eu[m.eperm[k]];
            float ke = MC2 * gm1(u.x, u.y, u.z);
            pw += u.w;
            if (S.E_bulk <= 0.0f || ke < S.E_bulk) { pwb += u.w; pkb += u.w * ke; }
        }
        for (int k = lane; k < ni; k += 32) {
            int sl = m.iperm[k];
            pq += (float)(m.ist[sl] & 0xff) + m.iu[sl].w;
        }
        We = wsum(pw); Wb = wsum(pwb); Kb = wsum(pkb); Q = wsum(pq);
    }
    const double n_e = We * S.n_ref, n_i = (double)ni * wi * S.n_ref;
    const double Te = Wb > 0.0 ? (2.0 / 3.0) * Kb / Wb : 0.0;
    const double zbar = ni > 0 ? Q / ni : 0.0;
    if (lane < NZ) m.dE[lane] = ipd_shift(S.ipd, lane, n_e, n_i, Te, zbar);
    const float lnL = S.coulomb_log > 0.0f ? S.coulomb_log : coulomb_log(n_e, Te, zbar);
    __syncwarp();

    // ---- binary collisions (Sec. IV): e-e, then e-i; exact energy restore ----
    const bool coll = (flags & 3u) != 0;
    double Kpre = 0.0;
    if (coll) {
        float pk = 0.f;
        for (int k = lane; k < ne; k += 32) { float4 u = m.eu[m.eperm[k]]; pk += u.w * MC2 * gm1(u.x, u.y, u.z); }
        float pki = 0.f;
        for (int k = lane; k < ni; k += 32) { float4 u = m.iu[m.iperm[k]]; pki += MC2 * mi * gm1(u.x, u.y, u.z); }
        Kpre = wsum(pk) + (double)wi * wsum(pki);
    }
    if ((flags & 1u) && ne >= 2) {
        const int start = (ne & 1) ? 3 : 0;
        const float ne_f = (float)n_e;
        auto ee = [&](int pa, int pb, float dtc) {
            int sa = m.eperm[pa], sb = m.eperm[pb];
            float4 A = m.eu[sa], B = m.eu[sb];
            float3 ua = make_float3(A.x, A.y, A.z), ub = make_float3(B.x, B.y, B.z);
            U4 r = draw(seed, m.eid[pa], step, PU_COLL_EE);
            if (binary_collision(ua, ub, 1.0f, 1.0f, -1.0f, -1.0f, A.w, B.w, ne_f, lnL, dtc,
                                 u01(r.x), u01(r.y), u01(r.z), u01(r.w))) lt.coll_ee++;
            m.eu[sa] = make_float4(ua.x, ua.y, ua.z, A.w);
            m.eu[sb] = make_float4(ub.x, ub.y, ub.z, B.w);
        };
        if ((ne & 1) && lane == 0) {
            ee(0, 1, 0.5f * S.dt);
            ee(1, 2, 0.5f * S.dt);
            ee(2, 0, 0.5f * S.dt);
        }
        const int npairs = (ne - start) >> 1;
        for (int p = lane; p < npairs; p += 32) ee(start + 2 * p, start + 2 * p + 1, S.dt);
        __syncwarp();
    }
    if ((flags & 2u) && ne >= 1 && ni >= 1) {
        const bool e_long = ne >= ni;
        const int nlong = e_long ? ne : ni, nshort = e_long ? ni : ne;
        for (int base = 0; base < nlong; base += nshort) {
            int cnt = min(nshort, nlong - base);
            for (int t = lane; t < cnt; t += 32) {
                int pe = e_long ? base + t : t;
                int pi = e_long ? t : base + t;
                int se = m.eperm[pe], si = m.iperm[pi];
                float4 A = m.eu[se], B = m.iu[si];
                float q = (float)(m.ist[si] & 0xff) + B.w;
                float npair = e_long ? (float)(n_i * fmaxf(A.w, wi) / wi) : (float)(n_e * fmaxf(A.w, wi) / A.w);
                U4 r = e_long ? draw(seed, m.eid[pe], step, PU_COLL_EI)
                              : draw(seed, (unsigned long long)m.iid[pi], step, PU_COLL_IE);
                float3 ua = make_float3(A.x, A.y, A.z), ub = make_float3(B.x, B.y, B.z);
                if (binary_collision(ua, ub, 1.0f, mi, -1.0f, q, A.w, wi, npair, lnL, S.dt,
                                     u01(r.x), u01(r.y), u01(r.z), u01(r.w))) lt.coll_ei++;
                m.eu[se] = make_float4(ua.x, ua.y, ua.z, A.w);
                m.iu[si] = make_float4(ub.x, ub.y, ub.z, B.w);
            }
            __syncwarp();
        }
    }
    if (coll && ne >= 1) {
        float pk = 0.f, pki = 0.f;
        for (int k = lane; k < ne; k += 32) { float4 u = m.eu[m.eperm[k]]; pk += u.w * MC2 * gm1(u.x, u.y, u.z); }
        for (int k = lane; k < ni; k += 32) { float4 u = m.iu[m.iperm[k]]; pki += MC2 * mi * gm1(u.x, u.y, u.z); }
        double Ke = wsum(pk), Ki = (double)wi * wsum(pki);
        if (Ke > 0.0) {
            double f = 1.0 + (Kpre - Ke - Ki) / Ke;
            if (f > 0.0) {
                float ff = (float)f;
                for (int k = lane; k < ne; k += 32) {
                    float4 u = m.eu[k];
                    scale_kinetic(u.x, u.y, u.z, ff);
                    m.eu[k] = u;
                }
            }
        }
        __syncwarp();
    }

    // ---- Lotz impact ionization, cell-average probability (Eq. 3) ----
    int nnew = 0, nnew_imp = 0;
    double Wnew_imp = 0.0;
    if ((flags & 4u) && ne >= 1 && ni >= 1) {
        unsigned pmask = 0;
        for (int k = lane; k < ni; k += 32) { int Z = m.ist[k] & 0xff; if (Z < ZNUC) pmask |= 1u << Z; }
        for (int o = 16; o > 0; o >>= 1) pmask |= __shfl_xor_sync(FULL, pmask, o);
        float pk = 0.f;
        for (int k = lane; k < ne; k += 32) { float4 u = m.eu[m.eperm[k]]; pk += u.w * MC2 * gm1(u.x, u.y, u.z); }
        const double Kt = wsum(pk);
        const double cfac = (double)S.dt * kCcmPerFs * S.n_ref;
        for (int z = 0; z < ZNUC; ++z) {
            if (!(pmask & (1u << z))) continue;
            float pr = 0.f;
            const float dEz = m.dE[z];
            for (int k = lane; k < ne; k += 32) {
                float4 u = m.eu[m.eperm[k]];
                float u2 = u.x * u.x + u.y * u.y + u.z * u.z;
                float g1 = u2 / (sqrtf(1.0f + u2) + 1.0f);
                float beta = sqrtf(u2) / (1.0f + g1);
                pr += u.w * beta * lotz_sigma(T, z, dEz, MC2 * g1);
            }
            double P = cfac * wsum(pr);
            if (lane == 0) m.Pz[z] = P;
            if (P > 1.0) lt.pgt1 += lane == 0;
        }
        __syncwarp();
        double carry = 0.0, paid = 0.0;
        for (int b0 = 0; b0 < ni; b0 += 32) {
            int t = b0 + lane;
            bool cand = false;
            double cost = 0.0;
            int sl = 0, Z = 0, nK = 0;
            if (t < ni) {
                sl = m.iperm[t];
                int st = m.ist[sl];
                Z = st & 0xff; nK = (st >> 8) & 0xff;
                if (Z < ZNUC) {
                    U4 r = draw(seed, (unsigned long long)m.iid[t], step, PU_ION);
                    if ((double)u01(r.x) < m.Pz[Z]) {
                        cand = true;
                        cost = (double)wi * (double)removal_energy(T, Z, nK, m.dE[Z]);
                    }
                }
            }
            double incl = carry + wscan_incl(cost, lane);
            bool acc = cand && incl <= Kt;
            if (cand && !acc) lt.ion_rej++;
            unsigned bal = __ballot_sync(FULL, acc);
            if (acc) {
                int so = outer_shell(ZNUC - Z, nK);
                lose_electron(Z, nK, so);
                m.ist[sl] = Z | (nK << 8);
                int pos = nnew + __popc(bal & ((1u << lane) - 1u));
                if (pos < a.cap_new) {
                    NewE q; q.ux = q.uy = q.uz = 0.0f; q.w = wi; q.meta = sl | (KIND_IMPACT << 16);
                    m.nw[pos] = q;
                } else {
                    atomicOr(a.err, ERR_NEW_OVERFLOW);
                }
                lt.ion++;
            }
            paid += wsum(acc ? cost : 0.0);
            nnew += __popc(bal);
            carry = __shfl_sync(FULL, incl, 31);
        }
        nnew = min(nnew, a.cap_new);
        nnew_imp = nnew;
        Wnew_imp = (double)nnew_imp * wi;
        if (paid > 0.0) {
            float f = (float)(1.0 - paid / Kt);
            for (int k = lane; k < ne; k += 32) {
                float4 u = m.eu[k];
                scale_kinetic(u.x, u.y, u.z, f);
                m.eu[k] = u;
            }
            tal_ion += paid;
        }
        __syncwarp();
    }

    // ---- EOS-clamped three-body recombination (Sec. IV) ----
    if ((flags & 8u) && ni >= 1) {
        float pq = 0.f;
        for (int k = lane; k < ni; k += 32) { int sl = m.iperm[k]; pq += (float)(m.ist[sl] & 0xff) + m.iu[sl].w; }
        const double zb = wsum(pq) / ni;
        float pwb = 0.f, pkb = 0.f, pwx = 0.f;
        for (int k = lane; k < ne; k += 32) {
            float4 u = m.eu[m.eperm[k]];
            float ke = MC2 * gm1(u.x, u.y, u.z);
            pwx += u.w;
            if (S.E_bulk <= 0.0f || ke < S.E_bulk) { pwb += u.w; pkb += u.w * ke; }
        }
        double Wb2 = wsum(pwb) + Wnew_imp, Kb2 = wsum(pkb), Wex = wsum(pwx);
        double Te2 = Wb2 > 0.0 ? (2.0 / 3.0) * Kb2 / Wb2 : 0.0;
        float zeos = eos_lookup(*a.eos, (float)n_i, (float)Te2);
        int Kev = zb > zeos ? (int)floor((zb - zeos) * ni + 0.5) : 0;
        int pel = 0;
        for (int k = lane; k < ni; k += 32) pel += m.ist[k] & 0xff;
        int elig = wsum_i(pel);
        Kev = min(Kev, elig);
        Kev = min(Kev, (int)floor(Wex / wi + 1e-9));
        if (Kev > 0) {
            int *nrec = (int *)m.ikey;            // sort keys are no longer needed
            double *take = (double *)m.ekey;
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
            const double Wrem = (double)Kev * wi;
            double carry = 0.0;
            float premKE = 0.f;
            for (int b0 = 0; b0 < ne; b0 += 32) {
                int t = b0 + lane;
                double w = 0.0;
                float ke = 0.f;
                if (t < ne) { float4 u = m.eu[m.eperm[t]]; w = u.w; ke = MC2 * gm1(u.x, u.y, u.z); }
                double incl = carry + wscan_incl(w, lane);
                double before = incl - w;
                double tk = fmin(fmax(Wrem - before, 0.0), w);
                if (t < ne) take[t] = tk;
                premKE += (float)tk * ke;
                carry = __shfl_sync(FULL, incl, 31);
            }
            __syncwarp();
            double remKE = wsum(premKE);
            float pb = 0.f;
            for (int k = lane; k < ni; k += 32) {
                int st = m.ist[m.iperm[k]];
                int Z = st & 0xff, nK = (st >> 8) & 0xff;
                for (int r = 1; r <= nrec[k]; ++r) pb += wi * removal_energy(T, Z - r, nK, m.dE[Z - r]);
            }
            double bind = wsum(pb);
            float pkr = 0.f;
            for (int k = lane; k < ne; k += 32) {
                float4 u = m.eu[m.eperm[k]];
                float ke = MC2 * gm1(u.x, u.y, u.z);
                if (S.E_bulk <= 0.0f || ke < S.E_bulk) pkr += (float)((double)u.w - take[k]) * ke;
            }
            double Krem = wsum(pkr);
            if (Krem > 0.0) {
                float f = (float)(1.0 + (remKE + bind) / Krem);
                for (int k = lane; k < ne; k += 32) {
                    int sl = m.eperm[k];
                    float4 u = m.eu[sl];
                    float ke = MC2 * gm1(u.x, u.y, u.z);
                    bool bulk = S.E_bulk <= 0.0f || ke < S.E_bulk;
                    double tk = take[k];
                    double wn = (double)u.w - tk;
                    bool dead = tk > 0.0 && wn <= 0.0;
                    u.w = dead ? 0.0f : (float)wn;
                    if (bulk && !dead) scale_kinetic(u.x, u.y, u.z, f);
                    m.eu[sl] = u;
                }
                for (int k = lane; k < ni; k += 32) {
                    int sl = m.iperm[k];
                    int st = m.ist[sl];
                    m.ist[sl] = st - nrec[k];
                }
                tal_ion -= bind;
                lt.rec += lane == 0 ? Kev : 0;
            }
            __syncwarp();
        }
    }

    // ---- rad step: subshell photoionization (Eq. 2), then K-vacancy decay ----
    if (rad && (flags & (16u | 32u)) && ni >= 1) {
        const int nb = S.nb;
        const float dtr = S.rad_every * S.dt;
        double *ph = nb ? a.photons + S.ph_off + (size_t)lc * nb : nullptr;
        if ((flags & 16u) && nb) {
            double n0[MAXB], used[MAXB];
            int carry[MAXB];
            for (int b = 0; b < nb; ++b) { n0[b] = ph[b]; used[b] = 0.0; carry[b] = 0; }
            const float cph = (float)(kCcmPerFs * dtr * S.n_ref);
            for (int b0 = 0; b0 < ni; b0 += 32) {
                int t = b0 + lane;
                int sub = -1, bin = -1, sl = 0, Z = 0, nK = 0;
                float edge = 0.f, rc = 0.f, rp = 0.f;
                if (t < ni) {
                    sl = m.iperm[t];
                    int st = m.ist[sl];
                    Z = st & 0xff; nK = (st >> 8) & 0xff;
                    int occ[NS];
                    if (Z < ZNUC && occupancy(ZNUC - Z, nK, occ)) {
                        U4 ra = draw(seed, (unsigned long long)m.iid[t], step, PU_PHOTO_A);
                        U4 rb = draw(seed, (unsigned long long)m.iid[t], step, PU_PHOTO_B);
                        float rs[NS] = {u01(ra.x), u01(ra.y), u01(ra.z), u01(ra.w), u01(rb.x)};
                        float Ps = 0.f;
                        for (int q = 0; q < NS; ++q) {
                            if (!occ[q]) continue;
                            float ed = lowered_binding(T, Z, q, m.dE[Z]);
                            float acc = 0.f;
                            for (int b = 0; b < nb; ++b)
                                if (S.hv_b[b] > ed) acc += (float)n0[b] * S.sig_b[q][b];
                            float P = cph * occ[q] * acc;
                            if (rs[q] < P) { sub = q; Ps = P; edge = ed; break; }
                        }
                        if (sub >= 0) {
                            float target = u01(rb.y) * Ps, cum = 0.f;
                            int lastpos = -1;
                            for (int b = 0; b < nb; ++b) {
                                float c = S.hv_b[b] > edge ? cph * occ[sub] * (float)n0[b] * S.sig_b[sub][b] : 0.f;
                                if (c > 0.f) lastpos = b;
                                cum += c;
                                if (cum > target) { bin = b; break; }
                            }
                            if (bin < 0) bin = lastpos;
                            rc = u01(rb.z); rp = u01(rb.w);
                        }
                    }
                }
                double g = 0.0;
                for (int b = 0; b < nb; ++b) {
                    bool eb = bin == b && sub >= 0;
                    unsigned bal = __ballot_sync(FULL, eb);
                    if (eb) {
                        int rank = carry[b] + __popc(bal & ((1u << lane) - 1u));
                        g = fmin((double)wi, fmax(0.0, n0[b] - (double)rank * wi));
                    }
                    carry[b] += __popc(bal);
                }
                bool ev = sub >= 0 && bin >= 0 && g > 0.0;
                if (ev) {
                    if (g == (double)wi) {
                        lose_electron(Z, nK, sub);
                    } else {
                        float zf = m.iu[sl].w + (float)(g / wi);
                        if (zf >= 1.0f) {
                            zf -= 1.0f;
                            int so = outer_shell(ZNUC - Z, nK);
                            if (so >= 0) lose_electron(Z, nK, so);
                        }
                        m.iu[sl].w = zf;
                        lt.part++;
                    }
                    m.ist[sl] = Z | (nK << 8);
                    lt.ph[sub]++;
                }
                for (int b = 0; b < nb; ++b) used[b] += wsum(ev && bin == b ? g : 0.0);
                tal_ion += wsum(ev ? g * edge : 0.0);
                unsigned bal = __ballot_sync(FULL, ev);
                if (ev) {
                    int pos = nnew + __popc(bal & ((1u << lane) - 1u));
                    if (pos < a.cap_new) {
                        float3 u = iso_momentum(S.hv_b[bin] - edge, rc, rp);
                        NewE q; q.ux = u.x; q.uy = u.y; q.uz = u.z; q.w = (float)g;
                        q.meta = sl | (KIND_PHOTO << 16);
                        m.nw[pos] = q;
                    } else {
                        atomicOr(a.err, ERR_NEW_OVERFLOW);
                    }
                }
                nnew = min(nnew + __popc(bal), a.cap_new);
            }
            __syncwarp();
            if (lane == 0)
                for (int b = 0; b < nb; ++b) ph[b] = n0[b] - used[b];
            __syncwarp();
        }
        if (flags & 32u) {
            double addph[MAXB];
            for (int b = 0; b < MAXB; ++b) addph[b] = 0.0;
            for (int b0 = 0; b0 < ni; b0 += 32) {
                int t = b0 + lane;
                int kind = 0, sl = 0, Z = 0;
                float EA = 0.f, rc = 0.f, rp = 0.f, Eka = 0.f;
                if (t < ni) {
                    sl = m.iperm[t];
                    int st = m.ist[sl];
                    Z = st & 0xff;
                    int nK = (st >> 8) & 0xff;
                    int nbd = ZNUC - Z, occ[NS];
                    if (nK > 0 && occupancy(nbd, nK, occ)) {
                        float tau = T.tauK[nbd][nK - 1];
                        if (tau > 0.f) {
                            U4 r = draw(seed, (unsigned long long)m.iid[t], step, PU_DECAY);
                            if (u01(r.x) < dtr / tau) {
                                float om = T.omegaK[nbd][nK - 1];
                                int nl = occ[1] + occ[2];
                                if (u01(r.y) < 1.0f - om) {
                                    if (nl >= 2) {
                                        float e2s = lowered_binding(T, Z, 1, m.dE[Z]);
                                        float e2p = lowered_binding(T, Z, 2, m.dE[Z]);
                                        EA = fmaxf(T.E_Ka[Z] - (occ[1] * e2s + occ[2] * e2p) / nl, 0.0f);
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
                        float3 u = iso_momentum(EA, rc, rp);
                        NewE q; q.ux = u.x; q.uy = u.y; q.uz = u.z; q.w = wi; q.meta = sl | (KIND_AUGER << 16);
                        m.nw[pos] = q;
                    } else {
                        atomicOr(a.err, ERR_NEW_OVERFLOW);
                    }
                    lt.aug++;
                }
                nnew = min(nnew + __popc(bal), a.cap_new);
                int hit = -1;
                if (kind == 2) {
                    lt.ka++;
                    for (int b = 0; b < nb; ++b)
                        if (Eka >= S.hv_b[b] - S.bin_hw && Eka < S.hv_b[b] + S.bin_hw) { hit = b; break; }
                }
                for (int b = 0; b < nb; ++b)
                    addph[b] += wsum(hit == b ? (double)wi * Eka / S.hv_b[b] : 0.0);
                tal_ka += wsum(kind == 2 && hit < 0 ? (double)wi * Eka : 0.0);
                tal_ion -= wsum(kind == 1 ? (double)wi * EA : (kind == 2 ? (double)wi * Eka : 0.0));
            }
            if (lane == 0 && nb)
                for (int b = 0; b < nb; ++b) ph[b] += addph[b];
            __syncwarp();
        }
    }

    // ---- Boris push + charge-conserving deposit of every particle ----
    double esc = 0.0;
    if (S.ny > 1) cell_push_deposit<2>(a, S, m, g, cx, cy, e0, ne, i0, ni, nnew, lane, esc, lt);
    else cell_push_deposit<1>(a, S, m, g, cx, cy, e0, ne, i0, ni, nnew, lane, esc, lt);
    tal_esc = wsum(esc);

    // ---- tallies ----
    int c_ee = wsum_i(lt.coll_ee), c_ei = wsum_i(lt.coll_ei), c_ion = wsum_i(lt.ion), c_rej = wsum_i(lt.ion_rej);
    int c_rec = wsum_i(lt.rec), c_part = wsum_i(lt.part), c_aug = wsum_i(lt.aug), c_ka = wsum_i(lt.ka);
    int c_pg = wsum_i(lt.pgt1), c_ee_esc = wsum_i(lt.esc_e), c_ei_esc = wsum_i(lt.esc_i);
    int c_ph[NS];
    for (int q = 0; q < NS; ++q) c_ph[q] = wsum_i(lt.ph[q]);
    if (lane == 0) {
        SlabTally *tl = a.tally + s;
        if (tal_ion != 0.0) atomicAdd(&tl->ion, tal_ion);
        if (tal_ka != 0.0) atomicAdd(&tl->ka_esc, tal_ka);
        if (tal_esc != 0.0) atomicAdd(&tl->esc, tal_esc);
        unsigned long long *c = tl->cnt;
        if (c_ion) atomicAdd(c + C_ION, (unsigned long long)c_ion);
        if (c_rej) atomicAdd(c + C_ION_REJ, (unsigned long long)c_rej);
        if (c_rec) atomicAdd(c + C_REC, (unsigned long long)c_rec);
        for (int q = 0; q < NS; ++q) if (c_ph[q]) atomicAdd(c + C_PH0 + q, (unsigned long long)c_ph[q]);
        if (c_part) atomicAdd(c + C_PART, (unsigned long long)c_part);
        if (c_aug) atomicAdd(c + C_AUG, (unsigned long long)c_aug);
        if (c_ka) atomicAdd(c + C_KA, (unsigned long long)c_ka);
        if (c_pg) atomicAdd(c + C_PGT1, (unsigned long long)c_pg);
        if (c_ee_esc) atomicAdd(c + C_ESC_E, (unsigned long long)c_ee_esc);
        if (c_ei_esc) atomicAdd(c + C_ESC_I, (unsigned long long)c_ei_esc);
        if (c_ee) atomicAdd(c + C_EE, (unsigned long long)c_ee);
        if (c_ei) atomicAdd(c + C_EI, (unsigned long long)c_ei);
    }
    __syncwarp();
}

// One warp per cell, cells taken from a shared counter.  Cells whose
// population exceeds this launch's shared-memory capacity go to a list for
// the large-cell launch.
__global__ void __launch_bounds__(256) k_cell(CellArgs a)
{
    extern __shared__ __align__(16) char smem[];
    __shared__ Tables T;
    for (int k = threadIdx.x; k < (int)(sizeof(Tables) / 4); k += blockDim.x)
        ((float *)&T)[k] = ((const float *)a.tab)[k];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpMem m = carve(smem + (size_t)warp * warp_mem_bytes(a.cap_ce, a.cap_ci, a.cap_new),
                      a.cap_ce, a.cap_ci, a.cap_new);
    const int total = a.list ? *a.n_list : a.ncell;
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(a.work, 1);
        w = __shfl_sync(FULL, w, 0);
        if (w >= total) break;
        int g = a.list ? a.list[w] : w;
        int ne = a.cs_e[g + 1] - a.cs_e[g], ni = a.cs_i[g + 1] - a.cs_i[g];
        if (ne > a.cap_ce || ni > a.cap_ci || 3 * ni > a.cap_new) {
            if (a.ovf_list) {
                if (lane == 0) a.ovf_list[atomicAdd(a.ovf_count, 1)] = g;
            } else {
                // no larger pass left: report, and drop the cell's particles so
                // that the next sort stays consistent
                if (lane == 0) atomicOr(a.err, ERR_CELL_OVERFLOW);
                for (int k = a.cs_e[g] + lane; k < a.cs_e[g + 1]; k += 32) a.ekey[k] = -1;
                for (int k = a.cs_i[g] + lane; k < a.cs_i[g + 1]; k += 32) a.ikey[k] = -1;
            }
            continue;
        }
        process_cell(a, m, T, g, lane);
    }
}

}  // namespace pic
