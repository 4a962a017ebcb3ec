// Grid-level kernels: photon march, counting sort (scan + scatter), Yee
// field update, particle loading and diagnostic reductions.
#pragma once
#include "pic_dev.cuh"

namespace pic {

// ---------------------------------------------------------------------
// photon march (every rad step): the photon number of every cell and bin
// moves c dt_rad along +x, split linearly between the two destination
// cells; the region x < 0 carries the pulse at retarded time; what passes
// x = L is transmitted.  One block per (slab, row).
// ---------------------------------------------------------------------
struct MarchArgs {
    const SlabDev *slabs;
    const unsigned *steps;
    const int *row_slab, *row_idx;   // per block
    ph2 *photons;
    SlabTally *tally;
};

__device__ __forceinline__ double pulse_source(const SlabDev &S, int b, double tau, int row)
{
    double I;
    if (S.shape == 1) I = fabs(tau - S.t_peak) <= 0.5 * S.fwhm ? S.I_peak : 0.0;
    else { double d = (tau - S.t_peak) / S.fwhm; I = S.I_peak * exp(-4.0 * 0.6931471805599453 * d * d); }
    double n = I / (kCcmPerFs * 1e15 * (double)S.hv_b[b] * kQe) / S.nb;      // cm^-3
    if (S.spot_sigma > 0.0 && S.ny > 1) {
        double y = (row + 0.5) * (double)S.dy - 0.5 * S.ny * (double)S.dy;
        n *= exp(-0.5 * y * y / (S.spot_sigma * S.spot_sigma));
    }
    return n / S.n_ref;
}

__global__ void k_march(MarchArgs a)
{
    extern __shared__ double srow[];
    __shared__ double red[2][32];
    const int s = a.row_slab[blockIdx.x], row = a.row_idx[blockIdx.x];
    const SlabDev &S = a.slabs[s];
    const unsigned step = a.steps[s];
    if (!S.active || !(S.flags & 16u) || S.nb == 0 || S.rad_every <= 0 || (step % (unsigned)S.rad_every) != 0) return;
    const int nx = S.nx, nb = S.nb;
    const double dtr = (double)S.rad_every * S.dt;
    const double sh = kCnmPerFs * dtr / S.dx;
    const int m = (int)floor(sh);
    const double f = sh - m;
    const double tprev = (double)step * S.dt - dtr;
    ph2 *ph = a.photons + S.ph_off + (size_t)row * nx * nb;
    for (int b = 0; b < nb; ++b) {
        for (int k = threadIdx.x; k < nx; k += blockDim.x) {
            ph2 v = ph[(size_t)k * nb + b];
            srow[k] = (double)v.hi + (double)v.lo;
        }
        __syncthreads();
        double trans = 0.0, inc = 0.0;
        for (int k = threadIdx.x; k < nx; k += blockDim.x) {
            int j0 = k - m, j1 = k - m - 1;
            double v0 = j0 >= 0 ? srow[j0] : pulse_source(S, b, tprev - (j0 + 0.5) * S.dx / kCnmPerFs, row);
            double v1 = j1 >= 0 ? srow[j1] : pulse_source(S, b, tprev - (j1 + 0.5) * S.dx / kCnmPerFs, row);
            double nv = (1.0 - f) * v0 + f * v1;
            real hi = (real)nv;
            ph[(size_t)k * nb + b] = ph2{hi, (real)(nv - (double)hi)};
            if (j0 < 0) inc += (1.0 - f) * v0;
            if (j1 < 0) inc += f * v1;
        }
        // sources whose destinations lie beyond the last cell
        for (int j = -(m + 1) + (int)threadIdx.x; j < nx; j += blockDim.x) {
            int d0 = j + m, d1 = j + m + 1;
            if (d1 < nx) continue;
            double v = j >= 0 ? srow[j] : pulse_source(S, b, tprev - (j + 0.5) * S.dx / kCnmPerFs, row);
            if (d0 >= nx) { trans += (1.0 - f) * v; if (j < 0) inc += (1.0 - f) * v; }
            trans += f * v;
            if (j < 0) inc += f * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            trans += __shfl_down_sync(0xffffffffu, trans, o);
            inc += __shfl_down_sync(0xffffffffu, inc, o);
        }
        if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = trans; red[1][threadIdx.x >> 5] = inc; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0, in = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t += red[0][w]; in += red[1][w]; }
            if (t != 0.0) atomicAdd(&a.tally[s].trans, t * S.hv_b[b]);
            if (in != 0.0) atomicAdd(&a.tally[s].inc, in * S.hv_b[b]);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------
// exclusive scan of the per-cell counts of both species (3 phases)
// ---------------------------------------------------------------------
constexpr int SCAN_T = 1024, SCAN_ITEMS = 4, SCAN_TILE = SCAN_T * SCAN_ITEMS;

__device__ __forceinline__ int block_excl_scan(int v, int *sh, int &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) { int t = __shfl_up_sync(0xffffffffu, x, o); if (lane >= o) x += t; }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int y = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) { int t = __shfl_up_sync(0xffffffffu, y, o); if (lane >= o) y += t; }
        sh[lane] = y;
    }
    __syncthreads();
    int pre = warp ? sh[warp - 1] : 0;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return pre + x - v;
}

// hist[sp][b]: cells whose count n has b = bit length of n (0 for empty,
// b in 1..15 for n in [2^(b-1), 2^b), 15 also for anything larger)
constexpr int NHIST = 16;
struct ScanArgs { const int *cnt[2]; int *cs[2]; int *bsum[2]; int *maxc[2]; int *hist[2]; int n; int nblk; };

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(ScanArgs a)
{
    __shared__ int sh[32];
    const int sp = blockIdx.y;
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) if (base + k < a.n) v += a.cnt[sp][base + k];
    int tot;
    block_excl_scan(v, sh, tot);
    if (threadIdx.x == 0) a.bsum[sp][blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_blocks(ScanArgs a)
{
    __shared__ int sh[32];
    const int sp = blockIdx.y;
    int carry = 0;
    for (int b0 = 0; b0 < a.nblk; b0 += SCAN_T) {
        int i = b0 + threadIdx.x;
        int v = i < a.nblk ? a.bsum[sp][i] : 0;
        int tot;
        int ex = block_excl_scan(v, sh, tot);
        if (i < a.nblk) a.bsum[sp][i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) a.cs[sp][a.n] = carry;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_final(ScanArgs a)
{
    __shared__ int sh[32];
    __shared__ int hs[NHIST];
    const int sp = blockIdx.y;
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    if (threadIdx.x < NHIST) hs[threadIdx.x] = 0;
    __syncthreads();
    int v[SCAN_ITEMS], sum = 0, mx = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < a.n ? a.cnt[sp][base + k] : 0;
        sum += v[k];
        mx = max(mx, v[k]);
        if (v[k] > 0) atomicAdd(hs + min(32 - __clz(v[k]), NHIST - 1), 1);
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(a.maxc[sp], mx);
    __syncthreads();
    if (threadIdx.x < NHIST && hs[threadIdx.x]) atomicAdd(a.hist[sp] + threadIdx.x, hs[threadIdx.x]);
    int tot;
    int ex = block_excl_scan(sum, sh, tot) + a.bsum[sp][blockIdx.x];
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < a.n) a.cs[sp][base + k] = ex;
        ex += v[k];
    }
}

// ---------------------------------------------------------------------
// scatter into cell order (order inside a cell is irrelevant: every later
// decision is keyed by particle id)
// ---------------------------------------------------------------------
struct ScatterArgs {
    const real4 *s0, *s1;
    const int *key;
    const int *n_sorted;     // cs_old[ncell]
    const int *n_extra;      // appended this step (NULL: none)
    const int *cs_new;
    int *fill;
    real4 *d0, *d1;
    int cap;                 // slots beyond the capacity never hold particles
};

__global__ void k_scatter(ScatterArgs a)
{
    const int n = min(*a.n_sorted + (a.n_extra ? *a.n_extra : 0), a.cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int c = a.key[k];
        if (c < 0) continue;
        int d = a.cs_new[c] + atomicAdd(a.fill + c, 1);
        a.d0[d] = a.s0[k];
        a.d1[d] = a.s1[k];
    }
}

__global__ void k_count(const int *key, const int *n_ptr, int *cnt)
{
    const int n = *n_ptr;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int c = key[k];
        if (c >= 0) atomicAdd(cnt + c, 1);
    }
}

// ---------------------------------------------------------------------
// Yee field update, all slabs at once; y periodic, Mur in x.  One update per
// step (nsub = 1) at the slab's field speed cf, the largest the step resolves.
// E is double buffered so the Mur boundary can read old interior values.
// ---------------------------------------------------------------------
struct FieldArgs {
    const SlabDev *slabs;
    const int *pt_slab;      // slab of every grid point
    int npts;
    const real *Ein;        // [3][npts]
    real *Eout;             // [3][npts]
    real *B;                // [3][npts]
    const unsigned long long *J;   // [3][npts] fixed point
    int sub;                 // update index within the step (always 0: nsub = 1)
};

__global__ void k_b_half(FieldArgs a)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.npts; p += gridDim.x * blockDim.x) {
        const int s = a.pt_slab[p];
        const SlabDev &S = a.slabs[s];
        const int W = S.nx + 1, q = p - S.fld_off;
        // points past the slab's own (a batch slot wider than the slab) stay zero
        if (!S.active || !(S.flags & 128u) || a.sub >= S.nsub || q >= W * S.ny) continue;
        const int j = q / W, i = q - j * W;
        const int jp = (j + 1) % S.ny;
        const real h = RF(0.5) * S.dt / S.nsub * S.cf;
        const int n = a.npts;
        const real *ex = a.Ein, *ey = a.Ein + n, *ez = a.Ein + 2 * n;
        real *bx = a.B, *by = a.B + n, *bz = a.B + 2 * n;
        const int o = S.fld_off, r = o + j * W, rp = o + jp * W;
        bx[p] -= h * (ez[rp + i] - ez[r + i]) / S.dy;
        if (i < S.nx) {
            by[p] += h * (ez[r + i + 1] - ez[r + i]) / S.dx;
            bz[p] -= h * ((ey[r + i + 1] - ey[r + i]) / S.dx - (ex[rp + i] - ex[r + i]) / S.dy);
        }
    }
}

__global__ void k_e_full(FieldArgs a)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.npts; p += gridDim.x * blockDim.x) {
        const int s = a.pt_slab[p];
        const SlabDev &S = a.slabs[s];
        const int n = a.npts;
        const real *exi = a.Ein, *eyi = a.Ein + n, *ezi = a.Ein + 2 * n;
        real *exo = a.Eout, *eyo = a.Eout + n, *ezo = a.Eout + 2 * n;
        const int W = S.nx + 1, q = p - S.fld_off;
        if (!S.active || !(S.flags & 128u) || a.sub >= S.nsub || q >= W * S.ny) {
            exo[p] = exi[p]; eyo[p] = eyi[p]; ezo[p] = ezi[p];
            continue;
        }
        const int j = q / W, i = q - j * W;
        const int jm = (j - 1 + S.ny) % S.ny;
        const int o = S.fld_off, r = o + j * W, rm = o + jm * W;
        // Cf: speed of the curl terms; C: c, the velocity unit of J
        const real dtf = S.dt / S.nsub, C = (real)kCnmPerFs, Cf = S.cf, kap = S.kappa_f;
        const real *bx = a.B, *by = a.B + n, *bz = a.B + 2 * n;
        const unsigned long long *Jx = a.J, *Jy = a.J + n, *Jz = a.J + 2 * n;
        const real sx = S.dx / S.dt, sy = S.ny > 1 ? S.dy / S.dt : C;
        // fixed point (JFIX) back to real: high and low 32 bits separately
        auto jv = [&](const unsigned long long *Jc, int idx, real scale) {
            long long v = (long long)Jc[idx];
            real hi = (real)(int)(v >> 32) * RF(4294967296.0);
            real lo = (real)(unsigned)(v & 0xffffffffll);
            return (hi + lo) * (real)(1.0 / JFIX) * scale;
        };
        // the current the update sees: (1/4, 1/2, 1/4) along x over the
        // component's own points (nx faces for Jx, nx + 1 nodes for Jy, Jz;
        // nothing beyond the slab) and along y (periodic) in 2D
        const int rp1 = o + ((j + 1) % S.ny) * W;
        auto js = [&](const unsigned long long *Jc, int ii, int imax, real scale) {
            real acc = RF(0.0);
            for (int b = 0; b < 3; ++b) {
                if (S.ny == 1 && b != 1) continue;
                const int rr = b == 0 ? rm : (b == 1 ? r : rp1);
                const real wy = S.ny == 1 ? RF(1.0) : (b == 1 ? RF(0.5) : RF(0.25));
                for (int d = -1; d <= 1; ++d) {
                    const int ix = ii + d;
                    if (ix < 0 || ix > imax) continue;
                    acc += wy * (d == 0 ? RF(0.5) : RF(0.25)) * jv(Jc, rr + ix, scale);
                }
            }
            return acc;
        };
        auto ey_new = [&](int ii) {
            return eyi[r + ii] + dtf * (-Cf * (bz[r + ii] - bz[r + ii - 1]) / S.dx - kap * js(Jy, ii, S.nx, sy));
        };
        auto ez_new = [&](int ii) {
            return ezi[r + ii] + dtf * (Cf * ((by[r + ii] - by[r + ii - 1]) / S.dx - (bx[r + ii] - bx[rm + ii]) / S.dy)
                                        - kap * js(Jz, ii, S.nx, C));
        };
        if (i < S.nx)
            exo[p] = exi[p] + dtf * (Cf * (bz[r + i] - bz[rm + i]) / S.dy - kap * js(Jx, i, S.nx - 1, sx));
        else
            exo[p] = exi[p];
        if (i >= 1 && i < S.nx) {
            eyo[p] = ey_new(i);
            ezo[p] = ez_new(i);
        } else if (i == 0) {
            real y1 = S.nx > 1 ? ey_new(1) : eyi[r + 1], z1 = S.nx > 1 ? ez_new(1) : ezi[r + 1];
            eyo[p] = eyi[r + 1] + S.mur * (y1 - eyi[r]);
            ezo[p] = ezi[r + 1] + S.mur * (z1 - ezi[r]);
        } else {
            const int l = S.nx - 1;
            real yl = l >= 1 ? ey_new(l) : eyi[r + l], zl = l >= 1 ? ez_new(l) : ezi[r + l];
            eyo[p] = eyi[r + l] + S.mur * (yl - eyi[r + S.nx]);
            ezo[p] = ezi[r + l] + S.mur * (zl - ezi[r + S.nx]);
        }
    }
}

// end of a step: every running slab's step count advances; a slab that
// went beyond its electron budget this step stops (its particles are dropped
// by the next push); the per-slab append counts start again from zero
__global__ void k_advance(unsigned *steps, SlabDev *slabs, int nslab, int *slab_app, const int *slab_err)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslab) return;
    slab_app[s] = 0;
    if (!slabs[s].active) return;
    if (slab_err[s]) slabs[s].active = 0;
    else steps[s] += 1u;
}

// keys of the sorted particles for a re-sort: their own cell, or -1 when
// the cell's slab is retired
__global__ void k_cell_keys(const int *cs, int ncell, const int *cell_slab, const SlabDev *slabs, int *key)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ncell; g += gridDim.x * blockDim.x) {
        int k = slabs[cell_slab[g]].active ? g : -1;
        for (int i = cs[g]; i < cs[g + 1]; ++i) key[i] = k;
    }
}

// ---------------------------------------------------------------------
// diagnostics
// ---------------------------------------------------------------------
struct DiagArgs {
    const real4 *e0, *e1, *i0, *i1;
    const int *e_lo, *e_hi, *i_lo, *i_hi;   // particle range of the slab (device)
    double m_ion;
    double *out;                 // [0] W_e, [1] KE_e, [2] KE_i, [3] N_i, [4..4+NZ) csd, then eedf
    int n_E;
    double E_lo, E_max;
};

// per-thread sums in single / double-float precision, block-reduced; the
// histogram bins in shared memory
__global__ void k_diag(DiagArgs a)
{
    extern __shared__ real sdf[];          // [4 + NZ + n_E] block partials
    const int nv = 4 + NZ + a.n_E;
    real *sd = sdf;
    for (int k = threadIdx.x; k < nv; k += blockDim.x) sd[k] = RF(0.0);
    __syncthreads();
    const int eb = *a.e_lo, ne = *a.e_hi - eb, ib = *a.i_lo, ni = *a.i_hi - ib;
    const real lo_e = (real)a.E_lo, inv_lr = (real)(a.n_E / log(a.E_max / a.E_lo));
    dd w_s = dd_zero(), ke_s = dd_zero(), ki_s = dd_zero();
    int n_s = 0;
    const real MC2 = (real)kMeC2, mi = (real)a.m_ion;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += gridDim.x * blockDim.x) {
        real4 P0 = a.e0[eb + k], P1 = a.e1[eb + k];
        real ke = MC2 * gm1(P0.z, P0.w, P1.x);
        real w = P1.y;
        w_s = dd_addf(w_s, w);
        ke_s = dd_addf(ke_s, w * ke);
        int b = ke <= lo_e ? 0 : (int)r_floor(r_log(ke / lo_e) * inv_lr);
        b = b < 0 ? 0 : (b >= a.n_E ? a.n_E - 1 : b);
        atomicAdd(sd + 4 + NZ + b, w);
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ni; k += gridDim.x * blockDim.x) {
        real4 P0 = a.i0[ib + k], P1 = a.i1[ib + k];
        ki_s = dd_addf(ki_s, MC2 * mi * gm1(P0.z, P0.w, P1.x));
        n_s += 1;
        int Z = rec_ist(P1) & 0xff;
        real zf = P1.y;
        atomicAdd(sd + 4 + Z, RF(1.0) - zf);
        if (zf > RF(0.0) && Z < ZNUC) atomicAdd(sd + 4 + Z + 1, zf);
    }
    for (int o = 16; o > 0; o >>= 1) {
        w_s = dd_add(w_s, dd{__shfl_down_sync(0xffffffffu, w_s.hi, o), __shfl_down_sync(0xffffffffu, w_s.lo, o)});
        ke_s = dd_add(ke_s, dd{__shfl_down_sync(0xffffffffu, ke_s.hi, o), __shfl_down_sync(0xffffffffu, ke_s.lo, o)});
        ki_s = dd_add(ki_s, dd{__shfl_down_sync(0xffffffffu, ki_s.hi, o), __shfl_down_sync(0xffffffffu, ki_s.lo, o)});
        n_s += __shfl_down_sync(0xffffffffu, n_s, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(a.out + 0, (double)w_s.hi + (double)w_s.lo);
        atomicAdd(a.out + 1, (double)ke_s.hi + (double)ke_s.lo);
        atomicAdd(a.out + 2, (double)ki_s.hi + (double)ki_s.lo);
        atomicAdd(a.out + 3, (double)n_s);
    }
    __syncthreads();
    for (int k = 4 + threadIdx.x; k < nv; k += blockDim.x)
        if (sd[k] != RF(0.0)) atomicAdd(a.out + k, (double)sd[k]);
}

// sum of squares of three components of one slab's grid points
__global__ void k_sumsq(const real *x, int npts, int off, int n, double *out)
{
    double v = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 3 * n; k += gridDim.x * blockDim.x) {
        real f = x[(size_t)(k / n) * npts + off + k % n];
        v += (double)f * f;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out, v);
}

__global__ void k_photon_energy(const ph2 *ph, int ncell, int nb, const real *hv, double *out)
{
    double v = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncell * nb; k += gridDim.x * blockDim.x)
        v += ((double)ph[k].hi + (double)ph[k].lo) * hv[k % nb];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out, v);
}

// the in-cell ordering of one cell (the cell kernel's warp_sort of the
// kernel instance RMAX), run by one warp on given keys and ids:
// order[k] = slot at position k
template <int RMAX>
__global__ void k_order_check(const unsigned long long *key_in, const unsigned long long *id_in, int n,
                              unsigned short *order)
{
    extern __shared__ __align__(16) char sm[];
    unsigned long long *key = (unsigned long long *)sm;                  // [n]
    unsigned long long *id = key + n;                                     // [n]
    unsigned long long *buf = id + n;                                     // [2 n]
    int *hist = (int *)(buf + 2 * n);                                     // [256]
    unsigned short *slot = (unsigned short *)(hist + 256);               // [n]
    const int lane = threadIdx.x;
    for (int k = lane; k < n; k += 32) { key[k] = key_in[k]; id[k] = id_in[k]; slot[k] = (unsigned short)k; }
    __syncwarp();
    warp_sort<unsigned long long, RMAX>(key, id, slot, key, buf, hist, n, lane);
    for (int k = lane; k < n; k += 32) order[k] = slot[k];
}

// ---------------- initial plasma on the device ----------------
struct SeedArgs {
    real4 *p0, *p1;          // records (unsorted side)
    int *key;                // their cells
    long long n;             // particles of the species
    int nx, ny, ppc;
    int electrons;
    double sigma_u;          // sqrt(T / (m c^2)): spread of each momentum component
    double beam_frac, beam_u;
    float w;                 // electron weight
    int st;                  // ion state Z | nK << 8
    unsigned long long seed;
};

__device__ __forceinline__ double u01d(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

// particle i of the species: cell i / ppc (cell-major), id i; three draws of
// its own stream give the position, the beam choice and direction, and two
// Box-Muller pairs for the Maxwellian
__global__ void k_seed(SeedArgs a)
{
    const uint32_t pu = a.electrons ? PU_SEED_E : PU_SEED_I;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i / a.ppc);
        const U4 r0 = draw(a.seed, (unsigned long long)i, 0u, pu);
        const U4 r1 = draw(a.seed, (unsigned long long)i, 1u, pu);
        const real xi = u01(r0.x);
        const real eta = a.ny > 1 ? u01(r0.y) : RF(0.5);
        double ux, uy, uz;
        if (a.electrons && u01d(r0.z) < a.beam_frac) {
            const double c = 2.0 * u01d(r0.w) - 1.0, ph = 2.0 * kPi * u01d(r1.x);
            const double sn = sqrt(fmax(0.0, 1.0 - c * c));
            ux = a.beam_u * sn * cos(ph); uy = a.beam_u * sn * sin(ph); uz = a.beam_u * c;
        } else {
            const U4 r2 = draw(a.seed, (unsigned long long)i, 2u, pu);
            const double m1 = sqrt(-2.0 * log(u01d(r2.x))), t1 = 2.0 * kPi * u01d(r2.y);
            const double m2 = sqrt(-2.0 * log(u01d(r2.z))), t2 = 2.0 * kPi * u01d(r2.w);
            ux = a.sigma_u * m1 * cos(t1); uy = a.sigma_u * m1 * sin(t1); uz = a.sigma_u * m2 * cos(t2);
        }
        a.p0[i] = make_real4(xi, eta, (real)ux, (real)uy);
        a.p1[i] = a.electrons ? rec_e1((real)uz, (real)a.w, (uint64_t)i)
                              : rec_i1((real)uz, RF(0.0), (uint32_t)i, a.st);
        a.key[i] = g;
    }
}

// the cell kernel's double-float sum of n terms, run by one warp (lane-
// strided accumulation, then the fixed tree of wsum_dd): out = hi + lo
__global__ void k_dd_check(const float *x, int n, double *out)
{
    const int lane = threadIdx.x;
    dd acc = dd_zero();
    for (int k = lane; k < n; k += 32) acc = dd_addf(acc, (real)x[k]);
    acc = wsum_dd(acc);
    if (lane == 0) out[0] = (double)acc.hi + (double)acc.lo;
}

__global__ void k_philox_check(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    U4 r = philox(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
    out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
}

}  // namespace pic
