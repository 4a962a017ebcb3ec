// Boris push and charge-conserving deposit, one warp per cell.
//
// A cell's particles are visited in the canonical order the collision
// kernel recorded (the memory order inside a cell, left by the atomic
// scatter of the counting sort, is unspecified).  Lane L takes canonical
// positions L, L+32, ...; each lane stores its stencil contributions in a
// shared-memory column, lane k % 32 sums row k of each batch in a fixed
// order and keeps the running total of node k, and the cell's totals go to
// the global grid as 2^40 fixed point, whose addition is associative.  The
// current is therefore bit-reproducible.
#pragma once
#include "pic_cell.cuh"

namespace pic {

struct PushArgs {
    real4 *e0, *e1;
    int *ekey;
    const int *cs_e;
    real4 *i0, *i1;
    int *ikey;
    const int *cs_i;
    int *cnt_e, *cnt_i;
    const int *append;        // electrons appended this step (after the sorted range)
    int cap_e;
    int ncell;
    const int *cell_slab;
    const SlabDev *slabs;
    SlabTally *tally;
    const real *fldE, *fldB;
    int npts;
    unsigned long long *J;
    int *err;
    int *work;
};


// CIC weights and indices of one particle on the staggered grid
struct GatherPt {
    int xn0, xn1, xh0, xh1;       // node / half-node columns
    real wn0, wn1, wh0, wh1;
    int yn0, yn1, yh0, yh1;       // rows (already wrapped)
    real vn0, vn1, vh0, vh1;
};

template <int DIM>
__device__ __forceinline__ GatherPt gather_pt(int nx, int ny, int cx, int cy, real xi, real eta)
{
    GatherPt p;
    p.xn0 = cx; p.xn1 = cx + 1; p.wn0 = RF(1.0) - xi; p.wn1 = xi;
    if (xi >= RF(0.5)) { p.xh0 = cx; p.xh1 = cx + 1; p.wh1 = xi - RF(0.5); }
    else { p.xh0 = cx - 1; p.xh1 = cx; p.wh1 = xi + RF(0.5); }
    p.wh0 = RF(1.0) - p.wh1;
    // half nodes exist for 0 <= i <= nx - 1: weight 0 (and a safe index) outside
    if (p.xh0 < 0) { p.xh0 = 0; p.wh0 = RF(0.0); }
    if (p.xh1 > nx - 1) { p.xh1 = nx - 1; p.wh1 = RF(0.0); }
    if (DIM == 2) {
        p.yn0 = cy; p.yn1 = cy + 1 == ny ? 0 : cy + 1; p.vn0 = RF(1.0) - eta; p.vn1 = eta;
        if (eta >= RF(0.5)) { p.yh0 = cy; p.yh1 = cy + 1 == ny ? 0 : cy + 1; p.vh1 = eta - RF(0.5); }
        else { p.yh0 = cy == 0 ? ny - 1 : cy - 1; p.yh1 = cy; p.vh1 = eta + RF(0.5); }
        p.vh0 = RF(1.0) - p.vh1;
    } else {
        p.yn0 = p.yn1 = p.yh0 = p.yh1 = 0;
        p.vn0 = RF(1.0); p.vn1 = RF(0.0); p.vh0 = RF(1.0); p.vh1 = RF(0.0);
    }
    return p;
}

__device__ __forceinline__ real interp4(const real *F, int W, int x0, int x1, real w0, real w1, int y0, int y1,
                                         real v0, real v1)
{
    const real *r0 = F + (size_t)y0 * W, *r1 = F + (size_t)y1 * W;
    return w0 * (v0 * __ldg(r0 + x0) + v1 * __ldg(r1 + x0)) + w1 * (v0 * __ldg(r0 + x1) + v1 * __ldg(r1 + x1));
}

// Per-warp staging of the stencil contributions: row k (node), column
// lane; the row pitch of 33 words keeps both the column stores and the row
// sums free of bank conflicts.
// (the FP64 build halves the warps per CTA: its rows are twice as wide)
constexpr int JROWS = 40, JPITCH = 33, PUSH_WARPS = sizeof(real) == 8 ? 4 : 8;

__device__ __forceinline__ void jput(real *col, int k, real v) { col[k * JPITCH] = v; }

// Row sums of one batch (fixed order: four interleaved partial sums, then
// pairwise), added to the running totals of the rows this lane owns:
// acc[0] <- row lane, acc[1] <- row lane + 32.
__device__ __forceinline__ void jrows(const real *sj, int nrows, int lane, real acc[2])
{
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h;
        if (k < nrows) {
            const real *r = sj + k * JPITCH;
            real s0 = RF(0.0), s1 = RF(0.0), s2 = RF(0.0), s3 = RF(0.0);
#pragma unroll
            for (int j = 0; j < 32; j += 4) { s0 += r[j]; s1 += r[j + 1]; s2 += r[j + 2]; s3 += r[j + 3]; }
            acc[h] += (s0 + s1) + (s2 + s3);
        }
    }
    __syncwarp();
}

// 2D Esirkepov weights of one sub-cell move (offsets relative to the cell,
// stencil nodes -1..2); order of the sums: jx[a][b] (12), jy[a][b] (12),
// jz[a][b] (16)
__device__ __forceinline__ void esirkepov2_w(real x0, real y0, real x1, real y1, real qw, real qwbz,
                                             real *col)
{
    real S0x[4], S1x[4], S0y[4], S1y[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        S0x[a] = cic_w(x0, a - 1); S1x[a] = cic_w(x1, a - 1);
        S0y[a] = cic_w(y0, a - 1); S1y[a] = cic_w(y1, a - 1);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        real acc_x = RF(0.0);
        real sy = S0y[b] + RF(0.5) * (S1y[b] - S0y[b]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            acc_x += (S1x[a] - S0x[a]) * sy;
            jput(col, a * 4 + b, -qw * acc_x);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        real acc_y = RF(0.0);
        real dsx = S1x[a] - S0x[a];
        real sx = S0x[a] + RF(0.5) * dsx;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            acc_y += (S1y[b] - S0y[b]) * sx;
            jput(col, 12 + a * 3 + b, -qw * acc_y);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            real dsy = S1y[b] - S0y[b];
            real wz = S0x[a] * S0y[b] + RF(0.5) * dsx * S0y[b] + RF(0.5) * S0x[a] * dsy + dsx * dsy * (RF(1.0) / RF(3.0));
            jput(col, 24 + a * 4 + b, qwbz * wz);
        }
    }
}

// 1D: jx at 3 half nodes (0..2), jy (3..6), jz (7..10) at 4 nodes
__device__ __forceinline__ void esirkepov1_w(real x0, real x1, real qw, real qwby, real qwbz, real *col)
{
    real S0x[4], S1x[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) { S0x[a] = cic_w(x0, a - 1); S1x[a] = cic_w(x1, a - 1); }
    real acc_x = RF(0.0);
#pragma unroll
    for (int a = 0; a < 3; ++a) { acc_x += S1x[a] - S0x[a]; jput(col, a, -qw * acc_x); }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        real sv = RF(0.5) * (S0x[a] + S1x[a]);
        jput(col, 3 + a, qwby * sv);
        jput(col, 7 + a, qwbz * sv);
    }
}

__device__ __forceinline__ long long wsum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ void jglobal(unsigned long long *J, real v)
{
    if (v != RF(0.0)) atomicAdd(J, (unsigned long long)fix40(v));
}

// The 3 x 3 grid points around cell (cx, cy) (columns cx-1..cx+1, rows
// cy-1..cy+1 wrapped in y; one row repeated in 1D) of the six field
// components, [component][row][column]: every CIC gather of a particle in
// the cell reads inside it.  Columns outside [0, nx] hold 0 (their weight is
// 0).  One warp fills it, 54 loads per cell instead of 24 per particle.
constexpr int TILE = 54;

template <int DIM>
__device__ __forceinline__ void load_tile(real *tile, const SlabDev &S, const real *fe, const real *fb, int npts,
                                          int cx, int cy, int lane)
{
    const int W = S.nx + 1;
    for (int t = lane; t < TILE; t += 32) {
        const int comp = t / 9, r = (t % 9) / 3, l = t % 3;
        const int gx = cx - 1 + l;
        int gy = 0;
        if (DIM == 2) { gy = cy - 1 + r; gy = gy < 0 ? gy + S.ny : (gy >= S.ny ? gy - S.ny : gy); }
        const real *F = comp < 3 ? fe + (size_t)comp * npts : fb + (size_t)(comp - 3) * npts;
        tile[t] = (gx >= 0 && gx <= S.nx) ? __ldg(F + (size_t)gy * W + gx) : RF(0.0);
    }
}

// interp4 on a tile component: columns / rows are tile-local
__device__ __forceinline__ real tinterp(const real *T, int x0, int x1, real w0, real w1, int y0, int y1,
                                         real v0, real v1)
{
    return w0 * (v0 * T[y0 * 3 + x0] + v1 * T[y1 * 3 + x0]) + w1 * (v0 * T[y0 * 3 + x1] + v1 * T[y1 * 3 + x1]);
}

// One particle: gather, Boris, move; returns the next local cell, -1 when
// it left through an x boundary, -2 when its move is not finite.  The
// fields come from global memory, or from the cell's tile when tile != NULL
// (the same values and the same arithmetic).
template <int DIM>
__device__ __forceinline__ int move_particle(const SlabDev &S, const real *fe, const real *fb, int npts,
                                             const real *tile, int cx, int cy, real &xi, real &eta, real &ux,
                                             real &uy, real &uz, real qm, real &xn, real &yn)
{
    const int W = S.nx + 1;
    GatherPt p = gather_pt<DIM>(S.nx, S.ny, cx, cy, xi, eta);
    real ex, ey, ez, bx, by, bz;
    if (tile) {
        // tile columns: nodes cx, cx+1 -> 1, 2; half nodes (cx-1, cx) or (cx, cx+1)
        const int hx0 = xi >= RF(0.5) ? 1 : 0, hy0 = DIM == 2 ? (eta >= RF(0.5) ? 1 : 0) : 1;
        const int ny0 = DIM == 2 ? 1 : 1, ny1 = DIM == 2 ? 2 : 1, hy1 = DIM == 2 ? hy0 + 1 : 1;
        ex = tinterp(tile + 0, hx0, hx0 + 1, p.wh0, p.wh1, ny0, ny1, p.vn0, p.vn1);
        ey = tinterp(tile + 9, 1, 2, p.wn0, p.wn1, hy0, hy1, p.vh0, p.vh1);
        ez = tinterp(tile + 18, 1, 2, p.wn0, p.wn1, ny0, ny1, p.vn0, p.vn1);
        bx = tinterp(tile + 27, 1, 2, p.wn0, p.wn1, hy0, hy1, p.vh0, p.vh1);
        by = tinterp(tile + 36, hx0, hx0 + 1, p.wh0, p.wh1, ny0, ny1, p.vn0, p.vn1);
        bz = tinterp(tile + 45, hx0, hx0 + 1, p.wh0, p.wh1, hy0, hy1, p.vh0, p.vh1);
    } else {
        ex = interp4(fe, W, p.xh0, p.xh1, p.wh0, p.wh1, p.yn0, p.yn1, p.vn0, p.vn1);
        ey = interp4(fe + npts, W, p.xn0, p.xn1, p.wn0, p.wn1, p.yh0, p.yh1, p.vh0, p.vh1);
        ez = interp4(fe + 2 * npts, W, p.xn0, p.xn1, p.wn0, p.wn1, p.yn0, p.yn1, p.vn0, p.vn1);
        bx = interp4(fb, W, p.xn0, p.xn1, p.wn0, p.wn1, p.yh0, p.yh1, p.vh0, p.vh1);
        by = interp4(fb + npts, W, p.xh0, p.xh1, p.wh0, p.wh1, p.yn0, p.yn1, p.vn0, p.vn1);
        bz = interp4(fb + 2 * npts, W, p.xh0, p.xh1, p.wh0, p.wh1, p.yh0, p.yh1, p.vh0, p.vh1);
    }
    boris(ux, uy, uz, ex, ey, ez, bx, by, bz, qm, S.dt);
    real ig = r_rsqrt(RF(1.0) + ux * ux + uy * uy + uz * uz);
    const real c = (real)kCnmPerFs;
    xn = xi + ux * ig * c * S.dt / S.dx;
    yn = DIM == 2 ? eta + uy * ig * c * S.dt / S.dy : eta;
    if (!(r_fabs(xn - xi) < RF(64.0) && r_fabs(yn - eta) < RF(64.0))) return -2;
    real fx = r_floor(xn), fy = r_floor(yn);
    int ncx = cx + (int)fx;
    int ncy = DIM == 2 ? cy + (int)fy : 0;
    if (DIM == 2) { if (ncy < 0) ncy += S.ny; else if (ncy >= S.ny) ncy -= S.ny; }
    return (ncx < 0 || ncx >= S.nx) ? -1 : ncy * S.nx + ncx;
}

__device__ __forceinline__ void wrap_offsets(real xn, real yn, real &xi, real &eta)
{
    const real below1 = kBelow1;
    xi = xn - r_floor(xn);
    eta = yn - r_floor(yn);
    if (xi >= RF(1.0)) xi = below1;
    if (eta >= RF(1.0)) eta = below1;
}

template <int DIM>
__device__ void push_cell(const PushArgs &a, const SlabDev &S, int s, int g, int lane, real *sj, real *tile,
                          dd &esc, int &esc_e, int &esc_i)
{
    constexpr int NJ = DIM == 2 ? 40 : 11;
    const int lc = g - S.cell0;
    const int cx = lc % S.nx, cy = lc / S.nx;
    const bool do_push = S.flags & 64u, do_dep = (S.flags & 128u) != 0;
    const real *fe = a.fldE + S.fld_off, *fb = a.fldB + S.fld_off;
    const real MC2 = (real)kMeC2;
    real acc[2] = {RF(0.0), RF(0.0)};
    if (do_push) {
        __syncwarp();
        load_tile<DIM>(tile, S, fe, fb, a.npts, cx, cy, lane);
        __syncwarp();
    }

    for (int pass = 0; pass < 2; ++pass) {
        const bool elec = pass == 0;
        const int k0 = elec ? a.cs_e[g] : a.cs_i[g], k1 = elec ? a.cs_e[g + 1] : a.cs_i[g + 1];
        real4 *R0 = elec ? a.e0 : a.i0, *R1 = elec ? a.e1 : a.i1;
        int *key = elec ? a.ekey : a.ikey;
        int *cnt = elec ? a.cnt_e : a.cnt_i;
        const int n = k1 - k0;
        // every lane runs the same number of iterations (the warp reductions
        // of the deposit need all 32 lanes)
        for (int base = 0; base < n; base += 32) {
            const bool have = base + lane < n;
            // the collision kernel left each cell's records in canonical order
            const int k = have ? k0 + base + lane : k0;
            int nk = -1;
            real x0 = RF(0.), y0 = RF(0.), x1 = RF(0.), y1 = RF(0.), qw = RF(0.), qwby = RF(0.), qwbz = RF(0.);
            bool dep_short = false;
            if (have) {
                real4 P0 = R0[k], P1 = R1[k];
                if (elec ? P1.y <= RF(0.0) : (rec_ist(P1) & 0xff) == 0xff) {
                    nk = -1;                                   // recombined away, or dropped
                } else if (!do_push) {
                    nk = g;
                } else {
                    real q, m, w;
                    if (elec) { q = -RF(1.0); m = RF(1.0); w = P1.y; }
                    else { q = (real)(rec_ist(P1) & 0xff) + P1.y; m = S.m_ion; w = S.w_ion; }
                    real xi = P0.x, eta = P0.y, ux = P0.z, uy = P0.w, uz = P1.x, xn, yn;
                    real ke = MC2 * m * gm1(ux, uy, uz);
                    int nc = move_particle<DIM>(S, fe, fb, a.npts, tile, cx, cy, xi, eta, ux, uy, uz, q / m, xn, yn);
                    if (nc == -2) {
                        nk = -1;
                        atomicOr(a.err, ERR_NUMERIC);
                    } else {
                        if (do_dep) {
                            real ig = r_rsqrt(RF(1.0) + ux * ux + uy * uy + uz * uz);
                            qw = q * w; qwby = qw * uy * ig; qwbz = qw * uz * ig;
                            if (r_fabs(xn - xi) < RF(1.0) && r_fabs(yn - eta) < RF(1.0)) {
                                dep_short = true;
                                x0 = xi; y0 = eta; x1 = xn; y1 = yn;
                            } else {
                                SlabGrid gr;
                                gr.nx = S.nx; gr.ny = S.ny; gr.W = S.nx + 1; gr.fe = fe; gr.fb = fb;
                                gr.npts = a.npts; gr.fo = S.fld_off;
                                deposit_long(gr, a.J, a.npts, S.fld_off, cx, cy, xi, eta, xn, yn, qw, qwby, qwbz);
                            }
                        }
                        if (nc == -1) {
                            esc = dd_addf(esc, w * ke);
                            if (elec) esc_e++; else esc_i++;
                        } else {
                            nk = S.cell0 + nc;
                        }
                        wrap_offsets(xn, yn, xi, eta);
                        R0[k] = make_real4(xi, eta, ux, uy);
                        reinterpret_cast<real *>(R1 + k)[0] = uz;
                    }
                }
                key[k] = nk;
            }
            if (do_dep) {
                if (!dep_short) { qw = qwby = qwbz = RF(0.0); x0 = x1 = RF(0.5); y0 = y1 = RF(0.5); }
                if constexpr (DIM == 2) esirkepov2_w(x0, y0, x1, y1, qw, qwbz, sj + lane);
                else esirkepov1_w(x0, x1, qw, qwby, qwbz, sj + lane);
                jrows(sj, NJ, lane, acc);
            }
            // aggregated count of the next cell
            unsigned peers = __match_any_sync(FULL, have ? nk : -2);
            if (have && nk >= 0 && lane == __ffs(peers) - 1) atomicAdd(cnt + nk, __popc(peers));
        }
    }

    if (do_dep) {
        const int fo = S.fld_off, W = S.nx + 1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = lane + 32 * h;
            if (k >= NJ || acc[h] == RF(0.0)) continue;
            if (DIM == 2) {
                int p, q, comp;
                if (k < 12) { comp = 0; p = k / 4; q = k % 4; }
                else if (k < 24) { comp = 1; p = (k - 12) / 3; q = (k - 12) % 3; }
                else { comp = 2; p = (k - 24) / 4; q = (k - 24) % 4; }
                const int i = cx - 1 + p;
                int j = cy - 1 + q;
                j = j < 0 ? j + S.ny : (j >= S.ny ? j - S.ny : j);
                const bool ok = comp == 0 ? (i >= 0 && i < S.nx) : (i >= 0 && i <= S.nx);
                if (ok) jglobal(a.J + (size_t)comp * a.npts + fo + (size_t)j * W + i, acc[h]);
            } else {
                int comp, p;
                if (k < 3) { comp = 0; p = k; } else if (k < 7) { comp = 1; p = k - 3; } else { comp = 2; p = k - 7; }
                const int i = cx - 1 + p;
                const bool ok = comp == 0 ? (i >= 0 && i < S.nx) : (i >= 0 && i <= S.nx);
                if (ok) jglobal(a.J + (size_t)comp * a.npts + fo + i, acc[h]);
            }
        }
    }
}

__device__ void push_flush(const PushArgs &a, int slab, dd &esc, int &esc_e, int &esc_i, int lane)
{
    dd e = wsum_dd(esc);
    int ce = wsum_i(esc_e), ci = wsum_i(esc_i);
    if (slab >= 0 && lane == 0) {
        SlabTally *tl = a.tally + slab;
        if (dd_f(e) != RF(0.0)) atomicAdd(&tl->esc, (double)e.hi + (double)e.lo);
        if (ce) atomicAdd(tl->cnt + C_ESC_E, (unsigned long long)ce);
        if (ci) atomicAdd(tl->cnt + C_ESC_I, (unsigned long long)ci);
    }
    esc = dd_zero();
    esc_e = esc_i = 0;
}

__global__ void __launch_bounds__(32 * PUSH_WARPS, 2) k_push(PushArgs a)
{
    __shared__ real s_j[PUSH_WARPS][JROWS * JPITCH];
    __shared__ real s_t[PUSH_WARPS][TILE];
    const int lane = threadIdx.x & 31;
    real *sj = s_j[threadIdx.x >> 5];
    real *tile = s_t[threadIdx.x >> 5];
    int cur = -1;
    dd esc = dd_zero();
    int esc_e = 0, esc_i = 0;
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(a.work, 1);
        w = __shfl_sync(FULL, w, 0);
        if (w >= a.ncell) break;
        const int g = w;
        if (a.cs_e[g + 1] == a.cs_e[g] && a.cs_i[g + 1] == a.cs_i[g]) continue;
        const int s = __ldg(a.cell_slab + g);
        if (s != cur) { push_flush(a, cur, esc, esc_e, esc_i, lane); cur = s; }
        const SlabDev &S = a.slabs[s];
        if (!S.active) {              // retired slab: its particles leave
            for (int k = a.cs_e[g] + lane; k < a.cs_e[g + 1]; k += 32) a.ekey[k] = -1;
            for (int k = a.cs_i[g] + lane; k < a.cs_i[g + 1]; k += 32) a.ikey[k] = -1;
            continue;
        }
        if (S.ny > 1) push_cell<2>(a, S, s, g, lane, sj, tile, esc, esc_e, esc_i);
        else push_cell<1>(a, S, s, g, lane, sj, tile, esc, esc_e, esc_i);
    }
    push_flush(a, cur, esc, esc_e, esc_i, lane);
}

// Electrons created this step sit after the sorted range with their cell in
// the key; they are pushed one per thread and deposit straight to global
// memory (integer atomics, so the order does not matter).
__global__ void k_push_new(PushArgs a)
{
    const int sorted = a.cs_e[a.ncell];
    const int n = min(*a.append, a.cap_e - sorted);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int k = sorted + t;
        const int g = a.ekey[k];
        if (g < 0) continue;
        const int s = __ldg(a.cell_slab + g);
        const SlabDev &S = a.slabs[s];
        const int lc = g - S.cell0, cx = lc % S.nx, cy = lc / S.nx;
        real4 P0 = a.e0[k], P1 = a.e1[k];
        int nk = g;
        if (S.flags & 64u) {
            const real *fe = a.fldE + S.fld_off, *fb = a.fldB + S.fld_off;
            real xi = P0.x, eta = P0.y, ux = P0.z, uy = P0.w, uz = P1.x, xn, yn;
            real ke = (real)kMeC2 * gm1(ux, uy, uz);
            int nc = S.ny > 1 ? move_particle<2>(S, fe, fb, a.npts, nullptr, cx, cy, xi, eta, ux, uy, uz, -RF(1.0), xn, yn)
                              : move_particle<1>(S, fe, fb, a.npts, nullptr, cx, cy, xi, eta, ux, uy, uz, -RF(1.0), xn, yn);
            if (nc == -2) {
                nk = -1;
                atomicOr(a.err, ERR_NUMERIC);
            } else {
                if (S.flags & 128u) {
                    real qw = -P1.y;
                    real ig = r_rsqrt(RF(1.0) + ux * ux + uy * uy + uz * uz);
                    SlabGrid gr;
                    gr.nx = S.nx; gr.ny = S.ny; gr.W = S.nx + 1; gr.fe = fe; gr.fb = fb;
                    gr.npts = a.npts; gr.fo = S.fld_off;
                    deposit_long(gr, a.J, a.npts, S.fld_off, cx, cy, xi, eta, xn, yn, qw, qw * uy * ig, qw * uz * ig);
                }
                if (nc == -1) {
                    nk = -1;
                    atomicAdd(&a.tally[s].esc, (double)(P1.y * ke));
                    atomicAdd(a.tally[s].cnt + C_ESC_E, 1ull);
                } else {
                    nk = S.cell0 + nc;
                }
                wrap_offsets(xn, yn, xi, eta);
                a.e0[k] = make_real4(xi, eta, ux, uy);
                reinterpret_cast<real *>(a.e1 + k)[0] = uz;
            }
        }
        a.ekey[k] = nk;
        if (nk >= 0) atomicAdd(a.cnt_e + nk, 1);
    }
}

}  // namespace pic
