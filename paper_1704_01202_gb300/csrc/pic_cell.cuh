// Building blocks of the per-cell hot path: one warp owns one cell and runs,
// in order, the canonical random ordering of its particles, the cell
// moments (double-float sums), binary e-e and e-i collisions, Lotz impact
// ionization, EOS-clamped recombination and, on rad steps, subshell
// photoionization and K-vacancy decay (k_cell); the Boris push and the
// charge-conserving deposit of the cell's particles follow in a second
// kernel in the same canonical order (k_push).  Particles are staged in
// shared memory; their positions stay in global memory until the push.
//
// Determinism: every random number is keyed by (slab seed, particle id,
// step, purpose) and every ordering comes from a sort on Philox keys, so
// the result of a cell does not depend on where its particles sit in memory
// or on which warp handles it.  Sums run lane-strided over the canonical
// order with a fixed reduction tree; the current goes to global memory as
// 64-bit fixed point, whose addition is associative.
#pragma once
#include "pic_dev.cuh"

namespace pic {

constexpr unsigned FULL = 0xffffffffu;
// fixed-point scale of J: 2^40 (|J| < 2^22 per node); the FP64 build keeps
// 2^48 (|J| < 2^14), eight more bits for its 1e-12 comparison
constexpr double JFIX = sizeof(real) == 8 ? 281474976710656.0 : 1099511627776.0;

struct NewE {            // an electron created in this cell this step
    real ux, uy, uz, w;
    int meta;            // ion slot | kind << 16
};

struct CellArgs {
    real4 *e0, *e1;     // electrons (xi, eta, ux, uy), (uz, w, id_lo, id_hi)
    int *ekey;           // next cell of each electron slot (-1: gone)
    const int *cs_e;     // cell start of electrons [ncell + 1]
    real4 *i0, *i1;     // ions (xi, eta, ux, uy), (uz, zfrac, id, Z | nK << 8)
    int *ikey;
    const int *cs_i;
    int *cnt_e, *cnt_i;  // per-cell counts of the next sort
    int *append;         // electrons appended this step
    int cap_e;           // electron capacity
    int *slab_app;       // [slab] electrons appended this step (budgeted slabs)
    int *slab_err;       // [slab] ERR_CAPACITY once a slab went beyond its budget
    int ncell;           // total cells (all slabs)
    const int *cell_slab;
    const SlabDev *slabs;
    const unsigned *steps;
    SlabTally *tally;
    ph2 *photons;
    const real *fldE;   // [3][npts] ex ey ez
    const real *fldB;   // [3][npts] bx by bz
    int npts;
    unsigned long long *J;   // [3][npts] fixed point
    const Tables *tab;
    const EosTable *eos;
    int *err;
    int *work;           // work counter
    const int *list;     // cell list (NULL: all cells)
    const int *n_list;   // number of cells in the list (device)
    int *ovf_list, *ovf_count;   // cells too large for this pass
    int cap_ce, cap_ci, cap_new; // per-cell capacities (staging; created electrons)
    NewE *nw;            // created-electron scratch: cap_new entries per warp of the launch
    unsigned long long *gw;  // global staging: warp_gmem_words(cap_ce, cap_ci) words per warp
};

// warp reductions: a fixed tree, result broadcast from lane 0 so every lane
// holds the same bits
__device__ __forceinline__ real wsum_f(real v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    return __shfl_sync(FULL, v, 0);
}

__device__ __forceinline__ dd wsum_dd(dd v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dd t{__shfl_down_sync(FULL, v.hi, o), __shfl_down_sync(FULL, v.lo, o)};
        v = dd_add(v, t);
    }
    return dd{__shfl_sync(FULL, v.hi, 0), __shfl_sync(FULL, v.lo, 0)};
}

__device__ __forceinline__ int wsum_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    return __shfl_sync(FULL, v, 0);
}

// inclusive prefix over the lanes (fixed order)
__device__ __forceinline__ real wscan_f(real v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        real t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ dd wscan_dd(dd v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        dd t{__shfl_up_sync(FULL, v.hi, o), __shfl_up_sync(FULL, v.lo, o)};
        if (lane >= o) v = dd_add(v, t);
    }
    return v;
}

__device__ __forceinline__ dd wbcast_dd(dd v, int src)
{
    return dd{__shfl_sync(FULL, v.hi, src), __shfl_sync(FULL, v.lo, src)};
}

// Sort of the cells larger than the register sorts take (n > radix_min of
// the kernel instance): a stable LSD radix sort (four 8-bit digits) of the
// keys' high 32 bits packed with the slot, then the rare runs of equal high
// words reordered by (low word, id) by one lane.  buf holds 2 n packed
// entries, hist 256 counters.
__host__ __device__ constexpr int radix_min(int rmax) { return rmax > 512 ? rmax : 512; }

// the cell-kernel instance (largest register sort) of a staging of ce
// electrons and ci ions per cell
__host__ __device__ constexpr int rmax_for(int ce, int ci)
{
    return ce <= 128 && ci <= 128 ? 128 : (ce <= 512 && ci <= 512 ? 512 : 1024);
}

template <class IdT>
__device__ void warp_radix(const unsigned long long *key, IdT *id, unsigned short *slot, unsigned long long *tmp,
                           unsigned long long *buf, int *hist, int n, int lane)
{
    unsigned long long *A = buf, *B = buf + n;
    for (int k = lane; k < n; k += 32) A[k] = (key[k] & 0xffffffff00000000ull) | (unsigned long long)k;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 32 + 8 * pass;
        for (int b = lane; b < 256; b += 32) hist[b] = 0;
        __syncwarp();
        for (int k = lane; k < n; k += 32) atomicAdd(hist + (int)((A[k] >> shift) & 255u), 1);
        __syncwarp();
        // exclusive scan of the 256 counts: eight per lane, then across lanes
        int c[8], run = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) { c[q] = hist[lane * 8 + q]; run += c[q]; }
        int incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        int off = incl - run;
#pragma unroll
        for (int q = 0; q < 8; ++q) { hist[lane * 8 + q] = off; off += c[q]; }
        __syncwarp();
        // stable scatter, 32 entries at a time in order
        for (int base = 0; base < n; base += 32) {
            const int k = base + lane;
            const bool act = k < n;
            const unsigned long long v = act ? A[k] : 0ull;
            const int d = act ? (int)((v >> shift) & 255u) : -1;
            const unsigned peers = __match_any_sync(FULL, d);
            const int at = act ? hist[d] + __popc(peers & ((1u << lane) - 1u)) : 0;
            __syncwarp();
            if (act) {
                B[at] = v;
                if (lane == __ffs(peers) - 1) hist[d] += __popc(peers);
            }
            __syncwarp();
        }
        unsigned long long *t = A; A = B; B = t;
    }
    // equal high words (rare): order those runs by (low word, id)
    bool tie = false;
    for (int k = lane; k + 1 < n; k += 32) tie |= (A[k] >> 32) == (A[k + 1] >> 32);
    if (__any_sync(FULL, tie) && lane == 0) {
        for (int k = 1; k < n; ++k) {
            unsigned long long v = A[k];
            int j = k - 1;
            while (j >= 0 && (A[j] >> 32) == (v >> 32)) {
                const int sa = (int)(A[j] & 0xffffu), sb = (int)(v & 0xffffu);
                const bool gt = key[sa] > key[sb] || (key[sa] == key[sb] && id[sa] > id[sb]);
                if (!gt) break;
                A[j + 1] = A[j];
                --j;
            }
            A[j + 1] = v;
        }
    }
    __syncwarp();
    for (int k = lane; k < n; k += 32) slot[k] = (unsigned short)(A[k] & 0xffffu);
    __syncwarp();
    for (int k = lane; k < n; k += 32) tmp[k] = (unsigned long long)id[slot[k]];
    __syncwarp();
    for (int k = lane; k < n; k += 32) id[k] = (IdT)tmp[k];
    __syncwarp();
}

// Sort of up to 32 E entries in registers, E per lane (entry lane * E + j):
// the bitonic network over (key high 48 bits | slot) words, compare-exchange
// through warp shuffles across lanes and in place within a lane.  That is
// the (key, id) order unless two keys share their high 48 bits (probability
// ~n^2 / 2^49 per cell); such runs are then put in (key, id) order by one
// lane.  slot[k] gets the slot at position k, id[] the ids in that order
// (through tmp, n entries of scratch, which may be the key array).
template <int E, int S>
__device__ __forceinline__ void reg_cmpx_in_lane(unsigned long long (&v)[E], int lane, int size)
{
    if constexpr (S < E) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            if ((j & S) != 0) continue;
            const bool asc = ((lane * E + j) & size) == 0;
            const unsigned long long a = v[j], b = v[j ^ S];
            if ((a > b) == asc) { v[j] = b; v[j ^ S] = a; }
        }
    }
}

// runs of equal high 48 key bits of a (high 48 bits, slot) order into
// (key, id) order: insertion within each run, by one lane
template <class IdT>
__device__ void order_ties(const unsigned long long *key, const IdT *id, unsigned short *slot, int n)
{
    for (int k = 1; k < n; ++k) {
        const int sb = slot[k];
        const unsigned long long kb = key[sb];
        int j = k - 1;
        while (j >= 0) {
            const int sa = slot[j];
            const unsigned long long ka = key[sa];
            if ((ka >> 16) != (kb >> 16)) break;
            if (!(ka > kb || (ka == kb && id[sa] > id[sb]))) break;
            slot[j + 1] = (unsigned short)sa;
            --j;
        }
        slot[j + 1] = (unsigned short)sb;
    }
}

template <int E, class IdT>
__device__ __forceinline__ void warp_sort_reg(const unsigned long long *key, IdT *id, unsigned short *slot,
                                              unsigned long long *tmp, int n, int lane)
{
    unsigned long long v[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int k = lane * E + j;
        v[j] = k < n ? (key[k] & ~0xffffull) | (unsigned long long)k : ~0ull;
    }
    for (int size = 2; size <= 32 * E; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= E) {
                const int lm = stride / E;
#pragma unroll
                for (int j = 0; j < E; ++j) {
                    const int e = lane * E + j;
                    const unsigned long long o = __shfl_xor_sync(FULL, v[j], lm);
                    const bool keep_min = ((e & stride) == 0) == ((e & size) == 0);
                    v[j] = keep_min ? (o < v[j] ? o : v[j]) : (o > v[j] ? o : v[j]);
                }
            } else if (stride == 1) {
                reg_cmpx_in_lane<E, 1>(v, lane, size);
            } else if (stride == 2) {
                reg_cmpx_in_lane<E, 2>(v, lane, size);
            } else if (stride == 4) {
                reg_cmpx_in_lane<E, 4>(v, lane, size);
            } else if (stride == 8) {
                reg_cmpx_in_lane<E, 8>(v, lane, size);
            } else {
                reg_cmpx_in_lane<E, 16>(v, lane, size);
            }
        }
    }
    // neighbours with equal high words (the padding never compares: its
    // positions are >= n)
    bool tie = false;
#pragma unroll
    for (int j = 0; j + 1 < E; ++j)
        tie |= lane * E + j + 1 < n && (v[j] >> 16) == (v[j + 1] >> 16);
    const unsigned long long nx = __shfl_down_sync(FULL, v[0], 1);
    tie |= lane < 31 && lane * E + E < n && (v[E - 1] >> 16) == (nx >> 16);
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int k = lane * E + j;
        if (k < n) slot[k] = (unsigned short)(v[j] & 0xffffu);
    }
    __syncwarp();
    if (__any_sync(FULL, tie)) {
        if (lane == 0) order_ties<IdT>(key, id, slot, n);
        __syncwarp();
    }
    for (int k = lane; k < n; k += 32) tmp[k] = (unsigned long long)id[slot[k]];
    __syncwarp();
    for (int k = lane; k < n; k += 32) id[k] = (IdT)tmp[k];
    __syncwarp();
}

// the larger register sorts out of line: their 16-32 key registers would
// otherwise raise the register pressure of the whole cell kernel
template <int E, class IdT>
__device__ __noinline__ void warp_sort_reg_call(const unsigned long long *key, IdT *id, unsigned short *slot,
                                                unsigned long long *tmp, int n, int lane)
{
    warp_sort_reg<E, IdT>(key, id, slot, tmp, n, lane);
}

// The in-cell canonical order, ascending (key, id): in registers up to
// RMAX entries (128, 512 or 1024: the kernel instance), the radix sort
// above radix_min(RMAX).  slot[] must hold 0..n-1 on entry; n is at most
// RMAX when rbuf is NULL (the staging of a kernel instance without the
// radix buffer never holds more).
template <class IdT, int RMAX = 512>
__device__ void warp_sort(unsigned long long *key, IdT *id, unsigned short *slot, unsigned long long *tmp,
                          unsigned long long *rbuf, int *rhist, int n, int lane)
{
    if (n > radix_min(RMAX)) { warp_radix<IdT>(key, id, slot, tmp, rbuf, rhist, n, lane); return; }
    if (n <= 32) warp_sort_reg<1, IdT>(key, id, slot, tmp, n, lane);
    else if (n <= 64) warp_sort_reg<2, IdT>(key, id, slot, tmp, n, lane);
    else if (n <= 128) warp_sort_reg<4, IdT>(key, id, slot, tmp, n, lane);
    else if constexpr (RMAX > 128) {
        if (n <= 256) warp_sort_reg_call<8, IdT>(key, id, slot, tmp, n, lane);
        else if (n <= 512) warp_sort_reg_call<16, IdT>(key, id, slot, tmp, n, lane);
        else if constexpr (RMAX > 512) warp_sort_reg_call<32, IdT>(key, id, slot, tmp, n, lane);
    }
}

__device__ __forceinline__ real cic_w(real x, int node)
{
    real d = r_fabs(x - (real)node);
    return d < RF(1.0) ? RF(1.0) - d : RF(0.0);
}

// per-warp shared memory carve-up
struct WarpMem {
    real4 *eu;                 // [cap_ce] ux uy uz w (slot order)
    unsigned long long *ekey;   // [cap_ce] sort key, later reused as real take
    unsigned long long *eid;    // [cap_ce] ids in canonical order
    unsigned short *eperm;      // [cap_ce] canonical position -> slot
    real2 *epos;               // [cap_ce] positions in the cell (slot order)
    real2 *ipos;               // [cap_ci] ion positions in the cell (slot order)
    real4 *iu;                 // [cap_ci] ux uy uz zfrac (slot order)
    int *ist;                   // [cap_ci] Z | nK << 8 (slot order)
    unsigned long long *ikey;   // [cap_ci] sort key, later reused as nrec
    unsigned int *iid;          // [cap_ci] ids in canonical order
    unsigned short *iperm;      // [cap_ci]
    NewE *nw;                   // [cap_new] in global memory: the warp's slice of the scratch
    real *dE;                  // [16] continuum lowering per charge state
    real *Pz;                  // [16] impact-ionization probability per charge
    real4 *lz;                 // [NS] Lotz constants of one charge state: P, 1/P, ln P, a q
    unsigned long long *rbuf;   // [2 max(cap_ce, cap_ci)] radix sort (only when a cell can exceed radix_min)
    int *rhist;                 // [256]
    dd *ph;                     // [2 MAXB] photon bin scratch
    int *phc;                   // [MAXB] events per bin so far
};

// shared-memory pieces start on 16 B (FP32) or 32 B (FP64: real4 is 32 B);
// the sort-key storage later holds a real2 per electron
constexpr size_t kSmAlign = sizeof(real4) > 16 ? 32 : 16;
constexpr size_t kKeyBytes = sizeof(real2) > 8 ? sizeof(real2) : 8;
__host__ __device__ inline size_t amem(size_t x) { return (x + kSmAlign - 1) & ~(kSmAlign - 1); }

// Shared memory of one warp staging up to ce electrons and ci ions.  The
// electrons a cell creates in a step (up to 3 per ion: impact, photo- and
// Auger ionization) are rare; they live in the warp's slice of a global
// scratch, which keeps the staging of large cells small.  The instances
// for cells above 128 entries, whose staging limits the warps resident on
// an SM, also keep the electron ids (read once per collision), the sort
// keys (later the per-electron scratch of the Lotz sums and of
// recombination), the positions (read back once, at the write-back) and
// the radix buffer there (warp_gmem_words 8-byte words a warp).
__host__ __device__ inline bool ids_in_gmem(int ce, int ci) { return rmax_for(ce, ci) > 128; }

__host__ __device__ inline size_t warp_gmem_words(int ce, int ci)
{
    if (!ids_in_gmem(ce, ci)) return 0;
    const int cm = ce > ci ? ce : ci;
    return (size_t)ce * (1 + kKeyBytes / 8 + sizeof(real2) / 8) +
           (cm > radix_min(rmax_for(ce, ci)) ? 2 * (size_t)cm : 0);
}

__host__ __device__ inline size_t warp_mem_bytes(int ce, int ci)
{
    const bool g = ids_in_gmem(ce, ci);
    size_t b = 0;
    b += amem((size_t)ce * sizeof(real4)) +
         (g ? 0 : amem((size_t)ce * kKeyBytes) + amem((size_t)ce * 8) + amem((size_t)ce * sizeof(real2))) +
         amem((size_t)ce * 2) + amem((size_t)ci * sizeof(real2));
    b += amem((size_t)ci * sizeof(real4)) + amem((size_t)ci * 4) + amem((size_t)ci * 8) + amem((size_t)ci * 4)
         + amem((size_t)ci * 2);
    b += amem(16 * sizeof(real)) * 2 + amem(NS * sizeof(real4)) + amem(2 * MAXB * sizeof(dd)) + amem(MAXB * 4);
    const int cm = ce > ci ? ce : ci;
    if (cm > radix_min(rmax_for(ce, ci))) b += (g ? 0 : amem((size_t)cm * 16)) + 256 * 4;
    return b;
}

// gw: the warp's slice of the global staging (warp_gmem_words words)
__device__ inline WarpMem carve(char *base, int ce, int ci, NewE *nw, unsigned long long *gw)
{
    const bool g = ids_in_gmem(ce, ci);
    WarpMem m;
    char *p = base;
    m.eu = (real4 *)p; p += amem((size_t)ce * sizeof(real4));
    if (g) {
        m.eid = gw;
        m.ekey = gw + ce;
        m.epos = reinterpret_cast<real2 *>(gw + (size_t)ce * (1 + kKeyBytes / 8));
    } else {
        m.ekey = (unsigned long long *)p; p += amem((size_t)ce * kKeyBytes);
        m.eid = (unsigned long long *)p; p += amem((size_t)ce * 8);
        m.epos = (real2 *)p; p += amem((size_t)ce * sizeof(real2));
    }
    m.eperm = (unsigned short *)p; p += amem((size_t)ce * 2);
    m.ipos = (real2 *)p; p += amem((size_t)ci * sizeof(real2));
    m.iu = (real4 *)p; p += amem((size_t)ci * sizeof(real4));
    m.ist = (int *)p; p += amem((size_t)ci * 4);
    m.ikey = (unsigned long long *)p; p += amem((size_t)ci * 8);
    m.iid = (unsigned int *)p; p += amem((size_t)ci * 4);
    m.iperm = (unsigned short *)p; p += amem((size_t)ci * 2);
    m.nw = nw;
    m.dE = (real *)p; p += amem(16 * sizeof(real));
    m.Pz = (real *)p; p += amem(16 * sizeof(real));
    m.lz = (real4 *)p; p += amem(NS * sizeof(real4));
    m.ph = (dd *)p; p += amem(2 * MAXB * sizeof(dd));
    m.phc = (int *)p; p += amem(MAXB * 4);
    const int cm = ce > ci ? ce : ci;
    m.rbuf = nullptr; m.rhist = nullptr;
    if (cm > radix_min(rmax_for(ce, ci))) {
        if (g) m.rbuf = gw + (size_t)ce * (1 + kKeyBytes / 8 + sizeof(real2) / 8);
        else { m.rbuf = (unsigned long long *)p; p += amem((size_t)cm * 16); }
        m.rhist = (int *)p;
    }
    return m;
}

// ---------------------------------------------------------------------
// field gather (CIC from the staggered Yee grid; zero outside [0, nx])
// ---------------------------------------------------------------------
struct SlabGrid {
    int nx, ny, W;       // W = nx + 1 points per row
    const real *fe;     // ex of this slab (ey, ez follow with stride npts)
    const real *fb;     // bx of this slab
    int npts;            // stride between components
    int fo;              // first grid point of the slab
};

__device__ __forceinline__ real grid_interp(const real *F, const SlabGrid &g, int cx, int cy,
                                             real xi, real eta, bool hx, bool hy)
{
    real xs = xi - (hx ? RF(0.5) : RF(0.0)), ys = eta - (hy ? RF(0.5) : RF(0.0));
    int ax = (int)r_floor(xs), ay = (int)r_floor(ys);
    real fx = xs - (real)ax, fy = ys - (real)ay;
    int imax = hx ? g.nx - 1 : g.nx;
    real v = RF(0.0);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        int i = cx + ax + a;
        if (i < 0 || i > imax) continue;
        real wx = a ? fx : RF(1.0) - fx;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            int j = cy + ay + b;
            j %= g.ny; if (j < 0) j += g.ny;
            real wy = b ? fy : RF(1.0) - fy;
            v += wx * wy * __ldg(F + (size_t)j * g.W + i);
        }
    }
    return v;
}

// ---------------------------------------------------------------------
// current deposit
// ---------------------------------------------------------------------
struct JAcc2 { real x[3][4], y[4][3], z[4][4]; };
struct JAcc1 { real x[3], y[4], z[4]; };

// v * 2^40 rounded to a 64-bit integer with FP32 and integer instructions
// only (|v| < 2^22): the high part is split off exactly at 2^31 (the
// FP64 build rounds v * JFIX directly)
__device__ __forceinline__ long long fix40(real v)
{
#ifdef PIC_FP64
    return __double2ll_rn(v * JFIX);
#else
    float x = v * 1099511627776.0f;                     // exact: power-of-two scale
    float qh = truncf(x * 4.656612873077393e-10f);      // x / 2^31, integer part
    float r = fmaf(-qh, 2147483648.0f, x);               // exact remainder, |r| < 2^31
    long long lo = (long long)__float2int_rn(fminf(fmaxf(r, -2147483520.0f), 2147483520.0f));
    return ((long long)(int)qh << 31) + lo;
#endif
}

__device__ __forceinline__ void jatomic(unsigned long long *J, real v)
{
    if (v != RF(0.0)) atomicAdd(J, (unsigned long long)fix40(v));
}

// Esirkepov weights of one sub-cell move, stencil anchored at cell (ax, ay)
// offsets -1..2; start (x0, y0), end (x1, y1) relative to the anchor cell
__device__ __forceinline__ void esirkepov2(real x0, real y0, real x1, real y1, real qw, real qwbz,
                                           real frac, JAcc2 &A)
{
    real S0x[4], S1x[4], S0y[4], S1y[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        S0x[a] = cic_w(x0, a - 1); S1x[a] = cic_w(x1, a - 1);
        S0y[a] = cic_w(y0, a - 1); S1y[a] = cic_w(y1, a - 1);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        real acc = RF(0.0);
        real sy = S0y[b] + RF(0.5) * (S1y[b] - S0y[b]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            acc += (S1x[a] - S0x[a]) * sy;
            A.x[a][b] -= qw * acc;
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        real acc = RF(0.0);
        real dsx = S1x[a] - S0x[a];
        real sx = S0x[a] + RF(0.5) * dsx;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            acc += (S1y[b] - S0y[b]) * sx;
            A.y[a][b] -= qw * acc;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            real dsy = S1y[b] - S0y[b];
            real wz = S0x[a] * S0y[b] + RF(0.5) * dsx * S0y[b] + RF(0.5) * S0x[a] * dsy + dsx * dsy * (RF(1.0) / RF(3.0));
            A.z[a][b] += qwbz * wz * frac;
        }
    }
}

__device__ __forceinline__ void esirkepov1(real x0, real x1, real qw, real qwby, real qwbz, real frac, JAcc1 &A)
{
    real S0x[4], S1x[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) { S0x[a] = cic_w(x0, a - 1); S1x[a] = cic_w(x1, a - 1); }
    real acc = RF(0.0);
#pragma unroll
    for (int a = 0; a < 3; ++a) { acc += S1x[a] - S0x[a]; A.x[a] -= qw * acc; }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        real s = RF(0.5) * (S0x[a] + S1x[a]);
        A.y[a] += qwby * s * frac;
        A.z[a] += qwbz * s * frac;
    }
}

// a move of one cell or more: equal sub-cell segments, each deposited
// straight to global memory around its own start cell
__device__ __noinline__ void deposit_long(const SlabGrid &g, unsigned long long *J, int npts, int fo, int cx, int cy,
                             real x0, real y0, real x1, real y1, real qw, real qwby, real qwbz)
{
    real ax = r_fabs(x1 - x0), ay = g.ny > 1 ? r_fabs(y1 - y0) : RF(0.0);
    int nseg = (int)r_floor(r_fmax(ax, ay)) + 1;
    for (int k = 0; k < nseg; ++k) {
        real a0 = (real)k / nseg, a1 = (real)(k + 1) / nseg;
        real xa = x0 + a0 * (x1 - x0), xb = x0 + a1 * (x1 - x0);
        real ya = y0 + a0 * (y1 - y0), yb = y0 + a1 * (y1 - y0);
        int sx = (int)r_floor(xa), sy = g.ny > 1 ? (int)r_floor(ya) : 0;
        real f = RF(1.0) / nseg;
        if (g.ny == 1) {
            JAcc1 A = {};
            esirkepov1(xa - sx, xb - sx, qw, qwby, qwbz, f, A);
            for (int a = 0; a < 4; ++a) {
                int i = cx + sx - 1 + a;
                if (a < 3 && i >= 0 && i < g.nx) jatomic(J + fo + i, A.x[a]);
                if (i >= 0 && i <= g.nx) {
                    jatomic(J + npts + fo + i, A.y[a]);
                    jatomic(J + 2 * npts + fo + i, A.z[a]);
                }
            }
        } else {
            JAcc2 A = {};
            esirkepov2(xa - sx, ya - sy, xb - sx, yb - sy, qw, qwbz, f, A);
            for (int a = 0; a < 4; ++a) {
                int i = cx + sx - 1 + a;
                for (int b = 0; b < 4; ++b) {
                    int j = (cy + sy - 1 + b) % g.ny; if (j < 0) j += g.ny;
                    size_t o = (size_t)fo + (size_t)j * g.W + i;
                    if (a < 3 && i >= 0 && i < g.nx) jatomic(J + o, A.x[a][b]);
                    if (b < 3 && i >= 0 && i <= g.nx) jatomic(J + npts + o, A.y[a][b]);
                    if (i >= 0 && i <= g.nx) jatomic(J + 2 * npts + o, A.z[a][b]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------
// push of one particle: gather, Boris, move, deposit; returns the next
// cell (local index) or -1 when it left through an x boundary
// ---------------------------------------------------------------------
template <int DIM, class Acc>
__device__ __forceinline__ int push_one(const SlabDev &S, const SlabGrid &g, unsigned long long *J, int npts,
                                        int cx, int cy, real &xi, real &eta, real &ux, real &uy, real &uz,
                                        real qm, real qw, bool do_push, bool do_dep, Acc &A)
{
    if (!do_push) return cy * S.nx + cx;
    real ex = grid_interp(g.fe, g, cx, cy, xi, eta, true, false);
    real ey = grid_interp(g.fe + g.npts, g, cx, cy, xi, eta, false, true);
    real ez = grid_interp(g.fe + 2 * g.npts, g, cx, cy, xi, eta, false, false);
    real bx = grid_interp(g.fb, g, cx, cy, xi, eta, false, true);
    real by = grid_interp(g.fb + g.npts, g, cx, cy, xi, eta, true, false);
    real bz = grid_interp(g.fb + 2 * g.npts, g, cx, cy, xi, eta, true, true);
    boris(ux, uy, uz, ex, ey, ez, bx, by, bz, qm, S.dt);
    real ig = r_rsqrt(RF(1.0) + ux * ux + uy * uy + uz * uz);
    real bxv = ux * ig, byv = uy * ig, bzv = uz * ig;
    const real c = (real)kCnmPerFs;
    real xn = xi + bxv * c * S.dt / S.dx;
    real yn = DIM == 2 ? eta + byv * c * S.dt / S.dy : eta;
    if (!(r_fabs(xn - xi) < RF(64.0) && r_fabs(yn - eta) < RF(64.0))) return -2;   // not finite: dropped
    if (do_dep) {
        if (r_fabs(xn - xi) < RF(1.0) && r_fabs(yn - eta) < RF(1.0)) {
            if constexpr (DIM == 2) esirkepov2(xi, eta, xn, yn, qw, qw * bzv, RF(1.0), A);
            else esirkepov1(xi, xn, qw, qw * byv, qw * bzv, RF(1.0), A);
        } else {
            deposit_long(g, J, npts, g.fo, cx, cy, xi, eta, xn, yn, qw, qw * byv, qw * bzv);
        }
    }
    real fx = r_floor(xn), fy = r_floor(yn);
    int ncx = cx + (int)fx;
    int ncy = cy + (int)fy;
    xi = xn - fx;
    eta = yn - fy;
    const real below1 = kBelow1;
    if (xi >= RF(1.0)) xi = below1;
    if (eta >= RF(1.0)) eta = below1;
    if (DIM == 1) { ncy = 0; }
    else { ncy %= S.ny; if (ncy < 0) ncy += S.ny; }
    if (ncx < 0 || ncx >= S.nx) return -1;
    return ncy * S.nx + ncx;
}

}  // namespace pic
