// Host side of the C ABI declared in include/pic.h: the context, its device
// arena, the per-step launch sequence and the host <-> device copies.
//
// A context holds nslot slots.  Slot k owns cells [k*slot_cells,
// (k+1)*slot_cells) and grid points [k*slot_pts, (k+1)*slot_pts) of one
// global numbering, so each kernel runs once per step for every slab.
// pic_init makes a one-slot context (1D or 2D); pic_batch_init a context of
// 1D slots into which slabs are admitted, and from which they are retired,
// between steps.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pic.h"
#include "pic_dev.cuh"
#include "pic_cellk.cuh"
#include "pic_push.cuh"
#include "pic_grid.cuh"
#include "pic_rt.cuh"

using namespace pic;

namespace {

// device counters; [0, CNT_STEP_ZERO) are cleared at the start of a step
constexpr int CNT_APPEND = 0, CNT_WORK = 1, CNT_WORK_T1 = 2, CNT_WORK_BIG = 3, CNT_OVF = 4, CNT_OVF2 = 5,
              CNT_WORK_PUSH = 6, CNT_WORK_T2 = 7, CNT_OVF3 = 8, CNT_STEP_ZERO = 9, CNT_ERR = 10, CNT_MAXE = 11,
              CNT_MAXI = 12, CNT_NLOAD = 13, CNT_HIST_E = 16, CNT_HIST_I = CNT_HIST_E + NHIST,
              NCOUNTERS = CNT_HIST_I + NHIST;
constexpr int NEV = 6;   // timing events per step
// largest cell of the one-warp pass (the FP64 build's staging is twice as
// wide and takes half the populations into the same shared memory)
constexpr int BIG_CE = sizeof(real) == 8 ? 1024 : 2048, BIG_CI = sizeof(real) == 8 ? 256 : 512;

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// Most cells (and grid points) of a context: 2^27, sixteen times the large
// 2D slab, so that cell counts times photon bins (8) or field components
// stay inside 32-bit int indices on the device.
constexpr long long kMaxCells = 1LL << 27;

// smallest power of two >= x, from 32, at most 2^30 (no signed overflow)
int next_pow2(int x)
{
    int p = 32;
    while (p < x && p < (1 << 30)) p <<= 1;
    return p;
}

}  // namespace

struct pic_ctx {
    cudaStream_t stream = nullptr;
    bool own_arena = false;
    char *arena = nullptr;
    size_t arena_bytes = 0, used = 0;
    std::string err;

    bool batch = false;
    int nslot = 1, slot_cells = 0, slot_pts = 0, slot_rows = 1;
    std::vector<SlabDev> slabs;          // host copy of every slot's description
    std::vector<int> slot_state;         // 0 free, 1 active, 2 retired (emptied by the next step), 3 failed
    std::vector<pic_grid> grids;         // grid of each slot as given
    struct Pending {                     // admitted, particles not yet on the device
        int slot;
        std::vector<real4> e0, e1, i0, i1;
        std::vector<int> ek, ik;
    };
    std::vector<Pending> pending;
    int ncell = 0, npts = 0, nblk = 0, nrows = 0, max_row_nx = 0;
    int cap_e = 0, cap_i = 0;

    real4 *eA0, *eA1, *eB0, *eB1;
    real4 *iA0, *iA1, *iB0, *iB1;
    int *ekey, *ikey;
    int *csE[2], *csI[2];
    int cur = 0;
    int *cnt_e, *cnt_i, *fill_e, *fill_i, *bsum_e, *bsum_i;
    int *counters, *ovf_list, *ovf_list2, *cell_slab, *pt_slab, *row_slab, *row_idx;
    int *slab_app, *slab_err;            // [nslot] per-slab appends of the step; budget failures
    bool budgets = false;                // some slot has an electron budget
    SlabDev *d_slab;                     // [nslot]
    unsigned *d_steps;                   // [nslot]
    SlabTally *d_tally;                  // [nslot]
    Tables *d_tab;
    EosTable *d_eos;
    real *E[2], *B;
    int ecur = 0;
    unsigned long long *J;
    ph2 *photons;
    double *diag_buf;

    // cell-kernel tiers: tier 0 takes every cell with the staging sizes
    // below; cells that do not fit go to tier 1 (sized for the largest
    // cells, when that is larger), then to the one-warp large-cell pass
    int cap_ce = 128, cap_ci = 32, cap_new = 96, wpc = 4;
    int t1_ce = 0, t1_ci = 0, t1_wpc = 1;    // t1_ce == 0: no tier 1
    int t2_ce = 0, t2_ci = 0, t2_wpc = 1;    // t2_ce == 0: no tier 2
    size_t smem_main = 0, smem_t1 = 0, smem_t2 = 0, smem_big = 0;
    int nsm = 0, grid_main = 0, grid_t1 = 0, grid_t2 = 0, grid_big = 0, grid_push = 0;
    NewE *nw = nullptr;                  // created-electron scratch of the cell launches
    size_t nw_entries = 0;
    unsigned long long *gw = nullptr;    // global staging of the large-cell instances (ids, radix buffer)
    size_t gw_words = 0;
    int64_t launches = 0;
    bool loaded_e = false, loaded_i = false;
    std::vector<double> hv_tab, sigma;   // host copy of the photoionization table
    bool timing = false;
    std::vector<cudaEvent_t> ev;         // NEV events per recorded step
    size_t ev_used = 0;

    // CUDA graphs of two steps (the buffer swaps of a step pair cancel, so a
    // pair replays from the same state); one per buffer parity
    struct StepShape {
        const void *eA0, *iA0;
        int cur, ecur, grid_main, wpc, cap_ce, cap_ci, cap_new, nsub, t1_ce, t1_ci, t1_wpc, grid_t1;
        int t2_ce, t2_ci, t2_wpc, grid_t2;
        size_t smem_main;
        bool march, field, rt;
    };
    struct StepGraph {
        StepShape key{};
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0;
    };
    bool use_graphs = true;
    // autotuner: warps per CTA of the cell kernel, chosen per staging size
    struct Tuned { int ce, ci, wpc; float ms[4]; unsigned tried; bool done = false; };  // ms: mean of two
    cudaEvent_t cell_ev[2] = {nullptr, nullptr};    // around the cell kernels while tuning
    bool cell_ev_on = false;
    int64_t steps_done = 0;
    std::vector<Tuned> tuned;
    bool autotune = false;
    cudaStream_t cap_stream = nullptr;
    StepGraph graphs[2];
    int graph_next = 0;
    // radiation transport mode (pic_rt): device memory the context owns
    void *rt_mem = nullptr;
    size_t rt_bytes = 0;                 // its size (one block, checkpointed whole)
    int rt_nord = 0;
};

namespace {

pic_status fail(pic_ctx *c, pic_status st, const std::string &msg)
{
    if (c) c->err = msg;
    return st;
}

pic_status cuda_fail(pic_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, PIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);     \
    } while (0)

template <class T>
T *carve_arena(pic_ctx *c, size_t count)
{
    size_t b = al(count * sizeof(T));
    if (c->arena && c->used + b > c->arena_bytes) return nullptr;
    T *p = reinterpret_cast<T *>(c->arena + c->used);
    c->used += b;
    return p;
}

// Created-electron scratch of the cell launches, in entries: cap_new = 3 x
// the ions a tier stages (at most 768 below the large-cell pass, whose
// 1536 take one warp a CTA) for every warp resident at once, at most 16 a
// SM (the register-bound instances) on up to 192 SMs, and no more warps
// than cells (plus a CTA).  Launch grids are clamped to the slices.
size_t nw_scratch_entries(int ncell)
{
    const size_t warps = std::min<size_t>(192 * 16, (size_t)ncell + 64);
    return warps * 768;
}

// Global staging of the large-cell instances, in 8-byte words: 3072 a warp
// (ids, keys and positions of 1024 electrons in the FP32 build) for as many
// warps; the
// large cells' warps are few, and their grids are clamped to the slices.
size_t gw_scratch_words(int ncell)
{
    const size_t warps = std::min<size_t>(192 * 16, (size_t)ncell + 64);
    return warps * 3072;
}

size_t arena_need(int ncell, int npts, int nblk, int cap_e, int cap_i, int nslot, int nrows)
{
    size_t b = 0;
    b += 4 * al((size_t)cap_e * sizeof(real4)) + al((size_t)cap_e * 4);
    b += 4 * al((size_t)cap_i * sizeof(real4)) + al((size_t)cap_i * 4);
    b += 4 * al((size_t)(ncell + 1) * 4) + al((size_t)ncell * 16) + 2 * al((size_t)nblk * 4);
    b += al(NCOUNTERS * 4) + al((size_t)ncell * 4) * 3;
    b += al(sizeof(SlabDev) * (size_t)nslot) + 3 * al(4 * (size_t)nslot) + al(sizeof(SlabTally) * (size_t)nslot)
         + al(sizeof(Tables)) + al(sizeof(EosTable));
    b += 3 * al((size_t)npts * 3 * sizeof(real)) + al((size_t)npts * 3 * 8) + al((size_t)npts * 4);
    b += 2 * al((size_t)nrows * 4);
    b += al((size_t)ncell * PIC_MAX_BINS * sizeof(ph2));
    b += al(nw_scratch_entries(ncell) * sizeof(NewE)) + al(gw_scratch_words(ncell) * 8);
    b += al((4 + NZ + 4096 + 8) * 8);
    return b + 4096;
}

// photoionization cross section of the table at hv: log-log interpolation,
// held constant beyond the table ends
double sigma_table(const pic_ctx *c, int s, double hv)
{
    const int n = (int)c->hv_tab.size();
    const double *g = c->hv_tab.data(), *v = c->sigma.data() + (size_t)s * n;
    if (hv <= g[0]) return v[0];
    if (hv >= g[n - 1]) return v[n - 1];
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) { int m = (lo + hi) / 2; if (g[m] <= hv) lo = m; else hi = m; }
    if (v[lo] <= 0.0 || v[lo + 1] <= 0.0) {
        double f = (hv - g[lo]) / (g[lo + 1] - g[lo]);
        return v[lo] + f * (v[lo + 1] - v[lo]);
    }
    double f = std::log(hv / g[lo]) / std::log(g[lo + 1] / g[lo]);
    return std::exp(std::log(v[lo]) + f * std::log(v[lo + 1] / v[lo]));
}

// the cell-kernel instance for a launch staging up to ce electrons and ci
// ions per cell: in-register sorts up to 128, 512 or 1024 entries
typedef void (*CellKernel)(CellArgs);
CellKernel cell_kernel(int ce, int ci)
{
    const int r = rmax_for(ce, ci);
    return r == 128 ? k_cell<128> : (r == 512 ? k_cell<512> : k_cell<1024>);
}

// largest warps per CTA of the cell kernel whose staging fits 200 KB, at
// most 8 and at most what the instance's launch bounds allow
int max_wpc(int ce, int ci)
{
    const size_t per = warp_mem_bytes(ce, ci);
    int lim = 8;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, cell_kernel(ce, ci)) == cudaSuccess && fa.maxThreadsPerBlock >= 32)
        lim = std::min(lim, fa.maxThreadsPerBlock / 32);
    return std::max(1, (int)std::min<size_t>(lim, (200 * 1024) / per));
}

// CTAs of a persistent cell launch staging ce / ci: the resident ones on
// every SM, as many as the global scratches have warp slices for
int cell_grid(const pic_ctx *c, int occ, int wpc, int ce, int ci)
{
    size_t cap = c->nw_entries / ((size_t)wpc * 3 * ci);
    const size_t gw = warp_gmem_words(ce, ci);
    if (gw) cap = std::min(cap, c->gw_words / ((size_t)wpc * gw));
    return std::max(1, (int)std::min<size_t>((size_t)std::max(1, occ) * c->nsm, std::min<size_t>(cap, 1 << 30)));
}

pic_status cell_smem_attr(pic_ctx *c)
{
    // the opt-in maximum (less the kernel's static shared memory), so that
    // occupancy can be asked for any staging size
    int dev = 0, optin = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t m = std::max(std::max(c->smem_main, c->smem_t1), std::max(c->smem_t2, c->smem_big));
    for (CellKernel k : {k_cell<128>, k_cell<512>, k_cell<1024>}) {
        cudaFuncAttributes fa{};
        CK(cudaFuncGetAttributes(&fa, k));
        const size_t lim = optin > (int)fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : m;
        CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max(m, lim)));
    }
    return PIC_OK;
}

// Warps per CTA (up to max_wpc) that keep the most warps of the cell kernel
// resident per SM: with large cells the staging, not the registers, limits
// residency, and fewer warps per CTA can let more CTAs share an SM.  Ties
// go to the larger CTA.
int best_wpc(pic_ctx *c, int ce, int ci)
{
    if (cell_smem_attr(c) != PIC_OK) return max_wpc(ce, ci);
    const size_t per = warp_mem_bytes(ce, ci);
    int best = 1, best_warps = 0;
    for (int w = 1; w <= max_wpc(ce, ci); ++w) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cell_kernel(ce, ci), 32 * w, per * w) != cudaSuccess)
            continue;
        if (occ * w >= best_warps) { best_warps = occ * w; best = w; }
    }
    return best;
}

// warps per CTA of the tier-0 cell launch: shared memory, grid of resident CTAs
pic_status set_wpc(pic_ctx *c, int wpc)
{
    c->wpc = wpc;
    c->smem_main = warp_mem_bytes(c->cap_ce, c->cap_ci) * wpc;
    pic_status r = cell_smem_attr(c);
    if (r != PIC_OK) return r;
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cell_kernel(c->cap_ce, c->cap_ci), wpc * 32, c->smem_main));
    c->grid_main = cell_grid(c, occ, wpc, c->cap_ce, c->cap_ci);
    return PIC_OK;
}

// smallest power-of-two capacity (>= lo) that holds `share` of the non-empty
// cells of a histogram (bins of bit length)
int cap_for_share(const int *hist, double share, int lo)
{
    long long tot = 0;
    for (int b = 1; b < NHIST; ++b) tot += hist[b];
    if (tot == 0) return lo;
    long long acc = 0;
    for (int b = 1; b < NHIST; ++b) {
        acc += hist[b];
        if (acc >= share * tot) return std::max(lo, 1 << b);   // bin b holds n < 2^b
    }
    return std::max(lo, 1 << (NHIST - 1));
}

// v rounded up to a multiple of q, within [lo, hi]
int round_cap(int v, int q, int lo, int hi) { return std::min(hi, std::max(lo, (v + q - 1) / q * q)); }

// Staging sizes of the cell tiers from the last sort's cell populations.
// Tier 0 holds 75 % of the cells of each species (powers of two, at least
// 64 electrons / 32 ions).  The larger cells go up a chain of tiers sized
// for the largest cell x 1.25 (the cells grow between two re-sizings):
// tier 1 up to 1024 electrons / 256 ions (multiples of 128 / 32), tier 2
// above that up to the large-cell pass's 2048 / 512 (multiples of 256 /
// 64); each tier launched only when the one below cannot hold the largest
// cells.  A staging just large enough for its cells keeps the most warps
// resident on the SM, which the large cells' staging limits.  Warps per
// CTA of tier 0 from the autotuner's choice for its sizes, else the most
// that stay resident.
pic_status configure_cell_launch(pic_ctx *c, const int *hist_e, const int *hist_i, int max_e, int max_i)
{
    // the largest cells x 1.25, kept well inside int (the tiers stop at 2048)
    const int want_e = (int)std::min(max_e * 1.25 + 1.0, (double)(1 << 30));
    const int want_i = (int)std::min(max_i * 1.25 + 1.0, (double)(1 << 30));
    int ce = std::min(cap_for_share(hist_e, 0.75, 64), 1024);
    int ci = std::min(cap_for_share(hist_i, 0.75, 32), 256);
    ce = std::min(ce, std::min(next_pow2(std::max(64, want_e)), 1024));
    ci = std::min(ci, std::min(next_pow2(std::max(32, want_i)), 256));
    c->cap_ce = ce; c->cap_ci = ci; c->cap_new = 3 * ci;
    c->t1_ce = c->t1_ci = c->t2_ce = c->t2_ci = 0;
    c->smem_t1 = c->smem_t2 = 0;
    if (want_e > ce || want_i > ci) {
        c->t1_ce = round_cap(want_e, 128, ce, 1024);
        c->t1_ci = round_cap(want_i, 32, ci, 256);
        c->t1_wpc = best_wpc(c, c->t1_ce, c->t1_ci);
        c->smem_t1 = warp_mem_bytes(c->t1_ce, c->t1_ci) * c->t1_wpc;
        if (want_e > c->t1_ce || want_i > c->t1_ci) {
            c->t2_ce = round_cap(want_e, 256, c->t1_ce, BIG_CE);
            c->t2_ci = round_cap(want_i, 64, c->t1_ci, BIG_CI);
            c->t2_wpc = best_wpc(c, c->t2_ce, c->t2_ci);
            c->smem_t2 = warp_mem_bytes(c->t2_ce, c->t2_ci) * c->t2_wpc;
        }
    }
    int wpc = best_wpc(c, ce, ci);
    for (const auto &t : c->tuned)
        if (t.ce == ce && t.ci == ci && t.done) wpc = t.wpc;
    pic_status r = set_wpc(c, wpc);
    if (r != PIC_OK) return r;
    int occ = 0;
    if (c->t1_ce) {
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cell_kernel(c->t1_ce, c->t1_ci), c->t1_wpc * 32,
                                                         c->smem_t1));
        c->grid_t1 = cell_grid(c, occ, c->t1_wpc, c->t1_ce, c->t1_ci);
    }
    if (c->t2_ce) {
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cell_kernel(c->t2_ce, c->t2_ci), c->t2_wpc * 32,
                                                         c->smem_t2));
        c->grid_t2 = cell_grid(c, occ, c->t2_wpc, c->t2_ce, c->t2_ci);
    }
    return PIC_OK;
}

// arguments of one cell-kernel launch: tier 0 (all cells), tiers 1 and 2
// (the cells the tier below could not stage) or the large-cell pass (the
// rest).  The overflow lists alternate: tier 0 writes list 1, tier 1 reads
// it and writes list 2, tier 2 reads list 2 and writes list 1 again (tier 1
// has finished reading it), the large-cell pass reads the last one.
enum CellTier { TIER0, TIER1, TIER2, TIER_BIG };

CellArgs cell_args(pic_ctx *c, CellTier tier)
{
    CellArgs a{};
    a.e0 = c->eA0; a.e1 = c->eA1; a.ekey = c->ekey; a.cs_e = c->csE[c->cur];
    a.i0 = c->iA0; a.i1 = c->iA1; a.ikey = c->ikey; a.cs_i = c->csI[c->cur];
    a.cnt_e = c->cnt_e; a.cnt_i = c->cnt_i;
    a.append = c->counters + CNT_APPEND;
    a.cap_e = c->cap_e;
    a.slab_app = c->slab_app; a.slab_err = c->slab_err;
    a.ncell = c->ncell;
    a.cell_slab = c->cell_slab;
    a.slabs = c->d_slab;
    a.steps = c->d_steps;
    a.tally = c->d_tally;
    a.photons = c->photons;
    a.fldE = c->E[c->ecur];
    a.fldB = c->B;
    a.npts = c->npts;
    a.J = c->J;
    a.tab = c->d_tab;
    a.eos = c->d_eos;
    a.err = c->counters + CNT_ERR;
    a.nw = c->nw;
    a.gw = c->gw;
    if (tier == TIER0) {
        a.work = c->counters + CNT_WORK;
        a.list = nullptr; a.n_list = nullptr;
        a.ovf_list = c->ovf_list; a.ovf_count = c->counters + CNT_OVF;
        a.cap_ce = c->cap_ce; a.cap_ci = c->cap_ci; a.cap_new = c->cap_new;
    } else if (tier == TIER1) {
        a.work = c->counters + CNT_WORK_T1;
        a.list = c->ovf_list; a.n_list = c->counters + CNT_OVF;
        a.ovf_list = c->ovf_list2; a.ovf_count = c->counters + CNT_OVF2;
        a.cap_ce = c->t1_ce; a.cap_ci = c->t1_ci; a.cap_new = 3 * c->t1_ci;
    } else if (tier == TIER2) {
        a.work = c->counters + CNT_WORK_T2;
        a.list = c->ovf_list2; a.n_list = c->counters + CNT_OVF2;
        a.ovf_list = c->ovf_list; a.ovf_count = c->counters + CNT_OVF3;
        a.cap_ce = c->t2_ce; a.cap_ci = c->t2_ci; a.cap_new = 3 * c->t2_ci;
    } else {
        a.work = c->counters + CNT_WORK_BIG;
        if (c->t2_ce) { a.list = c->ovf_list; a.n_list = c->counters + CNT_OVF3; }
        else if (c->t1_ce) { a.list = c->ovf_list2; a.n_list = c->counters + CNT_OVF2; }
        else { a.list = c->ovf_list; a.n_list = c->counters + CNT_OVF; }
        a.ovf_list = nullptr; a.ovf_count = nullptr;
        a.cap_ce = BIG_CE; a.cap_ci = BIG_CI; a.cap_new = 3 * BIG_CI;
    }
    return a;
}

pic_status run_scan(pic_ctx *c, int species_mask, int dst)
{
    ScanArgs s{};
    int k = 0;
    if (species_mask & 1) {
        s.cnt[k] = c->cnt_e; s.cs[k] = c->csE[dst]; s.bsum[k] = c->bsum_e;
        s.maxc[k] = c->counters + CNT_MAXE; s.hist[k] = c->counters + CNT_HIST_E; ++k;
    }
    if (species_mask & 2) {
        s.cnt[k] = c->cnt_i; s.cs[k] = c->csI[dst]; s.bsum[k] = c->bsum_i;
        s.maxc[k] = c->counters + CNT_MAXI; s.hist[k] = c->counters + CNT_HIST_I; ++k;
    }
    for (int q = 0; q < k; ++q) {
        CK(cudaMemsetAsync(s.maxc[q], 0, sizeof(int), c->stream));
        CK(cudaMemsetAsync(s.hist[q], 0, sizeof(int) * NHIST, c->stream));
    }
    s.n = c->ncell;
    s.nblk = c->nblk;
    dim3 g1(c->nblk, k);
    k_scan_reduce<<<g1, SCAN_T, 0, c->stream>>>(s);
    k_scan_blocks<<<dim3(1, k), SCAN_T, 0, c->stream>>>(s);
    k_scan_final<<<g1, SCAN_T, 0, c->stream>>>(s);
    c->launches += 3;
    CK(cudaGetLastError());
    return PIC_OK;
}

cudaEvent_t *timing_slot(pic_ctx *c)
{
    if (!c->timing) return nullptr;
    if (c->ev_used + NEV > c->ev.size()) {
        for (int k = 0; k < NEV; ++k) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            c->ev.push_back(e);
        }
    }
    cudaEvent_t *p = c->ev.data() + c->ev_used;
    c->ev_used += NEV;
    return p;
}

// does any active slab have this process switched on
bool any_active(const pic_ctx *c, unsigned flag, bool need_pulse)
{
    for (int k = 0; k < c->nslot; ++k) {
        const SlabDev &S = c->slabs[k];
        if (S.active && (S.flags & flag) && (!need_pulse || S.nb > 0)) return true;
    }
    return false;
}

// everything a step's launch sequence depends on besides device memory
pic_ctx::StepShape step_shape(const pic_ctx *c)
{
    pic_ctx::StepShape k{};
    k.eA0 = c->eA0; k.iA0 = c->iA0; k.cur = c->cur; k.ecur = c->ecur;
    k.grid_main = c->grid_main; k.wpc = c->wpc; k.smem_main = c->smem_main;
    k.cap_ce = c->cap_ce; k.cap_ci = c->cap_ci; k.cap_new = c->cap_new;
    k.t1_ce = c->t1_ce; k.t1_ci = c->t1_ci; k.t1_wpc = c->t1_wpc; k.grid_t1 = c->grid_t1;
    k.t2_ce = c->t2_ce; k.t2_ci = c->t2_ci; k.t2_wpc = c->t2_wpc; k.grid_t2 = c->grid_t2;
    k.rt = c->slabs[0].rt != 0;
    k.march = !k.rt && any_active(c, PIC_F_PHOTO, true);
    k.field = any_active(c, PIC_F_FIELD, false);
    k.nsub = 1;
    for (int q = 0; q < c->nslot; ++q)
        if (c->slabs[q].active && (c->slabs[q].flags & PIC_F_FIELD)) k.nsub = std::max(k.nsub, c->slabs[q].nsub);
    return k;
}

bool same_shape(const pic_ctx::StepShape &a, const pic_ctx::StepShape &b)
{
    return a.eA0 == b.eA0 && a.iA0 == b.iA0 && a.cur == b.cur && a.ecur == b.ecur && a.grid_main == b.grid_main &&
           a.wpc == b.wpc && a.smem_main == b.smem_main && a.cap_ce == b.cap_ce && a.cap_ci == b.cap_ci &&
           a.cap_new == b.cap_new && a.march == b.march && a.field == b.field && a.nsub == b.nsub && a.rt == b.rt &&
           a.t1_ce == b.t1_ce && a.t1_ci == b.t1_ci && a.t1_wpc == b.t1_wpc && a.grid_t1 == b.grid_t1 &&
           a.t2_ce == b.t2_ce && a.t2_ci == b.t2_ci && a.t2_wpc == b.t2_wpc && a.grid_t2 == b.grid_t2;
}

// NVTX ranges around the launches of a step (header-only NVTX 3: nothing
// happens unless a profiler is attached): the step, then one nested range
// per phase; inside a graph capture they mark the capture
struct NvRanges {
    bool open = false;
    explicit NvRanges(const char *name) { nvtxRangePushA(name); }
    void phase(const char *name)
    {
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
    }
    ~NvRanges()
    {
        if (open) nvtxRangePop();
        nvtxRangePop();
    }
};

pic_status launch_step(pic_ctx *c)
{
    NvRanges nv("pic step");
    cudaStream_t st = c->stream;
    const pic_ctx::StepShape shape = step_shape(c);
    cudaEvent_t *ev = timing_slot(c);
    if (ev) CK(cudaEventRecord(ev[0], st));
    CK(cudaMemsetAsync(c->cnt_e, 0, sizeof(int) * 4 * (size_t)c->ncell, st));   // cnt_e cnt_i fill_e fill_i
    CK(cudaMemsetAsync(c->counters, 0, sizeof(int) * CNT_STEP_ZERO, st));          // append, work counters, lists
    CK(cudaMemsetAsync(c->J, 0, sizeof(unsigned long long) * 3 * (size_t)c->npts, st));
    if (shape.rt) {
        nv.phase("radiation transport");
        // radiation transport (single-slab contexts): the kernels return at
        // once on steps that are not rad steps
        const SlabDev &S = c->slabs[0];
        RtArgs ra{c->d_slab, c->d_steps, c->photons, c->d_tally};
        const int nrc = S.rt_nrx * S.rt_nry;
        k_rt_cells<<<(nrc + 127) / 128, 128, 0, st>>>(ra);
        const size_t smx = 3 * sizeof(double) * (RT_GHOST + S.rt_nrx);
        k_rt_sweep<<<S.rt_nord * S.nb * S.rt_nry, RT_THREADS, smx, st>>>(ra, 0);
        c->launches += 2;
        if (S.ny > 1) {
            const size_t smy = 3 * sizeof(double) * (RT_GHOST + S.rt_nry);
            k_rt_sweep<<<S.rt_nord * S.nb * S.rt_nrx, RT_THREADS, smy, st>>>(ra, 1);
            ++c->launches;
        }
        k_rt_publish<<<std::min((S.ncell + 255) / 256, c->nsm * 8), 256, 0, st>>>(ra);
        ++c->launches;
    } else if (shape.march) {
        nv.phase("photon march");
        MarchArgs m{c->d_slab, c->d_steps, c->row_slab, c->row_idx, c->photons, c->d_tally};
        k_march<<<c->nrows, 256, (size_t)c->max_row_nx * 8, st>>>(m);
        ++c->launches;
    }
    if (ev) CK(cudaEventRecord(ev[1], st));
    if (c->cell_ev_on) CK(cudaEventRecord(c->cell_ev[0], st));
    nv.phase("collisions and atomic processes");
    CellArgs a0 = cell_args(c, TIER0);
    cell_kernel(c->cap_ce, c->cap_ci)<<<c->grid_main, c->wpc * 32, c->smem_main, st>>>(a0);
    if (c->t1_ce) {
        CellArgs a1 = cell_args(c, TIER1);
        cell_kernel(c->t1_ce, c->t1_ci)<<<c->grid_t1, c->t1_wpc * 32, c->smem_t1, st>>>(a1);
        ++c->launches;
    }
    if (c->t2_ce) {
        CellArgs a2 = cell_args(c, TIER2);
        cell_kernel(c->t2_ce, c->t2_ci)<<<c->grid_t2, c->t2_wpc * 32, c->smem_t2, st>>>(a2);
        ++c->launches;
    }
    CellArgs ab = cell_args(c, TIER_BIG);
    cell_kernel(BIG_CE, BIG_CI)<<<c->grid_big, 32, c->smem_big, st>>>(ab);
    c->launches += 2;
    if (c->cell_ev_on) CK(cudaEventRecord(c->cell_ev[1], st));
    CK(cudaGetLastError());
    if (ev) CK(cudaEventRecord(ev[2], st));
    nv.phase("push and deposit");
    PushArgs pa{};
    pa.e0 = c->eA0; pa.e1 = c->eA1; pa.ekey = c->ekey; pa.cs_e = c->csE[c->cur];
    pa.i0 = c->iA0; pa.i1 = c->iA1; pa.ikey = c->ikey; pa.cs_i = c->csI[c->cur];
    pa.cnt_e = c->cnt_e; pa.cnt_i = c->cnt_i; pa.append = c->counters + CNT_APPEND; pa.cap_e = c->cap_e;
    pa.ncell = c->ncell; pa.cell_slab = c->cell_slab; pa.slabs = c->d_slab; pa.tally = c->d_tally;
    pa.fldE = c->E[c->ecur]; pa.fldB = c->B; pa.npts = c->npts; pa.J = c->J;
    pa.err = c->counters + CNT_ERR; pa.work = c->counters + CNT_WORK_PUSH;
    k_push<<<c->grid_push, 32 * PUSH_WARPS, 0, st>>>(pa);
    k_push_new<<<c->nsm * 2, 256, 0, st>>>(pa);
    c->launches += 2;
    CK(cudaGetLastError());
    if (ev) CK(cudaEventRecord(ev[3], st));
    const int nxt = c->cur ^ 1;
    nv.phase("counting sort");
    pic_status r = run_scan(c, 3, nxt);
    if (r != PIC_OK) return r;
    int sgrid = c->nsm * 8;
    ScatterArgs se{c->eA0, c->eA1, c->ekey, c->csE[c->cur] + c->ncell, c->counters + CNT_APPEND,
                   c->csE[nxt], c->fill_e, c->eB0, c->eB1, c->cap_e};
    k_scatter<<<sgrid, 256, 0, st>>>(se);
    ScatterArgs si{c->iA0, c->iA1, c->ikey, c->csI[c->cur] + c->ncell, nullptr, c->csI[nxt], c->fill_i, c->iB0, c->iB1,
                   c->cap_i};
    k_scatter<<<sgrid, 256, 0, st>>>(si);
    c->launches += 2;
    if (ev) CK(cudaEventRecord(ev[4], st));
    if (shape.field) {
        nv.phase("fields");
        const int nsub = shape.nsub;
        FieldArgs f{};
        f.slabs = c->d_slab; f.pt_slab = c->pt_slab; f.npts = c->npts; f.B = c->B; f.J = c->J;
        int fg = std::min((c->npts + 255) / 256, c->nsm * 16);
        for (int sub = 0; sub < nsub; ++sub) {
            f.sub = sub;
            f.Ein = c->E[c->ecur]; f.Eout = c->E[c->ecur ^ 1];
            k_b_half<<<fg, 256, 0, st>>>(f);
            k_e_full<<<fg, 256, 0, st>>>(f);
            c->ecur ^= 1;
            f.Ein = c->E[c->ecur];
            k_b_half<<<fg, 256, 0, st>>>(f);
            c->launches += 3;
        }
    }
    k_advance<<<(c->nslot + 127) / 128, 128, 0, st>>>(c->d_steps, c->d_slab, c->nslot, c->slab_app, c->slab_err);
    ++c->launches;
    CK(cudaGetLastError());
    if (ev) CK(cudaEventRecord(ev[5], st));
    std::swap(c->eA0, c->eB0); std::swap(c->eA1, c->eB1);
    std::swap(c->iA0, c->iB0); std::swap(c->iA1, c->iB1);
    c->cur = nxt;
    return PIC_OK;
}

pic_status read_device_error(pic_ctx *c)
{
    int e = 0;
    CK(cudaMemcpyAsync(&e, c->counters + CNT_ERR, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (e & ERR_CELL_OVERFLOW) return fail(c, PIC_ERR_CAPACITY, "a cell holds more particles than the large-cell pass can stage");
    if (e & ERR_CAPACITY) return fail(c, PIC_ERR_CAPACITY, "electron capacity exceeded");
    if (e & ERR_NEW_OVERFLOW) return fail(c, PIC_ERR_CAPACITY, "too many electrons created in one cell");
    if (e & ERR_NUMERIC) return fail(c, PIC_ERR_NUMERIC, "numeric error on device");
    return PIC_OK;
}

bool valid_grid(const pic_grid *g)
{
    using std::isfinite;
    return g && g->nx >= 2 && g->ny >= 1 && g->nx <= 8192 && g->dx_nm > 0 && isfinite(g->dx_nm) &&
           g->dy_nm > 0 && isfinite(g->dy_nm) && g->dt_fs > 0 && isfinite(g->dt_fs) && g->cfl > 0 &&
           isfinite(g->cfl) && (long long)(g->nx + 1) * g->ny <= kMaxCells;
}

// Particle capacities: the electrons a step creates (at most three per ion:
// impact, photo- and Auger ionization) are appended after the held ones and
// every particle index is 32-bit, so cap_e + 3 cap_i must stay below 2^31.
bool caps_fit(long long ce, long long ci) { return ce > 0 && ci > 0 && ce + 3 * ci <= 0x7fffffffLL; }

bool valid_species(const pic_species *s)
{
    using std::isfinite;
    return s && s->w_ion > 0 && isfinite(s->w_ion) && s->m_ion_me > 0 && isfinite(s->m_ion_me) &&
           s->n_ref_cm3 > 0 && isfinite(s->n_ref_cm3) && s->ipd_model >= 0 && s->ipd_model <= 2 &&
           !std::isnan(s->E_bulk_eV) && isfinite(s->coulomb_log);
}

bool valid_pulse(const pic_pulse *p)
{
    using std::isfinite;
    return p && (p->shape == 0 || p->shape == 1) && p->n_bins >= 1 && p->n_bins <= PIC_MAX_BINS &&
           p->hv_eV > 0 && isfinite(p->hv_eV) && p->fwhm_fs >= 0 && isfinite(p->fwhm_fs) &&
           p->bandwidth_eV >= 0 && isfinite(p->bandwidth_eV) && p->I_peak_Wcm2 >= 0 &&
           isfinite(p->I_peak_Wcm2) && isfinite(p->t_peak_fs) && !std::isnan(p->spot_sigma_nm);
}

// description of the slab of slot k, inactive until it is switched on
SlabDev make_slab(const pic_ctx *c, int k, const pic_grid *g, const pic_species *s)
{
    SlabDev S{};
    S.active = 0;
    S.nx = g->nx; S.ny = g->ny;
    S.cell0 = k * c->slot_cells; S.ncell = g->nx * g->ny;
    S.fld_off = k * c->slot_pts;
    S.ph_off = k * c->slot_cells * PIC_MAX_BINS;
    S.nb = 0;
    S.rad_every = g->rad_every; S.flags = s->flags; S.ipd = s->ipd_model; S.shape = 0;
    S.dx = (real)g->dx_nm; S.dy = (real)g->dy_nm; S.dt = (real)g->dt_fs;
    S.w_ion = (real)s->w_ion; S.m_ion = (real)s->m_ion_me; S.E_bulk = (real)s->E_bulk_eV;
    S.coulomb_log = (real)s->coulomb_log;
    S.n_ref = s->n_ref_cm3;
    const double E0 = kMeKg * kCms / (kQe * 1e-15);
    S.kappa_J = kQe * s->n_ref_cm3 * 1e6 * 1e-9 / (kEps0 * E0);
    S.nref_f = (real)S.n_ref;
    S.kappa_f = (real)S.kappa_J;
    // Field speed: c where the step resolves it (c dt within cfl of the Yee
    // limit), else the largest speed it resolves.  With c dt beyond the cell
    // size, fields subcycled at c with the current held fixed are seen by
    // the particles only every dt, and the transverse fields grow without
    // bound once collisions feed them noise; the continuity of the deposited
    // current, hence Gauss's law and the electrostatic fields, does not
    // depend on this speed.  One field update per step.
    double inv = 1.0 / (g->dx_nm * g->dx_nm) + (g->ny > 1 ? 1.0 / (g->dy_nm * g->dy_nm) : 0.0);
    const double cmax = g->cfl / (g->dt_fs * std::sqrt(inv));
    const double cf = kCnmPerFs < cmax ? kCnmPerFs : cmax;
    S.nsub = 1;
    S.cf = (real)cf;
    S.mur = (real)((cf * g->dt_fs - g->dx_nm) / (cf * g->dt_fs + g->dx_nm));
    S.seed = g->seed;
    return S;
}

void set_pulse(const pic_ctx *c, SlabDev &S, const pic_pulse *p)
{
    S.nb = p->n_bins;
    S.shape = p->shape;
    S.I_peak = p->I_peak_Wcm2; S.fwhm = p->fwhm_fs; S.t_peak = p->t_peak_fs; S.spot_sigma = p->spot_sigma_nm;
    S.bin_hw = (real)(0.5 * p->bandwidth_eV / p->n_bins);
    for (int b = 0; b < PIC_MAX_BINS; ++b) {
        double hv = b < p->n_bins ? p->hv_eV + p->bandwidth_eV * ((b + 0.5) / p->n_bins - 0.5) : 0.0;
        S.hv_b[b] = (real)hv;
        for (int q = 0; q < NS; ++q) S.sig_b[q][b] = b < p->n_bins ? (real)sigma_table(c, q, hv) : (real)0;
    }
}

// zero the fields, photons, tallies and step counter of slot k and upload
// its description
pic_status reset_slot(pic_ctx *c, int k)
{
    cudaStream_t st = c->stream;
    const SlabDev &S = c->slabs[k];
    for (int comp = 0; comp < 3; ++comp) {
        size_t o = (size_t)comp * c->npts + S.fld_off;
        CK(cudaMemsetAsync(c->E[0] + o, 0, sizeof(real) * c->slot_pts, st));
        CK(cudaMemsetAsync(c->E[1] + o, 0, sizeof(real) * c->slot_pts, st));
        CK(cudaMemsetAsync(c->B + o, 0, sizeof(real) * c->slot_pts, st));
    }
    CK(cudaMemsetAsync(c->photons + S.ph_off, 0, sizeof(ph2) * (size_t)c->slot_cells * PIC_MAX_BINS, st));
    CK(cudaMemcpyAsync(c->d_slab + k, &S, sizeof(SlabDev), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(c->d_steps + k, 0, sizeof(unsigned), st));
    CK(cudaMemsetAsync(c->slab_app + k, 0, sizeof(int), st));
    CK(cudaMemsetAsync(c->slab_err + k, 0, sizeof(int), st));
    CK(cudaMemsetAsync(c->d_tally + k, 0, sizeof(SlabTally), st));
    CK(cudaStreamSynchronize(st));      // the host copy of S may change after this call
    return PIC_OK;
}

// a context of nslot empty slots
pic_status ctx_create(pic_ctx **out, int nslot, int slot_cells, int slot_pts, int slot_rows, int max_row_nx,
                      int cap_e, int cap_i, const pic_tables *t, void *arena, size_t arena_bytes, void *stream)
{
    if (t->n_hv < 2 || !t->hv_tab || !t->sigma_photo || t->n_T < 1 || t->n_n < 1 || t->n_T > EOS_MAX_T ||
        t->n_n > EOS_MAX_N || !t->eos_T || !t->eos_n || !t->eos_Zbar)
        return PIC_ERR_TABLE;
    if ((long long)nslot * slot_cells > kMaxCells || (long long)nslot * slot_pts > kMaxCells) return PIC_ERR_ARG;
    pic_ctx *c = new pic_ctx();
    c->stream = (cudaStream_t)stream;
    c->nslot = nslot;
    c->slot_cells = slot_cells;
    c->slot_pts = slot_pts;
    c->slot_rows = slot_rows;
    c->ncell = nslot * slot_cells;
    c->npts = nslot * slot_pts;
    c->nrows = nslot * slot_rows;
    c->max_row_nx = max_row_nx;
    c->nblk = (c->ncell + SCAN_TILE - 1) / SCAN_TILE;
    c->cap_e = cap_e;
    c->cap_i = cap_i;
    c->slabs.assign(nslot, SlabDev{});
    c->slot_state.assign(nslot, 0);
    c->grids.assign(nslot, pic_grid{});
    c->hv_tab.assign(t->hv_tab, t->hv_tab + t->n_hv);
    c->sigma.assign(t->sigma_photo, t->sigma_photo + (size_t)NS * t->n_hv);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { pic_status r = cuda_fail(c, e, "device query"); delete c; return r; }

    size_t need = arena_need(c->ncell, c->npts, c->nblk, cap_e, cap_i, nslot, c->nrows);
    if (arena) {
        if (arena_bytes < need) { delete c; return PIC_ERR_OOM; }
        c->arena = (char *)arena;
        c->arena_bytes = arena_bytes;
    } else {
        e = cudaMalloc((void **)&c->arena, need);
        if (e != cudaSuccess) { delete c; return PIC_ERR_OOM; }
        c->own_arena = true;
        c->arena_bytes = need;
    }
    c->eA0 = carve_arena<real4>(c, cap_e); c->eA1 = carve_arena<real4>(c, cap_e);
    c->eB0 = carve_arena<real4>(c, cap_e); c->eB1 = carve_arena<real4>(c, cap_e);
    c->ekey = carve_arena<int>(c, cap_e);
    c->iA0 = carve_arena<real4>(c, cap_i); c->iA1 = carve_arena<real4>(c, cap_i);
    c->iB0 = carve_arena<real4>(c, cap_i); c->iB1 = carve_arena<real4>(c, cap_i);
    c->ikey = carve_arena<int>(c, cap_i);
    for (int k = 0; k < 2; ++k) { c->csE[k] = carve_arena<int>(c, c->ncell + 1); c->csI[k] = carve_arena<int>(c, c->ncell + 1); }
    c->cnt_e = carve_arena<int>(c, 4 * (size_t)c->ncell);
    c->cnt_i = c->cnt_e + c->ncell; c->fill_e = c->cnt_i + c->ncell; c->fill_i = c->fill_e + c->ncell;
    c->bsum_e = carve_arena<int>(c, c->nblk); c->bsum_i = carve_arena<int>(c, c->nblk);
    c->counters = carve_arena<int>(c, NCOUNTERS);
    c->ovf_list = carve_arena<int>(c, c->ncell);
    c->ovf_list2 = carve_arena<int>(c, c->ncell);
    c->cell_slab = carve_arena<int>(c, c->ncell);
    c->d_slab = carve_arena<SlabDev>(c, nslot);
    c->d_steps = carve_arena<unsigned>(c, nslot);
    c->slab_app = carve_arena<int>(c, nslot);
    c->slab_err = carve_arena<int>(c, nslot);
    c->d_tally = carve_arena<SlabTally>(c, nslot);
    c->d_tab = carve_arena<Tables>(c, 1);
    c->d_eos = carve_arena<EosTable>(c, 1);
    c->E[0] = carve_arena<real>(c, 3 * (size_t)c->npts);
    c->E[1] = carve_arena<real>(c, 3 * (size_t)c->npts);
    c->B = carve_arena<real>(c, 3 * (size_t)c->npts);
    c->J = carve_arena<unsigned long long>(c, 3 * (size_t)c->npts);
    c->pt_slab = carve_arena<int>(c, c->npts);
    c->row_slab = carve_arena<int>(c, c->nrows);
    c->row_idx = carve_arena<int>(c, c->nrows);
    c->photons = carve_arena<ph2>(c, (size_t)c->ncell * PIC_MAX_BINS);
    c->nw_entries = nw_scratch_entries(c->ncell);
    c->nw = carve_arena<NewE>(c, c->nw_entries);
    c->gw_words = gw_scratch_words(c->ncell);
    c->gw = carve_arena<unsigned long long>(c, c->gw_words);
    c->diag_buf = carve_arena<double>(c, 4 + NZ + 4096 + 8);
    if (!c->diag_buf) { pic_free(c); return PIC_ERR_OOM; }

    Tables T{};
    for (int q = 0; q < NS; ++q) { T.lotz_a[q] = (real)t->lotz_a[q]; T.lotz_b[q] = (real)t->lotz_b[q]; T.lotz_c[q] = (real)t->lotz_c[q]; }
    for (int z = 0; z < NZ; ++z) {
        for (int q = 0; q < NS; ++q) T.E_bind[z][q] = (real)t->E_bind[z][q];
        for (int k = 0; k < 2; ++k) { T.tauK[z][k] = (real)t->tauK[z][k]; T.omegaK[z][k] = (real)t->omegaK[z][k]; }
        T.E_Ka[z] = (real)t->E_Kalpha[z];
    }
    std::vector<EosTable> eos(1);
    eos[0].n_T = t->n_T; eos[0].n_n = t->n_n;
    for (int k = 0; k < t->n_T; ++k) eos[0].T[k] = (real)t->eos_T[k];
    for (int k = 0; k < t->n_n; ++k) eos[0].n[k] = (real)t->eos_n[k];
    for (int a = 0; a < t->n_n; ++a)
        for (int b = 0; b < t->n_T; ++b) eos[0].Z[a * t->n_T + b] = (real)t->eos_Zbar[(size_t)a * t->n_T + b];
    std::vector<int> cs(c->ncell), ps(c->npts), rs(c->nrows), ri(c->nrows);
    for (int g = 0; g < c->ncell; ++g) cs[g] = g / slot_cells;
    for (int p = 0; p < c->npts; ++p) ps[p] = p / slot_pts;
    for (int q = 0; q < c->nrows; ++q) { rs[q] = q / slot_rows; ri[q] = q % slot_rows; }
    std::vector<SlabDev> idle(nslot, SlabDev{});
    cudaStream_t st = c->stream;
    do {
        if ((e = cudaMemcpyAsync(c->d_tab, &T, sizeof(Tables), cudaMemcpyHostToDevice, st))) break;
        if ((e = cudaMemcpyAsync(c->d_eos, eos.data(), sizeof(EosTable), cudaMemcpyHostToDevice, st))) break;
        if ((e = cudaMemcpyAsync(c->d_slab, idle.data(), sizeof(SlabDev) * nslot, cudaMemcpyHostToDevice, st))) break;
        if ((e = cudaMemsetAsync(c->d_steps, 0, sizeof(unsigned) * nslot, st))) break;
        if ((e = cudaMemsetAsync(c->d_tally, 0, sizeof(SlabTally) * nslot, st))) break;
        if ((e = cudaMemcpyAsync(c->cell_slab, cs.data(), sizeof(int) * c->ncell, cudaMemcpyHostToDevice, st))) break;
        if ((e = cudaMemcpyAsync(c->pt_slab, ps.data(), sizeof(int) * c->npts, cudaMemcpyHostToDevice, st))) break;
        if ((e = cudaMemcpyAsync(c->row_slab, rs.data(), sizeof(int) * c->nrows, cudaMemcpyHostToDevice, st))) break;
        if ((e = cudaMemcpyAsync(c->row_idx, ri.data(), sizeof(int) * c->nrows, cudaMemcpyHostToDevice, st))) break;
        if ((e = cudaMemsetAsync(c->E[0], 0, sizeof(real) * 3 * (size_t)c->npts, st))) break;
        if ((e = cudaMemsetAsync(c->E[1], 0, sizeof(real) * 3 * (size_t)c->npts, st))) break;
        if ((e = cudaMemsetAsync(c->B, 0, sizeof(real) * 3 * (size_t)c->npts, st))) break;
        if ((e = cudaMemsetAsync(c->J, 0, sizeof(unsigned long long) * 3 * (size_t)c->npts, st))) break;
        if ((e = cudaMemsetAsync(c->photons, 0, sizeof(ph2) * (size_t)c->ncell * PIC_MAX_BINS, st))) break;
        if ((e = cudaMemsetAsync(c->counters, 0, sizeof(int) * NCOUNTERS, st))) break;
        if ((e = cudaMemsetAsync(c->csE[0], 0, sizeof(int) * (c->ncell + 1), st))) break;
        if ((e = cudaMemsetAsync(c->csE[1], 0, sizeof(int) * (c->ncell + 1), st))) break;
        if ((e = cudaMemsetAsync(c->csI[0], 0, sizeof(int) * (c->ncell + 1), st))) break;
        if ((e = cudaMemsetAsync(c->csI[1], 0, sizeof(int) * (c->ncell + 1), st))) break;
        e = cudaStreamSynchronize(st);    // the host tables above go out of scope
    } while (0);
    pic_status rc = PIC_OK;
    if (e != cudaSuccess) { rc = cuda_fail(c, e, "init copies"); pic_free(c); return rc; }
    c->smem_big = warp_mem_bytes(BIG_CE, BIG_CI);
    c->grid_big = cell_grid(c, 1, 1, BIG_CE, BIG_CI);
    e = cudaFuncSetAttribute(k_march, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8);
    if (e != cudaSuccess) { rc = cuda_fail(c, e, "march attribute"); pic_free(c); return rc; }
    {
        int he[NHIST] = {}, hi[NHIST] = {};
        if ((rc = configure_cell_launch(c, he, hi, 100, 25)) != PIC_OK) { pic_free(c); return rc; }
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_push, 32 * PUSH_WARPS, 0);
    if (e != cudaSuccess) { rc = cuda_fail(c, e, "push occupancy"); pic_free(c); return rc; }
    c->grid_push = std::max(1, occ) * c->nsm;
    *out = c;
    return PIC_OK;
}

// Host records of one slab from positions in cell units of its grid:
// (xi, eta, ux, uy), (uz, w | zfrac, id, state) and the global cell key.
pic_status build_records(pic_ctx *c, int slot, const pic_grid *g, bool electrons, int64_t n, const double *X,
                         const double *Y, const float *u, const float *w_or_zf, const uint64_t *eid,
                         const int32_t *Z, const int32_t *nK, const uint32_t *iid, std::vector<real4> &p0,
                         std::vector<real4> &p1, std::vector<int> &key)
{
    p0.resize(n); p1.resize(n); key.resize(n);
    const int cell0 = slot * c->slot_cells;
    // 0 ok, 1 position outside the slab, 2 ion state out of range
    auto fill = [&](int64_t lo, int64_t hi) -> int {
        for (int64_t k = lo; k < hi; ++k) {
            double fx = std::floor(X[k]), fy = g->ny > 1 ? std::floor(Y[k]) : 0.0;
            if (!(fx >= 0 && fx < g->nx && fy >= 0 && fy < g->ny)) return 1;
            real xi = (real)(X[k] - fx), eta = g->ny > 1 ? (real)(Y[k] - fy) : (real)Y[k];
            if (xi >= (real)1) xi = kBelow1;
            if (g->ny > 1 && eta >= (real)1) eta = kBelow1;
            key[k] = cell0 + (int)fy * g->nx + (int)fx;
            p0[k] = make_real4(xi, eta, u[3 * k], u[3 * k + 1]);
            if (electrons) {
                p1[k] = rec_e1(u[3 * k + 2], w_or_zf[k], eid[k]);
            } else {
                // charge 0..13, K vacancies at most the K electrons of the
                // lowest configuration of the bound electrons, fraction in [0, 1)
                if (Z[k] < 0 || Z[k] > ZNUC || nK[k] < 0 || nK[k] > std::min(2, ZNUC - Z[k]) ||
                    !(w_or_zf[k] >= 0.0f && w_or_zf[k] < 1.0f))
                    return 2;
                int stv = Z[k] | (nK[k] << 8);
                p1[k] = rec_i1(u[3 * k + 2], w_or_zf[k], iid[k], stv);
            }
        }
        return 0;
    };
    // large loads are split over host threads (disjoint ranges, same records)
    const int64_t per = 1 << 20;
    const int nt = (int)std::min<int64_t>(std::max(1u, std::thread::hardware_concurrency()), (n + per - 1) / per);
    std::vector<int> rc(std::max(nt, 1), 0);
    if (nt <= 1) {
        rc[0] = fill(0, n);
    } else {
        std::vector<std::thread> th;
        for (int t = 0; t < nt; ++t)
            th.emplace_back([&, t] { rc[t] = fill(n * t / nt, n * (t + 1) / nt); });
        for (auto &x : th) x.join();
    }
    for (int r : rc) {
        if (r == 1) return fail(c, PIC_ERR_ARG, "particle position outside the slab");
        if (r == 2) return fail(c, PIC_ERR_ARG, "ion state out of range");
    }
    return PIC_OK;
}

// replace all particles of one species by host records (single-slab load):
// records into the B buffers, count, scan, scatter into A
// the n records of one species on the unsorted side (B buffers, keys) into
// cell order on the sorted side
pic_status sort_species(pic_ctx *c, bool electrons, int64_t n)
{
    cudaStream_t st = c->stream;
    real4 *s0 = electrons ? c->eB0 : c->iB0, *s1 = electrons ? c->eB1 : c->iB1;
    real4 *d0 = electrons ? c->eA0 : c->iA0, *d1 = electrons ? c->eA1 : c->iA1;
    int *k = electrons ? c->ekey : c->ikey;
    int *cnt = electrons ? c->cnt_e : c->cnt_i, *fill = electrons ? c->fill_e : c->fill_i;
    int nn = (int)n;
    CK(cudaMemcpyAsync(c->counters + CNT_NLOAD, &nn, sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(cnt, 0, sizeof(int) * c->ncell, st));
    CK(cudaMemsetAsync(fill, 0, sizeof(int) * c->ncell, st));
    k_count<<<c->nsm * 4, 256, 0, st>>>(k, c->counters + CNT_NLOAD, cnt);
    pic_status r = run_scan(c, electrons ? 1 : 2, c->cur);
    if (r != PIC_OK) return r;
    ScatterArgs sa{s0, s1, k, c->counters + CNT_NLOAD, nullptr, electrons ? c->csE[c->cur] : c->csI[c->cur], fill, d0, d1,
                   electrons ? c->cap_e : c->cap_i};
    k_scatter<<<c->nsm * 4, 256, 0, st>>>(sa);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return PIC_OK;
}

pic_status load_species(pic_ctx *c, bool electrons, int64_t n, const std::vector<real4> &p0,
                        const std::vector<real4> &p1, const std::vector<int> &key)
{
    cudaStream_t st = c->stream;
    if (n > 0) {
        CK(cudaMemcpyAsync(electrons ? c->eB0 : c->iB0, p0.data(), sizeof(real4) * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(electrons ? c->eB1 : c->iB1, p1.data(), sizeof(real4) * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(electrons ? c->ekey : c->ikey, key.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    }
    return sort_species(c, electrons, n);
}

// Admission: host records are appended behind the sorted particles of each
// species, every sorted particle is keyed by its own cell (-1 when its slab
// is inactive), and one count / scan / scatter re-sorts all of them.
pic_status resort_with(pic_ctx *c, const std::vector<real4> &e0, const std::vector<real4> &e1,
                       const std::vector<int> &ek, const std::vector<real4> &i0, const std::vector<real4> &i1,
                       const std::vector<int> &ik)
{
    cudaStream_t st = c->stream;
    int ns[2] = {0, 0};
    CK(cudaMemcpyAsync(&ns[0], c->csE[c->cur] + c->ncell, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&ns[1], c->csI[c->cur] + c->ncell, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int nxt = c->cur ^ 1;
    for (int sp = 0; sp < 2; ++sp) {
        const bool el = sp == 0;
        const std::vector<real4> &h0 = el ? e0 : i0, &h1 = el ? e1 : i1;
        const std::vector<int> &hk = el ? ek : ik;
        const long long n0 = ns[sp], nadd = (long long)hk.size();
        if (n0 + nadd > (el ? c->cap_e : c->cap_i))
            return fail(c, PIC_ERR_CAPACITY, "particle capacity exceeded by admission");
        real4 *A0 = el ? c->eA0 : c->iA0, *A1 = el ? c->eA1 : c->iA1, *B0 = el ? c->eB0 : c->iB0, *B1 = el ? c->eB1 : c->iB1;
        int *key = el ? c->ekey : c->ikey, *cnt = el ? c->cnt_e : c->cnt_i, *fill = el ? c->fill_e : c->fill_i;
        const int *cs = el ? c->csE[c->cur] : c->csI[c->cur];
        k_cell_keys<<<c->nsm * 4, 256, 0, st>>>(cs, c->ncell, c->cell_slab, c->d_slab, key);
        if (nadd) {
            CK(cudaMemcpyAsync(A0 + n0, h0.data(), sizeof(real4) * nadd, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(A1 + n0, h1.data(), sizeof(real4) * nadd, cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(key + n0, hk.data(), sizeof(int) * nadd, cudaMemcpyHostToDevice, st));
        }
        const int tot = (int)(n0 + nadd);
        CK(cudaMemcpyAsync(c->counters + CNT_NLOAD, &tot, sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(cnt, 0, sizeof(int) * c->ncell, st));
        CK(cudaMemsetAsync(fill, 0, sizeof(int) * c->ncell, st));
        k_count<<<c->nsm * 4, 256, 0, st>>>(key, c->counters + CNT_NLOAD, cnt);
        pic_status r = run_scan(c, el ? 1 : 2, nxt);
        if (r != PIC_OK) return r;
        ScatterArgs sa{A0, A1, key, c->counters + CNT_NLOAD, nullptr, el ? c->csE[nxt] : c->csI[nxt], fill, B0, B1,
                       el ? c->cap_e : c->cap_i};
        k_scatter<<<c->nsm * 4, 256, 0, st>>>(sa);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));     // tot is read by the device; the next species reuses it
    }
    std::swap(c->eA0, c->eB0); std::swap(c->eA1, c->eB1);
    std::swap(c->iA0, c->iB0); std::swap(c->iA1, c->iB1);
    c->cur = nxt;
    return PIC_OK;
}

// drop the particles of retired slabs now (one re-sort) and free their slots
pic_status compact(pic_ctx *c)
{
    const std::vector<real4> no4;
    const std::vector<int> noi;
    pic_status r = resort_with(c, no4, no4, noi, no4, no4, noi);
    if (r != PIC_OK) return r;
    for (int k = 0; k < c->nslot; ++k)
        if (c->slot_state[k] == 2) c->slot_state[k] = 0;
    return PIC_OK;
}

bool any_retired(const pic_ctx *c)
{
    for (int k = 0; k < c->nslot; ++k)
        if (c->slot_state[k] == 2) return true;
    return false;
}

pic_status apply_pending(pic_ctx *c)
{
    if (c->pending.empty()) return PIC_OK;
    // the new records are appended behind every sorted particle, retired
    // ones included: drop those first when the buffers would overflow
    if (any_retired(c)) {
        size_t add_e = 0, add_i = 0;
        for (auto &p : c->pending) { add_e += p.ek.size(); add_i += p.ik.size(); }
        int ns[2] = {0, 0};
        CK(cudaMemcpyAsync(&ns[0], c->csE[c->cur] + c->ncell, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(&ns[1], c->csI[c->cur] + c->ncell, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (ns[0] + add_e > (size_t)c->cap_e || ns[1] + add_i > (size_t)c->cap_i) {
            pic_status r = compact(c);
            if (r != PIC_OK) return r;
        }
    }
    std::vector<real4> e0, e1, i0, i1;
    std::vector<int> ek, ik;
    for (auto &p : c->pending) {
        c->slabs[p.slot].active = 1;
        pic_status r = reset_slot(c, p.slot);
        if (r != PIC_OK) return r;
        e0.insert(e0.end(), p.e0.begin(), p.e0.end()); e1.insert(e1.end(), p.e1.begin(), p.e1.end());
        ek.insert(ek.end(), p.ek.begin(), p.ek.end());
        i0.insert(i0.end(), p.i0.begin(), p.i0.end()); i1.insert(i1.end(), p.i1.begin(), p.i1.end());
        ik.insert(ik.end(), p.ik.begin(), p.ik.end());
    }
    c->pending.clear();
    return resort_with(c, e0, e1, ek, i0, i1, ik);
}

// particles of one slot back on the host with the slot's cell starts
pic_status fetch_slot(pic_ctx *c, int slot, bool electrons, std::vector<real4> &p0, std::vector<real4> &p1,
                      std::vector<int> &cs)
{
    cudaStream_t st = c->stream;
    cs.resize(c->slot_cells + 1);
    const int *src = (electrons ? c->csE[c->cur] : c->csI[c->cur]) + (size_t)slot * c->slot_cells;
    CK(cudaMemcpyAsync(cs.data(), src, sizeof(int) * (c->slot_cells + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int lo = cs[0], n = cs[c->slot_cells] - lo;
    p0.resize(n); p1.resize(n);
    if (n) {
        CK(cudaMemcpyAsync(p0.data(), (electrons ? c->eA0 : c->iA0) + lo, sizeof(real4) * n, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(p1.data(), (electrons ? c->eA1 : c->iA1) + lo, sizeof(real4) * n, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    for (auto &v : cs) v -= lo;
    return PIC_OK;
}

pic_status counts_slot(pic_ctx *c, int slot, int64_t *n_e, int64_t *n_i)
{
    int v[4];
    const size_t a = (size_t)slot * c->slot_cells, b = a + c->slot_cells;
    CK(cudaMemcpyAsync(&v[0], c->csE[c->cur] + a, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&v[1], c->csE[c->cur] + b, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&v[2], c->csI[c->cur] + a, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&v[3], c->csI[c->cur] + b, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (n_e) *n_e = v[1] - v[0];
    if (n_i) *n_i = v[3] - v[2];
    return read_device_error(c);
}

// U is float (the ABI's particle arrays) or double (the full-precision read-back)
template <class U>
pic_status get_electrons_slot(pic_ctx *c, int slot, double *X, double *Y, U *u, U *w, uint64_t *id)
{
    std::vector<real4> p0, p1;
    std::vector<int> cs;
    pic_status r = fetch_slot(c, slot, true, p0, p1, cs);
    if (r != PIC_OK) return r;
    const SlabDev &S = c->slabs[slot];
    for (int cell = 0; cell < c->slot_cells; ++cell) {
        const int cx = cell % S.nx, cy = cell / S.nx;
        for (int k = cs[cell]; k < cs[cell + 1]; ++k) {
            X[k] = cx + (double)p0[k].x;
            Y[k] = S.ny > 1 ? cy + (double)p0[k].y : (double)p0[k].y;
            u[3 * k] = (U)p0[k].z; u[3 * k + 1] = (U)p0[k].w; u[3 * k + 2] = (U)p1[k].x;
            w[k] = (U)p1[k].y;
            id[k] = rec_eid(p1[k]);
        }
    }
    return PIC_OK;
}

template <class U>
pic_status get_ions_slot(pic_ctx *c, int slot, double *X, double *Y, U *u, U *zfrac, int32_t *Z,
                         int32_t *nK, uint32_t *id)
{
    std::vector<real4> p0, p1;
    std::vector<int> cs;
    pic_status r = fetch_slot(c, slot, false, p0, p1, cs);
    if (r != PIC_OK) return r;
    const SlabDev &S = c->slabs[slot];
    for (int cell = 0; cell < c->slot_cells; ++cell) {
        const int cx = cell % S.nx, cy = cell / S.nx;
        for (int k = cs[cell]; k < cs[cell + 1]; ++k) {
            X[k] = cx + (double)p0[k].x;
            Y[k] = S.ny > 1 ? cy + (double)p0[k].y : (double)p0[k].y;
            u[3 * k] = (U)p0[k].z; u[3 * k + 1] = (U)p0[k].w; u[3 * k + 2] = (U)p1[k].x;
            zfrac[k] = (U)p1[k].y;
            const int stv = rec_ist(p1[k]);
            id[k] = rec_iid(p1[k]);
            Z[k] = stv & 0xff;
            nK[k] = (stv >> 8) & 0xff;
        }
    }
    return PIC_OK;
}

pic_status diag_slot(pic_ctx *c, int slot, pic_diag *out)
{
    if (!out || out->n_E < 0 || out->n_E > 4096) return PIC_ERR_ARG;
    cudaStream_t st = c->stream;
    const SlabDev &S = c->slabs[slot];
    const int nE = out->n_E > 0 ? out->n_E : 1;
    const int nv = 4 + NZ + nE;
    CK(cudaMemsetAsync(c->diag_buf, 0, sizeof(double) * (nv + 3), st));
    DiagArgs d{};
    const size_t a = (size_t)slot * c->slot_cells, b = a + c->slot_cells;
    d.e0 = c->eA0; d.e1 = c->eA1; d.i0 = c->iA0; d.i1 = c->iA1;
    d.e_lo = c->csE[c->cur] + a; d.e_hi = c->csE[c->cur] + b;
    d.i_lo = c->csI[c->cur] + a; d.i_hi = c->csI[c->cur] + b;
    d.m_ion = S.m_ion; d.out = c->diag_buf; d.n_E = nE; d.E_lo = 0.1;
    d.E_max = out->E_max_eV > 0.1 ? out->E_max_eV : 1e4;
    k_diag<<<c->nsm * 4, 256, sizeof(real) * nv, st>>>(d);
    k_sumsq<<<c->nsm * 2, 256, 0, st>>>(c->E[c->ecur], c->npts, S.fld_off, c->slot_pts, c->diag_buf + nv);
    k_sumsq<<<c->nsm * 2, 256, 0, st>>>(c->B, c->npts, S.fld_off, c->slot_pts, c->diag_buf + nv);
    if (S.nb > 0 && S.rt) {
        k_rt_energy<<<c->nsm * 2, 256, 0, st>>>(c->d_slab + slot, c->photons, c->diag_buf + nv + 1);
    } else if (S.nb > 0) {
        const real *hv = reinterpret_cast<const real *>(reinterpret_cast<const char *>(c->d_slab + slot) +
                                                          offsetof(SlabDev, hv_b));
        k_photon_energy<<<c->nsm * 2, 256, 0, st>>>(c->photons + S.ph_off, S.ncell, S.nb, hv, c->diag_buf + nv + 1);
    }
    CK(cudaGetLastError());
    std::vector<double> h(nv + 3);
    SlabTally tl;
    unsigned step = 0;
    CK(cudaMemcpyAsync(h.data(), c->diag_buf, sizeof(double) * (nv + 3), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&tl, c->d_tally + slot, sizeof(SlabTally), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&step, c->d_steps + slot, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    int64_t ne = 0, ni = 0;
    pic_status r = counts_slot(c, slot, &ne, &ni);     // synchronizes the stream
    if (r != PIC_OK) return r;
    const double We = h[0], Ke = h[1], Ki = h[2], Ni = h[3];
    if (out->csd) for (int z = 0; z < NZ; ++z) out->csd[z] = Ni > 0 ? h[4 + z] / Ni : 0.0;
    double zb = 0.0;
    for (int z = 0; z < NZ; ++z) zb += z * (Ni > 0 ? h[4 + z] / Ni : 0.0);
    if (out->eedf && out->n_E > 0) for (int q = 0; q < out->n_E; ++q) out->eedf[q] = We > 0 ? h[4 + NZ + q] / We : 0.0;
    const double E0 = kMeKg * kCms / (kQe * 1e-15);
    out->t_fs = step * c->grids[slot].dt_fs;
    out->transmission = tl.inc > 0 ? tl.trans / tl.inc : 0.0;
    out->T_e_eV = We > 0 ? (2.0 / 3.0) * Ke / We : 0.0;
    out->n_e_cm3 = S.ncell > 0 ? We * S.n_ref / S.ncell : 0.0;
    out->Zbar = zb;
    out->ke_e = Ke;
    out->ke_i = Ki * S.w_ion;
    out->e_ion = tl.ion;
    out->e_phot = h[nv + 1];
    out->e_inc = tl.inc;
    out->e_trans = tl.trans;
    out->e_ka_esc = tl.ka_esc;
    out->e_esc = tl.esc;
    out->e_field = h[nv] * kEps0 * E0 * E0 / (2.0 * S.n_ref * 1e6 * kQe);
    out->e_back = tl.back;
    out->e_rt_num = tl.rt_num;
    out->e_rt_pend = tl.rt_pend;
    for (int q = 0; q < 16; ++q) out->counts[q] = tl.cnt[q];
    out->n_e = ne;
    out->n_i = ni;
    return read_device_error(c);
}

// Capture two steps into a graph (on a private stream: the context stream
// may be the legacy default stream, which cannot be captured).  The host
// side of the pair (buffer swaps) is undone, so the context is left as it
// was; the graph replays the pair.
pic_status capture_pair(pic_ctx *c, pic_ctx::StepGraph &g)
{
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    real4 *saved[8] = {c->eA0, c->eA1, c->eB0, c->eB1, c->iA0, c->iA1, c->iB0, c->iB1};
    const int cur = c->cur, ecur = c->ecur;
    const int64_t l0 = c->launches;
    const pic_ctx::StepShape key = step_shape(c);
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    cudaGraph_t graph = nullptr;
    pic_status r = PIC_OK;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        r = launch_step(c);
        if (r == PIC_OK) r = launch_step(c);
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
        if (e2 != cudaSuccess && r == PIC_OK) r = cuda_fail(c, e2, "cudaStreamEndCapture");
    } else {
        r = cuda_fail(c, e, "cudaStreamBeginCapture");
    }
    c->stream = user;
    c->eA0 = saved[0]; c->eA1 = saved[1]; c->eB0 = saved[2]; c->eB1 = saved[3];
    c->iA0 = saved[4]; c->iA1 = saved[5]; c->iB0 = saved[6]; c->iB1 = saved[7];
    c->cur = cur; c->ecur = ecur;
    const int64_t nl = c->launches - l0;
    c->launches = l0;
    if (r == PIC_OK) {
        if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (e != cudaSuccess) { g.exec = nullptr; r = cuda_fail(c, e, "cudaGraphInstantiate"); }
        g.key = key;
        g.launches = nl;
    }
    if (graph) cudaGraphDestroy(graph);
    return r;
}

pic_ctx::StepGraph *pair_graph(pic_ctx *c, pic_status &r)
{
    const pic_ctx::StepShape key = step_shape(c);
    for (auto &g : c->graphs)
        if (g.exec && same_shape(g.key, key)) return &g;
    pic_ctx::StepGraph &g = c->graphs[c->graph_next];
    c->graph_next ^= 1;
    r = capture_pair(c, g);
    return r == PIC_OK ? &g : nullptr;
}

// Autotuner: time the cell kernels of real steps with 1, 2, 4 and 8 warps
// per CTA (as many as fit) for the current staging sizes and keep the
// fastest.  The launch shape changes no result (every decision is keyed by
// particle and cell), so the steps it times are steps of the simulation.
// Each shape is timed twice, in the order 1 2 4 8 8 4 2 1, so that a slow
// drift of the step cost (cells filling up as the slab ionizes) cancels;
// the context's first step is not timed.  A call tunes with as many of its
// steps as it has; the search goes on in later calls until it is complete.
pic_ctx::Tuned *tuned_entry(pic_ctx *c)
{
    for (auto &t : c->tuned)
        if (t.ce == c->cap_ce && t.ci == c->cap_ci) return &t;
    return nullptr;
}

pic_status tune_step(pic_ctx *c, int n, int &k)
{
    pic_ctx::Tuned *t = tuned_entry(c);
    if (!t) {
        c->tuned.push_back(pic_ctx::Tuned{c->cap_ce, c->cap_ci, c->wpc, {0, 0, 0, 0}, 0});
        t = &c->tuned.back();
    }
    const int top = max_wpc(c->cap_ce, c->cap_ci);
    int shapes = 0;
    while (shapes < 4 && (1 << shapes) <= top) ++shapes;
    if (c->steps_done == 0 && k < n) {          // untimed first step of the context
        pic_status r = launch_step(c);
        if (r != PIC_OK) return r;
        ++k;
        ++c->steps_done;
    }
    if (!c->cell_ev[0]) {
        CK(cudaEventCreate(&c->cell_ev[0]));
        CK(cudaEventCreate(&c->cell_ev[1]));
    }
    pic_status r = PIC_OK;
    while (t->tried < (unsigned)(2 * shapes) && k < n && r == PIC_OK) {
        const int idx = t->tried < (unsigned)shapes ? (int)t->tried : 2 * shapes - 1 - (int)t->tried;
        if ((r = set_wpc(c, 1 << idx)) != PIC_OK) break;
        c->cell_ev_on = true;
        r = launch_step(c);
        c->cell_ev_on = false;
        if (r != PIC_OK) break;
        ++k;
        ++c->steps_done;
        float ms = 0.0f;
        if (cudaEventSynchronize(c->cell_ev[1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, c->cell_ev[0], c->cell_ev[1]) != cudaSuccess) {
            r = fail(c, PIC_ERR_CUDA, "autotune timing");
            break;
        }
        t->ms[idx] += 0.5f * ms;
        ++t->tried;
    }
    if (r != PIC_OK) return r;
    t->done = t->tried >= (unsigned)(2 * shapes);
    t->wpc = best_wpc(c, c->cap_ce, c->cap_ci);  // undecided: the default
    if (t->done) {
        float best = 3.4e38f;
        for (int q = 0; q < shapes; ++q)
            if (t->ms[q] < best) { best = t->ms[q]; t->wpc = 1 << q; }
    }
    return set_wpc(c, t->wpc);
}

// slabs that went beyond their electron budget were stopped on the device
// (k_advance): mark them failed on the host too
pic_status read_budget_failures(pic_ctx *c)
{
    std::vector<int> err(c->nslot);
    CK(cudaMemcpyAsync(err.data(), c->slab_err, sizeof(int) * c->nslot, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < c->nslot; ++k)
        if (err[k] && c->slot_state[k] == 1) {
            c->slot_state[k] = 3;
            c->slabs[k].active = 0;
        }
    return PIC_OK;
}

// Steps between two re-sizings of the cell tiers inside one pic_step call:
// ionization grows the cells, and cells that outgrow the tiers fall through
// to the one-warp large-cell pass.  Even, so that step pairs replay whole.
constexpr int RESIZE_EVERY = 32;

pic_status step_chunk(pic_ctx *c, int n);

pic_status step_n(pic_ctx *c, int n)
{
    pic_status r = apply_pending(c);
    if (r != PIC_OK) return r;
    c->launches = 0;
    for (int done = 0; done < n;) {
        const int m = std::min(n - done, RESIZE_EVERY);
        r = step_chunk(c, m);
        if (r != PIC_OK) return r;
        done += m;
    }
    // the first step after a retirement dropped the retired slabs' particles
    if (n > 0)
        for (int k = 0; k < c->nslot; ++k)
            if (c->slot_state[k] == 2) c->slot_state[k] = 0;
    return n > 0 && c->budgets ? read_budget_failures(c) : PIC_OK;
}

pic_status step_chunk(pic_ctx *c, int n)
{
    pic_status r = PIC_OK;
    // size the per-warp staging for the cells of the last sort
    int cn[NCOUNTERS];
    CK(cudaMemcpyAsync(cn, c->counters, sizeof(int) * NCOUNTERS, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (cn[CNT_MAXE] > 0 || cn[CNT_MAXI] > 0) {
        r = configure_cell_launch(c, cn + CNT_HIST_E, cn + CNT_HIST_I, cn[CNT_MAXE], cn[CNT_MAXI]);
        if (r != PIC_OK) return r;
    }
    int k = 0;
    if (c->autotune) {
        const pic_ctx::Tuned *t = tuned_entry(c);
        if (!t || !t->done) {
            r = tune_step(c, n, k);
            if (r != PIC_OK) return r;
        }
    }
    const int tuned_steps = k;        // counted by tune_step
    if (c->use_graphs && !c->timing && n - k >= 2) {
        pic_ctx::StepGraph *g = pair_graph(c, r);
        if (!g) return r;
        for (; k + 2 <= n; k += 2) {   // pairs of the remaining steps
            CK(cudaGraphLaunch(g->exec, c->stream));
            c->launches += g->launches;
        }
    }
    for (; k < n; ++k) {
        r = launch_step(c);
        if (r != PIC_OK) return r;
    }
    c->steps_done += n - tuned_steps;
    return PIC_OK;
}

bool batch_slot_ok(const pic_ctx *c, int slot) { return c && c->batch && slot >= 0 && slot < c->nslot; }

}  // namespace

extern "C" {

size_t pic_required_bytes(const pic_grid *g, const pic_species *s, int n_e_cap, int n_i_cap)
{
    if (!valid_grid(g) || !s) return 0;
    int ncell = g->nx * g->ny, npts = (g->nx + 1) * g->ny;
    int nblk = (ncell + SCAN_TILE - 1) / SCAN_TILE;
    int ce = n_e_cap > 0 ? n_e_cap : s->cap_e, ci = n_i_cap > 0 ? n_i_cap : s->cap_i;
    if (!caps_fit(ce, ci)) return 0;
    return arena_need(ncell, npts, nblk, ce, ci, 1, g->ny);
}

pic_status pic_init(pic_ctx **out, const pic_grid *g, const pic_species *s, const pic_tables *t, void *arena,
                    size_t arena_bytes, void *stream)
{
    if (!out || !t) return PIC_ERR_ARG;
    *out = nullptr;
    if (!valid_grid(g) || !valid_species(s) || !caps_fit(s->cap_e, s->cap_i)) return PIC_ERR_ARG;
    pic_ctx *c = nullptr;
    pic_status r = ctx_create(&c, 1, g->nx * g->ny, (g->nx + 1) * g->ny, g->ny, g->nx, s->cap_e, s->cap_i, t, arena,
                              arena_bytes, stream);
    if (r != PIC_OK) return r;
    c->grids[0] = *g;
    c->slabs[0] = make_slab(c, 0, g, s);
    c->slabs[0].active = 1;
    c->slot_state[0] = 1;
    if ((r = reset_slot(c, 0)) != PIC_OK) { pic_free(c); return r; }
    *out = c;
    return PIC_OK;
}

pic_status pic_source(pic_ctx *c, const pic_pulse *p)
{
    if (!c || !p) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "a batch context takes the pulse at admission");
    if (!valid_pulse(p)) return fail(c, PIC_ERR_ARG, "pulse out of range");
    set_pulse(c, c->slabs[0], p);
    CK(cudaMemcpyAsync(c->d_slab, &c->slabs[0], sizeof(SlabDev), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->photons, 0, sizeof(ph2) * (size_t)c->ncell * PIC_MAX_BINS, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

pic_status pic_load_electrons(pic_ctx *c, int64_t n, const double *X, const double *Y, const float *u,
                              const float *w, const uint64_t *id)
{
    if (!c || n < 0 || (n > 0 && (!X || !Y || !u || !w || !id))) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "a batch context loads particles at admission");
    if (n > c->cap_e) return fail(c, PIC_ERR_CAPACITY, "more electrons than the capacity");
    std::vector<real4> p0, p1;
    std::vector<int> key;
    pic_status r = build_records(c, 0, &c->grids[0], true, n, X, Y, u, w, id, nullptr, nullptr, nullptr, p0, p1, key);
    if (r == PIC_OK) r = load_species(c, true, n, p0, p1, key);
    if (r == PIC_OK) c->loaded_e = true;
    return r;
}

pic_status pic_seed(pic_ctx *c, const pic_seed_spec *sp)
{
    if (!c || !sp) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "a batch context loads particles at admission");
    if (sp->ppc_e < 1 || sp->ppc_i < 1 || sp->Z_init < 0 || sp->Z_init > 12 ||
        !(sp->T_e_eV >= 0 && std::isfinite(sp->T_e_eV)) || !(sp->T_i_eV >= 0 && std::isfinite(sp->T_i_eV)) ||
        !(sp->beam_frac >= 0 && sp->beam_frac <= 1) || !(sp->beam_E_eV >= 0 && std::isfinite(sp->beam_E_eV)))
        return fail(c, PIC_ERR_ARG, "seed spec out of range");
    const SlabDev &S = c->slabs[0];
    const long long ne = (long long)S.ncell * sp->ppc_e, ni = (long long)S.ncell * sp->ppc_i;
    if (ne > c->cap_e || ni > c->cap_i) return fail(c, PIC_ERR_CAPACITY, "seeded particles exceed the capacity");
    const double w_ion = (double)S.w_ion;
    const double gb = 1.0 + sp->beam_E_eV / kMeC2;
    for (int e = 1; e >= 0; --e) {
        SeedArgs a{};
        a.p0 = e ? c->eB0 : c->iB0; a.p1 = e ? c->eB1 : c->iB1; a.key = e ? c->ekey : c->ikey;
        a.n = e ? ne : ni; a.nx = S.nx; a.ny = S.ny; a.ppc = e ? sp->ppc_e : sp->ppc_i;
        a.electrons = e;
        a.sigma_u = e ? std::sqrt(sp->T_e_eV / kMeC2) : std::sqrt(sp->T_i_eV / ((double)S.m_ion * kMeC2));
        a.beam_frac = sp->beam_frac; a.beam_u = std::sqrt(gb * gb - 1.0);
        a.w = (float)(sp->Z_init * sp->ppc_i * w_ion / sp->ppc_e);
        a.st = sp->Z_init;
        a.seed = sp->seed;
        k_seed<<<c->nsm * 8, 256, 0, c->stream>>>(a);
        CK(cudaGetLastError());
        pic_status r = sort_species(c, e != 0, a.n);
        if (r != PIC_OK) return r;
    }
    c->loaded_e = c->loaded_i = true;
    return PIC_OK;
}

pic_status pic_load_ions(pic_ctx *c, int64_t n, const double *X, const double *Y, const float *u,
                         const float *zfrac, const int32_t *Z, const int32_t *nK, const uint32_t *id)
{
    if (!c || n < 0 || (n > 0 && (!X || !Y || !u || !zfrac || !Z || !nK || !id))) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "a batch context loads particles at admission");
    if (n > c->cap_i) return fail(c, PIC_ERR_CAPACITY, "more ions than the capacity");
    std::vector<real4> p0, p1;
    std::vector<int> key;
    pic_status r = build_records(c, 0, &c->grids[0], false, n, X, Y, u, zfrac, nullptr, Z, nK, id, p0, p1, key);
    if (r == PIC_OK) r = load_species(c, false, n, p0, p1, key);
    if (r == PIC_OK) c->loaded_i = true;
    return r;
}

pic_status pic_set_photons(pic_ctx *c, const double *ph)
{
    if (!c || !ph) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "single-slab call on a batch context");
    const int nb = c->slabs[0].nb;
    if (nb <= 0) return fail(c, PIC_ERR_STATE, "set a pulse first");
    size_t n = (size_t)c->ncell * nb;
    std::vector<ph2> h(n);
    for (size_t k = 0; k < n; ++k) {
        real hi = (real)ph[k];
        h[k] = ph2{hi, (real)(ph[k] - (double)hi)};
    }
    CK(cudaMemcpyAsync(c->photons, h.data(), sizeof(ph2) * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

pic_status pic_set_fields(pic_ctx *c, const float *f6)
{
    if (!c || !f6) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "single-slab call on a batch context");
    size_t n = (size_t)c->npts;
    std::vector<real> h(f6, f6 + 6 * n);
    CK(cudaMemcpyAsync(c->E[c->ecur], h.data(), sizeof(real) * 3 * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->B, h.data() + 3 * n, sizeof(real) * 3 * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

pic_status pic_step(pic_ctx *c, int n)
{
    if (!c || n < 0) return PIC_ERR_ARG;
    if (!c->batch && (!c->loaded_e || !c->loaded_i)) return fail(c, PIC_ERR_STATE, "load particles before stepping");
    return step_n(c, n);
}

pic_status pic_sync(pic_ctx *c)
{
    if (!c) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream));
    return read_device_error(c);
}

pic_status pic_counts(pic_ctx *c, int64_t *n_e, int64_t *n_i)
{
    if (!c) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "single-slab call on a batch context");
    return counts_slot(c, 0, n_e, n_i);
}

pic_status pic_get_electrons(pic_ctx *c, double *X, double *Y, float *u, float *w, uint64_t *id)
{
    if (!c) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "single-slab call on a batch context");
    return get_electrons_slot(c, 0, X, Y, u, w, id);
}

pic_status pic_get_ions(pic_ctx *c, double *X, double *Y, float *u, float *zfrac, int32_t *Z, int32_t *nK,
                        uint32_t *id)
{
    if (!c) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "single-slab call on a batch context");
    return get_ions_slot(c, 0, X, Y, u, zfrac, Z, nK, id);
}

pic_status pic_get_electrons64(pic_ctx *c, double *X, double *Y, double *u, double *w, uint64_t *id)
{
    if (!c) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "single-slab call on a batch context");
    return get_electrons_slot(c, 0, X, Y, u, w, id);
}

pic_status pic_get_ions64(pic_ctx *c, double *X, double *Y, double *u, double *zfrac, int32_t *Z, int32_t *nK,
                          uint32_t *id)
{
    if (!c) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "single-slab call on a batch context");
    return get_ions_slot(c, 0, X, Y, u, zfrac, Z, nK, id);
}

int pic_real_bytes(void) { return (int)sizeof(real); }

pic_status pic_get_photons(pic_ctx *c, double *ph)
{
    if (!c || !ph) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "single-slab call on a batch context");
    const int nb = c->slabs[0].nb;
    if (nb <= 0) return fail(c, PIC_ERR_STATE, "no pulse set");
    size_t n = (size_t)c->ncell * nb;
    std::vector<ph2> h(n);
    CK(cudaMemcpyAsync(h.data(), c->photons, sizeof(ph2) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k < n; ++k) ph[k] = (double)h[k].hi + (double)h[k].lo;
    return read_device_error(c);
}

pic_status pic_get_fields(pic_ctx *c, float *f6)
{
    if (!c || !f6) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "single-slab call on a batch context");
    size_t n = (size_t)c->npts;
    std::vector<real> h(6 * n);
    CK(cudaMemcpyAsync(h.data(), c->E[c->ecur], sizeof(real) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(h.data() + 3 * n, c->B, sizeof(real) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k < 6 * n; ++k) f6[k] = (float)h[k];
    return read_device_error(c);
}

pic_status pic_get_current(pic_ctx *c, double *j3)
{
    if (!c || !j3) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "single-slab call on a batch context");
    size_t n = (size_t)c->npts;
    std::vector<unsigned long long> raw(3 * n);
    CK(cudaMemcpyAsync(raw.data(), c->J, sizeof(unsigned long long) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const pic_grid &g = c->grids[0];
    const double fix = 1.0 / JFIX;
    const double sx = g.dx_nm / g.dt_fs;
    const double sy = g.ny > 1 ? g.dy_nm / g.dt_fs : kCnmPerFs;
    for (size_t k = 0; k < n; ++k) {
        j3[k] = (double)(long long)raw[k] * fix * sx;
        j3[n + k] = (double)(long long)raw[n + k] * fix * sy;
        j3[2 * n + k] = (double)(long long)raw[2 * n + k] * fix * kCnmPerFs;
    }
    return read_device_error(c);
}

pic_status pic_diagnostics(pic_ctx *c, pic_diag *out)
{
    if (!c) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "single-slab call on a batch context");
    return diag_slot(c, 0, out);
}

size_t pic_batch_required_bytes(int max_slabs, int slot_cells, int cap_e, int cap_i)
{
    if (max_slabs < 1 || slot_cells < 2 || slot_cells > 8192 || !caps_fit(cap_e, cap_i)) return 0;
    long long ncell = (long long)max_slabs * slot_cells, npts = (long long)max_slabs * (slot_cells + 1);
    if (npts > kMaxCells) return 0;
    int nblk = (int)((ncell + SCAN_TILE - 1) / SCAN_TILE);
    return arena_need((int)ncell, (int)npts, nblk, cap_e, cap_i, max_slabs, max_slabs);
}

pic_status pic_batch_init(pic_ctx **out, int max_slabs, int slot_cells, int cap_e, int cap_i, const pic_tables *t,
                          void *arena, size_t arena_bytes, void *stream)
{
    if (!out || !t) return PIC_ERR_ARG;
    *out = nullptr;
    if (pic_batch_required_bytes(max_slabs, slot_cells, cap_e, cap_i) == 0) return PIC_ERR_ARG;
    pic_ctx *c = nullptr;
    pic_status r = ctx_create(&c, max_slabs, slot_cells, slot_cells + 1, 1, slot_cells, cap_e, cap_i, t, arena,
                              arena_bytes, stream);
    if (r != PIC_OK) return r;
    c->batch = true;
    *out = c;
    return PIC_OK;
}

pic_status pic_batch_admit(pic_ctx *c, const pic_grid *g, const pic_species *s, const pic_pulse *p, int64_t n_e,
                           const double *eX, const double *eY, const float *eu, const float *ew, const uint64_t *eid,
                           int64_t n_i, const double *iX, const double *iY, const float *iu, const float *izf,
                           const int32_t *iZ, const int32_t *inK, const uint32_t *iid, int *slot_out)
{
    if (!c || !slot_out) return PIC_ERR_ARG;
    *slot_out = -1;
    if (!c->batch) return fail(c, PIC_ERR_STATE, "not a batch context");
    if (!valid_grid(g) || g->ny != 1 || g->nx > c->slot_cells || !valid_species(s))
        return fail(c, PIC_ERR_ARG, "slab does not fit a slot (1D, nx <= slot cells)");
    if (p && !valid_pulse(p)) return fail(c, PIC_ERR_ARG, "pulse out of range");
    if (n_e < 0 || n_i < 0 || (n_e && (!eX || !eY || !eu || !ew || !eid)) ||
        (n_i && (!iX || !iY || !iu || !izf || !iZ || !inK || !iid)))
        return fail(c, PIC_ERR_ARG, "particle arrays missing");
    int k = -1;
    for (int q = 0; q < c->nslot && k < 0; ++q)
        if (c->slot_state[q] == 0) k = q;
    if (k < 0 && any_retired(c)) {               // free the retired slots now
        pic_status r = apply_pending(c);
        if (r == PIC_OK) r = compact(c);
        if (r != PIC_OK) return r;
        for (int q = 0; q < c->nslot && k < 0; ++q)
            if (c->slot_state[q] == 0) k = q;
    }
    if (k < 0) return fail(c, PIC_ERR_CAPACITY, "no free slot");
    pic_ctx::Pending pd;
    pd.slot = k;
    pic_status r = build_records(c, k, g, true, n_e, eX, eY, eu, ew, eid, nullptr, nullptr, nullptr, pd.e0, pd.e1, pd.ek);
    if (r != PIC_OK) return r;
    r = build_records(c, k, g, false, n_i, iX, iY, iu, izf, nullptr, iZ, inK, iid, pd.i0, pd.i1, pd.ik);
    if (r != PIC_OK) return r;
    c->grids[k] = *g;
    c->slabs[k] = make_slab(c, k, g, s);
    if (p) set_pulse(c, c->slabs[k], p);
    c->slot_state[k] = 1;
    c->pending.push_back(std::move(pd));
    *slot_out = k;
    return PIC_OK;
}

pic_status pic_batch_retire(pic_ctx *c, int slot)
{
    if (!batch_slot_ok(c, slot)) return PIC_ERR_ARG;
    if (c->slot_state[slot] == 3) {              // failed: stopped on the device already
        c->slot_state[slot] = 2;
        return PIC_OK;
    }
    if (c->slot_state[slot] != 1) return fail(c, PIC_ERR_STATE, "slot is not active");
    for (size_t q = 0; q < c->pending.size(); ++q)
        if (c->pending[q].slot == slot) {          // admitted, never on the device
            c->pending.erase(c->pending.begin() + q);
            c->slabs[slot].active = 0;
            c->slot_state[slot] = 0;
            return PIC_OK;
        }
    c->slabs[slot].active = 0;
    CK(cudaMemcpyAsync(c->d_slab + slot, &c->slabs[slot], sizeof(SlabDev), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->slot_state[slot] = 2;
    return PIC_OK;
}

pic_status pic_batch_set_budget(pic_ctx *c, int slot, int64_t max_e)
{
    if (!batch_slot_ok(c, slot) || max_e < 0 || max_e > (int64_t)c->cap_e) return PIC_ERR_ARG;
    if (c->slot_state[slot] != 1) return fail(c, PIC_ERR_STATE, "slot is not active");
    c->slabs[slot].budget_e = (int)max_e;
    if (max_e > 0) c->budgets = true;
    for (const auto &p : c->pending)
        if (p.slot == slot) return PIC_OK;      // uploaded with the admission
    CK(cudaMemcpyAsync(c->d_slab + slot, &c->slabs[slot], sizeof(SlabDev), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

pic_status pic_batch_slot(pic_ctx *c, int slot, int *state, uint32_t *step)
{
    if (!batch_slot_ok(c, slot)) return PIC_ERR_ARG;
    if (state) *state = c->slot_state[slot];
    if (step) {
        CK(cudaMemcpyAsync(step, c->d_steps + slot, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return PIC_OK;
}

pic_status pic_batch_diagnostics(pic_ctx *c, int slot, pic_diag *out)
{
    if (!batch_slot_ok(c, slot)) return PIC_ERR_ARG;
    if (c->slot_state[slot] != 1) return fail(c, PIC_ERR_STATE, "slot is not active");
    pic_status r = apply_pending(c);
    if (r != PIC_OK) return r;
    return diag_slot(c, slot, out);
}

pic_status pic_batch_counts(pic_ctx *c, int slot, int64_t *n_e, int64_t *n_i)
{
    if (!batch_slot_ok(c, slot)) return PIC_ERR_ARG;
    pic_status r = apply_pending(c);
    if (r != PIC_OK) return r;
    return counts_slot(c, slot, n_e, n_i);
}

pic_status pic_batch_get_electrons(pic_ctx *c, int slot, double *X, double *Y, float *u, float *w, uint64_t *id)
{
    if (!batch_slot_ok(c, slot)) return PIC_ERR_ARG;
    if (c->slot_state[slot] != 1) return fail(c, PIC_ERR_STATE, "slot is not active");
    pic_status r = apply_pending(c);
    if (r != PIC_OK) return r;
    return get_electrons_slot(c, slot, X, Y, u, w, id);
}

pic_status pic_batch_get_ions(pic_ctx *c, int slot, double *X, double *Y, float *u, float *zfrac, int32_t *Z,
                              int32_t *nK, uint32_t *id)
{
    if (!batch_slot_ok(c, slot)) return PIC_ERR_ARG;
    if (c->slot_state[slot] != 1) return fail(c, PIC_ERR_STATE, "slot is not active");
    pic_status r = apply_pending(c);
    if (r != PIC_OK) return r;
    return get_ions_slot(c, slot, X, Y, u, zfrac, Z, nK, id);
}

int64_t pic_launch_count(const pic_ctx *c) { return c ? c->launches : 0; }

pic_status pic_autotune(pic_ctx *c, int enable, int *wpc_out, float *ms_out)
{
    if (!c) return PIC_ERR_ARG;
    if (enable >= 0) c->autotune = enable != 0;
    if (wpc_out) *wpc_out = c->wpc;
    if (ms_out) {
        for (int q = 0; q < 4; ++q) ms_out[q] = 0.0f;
        for (const auto &t : c->tuned)
            if (t.ce == c->cap_ce && t.ci == c->cap_ci)
                for (int q = 0; q < 4; ++q) ms_out[q] = t.ms[q];
    }
    return PIC_OK;
}

pic_status pic_use_graphs(pic_ctx *c, int enable)
{
    if (!c) return PIC_ERR_ARG;
    c->use_graphs = enable != 0;
    return PIC_OK;
}

pic_status pic_timing(pic_ctx *c, int enable, double *ms_out, int64_t *nsteps)
{
    if (!c) return PIC_ERR_ARG;
    if (ms_out) {
        CK(cudaStreamSynchronize(c->stream));
        for (int k = 0; k < NEV; ++k) ms_out[k] = 0.0;
        // groups: cell kernels, march (+ memsets), push, sort, fields, whole step
        const int from[NEV] = {1, 0, 2, 3, 4, 0}, to[NEV] = {2, 1, 3, 4, 5, 5};
        for (size_t b = 0; b + NEV <= c->ev_used; b += NEV)
            for (int k = 0; k < NEV; ++k) {
                float t;
                CK(cudaEventElapsedTime(&t, c->ev[b + from[k]], c->ev[b + to[k]]));
                ms_out[k] += t;
            }
        if (nsteps) *nsteps = (int64_t)(c->ev_used / NEV);
    }
    if (enable >= 0) {
        c->timing = enable != 0;
        c->ev_used = 0;
    }
    return PIC_OK;
}

pic_status pic_free(pic_ctx *c)
{
    if (!c) return PIC_ERR_ARG;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->own_arena && c->arena) cudaFree(c->arena);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (auto &g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaEvent_t e : c->cell_ev)
        if (e) cudaEventDestroy(e);
    if (c->rt_mem) cudaFree(c->rt_mem);
    delete c;
    return PIC_OK;
}

pic_status pic_rt(pic_ctx *c, const pic_rt_config *rt)
{
    if (!c || !rt) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "radiation transport runs on single-slab contexts");
    SlabDev &S = c->slabs[0];
    const int R = rt->coarsen, d2 = S.ny > 1;
    if (S.nb <= 0) return fail(c, PIC_ERR_STATE, "pic_rt needs a pulse (pic_source) first");
    if (R < 1 || S.nx % R || (d2 && S.ny % R) || S.nx / R > 4096 || (d2 && S.ny / R > 4096) || rt->n_polar < 0 ||
        rt->n_polar > 16 || (d2 && (rt->n_azimuth < 1 || rt->n_azimuth > 16)) || (rt->scheme != 0 && rt->scheme != 1))
        return fail(c, PIC_ERR_ARG, "invalid radiation transport setting");
    if (c->rt_mem) return fail(c, PIC_ERR_STATE, "radiation transport already on");
    // the beam enters through ghost nodes: c dt_rad may span at most the
    // RT_GHOST - 3 rad cells they hold along any axis
    {
        const double dtr = (double)S.rad_every * (double)S.dt;
        const double dmin = (d2 ? std::min((double)S.dx, (double)S.dy) : (double)S.dx) * R;
        if (!(kCnmPerFs * dtr <= (RT_GHOST - 3) * dmin))
            return fail(c, PIC_ERR_ARG, "radiation transport: c dt_rad spans more rad cells than the inflow holds");
    }
    const int nb = S.nb, nrx = S.nx / R, nry = d2 ? S.ny / R : 1, nrc = nrx * nry;
    const int naz = d2 ? rt->n_azimuth : 1, nord = 1 + rt->n_polar * naz;
    // ordinates: the beam along +x, then Gauss-Legendre nodes of mu =
    // cos(theta) (Newton on the Legendre recurrence) times azimuths in
    // (0, pi); weights: share of the sphere (the lower half folded in)
    std::vector<double> ord(3 * (size_t)nord, 0.0);
    ord[0] = 1.0;
    for (int k = 0; k < rt->n_polar; ++k) {
        const int n = rt->n_polar;
        double z = std::cos(kPi * (4.0 * k + 3.0) / (4.0 * n + 2.0)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double pm = 1.0, pc = z;                 // P_{j-1}, P_j
            for (int j = 2; j <= n; ++j) {
                const double pn = ((2.0 * j - 1.0) * z * pc - (j - 1.0) * pm) / j;
                pm = pc; pc = pn;
            }
            dp = n * (z * pc - pm) / (z * z - 1.0);   // P_n'
            const double step = pc / dp;
            z -= step;
            if (std::fabs(step) < 1e-15) break;
        }
        const double a = 2.0 / ((1.0 - z * z) * dp * dp);
        for (int j = 0; j < naz; ++j) {
            const int o = 1 + k * naz + j;
            ord[o] = z;
            ord[nord + o] = d2 ? std::sqrt(1.0 - z * z) * std::cos(kPi * (j + 0.5) / naz) : 0.0;
            ord[2 * (size_t)nord + o] = 0.5 * a / naz;
        }
    }
    const size_t nf = (size_t)nord * nb * nrc, ncell = (size_t)S.ncell;
    // the sum of the pieces carved below, each rounded up to 256 bytes
    const size_t bytes = 3 * al(nf * 8) + al((size_t)nrc * nb * 8) + al(ord.size() * 8) + al(ncell * nb * 4) +
                         2 * al(ncell * 8) + al(ncell * 4);
    char *mem = nullptr;
    CK(cudaMalloc(&mem, bytes));
    c->rt_mem = mem;
    c->rt_bytes = bytes;
    CK(cudaMemsetAsync(mem, 0, bytes, c->stream));
    char *q = mem;
    S.rt_F = (double *)q; q += al(nf * 8);
    S.rt_Gx = (double *)q; q += al(nf * 8);
    S.rt_Gy = (double *)q; q += al(nf * 8);
    S.rt_npub = (double *)q; q += al((size_t)nrc * nb * 8);
    double *d_ord = (double *)q; q += al(ord.size() * 8);
    S.rt_ord = d_ord;
    S.rt_chi = (float *)q; q += al(ncell * nb * 4);
    S.rt_emc = (double *)q; q += al(ncell * 8);
    S.rt_dE = (double *)q; q += al(ncell * 8);
    S.rt_w = (float *)q;
    S.rt = 1; S.rt_R = R; S.rt_nrx = nrx; S.rt_nry = nry; S.rt_nord = nord; S.rt_scheme = rt->scheme;
    S.rt_ncd = d2 ? R * R : R;
    c->rt_nord = nord;
    CK(cudaMemcpyAsync(d_ord, ord.data(), ord.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_slab, &S, sizeof(SlabDev), cudaMemcpyHostToDevice, c->stream));
    CK(cudaFuncSetAttribute(k_rt_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(3 * sizeof(double) * (RT_GHOST + std::max(nrx, nry)))));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

pic_status pic_rt_get(pic_ctx *c, double *F, double *Gx, double *Gy)
{
    if (!c || !F || !Gx || !Gy) return PIC_ERR_ARG;
    if (!c->rt_mem) return fail(c, PIC_ERR_STATE, "radiation transport is off");
    const SlabDev &S = c->slabs[0];
    const size_t nf = (size_t)S.rt_nord * S.nb * S.rt_nrx * S.rt_nry;
    CK(cudaMemcpyAsync(F, S.rt_F, nf * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(Gx, S.rt_Gx, nf * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(Gy, S.rt_Gy, nf * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return read_device_error(c);
}

pic_status pic_rt_set(pic_ctx *c, const double *F, const double *Gx, const double *Gy)
{
    if (!c || !F || !Gx || !Gy) return PIC_ERR_ARG;
    if (!c->rt_mem) return fail(c, PIC_ERR_STATE, "radiation transport is off");
    const SlabDev &S = c->slabs[0];
    const size_t nf = (size_t)S.rt_nord * S.nb * S.rt_nrx * S.rt_nry;
    CK(cudaMemcpyAsync(S.rt_F, F, nf * 8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(S.rt_Gx, Gx, nf * 8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(S.rt_Gy, Gy, nf * 8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

pic_status pic_rt_cells(pic_ctx *c, double *chi, double *emc, double *w, double *dE)
{
    if (!c || !chi || !emc || !w || !dE) return PIC_ERR_ARG;
    if (!c->rt_mem) return fail(c, PIC_ERR_STATE, "radiation transport is off");
    const SlabDev &S = c->slabs[0];
    const size_t n = (size_t)S.ncell;
    std::vector<float> hc(n * S.nb), hw(n);
    CK(cudaMemcpyAsync(hc.data(), S.rt_chi, hc.size() * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(hw.data(), S.rt_w, n * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(emc, S.rt_emc, n * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(dE, S.rt_dE, n * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k < hc.size(); ++k) chi[k] = hc[k];
    for (size_t k = 0; k < n; ++k) w[k] = hw[k];
    return read_device_error(c);
}

const char *pic_last_error(const pic_ctx *c) { return c ? c->err.c_str() : "no context"; }

pic_status pic_philox_check(const uint32_t *ctr, const uint32_t key[2], uint32_t *out, int n)
{
    if (!ctr || !key || !out || n <= 0) return PIC_ERR_ARG;
    uint32_t *d = nullptr;
    if (cudaMalloc(&d, sizeof(uint32_t) * 8 * (size_t)n) != cudaSuccess) return PIC_ERR_OOM;
    pic_status st = PIC_OK;
    if (cudaMemcpy(d, ctr, sizeof(uint32_t) * 4 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess) st = PIC_ERR_CUDA;
    if (st == PIC_OK) {
        k_philox_check<<<(n + 127) / 128, 128>>>(d, key[0], key[1], d + 4 * (size_t)n, n);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(out, d + 4 * (size_t)n, sizeof(uint32_t) * 4 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = PIC_ERR_CUDA;
    }
    cudaFree(d);
    return st;
}

pic_status pic_order_check(const uint64_t *key, const uint64_t *id, int n, int rmax, uint16_t *order)
{
    if (!key || !id || !order || n <= 0 || n > 4096 || !(rmax == 128 || rmax == 512 || rmax == 1024) ||
        (rmax == 128 && n > 128))
        return PIC_ERR_ARG;
    const size_t smem = (size_t)n * 32 + 256 * 4 + (size_t)n * 2;
    void (*kern)(const unsigned long long *, const unsigned long long *, int, unsigned short *) =
        rmax == 128 ? k_order_check<128> : (rmax == 512 ? k_order_check<512> : k_order_check<1024>);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return PIC_ERR_CUDA;
    char *d = nullptr;
    const size_t bytes = (size_t)n * 16 + (size_t)n * 2;
    if (cudaMalloc(&d, bytes) != cudaSuccess) return PIC_ERR_OOM;
    pic_status st = PIC_OK;
    unsigned long long *dk = (unsigned long long *)d, *di = dk + n;
    unsigned short *dout = (unsigned short *)(di + n);
    if (cudaMemcpy(dk, key, sizeof(uint64_t) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(di, id, sizeof(uint64_t) * n, cudaMemcpyHostToDevice) != cudaSuccess)
        st = PIC_ERR_CUDA;
    if (st == PIC_OK) {
        kern<<<1, 32, smem>>>(dk, di, n, dout);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(order, dout, sizeof(uint16_t) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = PIC_ERR_CUDA;
    }
    cudaFree(d);
    return st;
}

}  // extern "C"

namespace {

// ---------------- checkpoint / restore ----------------
// Host image of a single-slab context: a header, the sorted particle records
// with their cell starts, the current E and B, the photon numbers, the
// tallies, the step count and, in transport mode, the transport's block.
// The random streams are keyed by (seed, id, step, purpose), so nothing of
// the generator needs saving: a restored context continues bit for bit.
struct CkptHeader {
    char magic[8];
    int32_t version, real_bytes, nx, ny, nb, rt;
    int64_t n_e, n_i;
    uint32_t step, pad;
    double dx, dy, dt, w_ion;
    uint64_t rt_bytes, total;
};
constexpr char kCkptMagic[8] = {'P', 'I', 'C', 'C', 'K', 'P', 'T', '1'};

size_t ckpt_bytes(const pic_ctx *c, int64_t ne, int64_t ni)
{
    const size_t cs = 2 * sizeof(int) * (size_t)(c->ncell + 1);
    return sizeof(CkptHeader) + 2 * sizeof(real4) * (size_t)(ne + ni) + cs + 6 * sizeof(real) * (size_t)c->npts +
           sizeof(ph2) * (size_t)c->ncell * PIC_MAX_BINS + sizeof(SlabTally) + c->rt_bytes;
}

pic_status ckpt_counts(pic_ctx *c, int64_t *ne, int64_t *ni)
{
    int v[2];
    CK(cudaMemcpyAsync(&v[0], c->csE[c->cur] + c->ncell, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&v[1], c->csI[c->cur] + c->ncell, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *ne = v[0]; *ni = v[1];
    return PIC_OK;
}

}  // namespace

extern "C" {

size_t pic_checkpoint_bytes(pic_ctx *c)
{
    if (!c || c->batch || !c->loaded_e || !c->loaded_i) return 0;
    int64_t ne = 0, ni = 0;
    if (ckpt_counts(c, &ne, &ni) != PIC_OK) return 0;
    return ckpt_bytes(c, ne, ni);
}

pic_status pic_checkpoint(pic_ctx *c, void *host, size_t bytes)
{
    if (!c || !host) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "checkpoints are of single-slab contexts");
    if (!c->loaded_e || !c->loaded_i) return fail(c, PIC_ERR_STATE, "nothing loaded");
    pic_status r = read_device_error(c);
    if (r != PIC_OK) return r;
    int64_t ne = 0, ni = 0;
    if ((r = ckpt_counts(c, &ne, &ni)) != PIC_OK) return r;
    const size_t need = ckpt_bytes(c, ne, ni);
    if (bytes < need) return fail(c, PIC_ERR_ARG, "checkpoint buffer too small");
    const SlabDev &S = c->slabs[0];
    const pic_grid &g = c->grids[0];
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 1; h.real_bytes = (int)sizeof(real); h.nx = g.nx; h.ny = g.ny; h.nb = S.nb; h.rt = S.rt;
    h.n_e = ne; h.n_i = ni; h.dx = g.dx_nm; h.dy = g.dy_nm; h.dt = g.dt_fs; h.w_ion = (double)S.w_ion;
    h.rt_bytes = c->rt_bytes; h.total = need;
    cudaStream_t st = c->stream;
    CK(cudaMemcpyAsync(&h.step, c->d_steps, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    char *p = (char *)host + sizeof(CkptHeader);
    auto get = [&](const void *src, size_t n) -> cudaError_t {
        cudaError_t e = n ? cudaMemcpyAsync(p, src, n, cudaMemcpyDeviceToHost, st) : cudaSuccess;
        p += n;
        return e;
    };
    CK(get(c->eA0, sizeof(real4) * ne)); CK(get(c->eA1, sizeof(real4) * ne));
    CK(get(c->iA0, sizeof(real4) * ni)); CK(get(c->iA1, sizeof(real4) * ni));
    CK(get(c->csE[c->cur], sizeof(int) * (size_t)(c->ncell + 1)));
    CK(get(c->csI[c->cur], sizeof(int) * (size_t)(c->ncell + 1)));
    CK(get(c->E[c->ecur], sizeof(real) * 3 * (size_t)c->npts));
    CK(get(c->B, sizeof(real) * 3 * (size_t)c->npts));
    CK(get(c->photons, sizeof(ph2) * (size_t)c->ncell * PIC_MAX_BINS));
    CK(get(c->d_tally, sizeof(SlabTally)));
    if (c->rt_bytes) CK(get(c->rt_mem, c->rt_bytes));
    CK(cudaStreamSynchronize(st));
    std::memcpy(host, &h, sizeof(CkptHeader));
    return PIC_OK;
}

pic_status pic_restore(pic_ctx *c, const void *host, size_t bytes)
{
    if (!c || !host || bytes < sizeof(CkptHeader)) return PIC_ERR_ARG;
    if (c->batch) return fail(c, PIC_ERR_STATE, "checkpoints are of single-slab contexts");
    CkptHeader h;
    std::memcpy(&h, host, sizeof(CkptHeader));
    const SlabDev &S = c->slabs[0];
    const pic_grid &g = c->grids[0];
    if (std::memcmp(h.magic, kCkptMagic, 8) || h.version != 1 || h.real_bytes != (int)sizeof(real))
        return fail(c, PIC_ERR_ARG, "not a checkpoint of this build");
    if (h.nx != g.nx || h.ny != g.ny || h.dx != g.dx_nm || h.dy != g.dy_nm || h.dt != g.dt_fs ||
        h.w_ion != (double)S.w_ion || h.nb != S.nb || h.rt != S.rt || h.rt_bytes != c->rt_bytes)
        return fail(c, PIC_ERR_ARG, "checkpoint of another slab, pulse or transport setting");
    if (h.n_e < 0 || h.n_i < 0 || h.total != ckpt_bytes(c, h.n_e, h.n_i) || bytes < h.total)
        return fail(c, PIC_ERR_ARG, "checkpoint truncated");
    if (h.n_e > c->cap_e || h.n_i > c->cap_i) return fail(c, PIC_ERR_CAPACITY, "checkpoint exceeds the capacity");
    const char *p = (const char *)host + sizeof(CkptHeader);
    const int64_t ne = h.n_e, ni = h.n_i;
    std::vector<real4> e0(ne), e1(ne), i0(ni), i1(ni);
    std::vector<int> cse(c->ncell + 1), csi(c->ncell + 1);
    auto take = [&](void *dst, size_t n) { std::memcpy(dst, p, n); p += n; };
    take(e0.data(), sizeof(real4) * ne); take(e1.data(), sizeof(real4) * ne);
    take(i0.data(), sizeof(real4) * ni); take(i1.data(), sizeof(real4) * ni);
    take(cse.data(), sizeof(int) * cse.size()); take(csi.data(), sizeof(int) * csi.size());
    if (cse[0] != 0 || csi[0] != 0 || cse[c->ncell] != ne || csi[c->ncell] != ni)
        return fail(c, PIC_ERR_ARG, "checkpoint cell starts inconsistent");
    // the records index the device's atomic tables and current stencils: a
    // damaged image is refused (the loaders' rules) rather than read out of
    // bounds on the device
    auto in_cell = [](const real4 &q) { return q.x >= (real)0 && q.x < (real)1 && q.y >= (real)0 && q.y < (real)1; };
    for (int64_t k = 0; k < ne; ++k)
        if (!in_cell(e0[k])) return fail(c, PIC_ERR_ARG, "checkpoint electron record out of range");
    for (int64_t k = 0; k < ni; ++k) {
        const unsigned st = (unsigned)rec_ist(i1[k]), Z = st & 0xffu, nK = st >> 8;
        if (!in_cell(i0[k]) || Z > (unsigned)ZNUC || nK > (unsigned)std::min(2, ZNUC - (int)Z) ||
            !(i1[k].y >= (real)0 && i1[k].y < (real)1))
            return fail(c, PIC_ERR_ARG, "checkpoint ion record out of range");
    }
    std::vector<int> ke(ne), ki(ni);
    for (int g2 = 0; g2 < c->ncell; ++g2) {
        if (cse[g2 + 1] < cse[g2] || csi[g2 + 1] < csi[g2]) return fail(c, PIC_ERR_ARG, "checkpoint cell starts inconsistent");
        for (int k = cse[g2]; k < cse[g2 + 1]; ++k) ke[k] = g2;
        for (int k = csi[g2]; k < csi[g2 + 1]; ++k) ki[k] = g2;
    }
    pic_status r = load_species(c, true, ne, e0, e1, ke);
    if (r == PIC_OK) r = load_species(c, false, ni, i0, i1, ki);
    if (r != PIC_OK) return r;
    cudaStream_t st = c->stream;
    auto put = [&](void *dst, size_t n) -> cudaError_t {
        cudaError_t e = n ? cudaMemcpyAsync(dst, p, n, cudaMemcpyHostToDevice, st) : cudaSuccess;
        p += n;
        return e;
    };
    CK(put(c->E[c->ecur], sizeof(real) * 3 * (size_t)c->npts));
    CK(put(c->B, sizeof(real) * 3 * (size_t)c->npts));
    CK(put(c->photons, sizeof(ph2) * (size_t)c->ncell * PIC_MAX_BINS));
    CK(put(c->d_tally, sizeof(SlabTally)));
    if (c->rt_bytes) CK(put(c->rt_mem, c->rt_bytes));
    CK(cudaMemcpyAsync(c->d_steps, &h.step, sizeof(unsigned), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    c->loaded_e = c->loaded_i = true;
    return PIC_OK;
}

pic_status pic_dd_sum_check(const float *x, int n, double *out)
{
    if (!x || !out || n <= 0 || n > (1 << 24)) return PIC_ERR_ARG;
    char *d = nullptr;
    if (cudaMalloc(&d, sizeof(float) * (size_t)n + 16) != cudaSuccess) return PIC_ERR_OOM;
    float *dx = (float *)(d + 16);
    double *dout = (double *)d;
    pic_status st = PIC_OK;
    if (cudaMemcpy(dx, x, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess) st = PIC_ERR_CUDA;
    if (st == PIC_OK) {
        k_dd_check<<<1, 32>>>(dx, n, dout);
        if (cudaGetLastError() != cudaSuccess || cudaMemcpy(out, dout, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = PIC_ERR_CUDA;
    }
    cudaFree(d);
    return st;
}

// Scratch of pic_philox_check_static: counters then outputs, 4 words each.
static __device__ __align__(256) uint32_t g_philox_scratch[8 * PIC_PHILOX_STATIC_MAX];

pic_status pic_philox_check_static(const uint32_t *ctr, const uint32_t key[2], uint32_t *out, int n)
{
    if (!ctr || !key || !out || n <= 0 || n > PIC_PHILOX_STATIC_MAX) return PIC_ERR_ARG;
    // address of the scratch on each device, looked up once with that device current
    constexpr int MAX_DEV = 64;
    static uint32_t *addr[MAX_DEV] = {};
    static std::mutex lock;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return PIC_ERR_CUDA;
    uint32_t *d = nullptr;
    {
        std::lock_guard<std::mutex> g(lock);
        if (!addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_philox_scratch) != cudaSuccess || !p) return PIC_ERR_CUDA;
            addr[dev] = static_cast<uint32_t *>(p);
        }
        d = addr[dev];
    }
    if (cudaMemcpy(d, ctr, sizeof(uint32_t) * 4 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess) return PIC_ERR_CUDA;
    k_philox_check<<<(n + 127) / 128, 128>>>(d, key[0], key[1], d + 4 * (size_t)PIC_PHILOX_STATIC_MAX, n);
    if (cudaGetLastError() != cudaSuccess) return PIC_ERR_CUDA;
    if (cudaMemcpy(out, d + 4 * (size_t)PIC_PHILOX_STATIC_MAX, sizeof(uint32_t) * 4 * (size_t)n,
                   cudaMemcpyDeviceToHost) != cudaSuccess)
        return PIC_ERR_CUDA;
    return PIC_OK;
}

}  // extern "C"
