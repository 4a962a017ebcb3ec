// Radiation transport mode (Sec. II, Eqs. 1a and 1b): the photon field as
// photon densities in discrete ordinates on a rad grid rt_R times coarser
// than the PIC grid, advanced once per rad step before the cell kernel:
//   k_rt_cells    per rad cell: gather what the cells recorded at the last
//                 rad step (opacity, photon energy the photoionization
//                 events took, electron weight, K-alpha photons added to
//                 their bins), absorb every ordinate over dt_rad, book the
//                 energy absorbed beyond the events for the rad cell's bulk
//                 electrons (shared among its PIC cells by electron
//                 weight, given at their next rad step), emit the K-alpha
//                 photons isotropically into the diffuse ordinates
//   k_rt_sweep    advect every (ordinate, bin) line, along x and in 2D
//                 along y (periodic): the CIP scheme (value and slope,
//                 cubic Hermite at the departure point) or the march's
//                 linear split; contents crossing the x faces by the split
//                 rule, what CIP's update adds to that tallied as its gain
//   k_rt_publish  per PIC cell: the densities of its rad cell
// The field and its bookkeeping are double precision (a few MB, a small
// part of a step).  The kernels return at once on other steps.
#pragma once
#include "pic_dev.cuh"

namespace pic {

struct RtArgs {
    const SlabDev *slab;       // the context's one slab
    const unsigned *steps;
    ph2 *photons;              // [ncell][nb] the cells' photon numbers
    SlabTally *tally;
};

__device__ __forceinline__ bool rt_active(const SlabDev &S, unsigned step)
{
    return S.active && S.rt && S.nb > 0 && S.rad_every > 0 && (step % (unsigned)S.rad_every) == 0;
}

__device__ __forceinline__ double ph_val(const ph2 &v) { return (double)v.hi + (double)v.lo; }

__global__ void k_rt_cells(RtArgs a)
{
    const SlabDev &S = *a.slab;
    if (!rt_active(S, a.steps[0])) return;
    const int nb = S.nb, nrc = S.rt_nrx * S.rt_nry, R = S.rt_R, nord = S.rt_nord, ncd = S.rt_ncd;
    const double dtr = (double)S.rad_every * (double)S.dt;
    const double *wo = S.rt_ord + 2 * nord;
    double Apend = 0.0, kesc = 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrc; r += gridDim.x * blockDim.x) {
        const int rx = r % S.rt_nrx, ry = r / S.rt_nrx;
        const int ylo = S.ny > 1 ? ry * R : 0, yhi = S.ny > 1 ? ylo + R : 1;
        double chi[MAXB], ka[MAXB], emc = 0.0, W = 0.0;
        for (int b = 0; b < nb; ++b) { chi[b] = 0.0; ka[b] = 0.0; }
        for (int j = ylo; j < yhi; ++j)
            for (int i = rx * R; i < rx * R + R; ++i) {
                const int c = j * S.nx + i;
                emc += S.rt_emc[c];
                W += (double)S.rt_w[c];
                for (int b = 0; b < nb; ++b) {
                    chi[b] += (double)S.rt_chi[(size_t)c * nb + b];
                    ka[b] += ph_val(a.photons[S.ph_off + (size_t)c * nb + b]) - S.rt_npub[(size_t)r * nb + b];
                }
            }
        double A = 0.0;
        for (int b = 0; b < nb; ++b) {
            chi[b] /= ncd;
            ka[b] /= ncd;
            const double e = exp(-chi[b] * kCcmPerFs * dtr);
            for (int o = 0; o < nord; ++o) {
                const size_t q = ((size_t)o * nb + b) * nrc + r;
                const double f = S.rt_F[q];
                A += f * (1.0 - e) * ncd * (double)S.hv_b[b];
                S.rt_F[q] = f * e; S.rt_Gx[q] *= e; S.rt_Gy[q] *= e;
            }
        }
        Apend += A;
        const double dE = A - emc;
        if (dE != 0.0)
            for (int j = ylo; j < yhi; ++j)
                for (int i = rx * R; i < rx * R + R; ++i) {
                    const int c = j * S.nx + i;
                    S.rt_dE[c] += W > 0.0 ? dE * (double)S.rt_w[c] / W : dE / ncd;
                }
        for (int b = 0; b < nb; ++b) {
            if (ka[b] == 0.0) continue;
            if (nord > 1)
                for (int o = 1; o < nord; ++o) S.rt_F[((size_t)o * nb + b) * nrc + r] += ka[b] * wo[o];
            else
                kesc += ka[b] * ncd * (double)S.hv_b[b];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        Apend += __shfl_down_sync(0xffffffffu, Apend, o);
        kesc += __shfl_down_sync(0xffffffffu, kesc, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (Apend != 0.0) atomicAdd(&a.tally->rt_pend, Apend);
        if (kesc != 0.0) atomicAdd(&a.tally->ka_esc, kesc);
    }
}

// photon density of bin b entering x = 0 at time tau, height y (nm)
__device__ __forceinline__ double rt_src(const SlabDev &S, int b, double tau, double y)
{
    double I;
    if (S.shape == 1) I = fabs(tau - S.t_peak) <= 0.5 * S.fwhm ? S.I_peak : 0.0;
    else { const double d = (tau - S.t_peak) / S.fwhm; I = S.I_peak * exp(-4.0 * 0.6931471805599453 * d * d); }
    double n = I / (kCcmPerFs * 1e15 * (double)S.hv_b[b] * kQe) / S.nb;
    if (S.spot_sigma > 0.0 && S.ny > 1) {
        const double yc = y - 0.5 * S.ny * (double)S.dy;
        n *= exp(-0.5 * yc * yc / (S.spot_sigma * S.spot_sigma));
    }
    return n / S.n_ref;
}

constexpr int RT_GHOST = 64;      // inflow ghost nodes held (Courant numbers below 60)
constexpr int RT_THREADS = 256;

// One line per block: axis 0 along x (rows of the rad grid), axis 1 along
// y (columns, periodic).  Shared memory: the line's old values, slopes and
// transverse slopes, with inflow ghosts in front.
__global__ void k_rt_sweep(RtArgs a, int axis)
{
    extern __shared__ double rt_sm[];
    __shared__ double red[4][RT_THREADS / 32];
    const SlabDev &S = *a.slab;
    if (!rt_active(S, a.steps[0])) return;
    const int nb = S.nb, nord = S.rt_nord, nrx = S.rt_nrx, nry = S.rt_nry, nrc = nrx * nry;
    const int n = axis == 0 ? nrx : nry, nperp = axis == 0 ? nry : nrx;
    const int line = blockIdx.x;
    if (line >= nord * nb * nperp) return;
    const int o = line / (nb * nperp), b = (line / nperp) % nb, p = line % nperp;
    const double *ox = S.rt_ord, *oy = S.rt_ord + nord;
    const double dtr = (double)S.rad_every * (double)S.dt;
    const double dcell = (axis == 0 ? (double)S.dx : (double)S.dy) * S.rt_R;
    const double nu = kCnmPerFs * dtr * (axis == 0 ? ox[o] : oy[o]) / dcell;
    if (axis == 1 && nu == 0.0) return;
    const bool periodic = axis == 1;
    double *F = S.rt_F + ((size_t)o * nb + b) * nrc, *G = (axis == 0 ? S.rt_Gx : S.rt_Gy) + ((size_t)o * nb + b) * nrc;
    double *T = (axis == 0 ? S.rt_Gy : S.rt_Gx) + ((size_t)o * nb + b) * nrc;
    const size_t stride = axis == 0 ? 1 : (size_t)nrx, base = axis == 0 ? (size_t)p * nrx : (size_t)p;
    // shared: [RT_GHOST ghosts | n nodes] for f, g, t
    double *sf = rt_sm, *sg = rt_sm + RT_GHOST + n, *st = rt_sm + 2 * (RT_GHOST + n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sf[RT_GHOST + i] = F[base + i * stride];
        sg[RT_GHOST + i] = G[base + i * stride];
        st[RT_GHOST + i] = T[base + i * stride];
    }
    // inflow ghosts (the beam ordinate along x, nu > 0): the pulse at the
    // retarded time, slope by central difference of the same profile
    const bool beam_in = axis == 0 && o == 0 && nu > 0.0;
    const int m = (int)floor(fabs(nu));
    const int ng = beam_in ? min((int)floor(nu) + 3, RT_GHOST - 2) : 0;
    const double tprev = (double)a.steps[0] * (double)S.dt - dtr;
    const double y = ((double)p + 0.5) * (double)S.dy * S.rt_R;
    for (int q = threadIdx.x; q < RT_GHOST; q += blockDim.x) {
        double f = 0.0, g = 0.0;
        if (q < ng) {
            const int j = -1 - q;
            f = rt_src(S, b, tprev - (j + 0.5) * dcell / kCnmPerFs, y);
            g = 0.5 * (rt_src(S, b, tprev - (j + 1.5) * dcell / kCnmPerFs, y) -
                       rt_src(S, b, tprev - (j - 0.5) * dcell / kCnmPerFs, y));
        }
        sf[RT_GHOST - 1 - q] = f; sg[RT_GHOST - 1 - q] = g; st[RT_GHOST - 1 - q] = 0.0;
    }
    __syncthreads();
    // node j (any integer) of the old line: ghosts before 0 (nu > 0 inflow),
    // empty beyond the outflow face, wrapped when periodic
    auto node = [&](int j, double &f, double &g, double &t) {
        if (periodic) { j %= n; if (j < 0) j += n; f = sf[RT_GHOST + j]; g = sg[RT_GHOST + j]; t = st[RT_GHOST + j]; return; }
        if (j >= 0 && j < n) { f = sf[RT_GHOST + j]; g = sg[RT_GHOST + j]; t = st[RT_GHOST + j]; return; }
        if (nu > 0.0 && j < 0 && -j <= RT_GHOST) { f = sf[RT_GHOST + j]; g = sg[RT_GHOST + j]; t = 0.0; return; }
        f = 0.0; g = 0.0; t = 0.0;
    };
    double before = 0.0, after = 0.0, fin = 0.0, fout = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        before += sf[RT_GHOST + i];
        double fn, gn, tn;
        if (S.rt_scheme == 1) {
            const double fr = fabs(nu) - m;
            const int sg1 = nu >= 0.0 ? 1 : -1;
            double v0, v1, d0, d1;
            node(i - sg1 * m, v0, d0, d1);
            node(i - sg1 * (m + 1), v1, d0, d1);
            fn = (1.0 - fr) * v0 + fr * v1;
            gn = 0.0; tn = 0.0;
        } else {
            const double xd = (double)i - nu;
            const int k = (int)floor(xd);
            const double t = xd - k, t2 = t * t, t3 = t2 * t;
            double fa, ga, ta, fb, gb, tb;
            node(k, fa, ga, ta);
            node(k + 1, fb, gb, tb);
            fn = (2 * t3 - 3 * t2 + 1) * fa + (t3 - 2 * t2 + t) * ga + (-2 * t3 + 3 * t2) * fb + (t3 - t2) * gb;
            gn = (6 * t2 - 6 * t) * fa + (3 * t2 - 4 * t + 1) * ga + (-6 * t2 + 6 * t) * fb + (3 * t2 - 2 * t) * gb;
            tn = (1.0 - t) * ta + t * tb;
        }
        F[base + i * stride] = fn; G[base + i * stride] = gn; T[base + i * stride] = tn;
        after += fn;
    }
    if (!periodic) {
        // contents crossing the faces by the split rule: source node j's
        // content goes (1 - fr) to j + m and fr to j + m + 1 (mirrored)
        const double fr = fabs(nu) - m;
        const int sg1 = nu >= 0.0 ? 1 : -1;
        for (int j = -(m + 1) + (int)threadIdx.x; j < n + m + 1; j += blockDim.x) {
            if ((sg1 > 0 && j >= n) || (sg1 < 0 && j < 0)) continue;
            double v, d0, d1;
            node(j, v, d0, d1);
            if (v == 0.0) continue;
            const bool in_src = j < 0 || j >= n;
            const int dd[2] = {j + sg1 * m, j + sg1 * (m + 1)};
            const double part[2] = {(1.0 - fr) * v, fr * v};
            for (int q = 0; q < 2; ++q) {
                const bool inside = dd[q] >= 0 && dd[q] < n, far = sg1 > 0 ? dd[q] >= n : dd[q] < 0;
                if (in_src && (inside || far)) fin += part[q];
                if (far) fout += part[q];
            }
        }
    }
    double v4[4] = {before, after, fin, fout};
    for (int q = 0; q < 4; ++q) {
        double v = v4[q];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s4[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int q = 0; q < 4; ++q) s4[q] += red[q][w];
        const double unit = (double)S.rt_ncd * (double)S.hv_b[b];
        const double gain = s4[1] - s4[0] - s4[2] + s4[3];
        if (gain != 0.0) atomicAdd(&a.tally->rt_num, gain * unit);
        if (s4[2] != 0.0) atomicAdd(&a.tally->inc, s4[2] * unit);
        if (s4[3] != 0.0) atomicAdd(nu > 0.0 ? &a.tally->trans : &a.tally->back, s4[3] * unit);
    }
}

__global__ void k_rt_publish(RtArgs a)
{
    const SlabDev &S = *a.slab;
    if (!rt_active(S, a.steps[0])) return;
    const int nb = S.nb, nrc = S.rt_nrx * S.rt_nry, R = S.rt_R, nord = S.rt_nord;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < S.ncell; c += gridDim.x * blockDim.x) {
        const int i = c % S.nx, j = c / S.nx;
        const int r = (S.ny > 1 ? (j / R) * S.rt_nrx : 0) + i / R;
        const bool first = i % R == 0 && (S.ny == 1 || j % R == 0);
        for (int b = 0; b < nb; ++b) {
            double v = 0.0;
            for (int o = 0; o < nord; ++o) v += S.rt_F[((size_t)o * nb + b) * nrc + r];
            const real hi = (real)v, lo = (real)(v - (double)hi);
            a.photons[S.ph_off + (size_t)c * nb + b] = ph2{hi, lo};
            // the value the cells hold (the pair rounds v to ~48 bits), so that
            // only what the cells add to their bins counts as emission
            if (first) S.rt_npub[(size_t)r * nb + b] = (double)hi + (double)lo;
        }
    }
}

// photon energy in transport mode: the field, plus the photons the cells
// added to their bins since it was published
__global__ void k_rt_energy(const SlabDev *slab, const ph2 *photons, double *out)
{
    const SlabDev &S = *slab;
    const int nb = S.nb, nrc = S.rt_nrx * S.rt_nry, R = S.rt_R;
    const size_t nf = (size_t)S.rt_nord * nb * nrc;
    double e = 0.0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nf; q += (size_t)gridDim.x * blockDim.x)
        e += S.rt_F[q] * S.rt_ncd * (double)S.hv_b[(q / nrc) % nb];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < S.ncell; c += gridDim.x * blockDim.x) {
        const int i = c % S.nx, j = c / S.nx;
        const int r = (S.ny > 1 ? (j / R) * S.rt_nrx : 0) + i / R;
        for (int b = 0; b < nb; ++b)
            e += (ph_val(photons[S.ph_off + (size_t)c * nb + b]) - S.rt_npub[(size_t)r * nb + b]) * (double)S.hv_b[b];
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0 && e != 0.0) atomicAdd(out, e);
}

}  // namespace pic
