// Device building blocks of the GB300 collisional-PIC step: constants,
// counter-based random numbers, atomic-structure rules, cross sections,
// continuum lowering, binary collision kinematics and the Boris rotation.
// Every function here is an independent implementation from the paper's
// statement of the method (and the published algorithms it cites).
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace pic {

// ---------------- arithmetic type ----------------
// The library is built twice from these sources: the production build keeps
// particle state and arithmetic in FP32 (real = float); with PIC_FP64 the
// same kernels run in FP64 (real = double), a check of the device logic
// against the FP64 oracle free of single-precision rounding.  RF(x) is the
// literal x in the build's type; the r_* names are the math functions of
// that type (the FP32 build keeps its fast variants where it uses them).
#ifdef PIC_FP64
typedef double real;
struct __align__(32) real4 { double x, y, z, w; };
struct __align__(16) real2 { double x, y; };
struct real3 { double x, y, z; };
#define RF(x) (x)
#define r_sqrt sqrt
#define r_rsqrt rsqrt
#define r_log log
#define r_flog log
#define r_fexp exp
#define r_cospi cospi
#define r_sincospi sincospi
#define r_sincos sincos
#define r_cos cos
#define r_fmax fmax
#define r_fmin fmin
#define r_fabs fabs
#define r_floor floor
#define r_trunc trunc
#define r_cbrt cbrt
#define r_pow pow
#define r_fma fma
#else
typedef float real;
typedef float4 real4;
typedef float2 real2;
typedef float3 real3;
#define RF(x) x##f
#define r_sqrt sqrtf
#define r_rsqrt rsqrtf
#define r_log logf
#define r_flog __logf
#define r_fexp __expf
#define r_cospi cospif
#define r_sincospi sincospif
#define r_sincos sincosf
#define r_cos cosf
#define r_fmax fmaxf
#define r_fmin fminf
#define r_fabs fabsf
#define r_floor floorf
#define r_trunc truncf
#define r_cbrt cbrtf
#define r_pow powf
#define r_fma fmaf
#endif
__host__ __device__ __forceinline__ real4 make_real4(real x, real y, real z, real w)
{
    real4 r; r.x = x; r.y = y; r.z = z; r.w = w; return r;
}
__host__ __device__ __forceinline__ real3 make_real3(real x, real y, real z)
{
    real3 r; r.x = x; r.y = y; r.z = z; return r;
}
__host__ __device__ __forceinline__ real2 make_real2(real x, real y)
{
    real2 r; r.x = x; r.y = y; return r;
}

// Integer payloads kept in the real-typed words of a particle record: an
// electron's 64-bit id in (z, w) of the second word as two 32-bit halves
// (FP32) or in z (FP64); an ion's 32-bit id in z and its state in w.
__host__ __device__ __forceinline__ real bits_real(uint64_t b)
{
    real r;
#ifdef PIC_FP64
    memcpy(&r, &b, 8);
#else
    uint32_t v = (uint32_t)b;
    memcpy(&r, &v, 4);
#endif
    return r;
}
__host__ __device__ __forceinline__ uint64_t real_bits(real r)
{
#ifdef PIC_FP64
    uint64_t b;
    memcpy(&b, &r, 8);
    return b;
#else
    uint32_t v;
    memcpy(&v, &r, 4);
    return v;
#endif
}
__host__ __device__ __forceinline__ uint64_t rec_eid(const real4 &p1)
{
#ifdef PIC_FP64
    return real_bits(p1.z);
#else
    return real_bits(p1.z) | (real_bits(p1.w) << 32);
#endif
}
__host__ __device__ __forceinline__ real4 rec_e1(real uz, real w, uint64_t id)
{
#ifdef PIC_FP64
    return make_real4(uz, w, bits_real(id), RF(0.0));
#else
    return make_real4(uz, w, bits_real(id & 0xffffffffu), bits_real(id >> 32));
#endif
}
__host__ __device__ __forceinline__ uint32_t rec_iid(const real4 &p1) { return (uint32_t)real_bits(p1.z); }
__host__ __device__ __forceinline__ int rec_ist(const real4 &p1) { return (int)(uint32_t)real_bits(p1.w); }
__host__ __device__ __forceinline__ real4 rec_i1(real uz, real zf, uint32_t id, int st)
{
    return make_real4(uz, zf, bits_real(id), bits_real((uint32_t)st));
}
// largest value below 1 (positions inside a cell stay < 1)
constexpr real kBelow1 = sizeof(real) == 8 ? (real)0.99999999999999989 : (real)0.99999994f;

// ---------------- physical constants (CODATA 2018) ----------------
constexpr double kPi = 3.141592653589793;
constexpr real kPiR = (real)kPi;
constexpr double kCcmPerFs = 2.99792458e-5;     // c in cm/fs
constexpr double kCnmPerFs = 299.792458;        // c in nm/fs
constexpr double kMeC2 = 510998.95;             // eV
constexpr double kReCm = 2.8179403262e-13;      // classical electron radius
constexpr double kQe = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMeKg = 9.1093837015e-31;
constexpr double kCms = 299792458.0;
constexpr double kHbarCeVnm = 197.3269804;
constexpr real kPminEv = RF(1.0);                 // floor of a lowered binding

constexpr int NS = 5;           // 1s 2s 2p 3s 3p
constexpr int NZ = 14;          // charge states 0..13
constexpr int ZNUC = 13;
constexpr int MAXB = 8;         // photon bins

// Philox stream purposes (counter word 3)
enum : uint32_t { PU_PAIR_E = 1, PU_PAIR_I = 2, PU_COLL_EE = 3, PU_COLL_EI = 4,
                  PU_COLL_IE = 5, PU_ION = 6, PU_PHOTO_A = 7, PU_PHOTO_B = 8, PU_DECAY = 9,
                  PU_THERM = 10, PU_SEED_E = 11, PU_SEED_I = 12 };
// kinds of created electrons: id high word = ((step + 1) << 2) | kind
enum : uint32_t { KIND_IMPACT = 1, KIND_PHOTO = 2, KIND_AUGER = 3 };

// counters in the per-slab tally
enum { C_ION, C_ION_REJ, C_REC, C_PH0, C_PH1, C_PH2, C_PH3, C_PH4, C_PART, C_AUG, C_KA,
       C_PGT1, C_ESC_E, C_ESC_I, C_EE, C_EI, NCOUNT };

// device error word bits
enum : int { ERR_CELL_OVERFLOW = 1, ERR_CAPACITY = 2, ERR_NUMERIC = 4, ERR_NEW_OVERFLOW = 8 };

// ---------------- atomic tables (shared by all slabs) ----------------
// small tables indexed per particle (copied to shared memory by kernels)
struct Tables {
    real lotz_a[NS], lotz_b[NS], lotz_c[NS];
    real E_bind[NZ][NS];
    real tauK[NZ][2], omegaK[NZ][2], E_Ka[NZ];
};
// equation of state Zbar(n_i, T_e), read once per cell
constexpr int EOS_MAX_T = 1024, EOS_MAX_N = 16;
struct EosTable {
    int n_T, n_n;
    real T[EOS_MAX_T], n[EOS_MAX_N];
    real Z[EOS_MAX_N * EOS_MAX_T];
};

// ---------------- per-slab description ----------------
struct SlabDev {
    int active;             // 0: retired / never admitted (its particles are dropped)
    int nx, ny, cell0, ncell;
    int fld_off;            // first grid point of this slab in the field arrays
    int ph_off;             // first photon entry (cells * nb)
    int nb;                 // photon bins in use (0: no pulse)
    int rad_every;
    unsigned flags;
    int ipd;
    int nsub;               // field updates per step (1: the field speed below is resolved by dt)
    int shape;
    int budget_e;           // electron slots the slab may hold after a step (0: only the context's capacity)
    real dx, dy, dt;
    real w_ion, m_ion, E_bulk, coulomb_log;
    real mur;              // first-order Mur coefficient
    real cf;               // speed of the Yee update, nm/fs (c, or the largest speed dt resolves)
    double n_ref;           // cm^-3
    double kappa_J;         // J coupling of the normalized field equations
    real nref_f, kappa_f;  // the same in single precision for the kernels
    double I_peak, fwhm, t_peak, spot_sigma;
    unsigned long long seed;
    real hv_b[MAXB];
    real sig_b[NS][MAXB];
    real bin_hw;
    // radiation transport mode (single-slab contexts; rt = 0: the ballistic
    // march): discrete ordinates on a rad grid rt_R times coarser
    int rt, rt_R, rt_nrx, rt_nry, rt_nord, rt_scheme, rt_ncd;
    double *rt_F, *rt_Gx, *rt_Gy;    // [nord][nb][nry][nrx] photon density (n_ref units), CIP slopes
    double *rt_npub;                 // [nrc][nb] densities published to the cells
    const double *rt_ord;            // [3][nord]: x and y direction cosines, share of isotropic emission
    float *rt_chi;                   // [ncell][nb] opacity (cm^-1), written on rad steps by the cell kernel
    double *rt_emc, *rt_dE;          // [ncell] photon energy the events took; energy due to the bulk electrons
    float *rt_w;                     // [ncell] electron weight after the cell's rad step
};

struct SlabTally {
    double ion, ka_esc, esc, inc, trans;
    // radiation transport: energy leaving through x = 0, the transport
    // scheme's own gain, energy owed between the field and the electrons
    double back, rt_num, rt_pend;
    unsigned long long cnt[NCOUNT];
};

// photon number per cell and bin, stored as a pair hi + lo of the build type
struct ph2 { real hi, lo; };

// ---------------- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ----------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// uniform in (0,1): top 23 bits, centred, (k + 1/2) 2^-23: at most 24
// significant bits, so the same value in float and double
__device__ __forceinline__ real u01(uint32_t x) { return ((real)(x >> 9) + RF(0.5)) * (RF(1.0) / RF(8388608.0)); }

__device__ __forceinline__ U4 draw(unsigned long long seed, unsigned long long id, uint32_t step, uint32_t purpose)
{
    return philox((uint32_t)id, (uint32_t)(id >> 32), step, purpose, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// ---------------- atomic structure ----------------
__device__ __forceinline__ int cap_of(int s) { return (s == 2 || s == 4) ? 6 : 2; }

// lowest-energy filling of nb electrons with nk extra K vacancies; false if impossible
__device__ __forceinline__ bool occupancy(int nb, int nk, int occ[NS])
{
    int k = (nb < 2 ? nb : 2) - nk;
    if (nb < 0 || nk < 0 || k < 0) return false;
    occ[0] = k;
    int rest = nb - k;
#pragma unroll
    for (int s = 1; s < NS; ++s) {
        int t = rest < cap_of(s) ? rest : cap_of(s);
        occ[s] = t;
        rest -= t;
    }
    return rest == 0;
}

__device__ __forceinline__ int outer_shell(int nb, int nk)
{
    int occ[NS];
    if (!occupancy(nb, nk, occ)) return -1;
    for (int s = NS - 1; s >= 0; --s)
        if (occ[s] > 0) return s;
    return -1;
}

// (Z, nK) after one electron of subshell s leaves
__device__ __forceinline__ void lose_electron(int &Z, int &nK, int s)
{
    int nb = ZNUC - Z, occ[NS];
    occupancy(nb, nK, occ);
    int kocc = occ[0] - (s == 0 ? 1 : 0);
    int nb2 = nb - 1;
    Z += 1;
    nK = (nb2 < 2 ? nb2 : 2) - kocc;
}

__device__ __forceinline__ real lowered_binding(const Tables &T, int z, int s, real dE)
{
    real p = T.E_bind[z][s] - dE;
    return p > kPminEv ? p : kPminEv;
}

// energy to remove the outermost electron of (Z, nK), lowered by dE
__device__ __forceinline__ real removal_energy(const Tables &T, int Z, int nK, real dE)
{
    int s = outer_shell(ZNUC - Z, nK);
    return s < 0 ? RF(0.0) : lowered_binding(T, Z, s, dE);
}

// ---------------- continuum lowering (Sec. V) ----------------
// Eq. 4 (Ecker-Kroll, dense branch, C = 1) and Eq. 5 (Stewart-Pyatt with
// T_i = T_e and z* = Zbar).  Densities cm^-3, T eV, result eV.  Single
// precision: once per cell and charge state.
__device__ __forceinline__ real ipd_shift(int model, int z, real n_e, real n_i, real T_e, real zbar)
{
    const real e2_4pe0_eVnm = (real)(kQe / (4.0 * kPi * kEps0) * 1e9);   // e^2/(4 pi eps0) in eV nm
    if (model == 1) {
        real n = (n_e + n_i) * RF(1e-21);                  // nm^-3
        if (n <= RF(0.0)) return RF(0.0);
        real r = r_cbrt(RF(3.0) / (RF(4.0) * kPiR * n));       // nm
        return (z + 1) * e2_4pe0_eVnm / r;
    }
    if (model == 2) {
        if (T_e <= RF(0.0) || n_e <= RF(0.0)) return RF(0.0);
        // lambda_D in nm: eps0 T / (e n_e (Zbar+1)), T in eV, n in nm^-3
        const real eps0_over_e = (real)(kEps0 / kQe * 1e-9);      // lambda^2 [nm^2] = this * T[eV] / n[nm^-3]
        real lam = r_sqrt(eps0_over_e * T_e / (n_e * RF(1e-21) * (zbar + RF(1.0))));
        real K = (z + 1) * e2_4pe0_eVnm / (lam * T_e);
        return T_e / (RF(2.0) * (zbar + RF(1.0))) * (r_pow(RF(3.0) * (zbar + RF(1.0)) * K + RF(1.0), RF(2.0) / RF(3.0)) - RF(1.0));
    }
    return RF(0.0);
}

// Coulomb logarithm stand-in: ln(lambda_D / b_min), b_min = max(classical
// closest approach, de Broglie length at 3T), floored at 2
__device__ __forceinline__ real coulomb_log(real n_e, real T_e, real zbar)
{
    if (n_e <= RF(0.0) || T_e <= RF(0.0)) return RF(2.0);
    const real eps0_over_e = (real)(kEps0 / kQe * 1e-9);
    const real e2_4pe0_eVnm = (real)(kQe / (4.0 * kPi * kEps0) * 1e9);
    real lam = r_sqrt(eps0_over_e * T_e / (n_e * RF(1e-21)));
    real zz = zbar > RF(1.0) ? zbar : RF(1.0);
    real bcl = zz * e2_4pe0_eVnm / (RF(3.0) * T_e);
    real bqm = (real)kHbarCeVnm / (RF(2.0) * r_sqrt(RF(3.0) * T_e * (real)kMeC2));
    real L = r_log(lam / (bcl > bqm ? bcl : bqm));
    return L > RF(2.0) ? L : RF(2.0);
}

// ---------------- double-float sums ----------------
// Cell sums in a pair of floats (hi + lo, Knuth's TwoSum), ~44-bit
// precision on the FP32 pipes: GB300 has very little FP64 throughput (in
// the FP64 build the pair is two doubles).
struct dd { real hi, lo; };

__device__ __forceinline__ dd dd_add(dd a, dd b)
{
    real s = a.hi + b.hi;
    real bv = s - a.hi;
    real e = (a.hi - (s - bv)) + (b.hi - bv);
    e += a.lo + b.lo;
    real h = s + e;
    return dd{h, e - (h - s)};
}
__device__ __forceinline__ dd dd_addf(dd a, real b) { return dd_add(a, dd{b, RF(0.0)}); }
__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ real dd_f(dd a) { return a.hi + a.lo; }
__device__ __forceinline__ dd dd_zero() { return dd{RF(0.0), RF(0.0)}; }
__device__ __forceinline__ bool dd_le(dd a, dd b) { dd d = dd_sub(b, a); return d.hi > RF(0.0) || (d.hi == RF(0.0) && d.lo >= RF(0.0)); }

// ---------------- Lotz cross section (Eq. 3) ----------------
// sigma(E) = sum_s a_s q_s ln(E / P_s) / (E P_s) [1 - b_s exp(-c_s (E / P_s - 1))]
// over the occupied subshells s with E > P_s (q_s electrons, P_s the lowered
// binding); the sum runs in the cell kernel with per-cell constants of P_s.
__device__ __forceinline__ int subshell_occ(int nb, int s)
{
    // electrons of subshell s in the lowest-energy configuration of nb bound
    // electrons (no K vacancy): 1s 2s 2p 3s 3p filled in order
    const int start = s == 0 ? 0 : s == 1 ? 2 : s == 2 ? 4 : s == 3 ? 10 : 12;
    const int t = nb - start;
    return t <= 0 ? 0 : (t < cap_of(s) ? t : cap_of(s));
}

// EOS table, bilinear, clamped
__device__ __forceinline__ real eos_lookup(const EosTable &T, real n, real t)
{
    auto locate = [](const real *g, int m, real x, int &i0) -> real {
        if (m == 1 || x <= g[0]) { i0 = 0; return RF(0.0); }
        if (x >= g[m - 1]) { i0 = m - 2; return RF(1.0); }
        int lo = 0, hi = m - 1;
        while (hi - lo > 1) { int md = (lo + hi) >> 1; if (g[md] <= x) lo = md; else hi = md; }
        i0 = lo;
        return (x - g[lo]) / (g[lo + 1] - g[lo]);
    };
    int a, b;
    real fa = locate(T.n, T.n_n, n, a), fb = locate(T.T, T.n_T, t, b);
    int a1 = T.n_n > 1 ? a + 1 : a, b1 = T.n_T > 1 ? b + 1 : b;
    const real *Z = T.Z;
    real z00 = Z[a * T.n_T + b], z01 = Z[a * T.n_T + b1], z10 = Z[a1 * T.n_T + b], z11 = Z[a1 * T.n_T + b1];
    return (1 - fa) * ((1 - fb) * z00 + fb * z01) + fa * ((1 - fb) * z10 + fb * z11);
}

// ---------------- kinematics ----------------
// kinetic energy in units of m c^2 (gamma - 1 = u^2 / (gamma + 1))
__device__ __forceinline__ real gm1(real ux, real uy, real uz)
{
    real u2 = ux * ux + uy * uy + uz * uz;
    return u2 / (r_sqrt(RF(1.0) + u2) + RF(1.0));
}

// Multiply the kinetic energy of u by f = 1 - delta, direction kept.  The
// factor is carried as delta and 1 - |u'|/|u| is formed without
// cancellation, so small corrections are not lost to FP32 rounding of f.
__device__ __forceinline__ void scale_kinetic(real &ux, real &uy, real &uz, real delta)
{
    real g1 = gm1(ux, uy, uz);
    if (g1 == RF(0.0) || delta == RF(0.0)) return;
    real b = delta * g1 / (RF(2.0) + g1);
    real x = delta + b - delta * b;                   // 1 - (|u'|/|u|)^2
    real d = x / (RF(1.0) + r_sqrt(RF(1.0) - x));            // 1 - |u'|/|u|
    ux -= ux * d; uy -= uy * d; uz -= uz * d;
}

// One binary collision: Takizuka-Abe deflection tan(theta/2) ~ N(0, var),
// var = 2 pi (qa qb)^2 r_e^2 c n lnL dt / (mu^2 beta_rel^3), applied as a
// rotation of the centre-of-momentum momentum; weighted acceptance
// min(1, w_other / w_self).  Masses in m_e, u in units of m c of each.
__device__ __noinline__ bool binary_collision(real3 &ua, real3 &ub, real ma, real mb, real qa, real qb,
                                                 real wa, real wb, real n_l, real lnL, real dtc,
                                                 real r0, real r1, real r2, real r3)
{
    if (qa == RF(0.0) || qb == RF(0.0)) return false;
    // divisions by the same quantity are done once, as a reciprocal
    real ga = r_sqrt(RF(1.0) + ua.x * ua.x + ua.y * ua.y + ua.z * ua.z);
    real gb = r_sqrt(RF(1.0) + ub.x * ub.x + ub.y * ub.y + ub.z * ub.z);
    const real iga = RF(1.0) / ga, igb = RF(1.0) / gb;
    real dvx = ua.x * iga - ub.x * igb, dvy = ua.y * iga - ub.y * igb, dvz = ua.z * iga - ub.z * igb;
    real vrel = r_sqrt(dvx * dvx + dvy * dvy + dvz * dvz);
    if (vrel < RF(1e-10)) return false;
    real mu = ma * mb / (ma + mb);
    // constant part 2 pi r_e^2 c in cm^3/fs, evaluated in double once
    const real k0 = (real)(2.0 * kPi * kReCm * kReCm * kCcmPerFs);
    real q2 = qa * qb;
    real var = k0 * q2 * q2 * n_l * lnL * dtc / (mu * mu * vrel * vrel * vrel);
    real delta = r_sqrt(var) * r_sqrt(-RF(2.0) * r_log(r0)) * r_cospi(RF(2.0) * r1);
    real sphi, cphi;
    r_sincospi(RF(2.0) * r2, &sphi, &cphi);

    real pax = ma * ua.x, pay = ma * ua.y, paz = ma * ua.z;
    real Ea = ma * ga, Eb = mb * gb, E = Ea + Eb;
    const real iE = RF(1.0) / E;
    real bx = (pax + mb * ub.x) * iE, by = (pay + mb * ub.y) * iE, bz = (paz + mb * ub.z) * iE;
    real b2 = bx * bx + by * by + bz * bz;
    real gc = r_rsqrt(RF(1.0) - b2);
    real h = gc * gc / (gc + RF(1.0));
    real bp = bx * pax + by * pay + bz * paz;
    real c1 = h * bp - gc * Ea;
    real sx = pax + c1 * bx, sy = pay + c1 * by, sz = paz + c1 * bz;
    real p = r_sqrt(sx * sx + sy * sy + sz * sz);
    if (p == RF(0.0)) return false;
    const real ip = RF(1.0) / p;
    real nx = sx * ip, ny = sy * ip, nz = sz * ip;
    real d2 = delta * delta;
    const real id2 = RF(1.0) / (RF(1.0) + d2);
    real st = RF(2.0) * delta * id2, ct = (RF(1.0) - d2) * id2;
    // azimuth frame (e1, e2) about n: on the z axis while n is at least 30
    // degrees from it, on the x axis otherwise (no division by a small
    // component, so FP32 rounding is not amplified near the poles)
    real e1x, e1y, e1z, e2x, e2y, e2z;
    const real np2 = nx * nx + ny * ny;
    if (np2 >= RF(0.25)) {
        const real np = r_sqrt(np2), inp = RF(1.0) / np;
        e1x = nx * nz * inp; e1y = ny * nz * inp; e1z = -np;
        e2x = -ny * inp; e2y = nx * inp; e2z = RF(0.0);
    } else {
        const real nq = r_sqrt(ny * ny + nz * nz), inq = RF(1.0) / nq;
        e2x = RF(0.0); e2y = nz * inq; e2z = -ny * inq;
        e1x = nq; e1y = -nx * ny * inq; e1z = -nx * nz * inq;
    }
    real qx = p * (ct * nx + st * cphi * e1x + st * sphi * e2x);
    real qy = p * (ct * ny + st * cphi * e1y + st * sphi * e2y);
    real qz = p * (ct * nz + st * cphi * e1z + st * sphi * e2z);
    real Eas = r_sqrt(ma * ma + p * p), Ebs = r_sqrt(mb * mb + p * p);
    real bq = bx * qx + by * qy + bz * qz;
    real ca = h * bq + gc * Eas, cb = -h * bq + gc * Ebs;
    real wm = wa > wb ? wa : wb;
    if (r3 < wb / wm) {
        const real ima = RF(1.0) / ma;
        ua.x = (qx + ca * bx) * ima; ua.y = (qy + ca * by) * ima; ua.z = (qz + ca * bz) * ima;
    }
    if (r3 < wa / wm) {
        const real imb = RF(1.0) / mb;
        ub.x = (-qx + cb * bx) * imb; ub.y = (-qy + cb * by) * imb; ub.z = (-qz + cb * bz) * imb;
    }
    return true;
}

// relativistic Boris: q/m in e/m_e, dt fs, normalized fields
__device__ __forceinline__ void boris(real &ux, real &uy, real &uz, real ex, real ey, real ez,
                                      real bx, real by, real bz, real qm, real dt)
{
    real h = RF(0.5) * qm * dt;
    real mx = ux + h * ex, my = uy + h * ey, mz = uz + h * ez;
    real ig = r_rsqrt(RF(1.0) + mx * mx + my * my + mz * mz);
    real tx = h * bx * ig, ty = h * by * ig, tz = h * bz * ig;
    real t2 = tx * tx + ty * ty + tz * tz;
    real s = RF(2.0) / (RF(1.0) + t2);
    real px = mx + my * tz - mz * ty, py = my + mz * tx - mx * tz, pz = mz + mx * ty - my * tx;
    real qx = mx + (py * tz - pz * ty) * s, qy = my + (pz * tx - px * tz) * s, qz = mz + (px * ty - py * tx) * s;
    ux = qx + h * ex; uy = qy + h * ey; uz = qz + h * ez;
}

// isotropic momentum of kinetic energy ke (eV) for an electron
__device__ __forceinline__ real3 iso_momentum(real ke, real rc, real rp)
{
    real x = ke / (real)kMeC2;
    real um = r_sqrt(x * (RF(2.0) + x));
    real ct = RF(2.0) * rc - RF(1.0);
    real st = r_sqrt(r_fmax(RF(0.0), RF(1.0) - ct * ct));
    real sp, cp;
    r_sincos(RF(2.0) * kPiR * rp, &sp, &cp);
    return make_real3(um * st * cp, um * st * sp, um * ct);
}

}  // namespace pic
