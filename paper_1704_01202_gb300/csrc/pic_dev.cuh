// Device building blocks of the GB300 collisional-PIC step: constants,
// counter-based random numbers, atomic-structure rules, cross sections,
// continuum lowering, binary collision kinematics and the Boris rotation.
// Every function here is an independent implementation from the paper's
// statement of the method (and the published algorithms it cites).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pic {

// ---------------- physical constants (CODATA 2018) ----------------
constexpr double kPi = 3.141592653589793;
constexpr float kPiF = 3.14159265f;
constexpr double kCcmPerFs = 2.99792458e-5;     // c in cm/fs
constexpr double kCnmPerFs = 299.792458;        // c in nm/fs
constexpr double kMeC2 = 510998.95;             // eV
constexpr double kReCm = 2.8179403262e-13;      // classical electron radius
constexpr double kQe = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMeKg = 9.1093837015e-31;
constexpr double kCms = 299792458.0;
constexpr double kHbarCeVnm = 197.3269804;
constexpr float kPminEv = 1.0f;                 // floor of a lowered binding

constexpr int NS = 5;           // 1s 2s 2p 3s 3p
constexpr int NZ = 14;          // charge states 0..13
constexpr int ZNUC = 13;
constexpr int MAXB = 8;         // photon bins

// Philox stream purposes (counter word 3)
enum : uint32_t { PU_PAIR_E = 1, PU_PAIR_I = 2, PU_COLL_EE = 3, PU_COLL_EI = 4,
                  PU_COLL_IE = 5, PU_ION = 6, PU_PHOTO_A = 7, PU_PHOTO_B = 8, PU_DECAY = 9,
                  PU_THERM = 10 };
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
    float lotz_a[NS], lotz_b[NS], lotz_c[NS];
    float E_bind[NZ][NS];
    float tauK[NZ][2], omegaK[NZ][2], E_Ka[NZ];
};
// equation of state Zbar(n_i, T_e), read once per cell
constexpr int EOS_MAX_T = 1024, EOS_MAX_N = 16;
struct EosTable {
    int n_T, n_n;
    float T[EOS_MAX_T], n[EOS_MAX_N];
    float Z[EOS_MAX_N * EOS_MAX_T];
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
    float dx, dy, dt;
    float w_ion, m_ion, E_bulk, coulomb_log;
    float mur;              // first-order Mur coefficient
    float cf;               // speed of the Yee update, nm/fs (c, or the largest speed dt resolves)
    double n_ref;           // cm^-3
    double kappa_J;         // J coupling of the normalized field equations
    float nref_f, kappa_f;  // the same in single precision for the kernels
    double I_peak, fwhm, t_peak, spot_sigma;
    unsigned long long seed;
    float hv_b[MAXB];
    float sig_b[NS][MAXB];
    float bin_hw;
};

struct SlabTally {
    double ion, ka_esc, esc, inc, trans;
    unsigned long long cnt[NCOUNT];
};

// photon number per cell and bin, stored as a double-float pair
struct ph2 { float hi, lo; };

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

// uniform in (0,1): top 24 bits, centred; exact in float and double
__device__ __forceinline__ float u01(uint32_t x) { return ((float)(x >> 8) + 0.5f) * (1.0f / 16777216.0f); }

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

__device__ __forceinline__ float lowered_binding(const Tables &T, int z, int s, float dE)
{
    float p = T.E_bind[z][s] - dE;
    return p > kPminEv ? p : kPminEv;
}

// energy to remove the outermost electron of (Z, nK), lowered by dE
__device__ __forceinline__ float removal_energy(const Tables &T, int Z, int nK, float dE)
{
    int s = outer_shell(ZNUC - Z, nK);
    return s < 0 ? 0.0f : lowered_binding(T, Z, s, dE);
}

// ---------------- continuum lowering (Sec. V) ----------------
// Eq. 4 (Ecker-Kroll, dense branch, C = 1) and Eq. 5 (Stewart-Pyatt with
// T_i = T_e and z* = Zbar).  Densities cm^-3, T eV, result eV.  Single
// precision: once per cell and charge state.
__device__ __forceinline__ float ipd_shift(int model, int z, float n_e, float n_i, float T_e, float zbar)
{
    const float e2_4pe0_eVnm = (float)(kQe / (4.0 * kPi * kEps0) * 1e9);   // e^2/(4 pi eps0) in eV nm
    if (model == 1) {
        float n = (n_e + n_i) * 1e-21f;                  // nm^-3
        if (n <= 0.0f) return 0.0f;
        float r = cbrtf(3.0f / (4.0f * kPiF * n));       // nm
        return (z + 1) * e2_4pe0_eVnm / r;
    }
    if (model == 2) {
        if (T_e <= 0.0f || n_e <= 0.0f) return 0.0f;
        // lambda_D in nm: eps0 T / (e n_e (Zbar+1)), T in eV, n in nm^-3
        const float eps0_over_e = (float)(kEps0 / kQe * 1e-9);      // lambda^2 [nm^2] = this * T[eV] / n[nm^-3]
        float lam = sqrtf(eps0_over_e * T_e / (n_e * 1e-21f * (zbar + 1.0f)));
        float K = (z + 1) * e2_4pe0_eVnm / (lam * T_e);
        return T_e / (2.0f * (zbar + 1.0f)) * (powf(3.0f * (zbar + 1.0f) * K + 1.0f, 2.0f / 3.0f) - 1.0f);
    }
    return 0.0f;
}

// Coulomb logarithm stand-in: ln(lambda_D / b_min), b_min = max(classical
// closest approach, de Broglie length at 3T), floored at 2
__device__ __forceinline__ float coulomb_log(float n_e, float T_e, float zbar)
{
    if (n_e <= 0.0f || T_e <= 0.0f) return 2.0f;
    const float eps0_over_e = (float)(kEps0 / kQe * 1e-9);
    const float e2_4pe0_eVnm = (float)(kQe / (4.0 * kPi * kEps0) * 1e9);
    float lam = sqrtf(eps0_over_e * T_e / (n_e * 1e-21f));
    float zz = zbar > 1.0f ? zbar : 1.0f;
    float bcl = zz * e2_4pe0_eVnm / (3.0f * T_e);
    float bqm = (float)kHbarCeVnm / (2.0f * sqrtf(3.0f * T_e * (float)kMeC2));
    float L = logf(lam / (bcl > bqm ? bcl : bqm));
    return L > 2.0f ? L : 2.0f;
}

// ---------------- double-float sums ----------------
// Cell sums in a pair of floats (hi + lo, Knuth's TwoSum), ~44-bit
// precision on the FP32 pipes: GB300 has very little FP64 throughput.
struct dd { float hi, lo; };

__device__ __forceinline__ dd dd_add(dd a, dd b)
{
    float s = a.hi + b.hi;
    float bv = s - a.hi;
    float e = (a.hi - (s - bv)) + (b.hi - bv);
    e += a.lo + b.lo;
    float h = s + e;
    return dd{h, e - (h - s)};
}
__device__ __forceinline__ dd dd_addf(dd a, float b) { return dd_add(a, dd{b, 0.0f}); }
__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ float dd_f(dd a) { return a.hi + a.lo; }
__device__ __forceinline__ dd dd_zero() { return dd{0.0f, 0.0f}; }
__device__ __forceinline__ bool dd_le(dd a, dd b) { dd d = dd_sub(b, a); return d.hi > 0.0f || (d.hi == 0.0f && d.lo >= 0.0f); }

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
__device__ __forceinline__ float eos_lookup(const EosTable &T, float n, float t)
{
    auto locate = [](const float *g, int m, float x, int &i0) -> float {
        if (m == 1 || x <= g[0]) { i0 = 0; return 0.0f; }
        if (x >= g[m - 1]) { i0 = m - 2; return 1.0f; }
        int lo = 0, hi = m - 1;
        while (hi - lo > 1) { int md = (lo + hi) >> 1; if (g[md] <= x) lo = md; else hi = md; }
        i0 = lo;
        return (x - g[lo]) / (g[lo + 1] - g[lo]);
    };
    int a, b;
    float fa = locate(T.n, T.n_n, n, a), fb = locate(T.T, T.n_T, t, b);
    int a1 = T.n_n > 1 ? a + 1 : a, b1 = T.n_T > 1 ? b + 1 : b;
    const float *Z = T.Z;
    float z00 = Z[a * T.n_T + b], z01 = Z[a * T.n_T + b1], z10 = Z[a1 * T.n_T + b], z11 = Z[a1 * T.n_T + b1];
    return (1 - fa) * ((1 - fb) * z00 + fb * z01) + fa * ((1 - fb) * z10 + fb * z11);
}

// ---------------- kinematics ----------------
// kinetic energy in units of m c^2 (gamma - 1 = u^2 / (gamma + 1))
__device__ __forceinline__ float gm1(float ux, float uy, float uz)
{
    float u2 = ux * ux + uy * uy + uz * uz;
    return u2 / (sqrtf(1.0f + u2) + 1.0f);
}

// Multiply the kinetic energy of u by f = 1 - delta, direction kept.  The
// factor is carried as delta and 1 - |u'|/|u| is formed without
// cancellation, so small corrections are not lost to FP32 rounding of f.
__device__ __forceinline__ void scale_kinetic(float &ux, float &uy, float &uz, float delta)
{
    float g1 = gm1(ux, uy, uz);
    if (g1 == 0.0f || delta == 0.0f) return;
    float b = delta * g1 / (2.0f + g1);
    float x = delta + b - delta * b;                   // 1 - (|u'|/|u|)^2
    float d = x / (1.0f + sqrtf(1.0f - x));            // 1 - |u'|/|u|
    ux -= ux * d; uy -= uy * d; uz -= uz * d;
}

// One binary collision: Takizuka-Abe deflection tan(theta/2) ~ N(0, var),
// var = 2 pi (qa qb)^2 r_e^2 c n lnL dt / (mu^2 beta_rel^3), applied as a
// rotation of the centre-of-momentum momentum; weighted acceptance
// min(1, w_other / w_self).  Masses in m_e, u in units of m c of each.
__device__ __noinline__ bool binary_collision(float3 &ua, float3 &ub, float ma, float mb, float qa, float qb,
                                                 float wa, float wb, float n_l, float lnL, float dtc,
                                                 float r0, float r1, float r2, float r3)
{
    if (qa == 0.0f || qb == 0.0f) return false;
    // divisions by the same quantity are done once, as a reciprocal
    float ga = sqrtf(1.0f + ua.x * ua.x + ua.y * ua.y + ua.z * ua.z);
    float gb = sqrtf(1.0f + ub.x * ub.x + ub.y * ub.y + ub.z * ub.z);
    const float iga = 1.0f / ga, igb = 1.0f / gb;
    float dvx = ua.x * iga - ub.x * igb, dvy = ua.y * iga - ub.y * igb, dvz = ua.z * iga - ub.z * igb;
    float vrel = sqrtf(dvx * dvx + dvy * dvy + dvz * dvz);
    if (vrel < 1e-10f) return false;
    float mu = ma * mb / (ma + mb);
    // constant part 2 pi r_e^2 c in cm^3/fs, evaluated in double once
    const float k0 = (float)(2.0 * kPi * kReCm * kReCm * kCcmPerFs);
    float q2 = qa * qb;
    float var = k0 * q2 * q2 * n_l * lnL * dtc / (mu * mu * vrel * vrel * vrel);
    float delta = sqrtf(var) * sqrtf(-2.0f * logf(r0)) * cospif(2.0f * r1);
    float sphi, cphi;
    sincospif(2.0f * r2, &sphi, &cphi);

    float pax = ma * ua.x, pay = ma * ua.y, paz = ma * ua.z;
    float Ea = ma * ga, Eb = mb * gb, E = Ea + Eb;
    const float iE = 1.0f / E;
    float bx = (pax + mb * ub.x) * iE, by = (pay + mb * ub.y) * iE, bz = (paz + mb * ub.z) * iE;
    float b2 = bx * bx + by * by + bz * bz;
    float gc = rsqrtf(1.0f - b2);
    float h = gc * gc / (gc + 1.0f);
    float bp = bx * pax + by * pay + bz * paz;
    float c1 = h * bp - gc * Ea;
    float sx = pax + c1 * bx, sy = pay + c1 * by, sz = paz + c1 * bz;
    float p = sqrtf(sx * sx + sy * sy + sz * sz);
    if (p == 0.0f) return false;
    const float ip = 1.0f / p;
    float nx = sx * ip, ny = sy * ip, nz = sz * ip;
    float d2 = delta * delta;
    const float id2 = 1.0f / (1.0f + d2);
    float st = 2.0f * delta * id2, ct = (1.0f - d2) * id2;
    float e1x, e1y, e1z, e2x, e2y, e2z;
    float np = sqrtf(nx * nx + ny * ny);
    if (np > 0.0f) {
        const float inp = 1.0f / np;
        e1x = nx * nz * inp; e1y = ny * nz * inp; e1z = -np;
        e2x = -ny * inp; e2y = nx * inp; e2z = 0.0f;
    } else {
        e1x = 1.0f; e1y = 0.0f; e1z = 0.0f;
        e2x = 0.0f; e2y = 1.0f; e2z = 0.0f;
    }
    float qx = p * (ct * nx + st * cphi * e1x + st * sphi * e2x);
    float qy = p * (ct * ny + st * cphi * e1y + st * sphi * e2y);
    float qz = p * (ct * nz + st * cphi * e1z + st * sphi * e2z);
    float Eas = sqrtf(ma * ma + p * p), Ebs = sqrtf(mb * mb + p * p);
    float bq = bx * qx + by * qy + bz * qz;
    float ca = h * bq + gc * Eas, cb = -h * bq + gc * Ebs;
    float wm = wa > wb ? wa : wb;
    if (r3 < wb / wm) {
        const float ima = 1.0f / ma;
        ua.x = (qx + ca * bx) * ima; ua.y = (qy + ca * by) * ima; ua.z = (qz + ca * bz) * ima;
    }
    if (r3 < wa / wm) {
        const float imb = 1.0f / mb;
        ub.x = (-qx + cb * bx) * imb; ub.y = (-qy + cb * by) * imb; ub.z = (-qz + cb * bz) * imb;
    }
    return true;
}

// relativistic Boris: q/m in e/m_e, dt fs, normalized fields
__device__ __forceinline__ void boris(float &ux, float &uy, float &uz, float ex, float ey, float ez,
                                      float bx, float by, float bz, float qm, float dt)
{
    float h = 0.5f * qm * dt;
    float mx = ux + h * ex, my = uy + h * ey, mz = uz + h * ez;
    float ig = rsqrtf(1.0f + mx * mx + my * my + mz * mz);
    float tx = h * bx * ig, ty = h * by * ig, tz = h * bz * ig;
    float t2 = tx * tx + ty * ty + tz * tz;
    float s = 2.0f / (1.0f + t2);
    float px = mx + my * tz - mz * ty, py = my + mz * tx - mx * tz, pz = mz + mx * ty - my * tx;
    float qx = mx + (py * tz - pz * ty) * s, qy = my + (pz * tx - px * tz) * s, qz = mz + (px * ty - py * tx) * s;
    ux = qx + h * ex; uy = qy + h * ey; uz = qz + h * ez;
}

// isotropic momentum of kinetic energy ke (eV) for an electron
__device__ __forceinline__ float3 iso_momentum(float ke, float rc, float rp)
{
    float x = ke / (float)kMeC2;
    float um = sqrtf(x * (2.0f + x));
    float ct = 2.0f * rc - 1.0f;
    float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    float sp, cp;
    sincosf(2.0f * kPiF * rp, &sp, &cp);
    return make_float3(um * st * cp, um * st * sp, um * ct);
}

}  // namespace pic
