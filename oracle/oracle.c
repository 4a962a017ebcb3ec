/* FP64 CPU oracle of the per-step collisional PIC update for XFEL-heated
 * solid Al (Royle, Sentoku, Mancini, Paraschiv, Johzaki; PICLS).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline legs of the bench.  Plain, sequential per cell, written for
 * checking by eye against the paper, not for speed.  It shares no code with
 * the CUDA path.
 *
 * One step, in order (the paper leaves the order within a PIC step open;
 * Fig. 1 gives the radiation cycle):
 *   0. every rad_every-th step: photon march along +x (Sec. II, simplified
 *      to ballistic transport of the pulse, attenuated by photoionization)
 *   per cell, on the particles whose position lies in the cell:
 *   1. canonical random order of electrons and of ions (Philox keys)
 *   2. FP64 cell moments: densities, T_e = (2/3) E_ave (Sec. II), Zbar,
 *      continuum lowering (Sec. V, Eqs. 4, 5), Coulomb logarithm
 *   3. binary e-e then e-i collisions (Sec. IV, by citation: Takizuka-Abe
 *      pairing and angle, relativistic centre-of-momentum rotation)
 *   4. Lotz impact ionization with the cell-average probability and the
 *      constant-factor energy payment (Sec. IV, Eq. 3)
 *   5. EOS-clamped three-body recombination (Sec. IV)
 *   6. rad steps: subshell photoionization (Sec. III, Eq. 2, partial
 *      ionization) then K-vacancy decay with Auger/K-alpha branching
 *      (Sec. III)
 *   7. rad steps, only in the forced-thermalization variant (Sec. VI C):
 *      the cell's free electrons resampled from a Maxwellian at (2/3) E_ave,
 *      momentum and kinetic energy restored exactly
 *   then over all particles:
 *   8. relativistic Boris push, charge-conserving (Esirkepov) deposit
 *   9. Yee field update at the field speed the step resolves (see
 *      orc_field_speed) with the binomially smoothed current (see
 *      smooth_current), periodic in y, first-order Mur in x
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------- physical constants (CODATA 2018) ---------------- */
#define PI 3.14159265358979323846
static const double C_CM_FS = 2.99792458e-5;     /* speed of light, cm/fs */
static const double C_NM_FS = 299.792458;        /* nm/fs */
static const double ME_C2 = 510998.95;           /* eV */
static const double R_E_CM = 2.8179403262e-13;   /* classical electron radius */
static const double Q_E = 1.602176634e-19;       /* C */
static const double EPS0 = 8.8541878128e-12;     /* F/m */
static const double ME_KG = 9.1093837015e-31;      /* kg */
static const double C_SI = 299792458.0;          /* m/s */
static const double HBARC_EVNM = 197.3269804;    /* eV nm */
static const double P_MIN = 1.0;                 /* eV, floor of lowered binding */

/* Philox stream purposes (counter word 3) */
enum { PU_PAIR_E = 1, PU_PAIR_I = 2, PU_COLL_EE = 3, PU_COLL_EI = 4,
       PU_COLL_IE = 5, PU_ION = 6, PU_PHOTO_A = 7, PU_PHOTO_B = 8, PU_DECAY = 9,
       PU_THERM = 10 };
/* kinds of created electrons (high id word = ((step+1) << 2) | kind) */
enum { K_IMPACT = 1, K_PHOTO = 2, K_AUGER = 3 };

static const int SUB_CAP[ORC_NS] = {2, 2, 6, 2, 6};

/* ---------------- Philox4x32-10 (Salmon et al., SC'11) ---------------- */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in the open interval (0,1): the top 23 bits k, centred,
 * (k + 1/2) 2^-23.  Every such value has at most 24 significant bits, so
 * it is the same number in single and double precision (24 bits, (k + 1/2)
 * 2^-24, would need 25 bits for k >= 2^23 and round to k + 1 in single
 * precision, 1.0 at the top). */
double orc_u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

static void draw4(uint64_t seed, uint64_t id, uint32_t step, uint32_t purpose, double r[4])
{
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox(ctr, key, o);
    for (int k = 0; k < 4; ++k) r[k] = orc_u01(o[k]);
}

static uint64_t key64(uint64_t seed, uint64_t id, uint32_t step, uint32_t purpose)
{
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox(ctr, key, o);
    return ((uint64_t)o[0] << 32) | o[1];
}

/* ---------------- atomic structure helpers ---------------- */
/* Lowest-energy filling of nb bound electrons with nk extra K vacancies:
 * K holds min(nb,2)-nk, the rest fill 2s 2p 3s 3p in order (Sec. III: N_b
 * from the lowest-energy configuration; the K-vacancy count is the only
 * other state an ion carries). Returns 0 for an impossible state. */
int orc_occ(int nb, int nk, int occ[ORC_NS])
{
    int k = (nb < 2 ? nb : 2) - nk;
    if (nb < 0 || nk < 0 || k < 0) return 0;
    occ[0] = k;
    int rest = nb - k;
    for (int s = 1; s < ORC_NS; ++s) {
        int t = rest < SUB_CAP[s] ? rest : SUB_CAP[s];
        occ[s] = t;
        rest -= t;
    }
    return rest == 0;
}

static int outermost(int nb, int nk)
{
    int occ[ORC_NS];
    if (!orc_occ(nb, nk, occ)) return -1;
    for (int s = ORC_NS - 1; s >= 0; --s)
        if (occ[s] > 0) return s;
    return -1;
}

/* remove one electron of subshell s from (Z, nK): Z+1, K-vacancy count
 * recomputed so the remaining K occupancy is kept */
static void remove_electron(int *Z, int *nK, int s)
{
    int nb = 13 - *Z, occ[ORC_NS];
    orc_occ(nb, *nK, occ);
    int kocc = occ[0] - (s == 0 ? 1 : 0);
    int nb2 = nb - 1;
    *Z += 1;
    *nK = (nb2 < 2 ? nb2 : 2) - kocc;
}

/* IPD-lowered binding of subshell s in charge state z */
static double lowered(const orc_tables *t, int z, int s, double dE)
{
    double p = t->E_bind[z][s] - dE;
    return p > P_MIN ? p : P_MIN;
}

/* energy to remove the outermost electron of (Z, nK) */
static double ion_energy(const orc_tables *t, int Z, int nK, const double *dE)
{
    int s = outermost(13 - Z, nK);
    if (s < 0) return 0.0;
    return lowered(t, Z, s, dE[Z]);
}

/* ---------------- continuum lowering (Sec. V) ---------------- */
/* Eq. 4 (Ecker-Kroll, n > n_crit branch, C = 1) and Eq. 5 (Stewart-Pyatt,
 * T_i = T_e, z* = Zbar).  Densities in cm^-3, T in eV, result in eV. */
double orc_ipd(int model, int z, double n_e, double n_i, double T_e, double zbar)
{
    double e_4pe0 = Q_E / (4.0 * PI * EPS0);   /* V m */
    if (model == 1) {
        double n = (n_e + n_i) * 1e6;
        if (n <= 0.0) return 0.0;
        double r = cbrt(3.0 / (4.0 * PI * n));
        return (z + 1) * e_4pe0 / r;
    }
    if (model == 2) {
        if (T_e <= 0.0 || n_e <= 0.0) return 0.0;
        double lam = sqrt(EPS0 * T_e / (Q_E * n_e * 1e6 * (zbar + 1.0)));
        double K = (z + 1) * e_4pe0 / (lam * T_e);
        double zs = zbar;
        return T_e / (2.0 * (zs + 1.0)) * (pow(3.0 * (zs + 1.0) * K + 1.0, 2.0 / 3.0) - 1.0);
    }
    return 0.0;
}

/* ---------------- Lotz cross section (Eq. 3) ---------------- */
/* Charge state z in its lowest-energy configuration, every subshell binding
 * lowered by dE; a subshell adds nothing below its binding.  cm^2. */
double orc_lotz(const orc_tables *t, int z, double dE, double E)
{
    int occ[ORC_NS];
    if (z >= 13 || !orc_occ(13 - z, 0, occ)) return 0.0;
    double sig = 0.0;
    for (int s = 0; s < ORC_NS; ++s) {
        if (!occ[s]) continue;
        double P = lowered(t, z, s, dE);
        if (E <= P) continue;
        double x = E / P;
        sig += t->lotz_a[s] * occ[s] * log(x) / (E * P)
               * (1.0 - t->lotz_b[s] * exp(-t->lotz_c[s] * (x - 1.0)));
    }
    return sig;
}

/* Coulomb logarithm stand-in (the paper defers to its refs): ln(lambda_D /
 * b_min), b_min the larger of the classical distance of closest approach and
 * the de Broglie length at 3T, floored at 2. */
double orc_coulomb_log(double n_e, double T_e, double zbar)
{
    if (n_e <= 0.0 || T_e <= 0.0) return 2.0;
    double lam = sqrt(EPS0 * T_e / (Q_E * n_e * 1e6)) * 1e9;   /* nm */
    double zz = zbar > 1.0 ? zbar : 1.0;
    double bcl = zz * (Q_E / (4.0 * PI * EPS0)) * 1e9 / (3.0 * T_e); /* nm */
    double bqm = HBARC_EVNM / (2.0 * sqrt(3.0 * T_e * ME_C2));
    double b = bcl > bqm ? bcl : bqm;
    double L = log(lam / b);
    return L > 2.0 ? L : 2.0;
}

/* EOS table, bilinear on the given (n, T) grids, clamped at the ends */
static double interp1(const double *g, int n, double x, int *i0)
{
    if (n == 1 || x <= g[0]) { *i0 = 0; return 0.0; }
    if (x >= g[n - 1]) { *i0 = n - 2; return 1.0; }
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        int m = (lo + hi) / 2;
        if (g[m] <= x) lo = m; else hi = m;
    }
    *i0 = lo;
    return (x - g[lo]) / (g[lo + 1] - g[lo]);
}

double orc_eos(const orc_tables *t, double n_i, double T_e)
{
    int a, b;
    double fa = interp1(t->eos_n, t->n_n, n_i, &a);
    double fb = interp1(t->eos_T, t->n_T, T_e, &b);
    int a1 = t->n_n > 1 ? a + 1 : a, b1 = t->n_T > 1 ? b + 1 : b;
    const double *Z = t->eos_Z;
    double z00 = Z[a * t->n_T + b], z01 = Z[a * t->n_T + b1];
    double z10 = Z[a1 * t->n_T + b], z11 = Z[a1 * t->n_T + b1];
    return (1 - fa) * ((1 - fb) * z00 + fb * z01) + fa * ((1 - fb) * z10 + fb * z11);
}

/* ---------------- kinematics ---------------- */
static double gam(const double u[3]) { return sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]); }
/* kinetic energy m c^2 (gamma - 1), written as u^2/(gamma+1) */
static double kin(const double u[3], double m)
{
    double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return m * ME_C2 * u2 / (sqrt(1.0 + u2) + 1.0);
}

/* Scale the kinetic energy of momentum u by f (direction kept). */
static void scale_ke(double u[3], double f)
{
    double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (u2 == 0.0) return;
    double g1 = u2 / (sqrt(1.0 + u2) + 1.0);            /* gamma - 1 */
    double s = sqrt(f * (2.0 + f * g1) / (2.0 + g1));    /* |u'|/|u| */
    u[0] *= s; u[1] *= s; u[2] *= s;
}

/* One binary Coulomb collision (Takizuka-Abe angle, relativistic
 * centre-of-momentum rotation, weighted acceptance).  Momenta u in units of
 * m c of each particle, masses in m_e, charges in e, n_l in cm^-3, dtc in
 * fs; r[0..3] uniforms.  Returns 1 if a rotation was computed. */
int orc_collide(double ua[3], double ub[3], double ma, double mb, double qa,
                double qb, double wa, double wb, double n_l, double lnL,
                double dtc, const double r[4], double *np2_out)
{
    if (qa == 0.0 || qb == 0.0) return 0;
    double ga = gam(ua), gb = gam(ub);
    double dv[3] = {ua[0] / ga - ub[0] / gb, ua[1] / ga - ub[1] / gb, ua[2] / ga - ub[2] / gb};
    double vrel = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    if (vrel < 1e-10) return 0;
    double mu = ma * mb / (ma + mb);
    double var = 2.0 * PI * (qa * qb) * (qa * qb) * R_E_CM * R_E_CM * C_CM_FS * n_l * lnL * dtc
                 / (mu * mu * vrel * vrel * vrel);
    double delta = sqrt(var) * sqrt(-2.0 * log(r[0])) * cos(2.0 * PI * r[1]);
    double phi = 2.0 * PI * r[2];

    double pa[3], pb[3], P[3], bc[3];
    for (int k = 0; k < 3; ++k) { pa[k] = ma * ua[k]; pb[k] = mb * ub[k]; P[k] = pa[k] + pb[k]; }
    double Ea = ma * ga, Eb = mb * gb, E = Ea + Eb;
    for (int k = 0; k < 3; ++k) bc[k] = P[k] / E;
    double bc2 = bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2];
    double gc = 1.0 / sqrt(1.0 - bc2);
    double h = gc * gc / (gc + 1.0);                      /* (gc-1)/bc^2 */
    double bp = bc[0] * pa[0] + bc[1] * pa[1] + bc[2] * pa[2];
    double ps[3];
    for (int k = 0; k < 3; ++k) ps[k] = pa[k] + (h * bp - gc * Ea) * bc[k];
    double p = sqrt(ps[0] * ps[0] + ps[1] * ps[1] + ps[2] * ps[2]);
    if (p == 0.0) return 0;
    double n[3] = {ps[0] / p, ps[1] / p, ps[2] / p};
    double st = 2.0 * delta / (1.0 + delta * delta);
    double ct = (1.0 - delta * delta) / (1.0 + delta * delta);
    /* orthonormal (e1, e2) about n, the origin of the azimuth: built on the
     * z axis while n is at least 30 degrees from it (|n_xy|^2 >= 1/4), on
     * the x axis otherwise, so that the frame never divides by a small
     * component (any frame gives the same distribution of outcomes) */
    double e1[3], e2[3];
    double np2 = n[0] * n[0] + n[1] * n[1];
    if (np2_out) *np2_out = np2;
    if (np2 >= 0.25) {
        double np = sqrt(np2);
        e1[0] = n[0] * n[2] / np; e1[1] = n[1] * n[2] / np; e1[2] = -np;
        e2[0] = -n[1] / np; e2[1] = n[0] / np; e2[2] = 0.0;
    } else {
        double nq = sqrt(n[1] * n[1] + n[2] * n[2]);
        e2[0] = 0.0; e2[1] = n[2] / nq; e2[2] = -n[1] / nq;
        e1[0] = nq; e1[1] = -n[0] * n[1] / nq; e1[2] = -n[0] * n[2] / nq;
    }
    double cp = cos(phi), sp = sin(phi);
    double qa_s[3];
    for (int k = 0; k < 3; ++k)
        qa_s[k] = p * (ct * n[k] + st * cp * e1[k] + st * sp * e2[k]);
    double Eas = sqrt(ma * ma + p * p), Ebs = sqrt(mb * mb + p * p);
    double bq = bc[0] * qa_s[0] + bc[1] * qa_s[1] + bc[2] * qa_s[2];
    double pa2[3], pb2[3];
    for (int k = 0; k < 3; ++k) {
        pa2[k] = qa_s[k] + (h * bq + gc * Eas) * bc[k];
        pb2[k] = -qa_s[k] + (-h * bq + gc * Ebs) * bc[k];
    }
    double wm = wa > wb ? wa : wb;
    if (r[3] < wb / wm)
        for (int k = 0; k < 3; ++k) ua[k] = pa2[k] / ma;
    if (r[3] < wa / wm)
        for (int k = 0; k < 3; ++k) ub[k] = pb2[k] / mb;
    return 1;
}

/* relativistic Boris rotation, q/m in e/m_e, dt in fs, normalized fields */
void orc_boris(double u[3], const double e[3], const double b[3], double qm, double dt)
{
    double h = 0.5 * qm * dt;
    double um[3] = {u[0] + h * e[0], u[1] + h * e[1], u[2] + h * e[2]};
    double g = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    double t[3] = {h * b[0] / g, h * b[1] / g, h * b[2] / g};
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    double s[3] = {2 * t[0] / (1 + t2), 2 * t[1] / (1 + t2), 2 * t[2] / (1 + t2)};
    double up[3] = {um[0] + um[1] * t[2] - um[2] * t[1],
                    um[1] + um[2] * t[0] - um[0] * t[2],
                    um[2] + um[0] * t[1] - um[1] * t[0]};
    double uq[3] = {um[0] + up[1] * s[2] - up[2] * s[1],
                    um[1] + up[2] * s[0] - up[0] * s[2],
                    um[2] + up[0] * s[1] - up[1] * s[0]};
    u[0] = uq[0] + h * e[0]; u[1] = uq[1] + h * e[1]; u[2] = uq[2] + h * e[2];
}

/* ---------------- pairing order ---------------- */
typedef struct { uint64_t key, id; int idx; } keyrec;
static int cmp_keyrec(const void *a, const void *b)
{
    const keyrec *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

/* random permutation: ascending Philox key, ties broken by id */
void orc_pair_order(int n, const uint64_t *id, uint32_t step, uint32_t purpose,
                    uint64_t seed, int *perm)
{
    keyrec *k = malloc(sizeof(keyrec) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        k[i].key = key64(seed, id[i], step, purpose);
        k[i].id = id[i];
        k[i].idx = i;
    }
    qsort(k, n, sizeof(keyrec), cmp_keyrec);
    for (int i = 0; i < n; ++i) perm[i] = k[i].idx;
    free(k);
}

/* like-particle pairs over positions of the permuted list: odd n >= 3 puts
 * the first three in a triangle at half time step (Takizuka-Abe). */
int orc_ee_pairs(int n, int *pa, int *pb, double *frac)
{
    int m = 0, start = 0;
    if (n < 2) return 0;
    if (n % 2 == 1) {
        pa[0] = 0; pb[0] = 1; frac[0] = 0.5;
        pa[1] = 1; pb[1] = 2; frac[1] = 0.5;
        pa[2] = 2; pb[2] = 0; frac[2] = 0.5;
        m = 3; start = 3;
    }
    for (int k = start; k + 1 < n; k += 2) {
        pa[m] = k; pb[m] = k + 1; frac[m] = 1.0; ++m;
    }
    return m;
}

/* ---------------- deposit ---------------- */
static double cic(double X, int node) { double d = fabs(X - node); return d < 1.0 ? 1.0 - d : 0.0; }
static int wrapy(int j, int ny) { j %= ny; return j < 0 ? j + ny : j; }

static void dep_seg(int nx, int ny, double dx, double dy, double dt, double X0, double Y0,
                    double X1, double Y1, double vz, double vy, double qw, double frac, double *j3)
{
    double *jx = j3, *jy = j3 + (size_t)ny * (nx + 1), *jz = j3 + 2 * (size_t)ny * (nx + 1);
    int i0 = (int)floor(X0);
    double S0x[4], S1x[4], DSx[4];
    for (int a = 0; a < 4; ++a) {
        S0x[a] = cic(X0, i0 - 1 + a);
        S1x[a] = cic(X1, i0 - 1 + a);
        DSx[a] = S1x[a] - S0x[a];
    }
    if (ny == 1) {
        double acc = 0.0;
        for (int a = 0; a < 3; ++a) {
            acc += DSx[a];
            int i = i0 - 1 + a;
            if (i >= 0 && i < nx) jx[i] += -qw * (dx / dt) * acc;
        }
        for (int a = 0; a < 4; ++a) {
            int i = i0 - 1 + a;
            if (i < 0 || i > nx) continue;
            double s = 0.5 * (S0x[a] + S1x[a]);
            jy[i] += qw * vy * s * frac;
            jz[i] += qw * vz * s * frac;
        }
        return;
    }
    int j0 = (int)floor(Y0);
    double S0y[4], S1y[4], DSy[4];
    for (int b = 0; b < 4; ++b) {
        S0y[b] = cic(Y0, j0 - 1 + b);
        S1y[b] = cic(Y1, j0 - 1 + b);
        DSy[b] = S1y[b] - S0y[b];
    }
    for (int b = 0; b < 4; ++b) {
        int jj = wrapy(j0 - 1 + b, ny);
        double acc = 0.0;
        for (int a = 0; a < 3; ++a) {
            acc += DSx[a] * (S0y[b] + 0.5 * DSy[b]);
            int i = i0 - 1 + a;
            if (i >= 0 && i < nx) jx[(size_t)jj * (nx + 1) + i] += -qw * (dx / dt) * acc;
        }
    }
    for (int a = 0; a < 4; ++a) {
        int i = i0 - 1 + a;
        if (i < 0 || i > nx) continue;
        double acc = 0.0;
        for (int b = 0; b < 3; ++b) {
            acc += DSy[b] * (S0x[a] + 0.5 * DSx[a]);
            int jj = wrapy(j0 - 1 + b, ny);
            jy[(size_t)jj * (nx + 1) + i] += -qw * (dy / dt) * acc;
        }
        for (int b = 0; b < 4; ++b) {
            int jj = wrapy(j0 - 1 + b, ny);
            double wz = S0x[a] * S0y[b] + 0.5 * DSx[a] * S0y[b] + 0.5 * S0x[a] * DSy[b]
                        + DSx[a] * DSy[b] / 3.0;
            jz[(size_t)jj * (nx + 1) + i] += qw * vz * wz * frac;
        }
    }
}

/* Charge-conserving current of one particle moving (X0,Y0)->(X1,Y1) in one
 * step (cell units), split into equal segments shorter than one cell.
 * j3 = [jx, jy, jz] on [ny][nx+1], units e*n_ref*nm/fs; jx at (i+1/2, j),
 * jy at (i, j+1/2), jz at (i, j).  In 1D (ny == 1) jy, jz use the
 * time-averaged x shape. */
void orc_deposit(int nx, int ny, double dx, double dy, double dt, double X0,
                 double Y0, double X1, double Y1, double vz, double vy,
                 double qw, double *j3)
{
    double ax = fabs(X1 - X0), ay = ny > 1 ? fabs(Y1 - Y0) : 0.0;
    double m = ax > ay ? ax : ay;
    int nseg = (int)floor(m) + 1;
    for (int k = 0; k < nseg; ++k) {
        double a0 = (double)k / nseg, a1 = (double)(k + 1) / nseg;
        double xa = X0 + a0 * (X1 - X0), xb = X0 + a1 * (X1 - X0);
        double ya = Y0 + a0 * (Y1 - Y0), yb = Y0 + a1 * (Y1 - Y0);
        dep_seg(nx, ny, dx, dy, dt, xa, ya, xb, yb, vz, vy, qw, 1.0 / nseg, j3);
    }
}

/* CIC charge density of one particle on the node grid [ny][nx+1] */
void orc_rho(int nx, int ny, double X, double Y, double qw, double *rho)
{
    int i0 = (int)floor(X);
    for (int a = 0; a < 2; ++a) {
        int i = i0 + a;
        if (i < 0 || i > nx) continue;
        double sx = cic(X, i);
        if (ny == 1) { rho[i] += qw * sx; continue; }
        int j0 = (int)floor(Y);
        for (int b = 0; b < 2; ++b) {
            int jj = wrapy(j0 + b, ny);
            rho[(size_t)jj * (nx + 1) + i] += qw * sx * cic(Y, j0 + b);
        }
    }
}

/* ---------------- slab state ---------------- */
/* cs: momentum scale of the binary collisions the electron took part in
 * during the last step (the largest |u| of itself and its partners before
 * each collision; test bookkeeping, no part of the method) */
typedef struct { double X, Y, u[3], w; uint64_t id; int alive; double cs; } elec;
typedef struct { double X, Y, u[3], zf; uint32_t id; int Z, nK; } ionr;

struct orc_slab {
    orc_params p;
    orc_tables t;
    double *hv_tab, *sigma, *eos_T, *eos_n, *eos_Z;
    orc_pulse pulse;
    int have_pulse;
    double *hv_b, *sig_b;       /* per bin: photon energy, sigma[s][b] */
    elec *e; int ne, cap_e;
    ionr *ion; int ni;
    double *f;                  /* [6][ny][nx+1] ex ey ez bx by bz */
    double *j;                  /* [3][ny][nx+1] */
    double *ph;                 /* [ny][nx][nb] */
    /* radiation transport mode (orc_set_rt) */
    int rt_on;
    orc_rt rt;
    int nrx, nry, nrc, ncd, nord;
    double *o_mu, *o_vy, *o_w;  /* [nord] direction cosines in the plane, share of isotropic emission */
    double *F, *Gx, *Gy;        /* [nord][nb][nry][nrx] */
    double *n_pub;              /* [nrc][nb] densities published to the cells */
    double *c_chi, *c_emc, *c_w, *c_dE;   /* per PIC cell ([ncell][nb], [ncell] x 3) */
    uint32_t step;
    double tally[ORC_NT];
    uint64_t cnt[ORC_NC];
    double trace_rel;           /* > 0: decision trace on */
    orc_near *near; int nnear, capnear;
    uint64_t ndraw, ndec;
};

static double *dupd(const double *a, size_t n)
{
    double *b = malloc(sizeof(double) * (n ? n : 1));
    if (n) memcpy(b, a, sizeof(double) * n);
    return b;
}

orc_slab *orc_create(const orc_params *p, const orc_tables *t)
{
    orc_slab *s = calloc(1, sizeof(orc_slab));
    s->p = *p;
    s->t = *t;
    s->hv_tab = dupd(t->hv_tab, t->n_hv);
    s->sigma = dupd(t->sigma, (size_t)ORC_NS * t->n_hv);
    s->eos_T = dupd(t->eos_T, t->n_T);
    s->eos_n = dupd(t->eos_n, t->n_n);
    s->eos_Z = dupd(t->eos_Z, (size_t)t->n_T * t->n_n);
    s->t.hv_tab = s->hv_tab; s->t.sigma = s->sigma;
    s->t.eos_T = s->eos_T; s->t.eos_n = s->eos_n; s->t.eos_Z = s->eos_Z;
    size_t ng = (size_t)p->ny * (p->nx + 1);
    s->f = calloc(6 * ng, sizeof(double));
    s->j = calloc(3 * ng, sizeof(double));
    return s;
}

void orc_destroy(orc_slab *s)
{
    if (!s) return;
    free(s->hv_tab); free(s->sigma); free(s->eos_T); free(s->eos_n); free(s->eos_Z);
    free(s->hv_b); free(s->sig_b); free(s->e); free(s->ion); free(s->f); free(s->j); free(s->ph);
    free(s->near);
    free(s->o_mu); free(s->o_vy); free(s->o_w); free(s->F); free(s->Gx); free(s->Gy); free(s->n_pub);
    free(s->c_chi); free(s->c_emc); free(s->c_w); free(s->c_dE);
    free(s);
}

/* photoionization cross section of the table at hv: log-log interpolation,
 * held constant beyond the table ends */
static double sigma_at(const orc_tables *t, int sub, double hv)
{
    const double *g = t->hv_tab, *v = t->sigma + (size_t)sub * t->n_hv;
    int n = t->n_hv;
    if (hv <= g[0]) return v[0];
    if (hv >= g[n - 1]) return v[n - 1];
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) { int m = (lo + hi) / 2; if (g[m] <= hv) lo = m; else hi = m; }
    if (v[lo] <= 0.0 || v[lo + 1] <= 0.0) {
        double f = (hv - g[lo]) / (g[lo + 1] - g[lo]);
        return v[lo] + f * (v[lo + 1] - v[lo]);
    }
    double f = log(hv / g[lo]) / log(g[lo + 1] / g[lo]);
    return exp(log(v[lo]) + f * log(v[lo + 1] / v[lo]));
}

void orc_set_pulse(orc_slab *s, const orc_pulse *pl)
{
    int nb = pl->n_bins;
    s->pulse = *pl;
    s->have_pulse = 1;
    free(s->hv_b); free(s->sig_b); free(s->ph);
    s->hv_b = malloc(sizeof(double) * nb);
    s->sig_b = malloc(sizeof(double) * nb * ORC_NS);
    for (int b = 0; b < nb; ++b) {
        s->hv_b[b] = pl->hv + pl->bandwidth * ((b + 0.5) / nb - 0.5);
        for (int q = 0; q < ORC_NS; ++q) s->sig_b[q * nb + b] = sigma_at(&s->t, q, s->hv_b[b]);
    }
    s->ph = calloc((size_t)s->p.ny * s->p.nx * nb, sizeof(double));
}

void orc_set_step(orc_slab *s, uint32_t n) { s->step = n; }
uint32_t orc_get_step(const orc_slab *s) { return s->step; }

static void ensure_e(orc_slab *s, int n)
{
    if (n <= s->cap_e) return;
    int c = s->cap_e ? s->cap_e : 1024;
    while (c < n) c *= 2;
    s->e = realloc(s->e, sizeof(elec) * c);
    s->cap_e = c;
}

void orc_load_electrons(orc_slab *s, int n, const double *X, const double *Y,
                        const double *u, const double *w, const uint64_t *id)
{
    s->ne = 0;
    ensure_e(s, n);
    for (int k = 0; k < n; ++k) {
        elec *e = &s->e[k];
        e->X = X[k]; e->Y = Y[k];
        e->u[0] = u[3 * k]; e->u[1] = u[3 * k + 1]; e->u[2] = u[3 * k + 2];
        e->w = w[k]; e->id = id[k]; e->alive = 1; e->cs = 0.0;
    }
    s->ne = n;
}

void orc_load_ions(orc_slab *s, int n, const double *X, const double *Y,
                   const double *u, const double *zf, const int32_t *Z,
                   const int32_t *nK, const uint32_t *id)
{
    free(s->ion);
    s->ion = malloc(sizeof(ionr) * (n ? n : 1));
    for (int k = 0; k < n; ++k) {
        ionr *q = &s->ion[k];
        q->X = X[k]; q->Y = Y[k];
        q->u[0] = u[3 * k]; q->u[1] = u[3 * k + 1]; q->u[2] = u[3 * k + 2];
        q->zf = zf[k]; q->Z = Z[k]; q->nK = nK[k]; q->id = id[k];
    }
    s->ni = n;
}

int orc_n_electrons(const orc_slab *s) { return s->ne; }
void orc_get_electron_scales(const orc_slab *s, double *cs)
{
    for (int k = 0; k < s->ne; ++k) cs[k] = s->e[k].cs;
}
int orc_n_ions(const orc_slab *s) { return s->ni; }

void orc_get_electrons(const orc_slab *s, double *X, double *Y, double *u, double *w, uint64_t *id)
{
    for (int k = 0; k < s->ne; ++k) {
        const elec *e = &s->e[k];
        X[k] = e->X; Y[k] = e->Y;
        u[3 * k] = e->u[0]; u[3 * k + 1] = e->u[1]; u[3 * k + 2] = e->u[2];
        w[k] = e->w; id[k] = e->id;
    }
}

void orc_get_ions(const orc_slab *s, double *X, double *Y, double *u, double *zf,
                  int32_t *Z, int32_t *nK, uint32_t *id)
{
    for (int k = 0; k < s->ni; ++k) {
        const ionr *q = &s->ion[k];
        X[k] = q->X; Y[k] = q->Y;
        u[3 * k] = q->u[0]; u[3 * k + 1] = q->u[1]; u[3 * k + 2] = q->u[2];
        zf[k] = q->zf; Z[k] = q->Z; nK[k] = q->nK; id[k] = q->id;
    }
}

void orc_set_fields(orc_slab *s, const double *f6)
{
    memcpy(s->f, f6, sizeof(double) * 6 * (size_t)s->p.ny * (s->p.nx + 1));
}
void orc_get_fields(const orc_slab *s, double *f6)
{
    memcpy(f6, s->f, sizeof(double) * 6 * (size_t)s->p.ny * (s->p.nx + 1));
}
void orc_get_current(const orc_slab *s, double *j3)
{
    memcpy(j3, s->j, sizeof(double) * 3 * (size_t)s->p.ny * (s->p.nx + 1));
}
void orc_set_photons(orc_slab *s, const double *ph)
{
    if (s->have_pulse) memcpy(s->ph, ph, sizeof(double) * (size_t)s->p.ny * s->p.nx * s->pulse.n_bins);
}
void orc_get_photons(const orc_slab *s, double *ph)
{
    if (s->have_pulse) memcpy(ph, s->ph, sizeof(double) * (size_t)s->p.ny * s->p.nx * s->pulse.n_bins);
}

/* ---------------- photon march (every rad step) ---------------- */
static double pulse_I(const orc_pulse *pl, double tau)
{
    if (pl->shape == 1) return fabs(tau - pl->t_peak) <= 0.5 * pl->fwhm ? pl->I_peak : 0.0;
    double d = (tau - pl->t_peak) / pl->fwhm;
    return pl->I_peak * exp(-4.0 * log(2.0) * d * d);
}

/* photon number density (units n_ref) entering x = 0 at time tau in bin b */
static double source(const orc_slab *s, int b, double tau, int row)
{
    double I = pulse_I(&s->pulse, tau);                       /* W/cm^2 */
    double n = I / (C_CM_FS * 1e15 * s->hv_b[b] * Q_E) / s->pulse.n_bins;  /* cm^-3 */
    if (s->pulse.spot_sigma > 0.0 && s->p.ny > 1) {
        double y = (row + 0.5) * s->p.dy - 0.5 * s->p.ny * s->p.dy;
        n *= exp(-0.5 * y * y / (s->pulse.spot_sigma * s->pulse.spot_sigma));
    }
    return n / s->p.n_ref;
}

/* Advance the photon field by one rad step: every cell's content moves
 * c*dt_rad along +x, split linearly between the two destination cells;
 * the region x < 0 holds the pulse at retarded time; what passes x = L is
 * transmitted. */
static void march(orc_slab *s)
{
    int nx = s->p.nx, ny = s->p.ny, nb = s->pulse.n_bins;
    double dtr = s->p.rad_every * s->p.dt;
    double sh = C_NM_FS * dtr / s->p.dx;
    int m = (int)floor(sh);
    double f = sh - m;
    double tprev = (double)s->step * s->p.dt - dtr;
    double *col = malloc(sizeof(double) * nx);
    for (int row = 0; row < ny; ++row)
        for (int b = 0; b < nb; ++b) {
            double *ph = s->ph + (size_t)row * nx * nb;
            for (int k = 0; k < nx; ++k) col[k] = ph[(size_t)k * nb + b];
            double trans = 0.0, inc = 0.0;
            for (int k = 0; k < nx; ++k) ph[(size_t)k * nb + b] = 0.0;
            for (int j = -(m + 1); j < nx; ++j) {
                double v;
                if (j < 0) v = source(s, b, tprev - (j + 0.5) * s->p.dx / C_NM_FS, row);
                else v = col[j];
                if (v == 0.0) continue;
                int d0 = j + m, d1 = j + m + 1;
                double v0 = (1.0 - f) * v, v1 = f * v;
                if (j < 0) {
                    if (d0 >= 0) inc += v0;
                    if (d1 >= 0) inc += v1;
                }
                if (d0 >= nx) trans += v0; else if (d0 >= 0) ph[(size_t)d0 * nb + b] += v0;
                if (d1 >= nx) trans += v1; else if (d1 >= 0) ph[(size_t)d1 * nb + b] += v1;
            }
            s->tally[ORC_T_INC] += inc * s->hv_b[b];
            s->tally[ORC_T_TRANS] += trans * s->hv_b[b];
        }
    free(col);
}

/* ---------------- radiation transport (Sec. II, Eqs. 1a and 1b) ---------------- */
/* Gauss-Legendre nodes and weights on (-1, 1) (Newton on the Legendre
 * recurrence), nodes in descending order */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(PI * (i + 0.75) / (n + 0.5)), pp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            pp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-15) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

int orc_set_rt(orc_slab *s, const orc_rt *rt)
{
    const orc_params *p = &s->p;
    const int R = rt->coarsen, d2 = p->ny > 1;
    if (!s->have_pulse || R < 1 || p->nx % R || (d2 && p->ny % R) || rt->n_polar < 0 || rt->n_polar > 16 ||
        (d2 && (rt->n_azimuth < 1 || rt->n_azimuth > 16)) || (rt->scheme != 0 && rt->scheme != 1))
        return 1;
    s->rt = *rt;
    s->rt_on = 1;
    s->nrx = p->nx / R;
    s->nry = d2 ? p->ny / R : 1;
    s->nrc = s->nrx * s->nry;
    s->ncd = d2 ? R * R : R;
    const int naz = d2 ? rt->n_azimuth : 1;
    s->nord = 1 + rt->n_polar * naz;
    const int nb = s->pulse.n_bins;
    free(s->o_mu); free(s->o_vy); free(s->o_w);
    s->o_mu = calloc(s->nord, sizeof(double));
    s->o_vy = calloc(s->nord, sizeof(double));
    s->o_w = calloc(s->nord, sizeof(double));
    s->o_mu[0] = 1.0;                 /* the XFEL beam along +x: no share of isotropic emission */
    if (rt->n_polar > 0) {
        double *x = malloc(sizeof(double) * rt->n_polar), *a = malloc(sizeof(double) * rt->n_polar);
        gauss_legendre(rt->n_polar, x, a);
        for (int k = 0; k < rt->n_polar; ++k)
            for (int j = 0; j < naz; ++j) {
                const int o = 1 + k * naz + j;
                s->o_mu[o] = x[k];
                /* azimuth phi in (0, pi) about +x: n_z = sin(theta) sin(phi) >= 0,
                 * the lower hemisphere is its mirror image */
                s->o_vy[o] = d2 ? sqrt(1.0 - x[k] * x[k]) * cos(PI * (j + 0.5) / naz) : 0.0;
                s->o_w[o] = 0.5 * a[k] / naz;
            }
        free(x); free(a);
    }
    const size_t nf = (size_t)s->nord * nb * s->nrc, nc = (size_t)p->nx * p->ny;
    free(s->F); free(s->Gx); free(s->Gy); free(s->n_pub);
    free(s->c_chi); free(s->c_emc); free(s->c_w); free(s->c_dE);
    s->F = calloc(nf, sizeof(double));
    s->Gx = calloc(nf, sizeof(double));
    s->Gy = calloc(nf, sizeof(double));
    s->n_pub = calloc((size_t)s->nrc * nb, sizeof(double));
    s->c_chi = calloc(nc * nb, sizeof(double));
    s->c_emc = calloc(nc, sizeof(double));
    s->c_w = calloc(nc, sizeof(double));
    s->c_dE = calloc(nc, sizeof(double));
    return 0;
}

int orc_rt_ordinates(const orc_slab *s, double *mu, double *vy, double *w)
{
    for (int o = 0; o < s->nord; ++o) { mu[o] = s->o_mu[o]; vy[o] = s->o_vy[o]; w[o] = s->o_w[o]; }
    return s->nord;
}

void orc_rt_get(const orc_slab *s, double *F, double *Gx, double *Gy)
{
    const size_t nf = (size_t)s->nord * s->pulse.n_bins * s->nrc;
    memcpy(F, s->F, sizeof(double) * nf);
    memcpy(Gx, s->Gx, sizeof(double) * nf);
    memcpy(Gy, s->Gy, sizeof(double) * nf);
}

void orc_rt_set(orc_slab *s, const double *F, const double *Gx, const double *Gy)
{
    const size_t nf = (size_t)s->nord * s->pulse.n_bins * s->nrc;
    memcpy(s->F, F, sizeof(double) * nf);
    memcpy(s->Gx, Gx, sizeof(double) * nf);
    memcpy(s->Gy, Gy, sizeof(double) * nf);
}

void orc_rt_cells(const orc_slab *s, double *chi, double *emc, double *wcell, double *dEc)
{
    const size_t nc = (size_t)s->p.nx * s->p.ny;
    memcpy(chi, s->c_chi, sizeof(double) * nc * s->pulse.n_bins);
    memcpy(emc, s->c_emc, sizeof(double) * nc);
    memcpy(wcell, s->c_w, sizeof(double) * nc);
    memcpy(dEc, s->c_dE, sizeof(double) * nc);
}

/* cubic Hermite pieces on one node interval, unit spacing, t in [0, 1]:
 * value, slope, and integral from 0 to t */
static double herm(double f0, double g0, double f1, double g1, double t)
{
    const double t2 = t * t, t3 = t2 * t;
    return (2 * t3 - 3 * t2 + 1) * f0 + (t3 - 2 * t2 + t) * g0 + (-2 * t3 + 3 * t2) * f1 + (t3 - t2) * g1;
}
static double herm_d(double f0, double g0, double f1, double g1, double t)
{
    const double t2 = t * t;
    return (6 * t2 - 6 * t) * f0 + (3 * t2 - 4 * t + 1) * g0 + (-6 * t2 + 6 * t) * f1 + (3 * t2 - 2 * t) * g1;
}
static double herm_i(double f0, double g0, double f1, double g1, double t)
{
    const double t2 = t * t, t3 = t2 * t, t4 = t3 * t;
    return (0.5 * t4 - t3 + t) * f0 + (0.25 * t4 - 2.0 * t3 / 3.0 + 0.5 * t2) * g0 + (-0.5 * t4 + t3) * f1 +
           (0.25 * t4 - t3 / 3.0) * g1;
}

typedef struct {
    const double *f, *g;
    int n, periodic, ng;
    double nu;
    const double *fin, *gin;
} rtline;

/* value and slope of node j of a line (ghosts outside [0, n)) */
static void rt_node(const rtline *L, int j, double *fj, double *gj)
{
    if (L->periodic) { j %= L->n; if (j < 0) j += L->n; *fj = L->f[j]; *gj = L->g[j]; return; }
    if (j >= 0 && j < L->n) { *fj = L->f[j]; *gj = L->g[j]; return; }
    const int in_side = L->nu > 0 ? j < 0 : j >= L->n;
    if (in_side) {
        const int q = L->nu > 0 ? -j - 1 : j - L->n;
        if (q < L->ng && L->fin) { *fj = L->fin[q]; *gj = L->gin ? L->gin[q] : 0.0; }
        else { *fj = 0.0; *gj = 0.0; }
        return;
    }
    *fj = 0.0;                          /* beyond the outflow face: empty */
    *gj = 0.0;
}

/* integral of the Hermite reconstruction over [a, b] (node coordinates) */
static double rt_integral(const rtline *L, double a, double b)
{
    double acc = 0.0;
    int k = (int)floor(a);
    while (k < b) {
        const double lo = a > k ? a - k : 0.0, hi = b < k + 1 ? b - k : 1.0;
        if (hi > lo) {
            double f0, g0, f1, g1;
            rt_node(L, k, &f0, &g0);
            rt_node(L, k + 1, &f1, &g1);
            acc += herm_i(f0, g0, f1, g1, hi) - herm_i(f0, g0, f1, g1, lo);
        }
        ++k;
    }
    return acc;
}

/* contents crossing the two faces of a line in one shift by nu nodes, as
 * the linear split moves them (node j's content goes (1 - fr) to j + m and
 * fr to j + m + 1, mirrored for nu < 0): the inflow ghosts' parts that land
 * inside or beyond entered, every part that lands beyond the far face left */
static void split_flows(const rtline *L, int n, double nu, double *in, double *out)
{
    const double a = fabs(nu);
    const int m = (int)floor(a), sgn = nu >= 0 ? 1 : -1;
    const double fr = a - m;
    for (int j = -(m + 1); j < n + m + 1; ++j) {
        if ((sgn > 0 && j >= n) || (sgn < 0 && j < 0)) continue;
        double v, dummy;
        rt_node(L, j, &v, &dummy);
        if (v == 0.0) continue;
        const int in_src = j < 0 || j >= n;
        const int d[2] = {j + sgn * m, j + sgn * (m + 1)};
        const double part[2] = {(1.0 - fr) * v, fr * v};
        for (int q = 0; q < 2; ++q) {
            const int inside = d[q] >= 0 && d[q] < n, far = sgn > 0 ? d[q] >= n : d[q] < 0;
            if (in_src && (inside || far)) *in += part[q];
            if (far) *out += part[q];
        }
    }
}

void orc_rt_line(double *f, double *g, double *gt, int n, double nu, int scheme, int periodic,
                 const double *fin, const double *gin, int ng, double *in, double *out)
{
    double *f0 = malloc(sizeof(double) * n), *g0 = malloc(sizeof(double) * n), *t0 = malloc(sizeof(double) * n);
    memcpy(f0, f, sizeof(double) * n);
    memcpy(g0, g, sizeof(double) * n);
    if (gt) memcpy(t0, gt, sizeof(double) * n);
    else memset(t0, 0, sizeof(double) * n);
    rtline L = {f0, g0, n, periodic, ng, nu, fin, gin};
    rtline T = {t0, t0, n, periodic, ng, nu, NULL, NULL};   /* transverse slope: zero inflow */
    *in = *out = 0.0;
    if (scheme == 1) {
        /* the ballistic march's split: node j's content goes (1 - fr) to
         * j + m and fr to j + m + 1 (mirrored for nu < 0) */
        const double a = fabs(nu);
        const int m = (int)floor(a), sgn = nu >= 0 ? 1 : -1;
        const double fr = a - m;
        for (int i = 0; i < n; ++i) {
            double v0, v1, dummy;
            rt_node(&L, i - sgn * m, &v0, &dummy);
            rt_node(&L, i - sgn * (m + 1), &v1, &dummy);
            f[i] = (1.0 - fr) * v0 + fr * v1;
        }
        if (!periodic) split_flows(&L, n, nu, in, out);
        if (gt) memset(gt, 0, sizeof(double) * n);
        memset(g, 0, sizeof(double) * n);
    } else {
        for (int i = 0; i < n; ++i) {
            const double xd = i - nu;
            const int k = (int)floor(xd);
            const double t = xd - k;
            double fa, ga, fb, gb;
            rt_node(&L, k, &fa, &ga);
            rt_node(&L, k + 1, &fb, &gb);
            f[i] = herm(fa, ga, fb, gb, t);
            g[i] = herm_d(fa, ga, fb, gb, t);
            if (gt) {
                double ta, tb, dummy;
                rt_node(&T, k, &ta, &dummy);
                rt_node(&T, k + 1, &tb, &dummy);
                gt[i] = (1.0 - t) * ta + t * tb;
            }
        }
        /* faces crossed: the contents the shift carries across them, as the
         * linear split moves them (exact at integer Courant numbers, where
         * CIP is an exact shift too); what CIP's cubic update of the
         * interior adds to or removes from that is the scheme's own gain */
        if (!periodic) split_flows(&L, n, nu, in, out);
    }
    free(f0); free(g0); free(t0);
}

/* photon density (n_ref units) of bin b entering x = 0 at time tau, at height y (nm) */
static double rt_source(const orc_slab *s, int b, double tau, double y)
{
    double I = pulse_I(&s->pulse, tau);
    double n = I / (C_CM_FS * 1e15 * s->hv_b[b] * Q_E) / s->pulse.n_bins;
    if (s->pulse.spot_sigma > 0.0 && s->p.ny > 1) {
        double yc = y - 0.5 * s->p.ny * s->p.dy;
        n *= exp(-0.5 * yc * yc / (s->pulse.spot_sigma * s->pulse.spot_sigma));
    }
    return n / s->p.n_ref;
}

static int rt_cell(const orc_slab *s, int c)
{
    const int R = s->rt.coarsen, i = c % s->p.nx, j = c / s->p.nx;
    return (s->p.ny > 1 ? (j / R) * s->nrx : 0) + i / R;
}

/* One rad step of the radiation field, before the cells' physics of the
 * step: (1) gather what the cells recorded at the last rad step (opacity,
 * photon energy taken by photoionization, electron weight, K-alpha photons
 * added to their photon numbers); (2) absorb the field over dt_rad with
 * that opacity; (3) the energy absorbed beyond what the photoionization
 * events took is given to the bulk electrons of the rad cell (negative:
 * taken), shared among its PIC cells by electron weight, at their next
 * rad step; (4) K-alpha photons join the diffuse ordinates isotropically;
 * (5) advect every ordinate and bin (x, then y in 2D); (6) publish the
 * photon densities to the PIC cells. */
static void rt_step(orc_slab *s)
{
    const orc_params *p = &s->p;
    const int nb = s->pulse.n_bins, nrc = s->nrc, nord = s->nord, ncell = p->nx * p->ny, ncd = s->ncd;
    const double dtr = p->rad_every * p->dt;
    const double dxr = p->dx * s->rt.coarsen, dyr = p->dy * s->rt.coarsen;
    double *chi = calloc((size_t)nrc * nb, sizeof(double)), *ka = calloc((size_t)nrc * nb, sizeof(double));
    double *emc = calloc(nrc, sizeof(double)), *W = calloc(nrc, sizeof(double));
    /* (1) */
    for (int c = 0; c < ncell; ++c) {
        const int r = rt_cell(s, c);
        emc[r] += s->c_emc[c];
        W[r] += s->c_w[c];
        for (int b = 0; b < nb; ++b) {
            chi[(size_t)r * nb + b] += s->c_chi[(size_t)c * nb + b] / ncd;
            ka[(size_t)r * nb + b] += (s->ph[(size_t)c * nb + b] - s->n_pub[(size_t)r * nb + b]) / ncd;
        }
    }
    /* (2), (3) */
    for (int r = 0; r < nrc; ++r) {
        double A = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double e = exp(-chi[(size_t)r * nb + b] * C_CM_FS * dtr);
            for (int o = 0; o < nord; ++o) {
                const size_t q = ((size_t)o * nb + b) * nrc + r;
                A += s->F[q] * (1.0 - e) * ncd * s->hv_b[b];
                s->F[q] *= e; s->Gx[q] *= e; s->Gy[q] *= e;
            }
        }
        const double dE = A - emc[r];
        s->tally[ORC_T_RT_PEND] += A;      /* the events' photons were owed (see cell_physics) */
        if (dE == 0.0) continue;
        for (int c = 0; c < ncell; ++c) {
            if (rt_cell(s, c) != r) continue;
            s->c_dE[c] += W[r] > 0.0 ? dE * s->c_w[c] / W[r] : dE / ncd;
        }
    }
    /* (4) */
    for (int r = 0; r < nrc; ++r)
        for (int b = 0; b < nb; ++b) {
            const double k = ka[(size_t)r * nb + b];
            if (k == 0.0) continue;
            if (nord > 1) {
                for (int o = 1; o < nord; ++o) s->F[((size_t)o * nb + b) * nrc + r] += k * s->o_w[o];
            } else {
                s->tally[ORC_T_KA_ESC] += k * ncd * s->hv_b[b];
            }
        }
    /* (5) */
    const double tprev = (double)s->step * p->dt - dtr;
    const int mx = s->nrx > s->nry ? s->nrx : s->nry;
    double *f = malloc(sizeof(double) * mx), *g = malloc(sizeof(double) * mx), *gt = malloc(sizeof(double) * mx);
    for (int o = 0; o < nord; ++o)
        for (int b = 0; b < nb; ++b) {
            double *F = s->F + ((size_t)o * nb + b) * nrc, *Gx = s->Gx + ((size_t)o * nb + b) * nrc;
            double *Gy = s->Gy + ((size_t)o * nb + b) * nrc;
            double before = 0.0, after = 0.0, inflow = 0.0, outflow = 0.0;
            for (int r = 0; r < nrc; ++r) before += F[r];
            const double nux = C_NM_FS * dtr * s->o_mu[o] / dxr;
            for (int ry = 0; ry < s->nry; ++ry) {
                int ng = 0;
                double fin[64], gin[64];
                if (o == 0 && nux > 0) {
                    const double y = (ry + 0.5) * dyr;
                    ng = (int)floor(nux) + 3;
                    if (ng > 62) ng = 62;
                    for (int q = 0; q < ng; ++q) {
                        const int j = -1 - q;
                        const double xa = (j + 0.5) * dxr, xm = (j - 0.5) * dxr, xp = (j + 1.5) * dxr;
                        fin[q] = rt_source(s, b, tprev - xa / C_NM_FS, y);
                        gin[q] = 0.5 * (rt_source(s, b, tprev - xp / C_NM_FS, y) - rt_source(s, b, tprev - xm / C_NM_FS, y));
                    }
                }
                for (int rx = 0; rx < s->nrx; ++rx) {
                    f[rx] = F[(size_t)ry * s->nrx + rx]; g[rx] = Gx[(size_t)ry * s->nrx + rx];
                    gt[rx] = Gy[(size_t)ry * s->nrx + rx];
                }
                double in, out;
                orc_rt_line(f, g, gt, s->nrx, nux, s->rt.scheme, 0, ng ? fin : NULL, ng ? gin : NULL, ng, &in, &out);
                for (int rx = 0; rx < s->nrx; ++rx) {
                    F[(size_t)ry * s->nrx + rx] = f[rx]; Gx[(size_t)ry * s->nrx + rx] = g[rx];
                    Gy[(size_t)ry * s->nrx + rx] = gt[rx];
                }
                inflow += in;
                outflow += out;
                if (nux > 0) s->tally[ORC_T_TRANS] += out * ncd * s->hv_b[b];
                else s->tally[ORC_T_BACK] += out * ncd * s->hv_b[b];
            }
            s->tally[ORC_T_INC] += inflow * ncd * s->hv_b[b];
            if (s->nry > 1 && s->o_vy[o] != 0.0) {
                const double nuy = C_NM_FS * dtr * s->o_vy[o] / dyr;
                for (int rx = 0; rx < s->nrx; ++rx) {
                    for (int ry = 0; ry < s->nry; ++ry) {
                        f[ry] = F[(size_t)ry * s->nrx + rx]; g[ry] = Gy[(size_t)ry * s->nrx + rx];
                        gt[ry] = Gx[(size_t)ry * s->nrx + rx];
                    }
                    double in, out;
                    orc_rt_line(f, g, gt, s->nry, nuy, s->rt.scheme, 1, NULL, NULL, 0, &in, &out);
                    for (int ry = 0; ry < s->nry; ++ry) {
                        F[(size_t)ry * s->nrx + rx] = f[ry]; Gy[(size_t)ry * s->nrx + rx] = g[ry];
                        Gx[(size_t)ry * s->nrx + rx] = gt[ry];
                    }
                }
            }
            for (int r = 0; r < nrc; ++r) after += F[r];
            s->tally[ORC_T_RT_NUM] += (after - before - inflow + outflow) * ncd * s->hv_b[b];
        }
    free(f); free(g); free(gt);
    /* (6) */
    for (int r = 0; r < nrc; ++r)
        for (int b = 0; b < nb; ++b) {
            double n = 0.0;
            for (int o = 0; o < nord; ++o) n += s->F[((size_t)o * nb + b) * nrc + r];
            s->n_pub[(size_t)r * nb + b] = n;
        }
    for (int c = 0; c < ncell; ++c) {
        const int r = rt_cell(s, c);
        for (int b = 0; b < nb; ++b) s->ph[(size_t)c * nb + b] = s->n_pub[(size_t)r * nb + b];
    }
    free(chi); free(ka); free(emc); free(W);
}

/* ---------------- per-cell physics ---------------- */
typedef struct {
    double X, Y, u[3], w; uint64_t id;
} newe;

typedef struct {
    newe *ne; int n, cap;
    double tally_ion, ka_esc, rt_applied;
    uint64_t cnt[ORC_NC];
    /* decision trace of the cell (see orc_trace) */
    double rel; uint32_t step; int cell;
    orc_near *nr; int nn, ncap;
    uint64_t ndraw, ndec;
} cellout;

/* a decision x < thr (or x > thr): counted; recorded when within rel of
 * the threshold.  draw != 0 for Monte-Carlo draws. */
static void decide(cellout *o, int draw, int kind, int species, uint64_t id, double x, double thr)
{
    if (!(o->rel > 0.0)) return;
    if (draw) o->ndraw++; else o->ndec++;
    if (!(fabs(x - thr) <= o->rel * fabs(thr))) return;
    if (o->nn == o->ncap) {
        o->ncap = o->ncap ? 2 * o->ncap : 8;
        o->nr = realloc(o->nr, sizeof(orc_near) * o->ncap);
    }
    orc_near *q = &o->nr[o->nn++];
    q->step = o->step; q->cell = o->cell; q->kind = kind; q->species = species; q->id = id;
    q->x = x; q->thr = thr;
}

static void push_new(cellout *o, double X, double Y, const double u[3], double w, uint64_t id)
{
    if (o->n == o->cap) {
        o->cap = o->cap ? 2 * o->cap : 16;
        o->ne = realloc(o->ne, sizeof(newe) * o->cap);
    }
    newe *q = &o->ne[o->n++];
    q->X = X; q->Y = Y; q->u[0] = u[0]; q->u[1] = u[1]; q->u[2] = u[2]; q->w = w; q->id = id;
}

static void iso_u(double ke, double rc, double rp, double u[3])
{
    double x = ke / ME_C2;
    double um = sqrt(x * (2.0 + x));
    double ct = 2.0 * rc - 1.0;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = 2.0 * PI * rp;
    u[0] = um * st * cos(ph); u[1] = um * st * sin(ph); u[2] = um * ct;
}

/* Forced thermalization (Sec. VI C, the variant that thermalizes the photo-
 * and Auger electrons instantly): after the rad-step processes, the free
 * electrons of the cell, those created in this step included, get momenta
 * drawn from a Maxwellian at kT = (2/3) E_ave (E_ave the weighted mean
 * kinetic energy), each component normal with standard deviation
 * sqrt(kT / m c^2).  The draw's small excess of momentum and energy is then
 * removed: the mean momentum is shifted back to the cell's, and the
 * momenta relative to it are scaled by the one factor that restores the
 * cell's kinetic energy (Newton on the relativistic energy), so both are
 * conserved exactly. */
typedef struct { double *u; double w; uint64_t id; } eref;

static double therm_energy(const eref *r, int n, const double V[3], const double *d, double a, double *slope)
{
    double K = 0.0, dK = 0.0;
    for (int k = 0; k < n; ++k) {
        double u[3] = {V[0] + a * d[3 * k], V[1] + a * d[3 * k + 1], V[2] + a * d[3 * k + 2]};
        K += r[k].w * kin(u, 1.0);
        dK += r[k].w * ME_C2 * (u[0] * d[3 * k] + u[1] * d[3 * k + 1] + u[2] * d[3 * k + 2]) / gam(u);
    }
    *slope = dK;
    return K;
}

static void thermalize(orc_slab *S, const int *pe, int ne, cellout *o, uint64_t seed, uint32_t step)
{
    eref *r = malloc(sizeof(eref) * (ne + o->n + 1));
    int n = 0;
    for (int k = 0; k < ne; ++k) {
        elec *e = &S->e[pe[k]];
        if (e->alive && e->w > 0.0) { r[n].u = e->u; r[n].w = e->w; r[n].id = e->id; ++n; }
    }
    for (int k = 0; k < o->n; ++k)
        if (o->ne[k].w > 0.0) { r[n].u = o->ne[k].u; r[n].w = o->ne[k].w; r[n].id = o->ne[k].id; ++n; }
    double W = 0.0, K = 0.0, P[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < n; ++k) {
        W += r[k].w;
        K += r[k].w * kin(r[k].u, 1.0);
        for (int c = 0; c < 3; ++c) P[c] += r[k].w * r[k].u[c];
    }
    if (n < 2 || W <= 0.0 || K <= 0.0) { free(r); return; }
    const double T = (2.0 / 3.0) * K / W, sig = sqrt(T / ME_C2);
    double Pn[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < n; ++k) {
        double q[4];
        draw4(seed, r[k].id, step, PU_THERM, q);
        double a0 = sqrt(-2.0 * log(q[0])), a1 = sqrt(-2.0 * log(q[2]));
        r[k].u[0] = sig * a0 * cos(2.0 * PI * q[1]);
        r[k].u[1] = sig * a0 * sin(2.0 * PI * q[1]);
        r[k].u[2] = sig * a1 * cos(2.0 * PI * q[3]);
        for (int c = 0; c < 3; ++c) Pn[c] += r[k].w * r[k].u[c];
    }
    /* mean momentum back to the cell's; peculiar momenta d about it */
    double V[3], *d = malloc(sizeof(double) * 3 * n);
    for (int c = 0; c < 3; ++c) V[c] = P[c] / W;
    for (int k = 0; k < n; ++k)
        for (int c = 0; c < 3; ++c) d[3 * k + c] = r[k].u[c] - Pn[c] / W;
    /* scale d by a so that the kinetic energy is K (convex in a, root >= 0) */
    double a = 1.0;
    for (int it = 0; it < 60; ++it) {
        double slope, Ka = therm_energy(r, n, V, d, a, &slope);
        if (slope <= 0.0) break;
        double da = (Ka - K) / slope;
        a -= da;
        if (a < 0.0) a = 0.0;
        if (fabs(da) < 1e-15 * (a > 1e-300 ? a : 1.0)) break;
    }
    for (int k = 0; k < n; ++k)
        for (int c = 0; c < 3; ++c) r[k].u[c] = V[c] + a * d[3 * k + c];
    free(d);
    free(r);
}

static void cell_physics(orc_slab *S, int cell, int *eidx, int ne, int *iidx, int ni, cellout *o)
{
    const orc_params *p = &S->p;
    const orc_tables *t = &S->t;
    uint32_t step = S->step;
    uint64_t seed = p->seed;
    double wi = p->w_ion;
    int rad = p->rad_every > 0 && (step % (uint32_t)p->rad_every) == 0;

    /* 1. canonical order: ascending Philox key, ties by id */
    int *pe = malloc(sizeof(int) * (ne + 1)), *pi = malloc(sizeof(int) * (ni + 1));
    {
        uint64_t *ids = calloc((ne > ni ? ne : ni) + 1, sizeof(uint64_t));
        int *perm = malloc(sizeof(int) * (ne > ni ? ne : ni) + 8);
        for (int k = 0; k < ne; ++k) ids[k] = S->e[eidx[k]].id;
        orc_pair_order(ne, ids, step, PU_PAIR_E, seed, perm);
        for (int k = 0; k < ne; ++k) pe[k] = eidx[perm[k]];
        for (int k = 0; k < ni; ++k) ids[k] = S->ion[iidx[k]].id;
        orc_pair_order(ni, ids, step, PU_PAIR_I, seed, perm);
        for (int k = 0; k < ni; ++k) pi[k] = iidx[perm[k]];
        free(ids); free(perm);
    }

    for (int k = 0; k < ne; ++k) S->e[pe[k]].cs = 0.0;

    /* 1b. radiation transport mode, rad steps: the energy the radiation
     * field gave up to (or took from) this cell's share of its rad cell
     * goes to the bulk electrons by one factor on their kinetic energy
     * (Sec. II: uniform heating or cooling); at most 90 % of their energy
     * is taken, the rest waits for the next rad step */
    const int rtmode = S->rt_on && rad;
    if (rtmode) {
        const int nbr = S->pulse.n_bins;
        for (int b = 0; b < nbr; ++b) S->c_chi[(size_t)cell * nbr + b] = 0.0;
        S->c_emc[cell] = 0.0;
        const double dE = S->c_dE[cell];
        if (dE != 0.0) {
            double K = 0.0;
            for (int k = 0; k < ne; ++k) {
                const elec *e = &S->e[pe[k]];
                const double ke = kin(e->u, 1.0);
                if (p->E_bulk <= 0.0 || ke < p->E_bulk) K += e->w * ke;
            }
            if (K > 0.0) {
                const double dEa = dE < -0.9 * K ? -0.9 * K : dE;
                const double f = 1.0 + dEa / K;
                for (int k = 0; k < ne; ++k) {
                    elec *e = &S->e[pe[k]];
                    if (p->E_bulk <= 0.0 || kin(e->u, 1.0) < p->E_bulk) scale_ke(e->u, f);
                }
                S->c_dE[cell] = dE - dEa;
                o->rt_applied += dEa;
            }
        }
    }

    /* 2. moments (FP64) */
    double We = 0, Wb = 0, Kb = 0, Q = 0;
    for (int k = 0; k < ne; ++k) {
        elec *e = &S->e[pe[k]];
        double ke = kin(e->u, 1.0);
        We += e->w;
        if (p->E_bulk > 0.0) decide(o, 0, ORC_N_EBULK, 0, e->id, ke, p->E_bulk);
        if (p->E_bulk <= 0.0 || ke < p->E_bulk) { Wb += e->w; Kb += e->w * ke; }
    }
    for (int k = 0; k < ni; ++k) Q += S->ion[pi[k]].Z + S->ion[pi[k]].zf;
    double n_e = We * p->n_ref, n_i = ni * wi * p->n_ref;
    double Te = Wb > 0 ? (2.0 / 3.0) * Kb / Wb : 0.0;
    double zbar = ni > 0 ? Q / ni : 0.0;
    double dE[ORC_NZ];
    for (int z = 0; z < ORC_NZ; ++z) dE[z] = orc_ipd(p->ipd_model, z, n_e, n_i, Te, zbar);
    double lnL = p->coulomb_log > 0 ? p->coulomb_log : orc_coulomb_log(n_e, Te, zbar);

    /* kinetic energy of the cell before the collisions */
    int coll = (p->flags & (ORC_F_COLL_EE | ORC_F_COLL_EI)) != 0;
    double Kpre = 0.0;
    if (coll) {
        for (int k = 0; k < ne; ++k) Kpre += S->e[pe[k]].w * kin(S->e[pe[k]].u, 1.0);
        for (int k = 0; k < ni; ++k) Kpre += wi * kin(S->ion[pi[k]].u, p->m_ion);
    }

    /* 3a. e-e collisions */
    if ((p->flags & ORC_F_COLL_EE) && ne >= 2) {
        int *pa = malloc(sizeof(int) * (ne + 3)), *pb = malloc(sizeof(int) * (ne + 3));
        double *fr = malloc(sizeof(double) * (ne + 3));
        int np = orc_ee_pairs(ne, pa, pb, fr);
        for (int k = 0; k < np; ++k) {
            elec *a = &S->e[pe[pa[k]]], *b = &S->e[pe[pb[k]]];
            double r[4];
            {
                const double sa = sqrt(a->u[0] * a->u[0] + a->u[1] * a->u[1] + a->u[2] * a->u[2]);
                const double sb = sqrt(b->u[0] * b->u[0] + b->u[1] * b->u[1] + b->u[2] * b->u[2]);
                const double m = sa > sb ? sa : sb;
                if (m > a->cs) a->cs = m;
                if (m > b->cs) b->cs = m;
            }
            draw4(seed, a->id, step, PU_COLL_EE, r);
            if (a->w != b->w) {
                double wm = a->w > b->w ? a->w : b->w;
                decide(o, 1, ORC_N_COLL_ACC, 0, a->id, r[3], (a->w < wm ? a->w : b->w) / wm);
            }
            double np2 = -1.0;
            o->cnt[ORC_C_EE] += orc_collide(a->u, b->u, 1.0, 1.0, -1.0, -1.0, a->w, b->w,
                                            n_e, lnL, p->dt * fr[k], r, &np2);
            if (np2 >= 0.0) decide(o, 0, ORC_N_BASIS, 0, a->id, np2, 0.25);
        }
        free(pa); free(pb); free(fr);
    }
    /* 3b. e-i collisions: the longer list in order, the shorter cycled.
     * Density of a pair: the cycled species' density times
     * max(w_a, w_b) / w_cycled, so that with the acceptance min(1,
     * w_other/w_self) every real electron sees n_i and every real ion n_e
     * (Takizuka-Abe pairing with Nanbu-Yonemura weights). */
    if ((p->flags & ORC_F_COLL_EI) && ne >= 1 && ni >= 1) {
        int nmax = ne >= ni ? ne : ni;
        for (int k = 0; k < nmax; ++k) {
            elec *a; ionr *b; double r[4], npair;
            if (ne >= ni) {
                a = &S->e[pe[k]]; b = &S->ion[pi[k % ni]];
                draw4(seed, a->id, step, PU_COLL_EI, r);
                npair = n_i * (a->w > wi ? a->w : wi) / wi;
            } else {
                b = &S->ion[pi[k]]; a = &S->e[pe[k % ne]];
                draw4(seed, b->id, step, PU_COLL_IE, r);
                npair = n_e * (a->w > wi ? a->w : wi) / a->w;
            }
            if (a->w != wi) {
                double wm = a->w > wi ? a->w : wi;
                decide(o, 1, ORC_N_COLL_ACC, 0, a->id, r[3], (a->w < wm ? a->w : wi) / wm);
            }
            double np2 = -1.0;
            o->cnt[ORC_C_EI] += orc_collide(a->u, b->u, 1.0, p->m_ion, -1.0, b->Z + b->zf,
                                            a->w, wi, npair, lnL, p->dt, r, &np2);
            if (np2 >= 0.0) decide(o, 0, ORC_N_BASIS, 0, a->id, np2, 0.25);
        }
    }

    /* 3c. weighted pairs conserve energy only on average: restore the cell's
     * kinetic energy exactly by the constant-factor scaling of the electron
     * kinetic energies (the operator Sec. IV uses for ionization) */
    if (coll && ne >= 1) {
        double Ke = 0.0, Ki = 0.0;
        for (int k = 0; k < ne; ++k) Ke += S->e[pe[k]].w * kin(S->e[pe[k]].u, 1.0);
        for (int k = 0; k < ni; ++k) Ki += wi * kin(S->ion[pi[k]].u, p->m_ion);
        if (Ke > 0.0) {
            double f = 1.0 + (Kpre - Ke - Ki) / Ke;
            if (f > 0.0)
                for (int k = 0; k < ne; ++k) scale_ke(S->e[pe[k]].u, f);
        }
    }

    /* 4. Lotz impact ionization with cell-average probability per charge state */
    int nnew_imp = 0;
    if ((p->flags & ORC_F_IONIZE) && ne >= 1 && ni >= 1) {
        int present[ORC_NZ] = {0};
        for (int k = 0; k < ni; ++k) if (S->ion[pi[k]].Z < 13) present[S->ion[pi[k]].Z] = 1;
        double Pz[ORC_NZ] = {0};
        double Kt = 0.0;
        for (int k = 0; k < ne; ++k) Kt += S->e[pe[k]].w * kin(S->e[pe[k]].u, 1.0);
        for (int z = 0; z < 13; ++z) {
            if (!present[z]) continue;
            double R = 0.0;
            for (int k = 0; k < ne; ++k) {
                elec *e = &S->e[pe[k]];
                double g = gam(e->u);
                double beta = sqrt(e->u[0] * e->u[0] + e->u[1] * e->u[1] + e->u[2] * e->u[2]) / g;
                R += e->w * beta * orc_lotz(t, z, dE[z], kin(e->u, 1.0));
            }
            Pz[z] = p->dt * C_CM_FS * p->n_ref * R;
            if (Pz[z] > 1.0) o->cnt[ORC_C_PGT1]++;
        }
        double paid = 0.0;
        int stop = 0;
        for (int k = 0; k < ni; ++k) {
            ionr *q = &S->ion[pi[k]];
            if (q->Z >= 13) continue;
            double r[4];
            draw4(seed, q->id, step, PU_ION, r);
            decide(o, 1, ORC_N_ION_DRAW, 1, q->id, r[0], Pz[q->Z]);
            if (!(r[0] < Pz[q->Z])) continue;
            double I = ion_energy(t, q->Z, q->nK, dE);
            if (!stop) decide(o, 0, ORC_N_ION_PAY, -1, 0, paid + wi * I, Kt);
            if (stop || paid + wi * I > Kt) { stop = 1; o->cnt[ORC_C_ION_REJ]++; continue; }
            paid += wi * I;
            int s = outermost(13 - q->Z, q->nK);
            remove_electron(&q->Z, &q->nK, s);
            double u0[3] = {0, 0, 0};
            push_new(o, q->X, q->Y, u0, wi, ((uint64_t)(((step + 1u) << 2) | K_IMPACT) << 32) | q->id);
            o->cnt[ORC_C_ION]++;
            ++nnew_imp;
        }
        if (paid > 0.0) {
            double f = 1.0 - paid / Kt;
            for (int k = 0; k < ne; ++k) scale_ke(S->e[pe[k]].u, f);
            o->tally_ion += paid;
        }
    }

    /* 5. EOS-clamped three-body recombination */
    if ((p->flags & ORC_F_RECOMB) && ni >= 1) {
        double Q2 = 0.0;
        for (int k = 0; k < ni; ++k) Q2 += S->ion[pi[k]].Z + S->ion[pi[k]].zf;
        double zb = Q2 / ni;
        double Wb2 = 0.0, Kb2 = 0.0, Wex = 0.0;
        for (int k = 0; k < ne; ++k) {
            elec *e = &S->e[pe[k]];
            double ke = kin(e->u, 1.0);
            Wex += e->w;
            if (p->E_bulk <= 0.0 || ke < p->E_bulk) { Wb2 += e->w; Kb2 += e->w * ke; }
        }
        for (int k = o->n - nnew_imp; k < o->n; ++k) {  /* new zero-energy electrons */
            if (p->E_bulk <= 0.0 || 0.0 < p->E_bulk) Wb2 += o->ne[k].w;
        }
        double Te2 = Wb2 > 0 ? (2.0 / 3.0) * Kb2 / Wb2 : 0.0;
        double zeos = orc_eos(t, n_i, Te2);
        int Kev = 0;
        if (zb > zeos) {
            const double xk = (zb - zeos) * ni + 0.5;
            decide(o, 0, ORC_N_REC_K, -1, 0, xk, floor(xk + 0.5));
            Kev = (int)floor(xk);
        }
        /* events are dealt round-robin over the ions in canonical order; an
         * ion can take several in one step (no limit on the instantaneous
         * rate), at most as many as its charge */
        int elig = 0;
        for (int k = 0; k < ni; ++k) elig += S->ion[pi[k]].Z;
        if (Kev > elig) Kev = elig;
        int wcap = (int)floor(Wex / wi + 1e-9);
        if (Kev >= wcap) decide(o, 0, ORC_N_REC_CAP, -1, 0, Wex / wi, floor(Wex / wi + 0.5));
        if (Kev > wcap) Kev = wcap;
        if (Kev > 0) {
            int *nrec = calloc(ni, sizeof(int));
            int left = Kev;
            while (left > 0) {
                for (int k = 0; k < ni && left > 0; ++k)
                    if (S->ion[pi[k]].Z - nrec[k] >= 1) { nrec[k]++; --left; }
            }
            double Wrem = Kev * wi;
            /* electrons give up weight in canonical order */
            double *take = calloc(ne + 1, sizeof(double));
            double before = 0.0, remKE = 0.0;
            for (int k = 0; k < ne; ++k) {
                elec *e = &S->e[pe[k]];
                double tk = Wrem - before;
                decide(o, 0, ORC_N_REC_TAKE, -1, 0, before + e->w, Wrem);
                if (tk > e->w) tk = e->w;
                if (tk < 0.0) tk = 0.0;
                take[k] = tk;
                before += e->w;
                remKE += tk * kin(e->u, 1.0);
            }
            /* binding released: Z -> Z-1 -> ... for each event of an ion */
            double bind = 0.0;
            for (int k = 0; k < ni; ++k) {
                ionr *q = &S->ion[pi[k]];
                for (int r = 1; r <= nrec[k]; ++r)
                    bind += wi * ion_energy(t, q->Z - r, q->nK, dE);
            }
            /* bulk energy left to scale */
            double Krem = 0.0;
            for (int k = 0; k < ne; ++k) {
                elec *e = &S->e[pe[k]];
                double ke = kin(e->u, 1.0);
                if (p->E_bulk <= 0.0 || ke < p->E_bulk) Krem += (e->w - take[k]) * ke;
            }
            if (Krem > 0.0) {
                double f = 1.0 + (remKE + bind) / Krem;
                for (int k = 0; k < ne; ++k) {
                    elec *e = &S->e[pe[k]];
                    double ke = kin(e->u, 1.0);
                    int bulk = p->E_bulk <= 0.0 || ke < p->E_bulk;
                    e->w -= take[k];
                    if (take[k] > 0.0 && e->w <= 0.0) { e->w = 0.0; e->alive = 0; }
                    if (bulk && e->alive) scale_ke(e->u, f);
                }
                for (int k = 0; k < ni; ++k) S->ion[pi[k]].Z -= nrec[k];
                o->tally_ion -= bind;
                o->cnt[ORC_C_REC] += (uint64_t)Kev;
            }
            free(take); free(nrec);
        }
    }

    /* 6. rad step: photoionization then K-vacancy decay */
    if (rad && (p->flags & (ORC_F_PHOTO | ORC_F_DECAY)) && ni >= 1) {
        int nb = S->have_pulse ? S->pulse.n_bins : 0;
        double dtr = p->rad_every * p->dt;
        double *ph = nb ? S->ph + (size_t)cell * nb : NULL;
        if ((p->flags & ORC_F_PHOTO) && nb) {
            double cph = C_CM_FS * dtr * p->n_ref;
            double *n0 = malloc(sizeof(double) * nb);
            memcpy(n0, ph, sizeof(double) * nb);
            /* photons left in the bins for the events of this cell: the
             * cell's own photon numbers, or in transport mode a copy (the
             * field loses the absorbed photons through the opacity instead) */
            double *avail = rtmode ? malloc(sizeof(double) * nb) : ph;
            if (rtmode) memcpy(avail, ph, sizeof(double) * nb);
            double *chi = rtmode ? S->c_chi + (size_t)cell * nb : NULL;
            for (int k = 0; k < ni; ++k) {
                ionr *q = &S->ion[pi[k]];
                int nbd = 13 - q->Z, occ[ORC_NS];
                if (nbd <= 0 || !orc_occ(nbd, q->nK, occ)) continue;
                if (chi) {
                    /* opacity of the cell in each bin: sum over subshells
                     * of N_s sigma_s above the lowered edge (Eq. 2's
                     * absorption), for the radiation transport */
                    for (int q2 = 0; q2 < ORC_NS; ++q2) {
                        if (!occ[q2]) continue;
                        const double ed = lowered(t, q->Z, q2, dE[q->Z]);
                        for (int b = 0; b < nb; ++b)
                            if (S->hv_b[b] > ed) chi[b] += p->n_ref * wi * occ[q2] * S->sig_b[q2 * nb + b];
                    }
                }
                double ra[4], rb[4];
                draw4(seed, q->id, step, PU_PHOTO_A, ra);
                draw4(seed, q->id, step, PU_PHOTO_B, rb);
                double rs[ORC_NS] = {ra[0], ra[1], ra[2], ra[3], rb[0]};
                int sub = -1; double Ps = 0.0, edge = 0.0;
                for (int q2 = 0; q2 < ORC_NS; ++q2) {
                    if (!occ[q2]) continue;
                    double ed = lowered(t, q->Z, q2, dE[q->Z]);
                    double acc = 0.0;
                    for (int b = 0; b < nb; ++b) {
                        decide(o, 0, ORC_N_PH_EDGE, 1, q->id, S->hv_b[b], ed);
                        if (S->hv_b[b] > ed) acc += n0[b] * S->sig_b[q2 * nb + b];
                    }
                    double P = cph * occ[q2] * acc;
                    if (P > 0.0) decide(o, 1, ORC_N_PH_DRAW, 1, q->id, rs[q2], P);
                    if (rs[q2] < P) { sub = q2; Ps = P; edge = ed; break; }
                }
                if (sub < 0) continue;
                double target = rb[1] * Ps, cum = 0.0;
                int bin = -1, lastpos = -1;
                for (int b = 0; b < nb; ++b) {
                    double c = (S->hv_b[b] > edge) ? cph * occ[sub] * n0[b] * S->sig_b[sub * nb + b] : 0.0;
                    if (c > 0.0) lastpos = b;
                    cum += c;
                    if (c > 0.0) decide(o, 0, ORC_N_PH_BIN, 1, q->id, cum, target);
                    if (cum > target) { bin = b; break; }
                }
                if (bin < 0) bin = lastpos;
                if (bin < 0) continue;
                decide(o, 0, ORC_N_PH_PART, -1, 0, avail[bin], wi);
                double g = avail[bin] < wi ? avail[bin] : wi;
                if (g <= 0.0) continue;
                avail[bin] -= g;
                if (rtmode) {
                    /* the plasma takes these photons' energy now; the field
                     * gives it up through its opacity at the next transport
                     * step: owed until then */
                    S->c_emc[cell] += g * S->hv_b[bin];
                    o->rt_applied += g * S->hv_b[bin];
                }
                if (g == wi) {
                    remove_electron(&q->Z, &q->nK, sub);
                } else {
                    q->zf += g / wi;
                    o->cnt[ORC_C_PART]++;
                    decide(o, 0, ORC_N_PH_ZF, 1, q->id, q->zf, 1.0);
                    if (q->zf >= 1.0) {
                        q->zf -= 1.0;
                        int so = outermost(13 - q->Z, q->nK);
                        if (so >= 0) remove_electron(&q->Z, &q->nK, so);
                    }
                }
                double u[3];
                iso_u(S->hv_b[bin] - edge, rb[2], rb[3], u);
                push_new(o, q->X, q->Y, u, g, ((uint64_t)(((step + 1u) << 2) | K_PHOTO) << 32) | q->id);
                o->tally_ion += g * edge;
                o->cnt[ORC_C_PH0 + sub]++;
            }
            free(n0);
            if (rtmode) free(avail);
        }
        if (p->flags & ORC_F_DECAY) {
            for (int k = 0; k < ni; ++k) {
                ionr *q = &S->ion[pi[k]];
                if (q->nK <= 0) continue;
                int nbd = 13 - q->Z, occ[ORC_NS];
                if (!orc_occ(nbd, q->nK, occ)) continue;
                double tau = t->tauK[nbd][q->nK - 1];
                if (tau <= 0.0) continue;
                double r[4];
                draw4(seed, q->id, step, PU_DECAY, r);
                decide(o, 1, ORC_N_DECAY, 1, q->id, r[0], dtr / tau);
                if (!(r[0] < dtr / tau)) continue;
                double om = t->omegaK[nbd][q->nK - 1];
                int nl = occ[1] + occ[2];
                decide(o, 1, ORC_N_BRANCH, 1, q->id, r[1], 1.0 - om);
                if (r[1] < 1.0 - om) {
                    if (nl < 2) continue;
                    double e2s = lowered(t, q->Z, 1, dE[q->Z]), e2p = lowered(t, q->Z, 2, dE[q->Z]);
                    double EA = t->E_Ka[q->Z] - (occ[1] * e2s + occ[2] * e2p) / nl;
                    if (EA < 0.0) EA = 0.0;
                    int kocc = occ[0] + 1, nb2 = nbd - 1;
                    q->Z += 1;
                    q->nK = (nb2 < 2 ? nb2 : 2) - kocc;
                    double u[3];
                    iso_u(EA, r[2], r[3], u);
                    push_new(o, q->X, q->Y, u, wi, ((uint64_t)(((step + 1u) << 2) | K_AUGER) << 32) | q->id);
                    o->tally_ion -= wi * EA;
                    o->cnt[ORC_C_AUG]++;
                } else {
                    if (occ[2] < 1) continue;
                    double Eka = t->E_Ka[q->Z];
                    q->nK -= 1;
                    int hit = -1;
                    if (nb) {
                        double hw = 0.5 * S->pulse.bandwidth / nb;
                        for (int b = 0; b < nb; ++b)
                            if (Eka >= S->hv_b[b] - hw && Eka < S->hv_b[b] + hw) { hit = b; break; }
                    }
                    if (hit >= 0) ph[hit] += wi * Eka / S->hv_b[hit];
                    else o->ka_esc += wi * Eka;
                    o->tally_ion -= wi * Eka;
                    o->cnt[ORC_C_KA]++;
                }
            }
        }
    }
    /* 7. rad step, forced-thermalization variant */
    if (rad && (p->flags & ORC_F_THERM)) thermalize(S, pe, ne, o, seed, step);
    /* 8. transport mode: the cell's electron weight, its share of the next
     * heating of its rad cell */
    if (rtmode) {
        double W = 0.0;
        for (int k = 0; k < ne; ++k) if (S->e[pe[k]].alive) W += S->e[pe[k]].w;
        for (int k = 0; k < o->n; ++k) W += o->ne[k].w;
        S->c_w[cell] = W;
    }
    free(pe); free(pi);
}

/* ---------------- fields ---------------- */
static double kappa_J(const orc_slab *s)
{
    double E0 = ME_KG * C_SI / (Q_E * 1e-15);
    return Q_E * s->p.n_ref * 1e6 * 1e-9 / (EPS0 * E0);
}

#define IX(j, i) ((size_t)(j) * W + (i))
/* B half step: dB/dt = -curl E, times the field speed cf */
static void b_half(double *f, int nx, int ny, double dx, double dy, double h, double cf)
{
    int W = nx + 1;
    size_t ng = (size_t)ny * W;
    double *ex = f, *ey = f + ng, *ez = f + 2 * ng, *bx = f + 3 * ng, *by = f + 4 * ng, *bz = f + 5 * ng;
    for (int j = 0; j < ny; ++j) {
        int jp = (j + 1) % ny;
        for (int i = 0; i <= nx; ++i)
            bx[IX(j, i)] -= h * cf * (ez[IX(jp, i)] - ez[IX(j, i)]) / dy;
        for (int i = 0; i < nx; ++i) {
            by[IX(j, i)] += h * cf * (ez[IX(j, i + 1)] - ez[IX(j, i)]) / dx;
            bz[IX(j, i)] -= h * cf * ((ey[IX(j, i + 1)] - ey[IX(j, i)]) / dx
                                           - (ex[IX(jp, i)] - ex[IX(j, i)]) / dy);
        }
    }
}

/* E full step: dE/dt = cf curl B - kappa J; first-order Mur at x = 0, L */
static void e_full(double *f, const double *jc, int nx, int ny, double dx, double dy,
                   double dtf, double kap, double cf)
{
    int W = nx + 1;
    size_t ng = (size_t)ny * W;
    double *ex = f, *ey = f + ng, *ez = f + 2 * ng, *bx = f + 3 * ng, *by = f + 4 * ng, *bz = f + 5 * ng;
    const double *jx = jc, *jy = jc + ng, *jz = jc + 2 * ng;
    double mur = (cf * dtf - dx) / (cf * dtf + dx);
    for (int j = 0; j < ny; ++j) {
        int jm = (j - 1 + ny) % ny;
        double y0 = ey[IX(j, 0)], y1 = ey[IX(j, 1)], yn1 = ey[IX(j, nx - 1)], yn = ey[IX(j, nx)];
        double z0 = ez[IX(j, 0)], z1 = ez[IX(j, 1)], zn1 = ez[IX(j, nx - 1)], zn = ez[IX(j, nx)];
        for (int i = 0; i < nx; ++i)
            ex[IX(j, i)] += dtf * (cf * (bz[IX(j, i)] - bz[IX(jm, i)]) / dy - kap * jx[IX(j, i)]);
        for (int i = 1; i < nx; ++i) {
            ey[IX(j, i)] += dtf * (-cf * (bz[IX(j, i)] - bz[IX(j, i - 1)]) / dx - kap * jy[IX(j, i)]);
            ez[IX(j, i)] += dtf * (cf * ((by[IX(j, i)] - by[IX(j, i - 1)]) / dx
                                              - (bx[IX(j, i)] - bx[IX(jm, i)]) / dy)
                                   - kap * jz[IX(j, i)]);
        }
        ey[IX(j, 0)] = y1 + mur * (ey[IX(j, 1)] - y0);
        ez[IX(j, 0)] = z1 + mur * (ez[IX(j, 1)] - z0);
        ey[IX(j, nx)] = yn1 + mur * (ey[IX(j, nx - 1)] - yn);
        ez[IX(j, nx)] = zn1 + mur * (ez[IX(j, nx - 1)] - zn);
    }
}
#undef IX

/* Field speed of the Yee update: c where the particle step resolves it
 * (c dt within cfl times the Yee limit), otherwise the largest speed that
 * the step resolves.  The particle step c dt = 6 nm exceeds the 2-5 nm cells
 * of the workloads; subcycling the fields with the current held fixed let
 * the particles see the transverse waves only every dt, and the transverse
 * fields then grew exponentially once e-i collisions fed them noise (both
 * sides, within a few fs).  Gauss's law goes through the continuity of the
 * deposited current and does not involve cf, so the electrostatic and
 * sheath fields are unchanged; only light waves and magnetic induction are
 * slowed. */
double orc_field_speed(const orc_params *p)
{
    double inv = 1.0 / (p->dx * p->dx) + (p->ny > 1 ? 1.0 / (p->dy * p->dy) : 0.0);
    double cmax = p->cfl / (p->dt * sqrt(inv));
    return C_NM_FS < cmax ? C_NM_FS : cmax;
}

/* The current the field update sees: the deposited current smoothed by the
 * binomial (1/4, 1/2, 1/4) filter along x, and along y (periodic) in 2D,
 * each component over its own points (Jx on the nx faces of a row, Jy and
 * Jz on its nx + 1 nodes; nothing beyond the slab).  A linear filter of
 * constant weights commutes with the discrete divergence away from the x
 * boundaries, so Gauss's law holds there for the equally smoothed charge;
 * the smoothing damps the grid-scale modes through which cells many Debye
 * lengths wide heat numerically. */
static void smooth_current(const double *jc, double *out, int nx, int ny)
{
    const int W = nx + 1;
    const size_t ng = (size_t)ny * W;
    for (int c = 0; c < 3; ++c) {
        const double *src = jc + c * ng;
        double *dst = out + c * ng;
        const int imax = c == 0 ? nx - 1 : nx;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < W; ++i) {
                if (i > imax) { dst[(size_t)j * W + i] = 0.0; continue; }
                double acc = 0.0;
                for (int b = -1; b <= 1; ++b) {
                    if (ny == 1 && b != 0) continue;
                    const int jj = (j + b + ny) % ny;
                    const double wy = ny == 1 ? 1.0 : (b == 0 ? 0.5 : 0.25);
                    for (int a = -1; a <= 1; ++a) {
                        const int ii = i + a;
                        if (ii < 0 || ii > imax) continue;
                        acc += wy * (a == 0 ? 0.5 : 0.25) * src[(size_t)jj * W + ii];
                    }
                }
                dst[(size_t)j * W + i] = acc;
            }
    }
}

static void field_step(orc_slab *s)
{
    const orc_params *p = &s->p;
    const double cf = orc_field_speed(p), dt = p->dt, kap = kappa_J(s);
    const size_t ng = (size_t)p->ny * (p->nx + 1);
    double *js = (double *)malloc(sizeof(double) * 3 * ng);
    if (!js) abort();
    smooth_current(s->j, js, p->nx, p->ny);
    b_half(s->f, p->nx, p->ny, p->dx, p->dy, 0.5 * dt, cf);
    e_full(s->f, js, p->nx, p->ny, p->dx, p->dy, dt, kap, cf);
    b_half(s->f, p->nx, p->ny, p->dx, p->dy, 0.5 * dt, cf);
    free(js);
}

/* field at (X, Y): CIC from the staggered grid, zero outside [0, nx] */
static double grid_at(const double *F, int nx, int ny, double X, double Y, int hx, int hy)
{
    double xs = X - (hx ? 0.5 : 0.0), ys = Y - (hy ? 0.5 : 0.0);
    int i0 = (int)floor(xs), j0 = (int)floor(ys);
    double fx = xs - i0, fy = ys - j0;
    int imax = hx ? nx - 1 : nx;
    double v = 0.0;
    for (int a = 0; a < 2; ++a) {
        int i = i0 + a;
        if (i < 0 || i > imax) continue;
        double wx = a ? fx : 1.0 - fx;
        for (int b = 0; b < 2; ++b) {
            int jj = wrapy(j0 + b, ny);
            double wy = b ? fy : 1.0 - fy;
            v += wx * wy * F[(size_t)jj * (nx + 1) + i];
        }
    }
    return v;
}

static void gather(const orc_slab *s, double X, double Y, double e[3], double b[3])
{
    int nx = s->p.nx, ny = s->p.ny;
    size_t ng = (size_t)ny * (nx + 1);
    const double *f = s->f;
    e[0] = grid_at(f, nx, ny, X, Y, 1, 0);
    e[1] = grid_at(f + ng, nx, ny, X, Y, 0, 1);
    e[2] = grid_at(f + 2 * ng, nx, ny, X, Y, 0, 0);
    b[0] = grid_at(f + 3 * ng, nx, ny, X, Y, 0, 1);
    b[1] = grid_at(f + 4 * ng, nx, ny, X, Y, 1, 0);
    b[2] = grid_at(f + 5 * ng, nx, ny, X, Y, 1, 1);
}

/* push one particle; returns 0 if it left through an x boundary */
static int push_one(orc_slab *s, double *X, double *Y, double u[3], double qm, double qw)
{
    const orc_params *p = &s->p;
    double e[3], b[3];
    gather(s, *X, *Y, e, b);
    orc_boris(u, e, b, qm, p->dt);
    double g = gam(u);
    double X1 = *X + u[0] / g * C_NM_FS * p->dt / p->dx;
    double Y1 = p->ny > 1 ? *Y + u[1] / g * C_NM_FS * p->dt / p->dy : *Y;
    if (p->flags & ORC_F_FIELD)
        orc_deposit(p->nx, p->ny, p->dx, p->dy, p->dt, *X, *Y, X1, Y1,
                    u[2] / g * C_NM_FS, u[1] / g * C_NM_FS, qw, s->j);
    if (p->ny > 1) {
        Y1 = fmod(Y1, (double)p->ny);
        if (Y1 < 0.0) Y1 += p->ny;
        if (Y1 >= p->ny) Y1 -= p->ny;
    }
    *X = X1; *Y = Y1;
    return X1 >= 0.0 && X1 < p->nx;
}

/* ---------------- step ---------------- */
static int cell_of(const orc_slab *s, double X, double Y)
{
    int i = (int)floor(X), j = s->p.ny > 1 ? (int)floor(Y) : 0;
    return j * s->p.nx + i;
}

void orc_step(orc_slab *s, int nsteps, int nthreads)
{
    const orc_params *p = &s->p;
    int ncell = p->nx * p->ny;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int it = 0; it < nsteps; ++it) {
        int rad = p->rad_every > 0 && (s->step % (uint32_t)p->rad_every) == 0;
        if (rad && s->rt_on) rt_step(s);
        else if (rad && (p->flags & ORC_F_PHOTO) && s->have_pulse) march(s);

        /* bucket by cell (counting sort) */
        int *cse = calloc(ncell + 1, sizeof(int)), *csi = calloc(ncell + 1, sizeof(int));
        int *oe = malloc(sizeof(int) * (s->ne + 1)), *oi = malloc(sizeof(int) * (s->ni + 1));
        for (int k = 0; k < s->ne; ++k) cse[cell_of(s, s->e[k].X, s->e[k].Y) + 1]++;
        for (int k = 0; k < s->ni; ++k) csi[cell_of(s, s->ion[k].X, s->ion[k].Y) + 1]++;
        for (int c = 0; c < ncell; ++c) { cse[c + 1] += cse[c]; csi[c + 1] += csi[c]; }
        {
            int *fe = calloc(ncell, sizeof(int)), *fi = calloc(ncell, sizeof(int));
            for (int k = 0; k < s->ne; ++k) { int c = cell_of(s, s->e[k].X, s->e[k].Y); oe[cse[c] + fe[c]++] = k; }
            for (int k = 0; k < s->ni; ++k) { int c = cell_of(s, s->ion[k].X, s->ion[k].Y); oi[csi[c] + fi[c]++] = k; }
            free(fe); free(fi);
        }
        cellout *co = calloc(ncell, sizeof(cellout));
        for (int c = 0; c < ncell; ++c) { co[c].rel = s->trace_rel; co[c].step = s->step; co[c].cell = c; }
#pragma omp parallel for schedule(dynamic, 16)
        for (int c = 0; c < ncell; ++c)
            cell_physics(s, c, oe + cse[c], cse[c + 1] - cse[c], oi + csi[c], csi[c + 1] - csi[c], &co[c]);
        /* merge: new electrons in cell order, tallies */
        int add = 0;
        for (int c = 0; c < ncell; ++c) add += co[c].n;
        int ne_old = s->ne;
        ensure_e(s, s->ne + add);
        for (int c = 0; c < ncell; ++c) {
            for (int k = 0; k < co[c].n; ++k) {
                elec *e = &s->e[s->ne++];
                newe *q = &co[c].ne[k];
                e->X = q->X; e->Y = q->Y; e->u[0] = q->u[0]; e->u[1] = q->u[1]; e->u[2] = q->u[2];
                e->w = q->w; e->id = q->id; e->alive = 1; e->cs = 0.0;
            }
            s->tally[ORC_T_ION] += co[c].tally_ion;
            s->tally[ORC_T_KA_ESC] += co[c].ka_esc;
            s->tally[ORC_T_RT_PEND] -= co[c].rt_applied;
            for (int q = 0; q < ORC_NC; ++q) s->cnt[q] += co[c].cnt[q];
            s->ndraw += co[c].ndraw;
            s->ndec += co[c].ndec;
            for (int k = 0; k < co[c].nn; ++k) {
                if (s->nnear == s->capnear) {
                    s->capnear = s->capnear ? 2 * s->capnear : 64;
                    s->near = realloc(s->near, sizeof(orc_near) * s->capnear);
                }
                s->near[s->nnear++] = co[c].nr[k];
            }
            free(co[c].nr);
            free(co[c].ne);
        }
        (void)ne_old;
        free(co); free(cse); free(csi); free(oe); free(oi);

        /* push + deposit */
        size_t ng = (size_t)p->ny * (p->nx + 1);
        memset(s->j, 0, sizeof(double) * 3 * ng);
        if (p->flags & ORC_F_PUSH) {
            for (int k = 0; k < s->ne; ++k) {
                elec *e = &s->e[k];
                if (!e->alive) continue;
                double ke = kin(e->u, 1.0);
                if (!push_one(s, &e->X, &e->Y, e->u, -1.0, -e->w)) {
                    e->alive = 0;
                    s->tally[ORC_T_ESC] += e->w * ke;
                    s->cnt[ORC_C_ESC_E]++;
                }
            }
            int w = 0;
            for (int k = 0; k < s->ni; ++k) {
                ionr *q = &s->ion[k];
                double qc = q->Z + q->zf;
                double ke = kin(q->u, p->m_ion);
                int in = push_one(s, &q->X, &q->Y, q->u, qc / p->m_ion, qc * p->w_ion);
                if (!in) { s->tally[ORC_T_ESC] += p->w_ion * ke; s->cnt[ORC_C_ESC_I]++; continue; }
                s->ion[w++] = *q;
            }
            s->ni = w;
        }
        /* drop dead electrons */
        {
            int w = 0;
            for (int k = 0; k < s->ne; ++k) if (s->e[k].alive && s->e[k].w > 0.0) s->e[w++] = s->e[k];
            s->ne = w;
        }
        if (p->flags & ORC_F_FIELD) field_step(s);
        s->step++;
    }
}

void orc_tallies(orc_slab *s, double *t, uint64_t *c)
{
    const orc_params *p = &s->p;
    double kee = 0.0, kei = 0.0, ph = 0.0, fe = 0.0;
    for (int k = 0; k < s->ne; ++k) kee += s->e[k].w * kin(s->e[k].u, 1.0);
    for (int k = 0; k < s->ni; ++k) kei += p->w_ion * kin(s->ion[k].u, p->m_ion);
    if (s->have_pulse && s->rt_on) {
        /* the rad field, plus the K-alpha photons the cells added since it
         * was published */
        const int nb = s->pulse.n_bins;
        for (int o = 0; o < s->nord; ++o)
            for (int b = 0; b < nb; ++b)
                for (int r = 0; r < s->nrc; ++r)
                    ph += s->F[((size_t)o * nb + b) * s->nrc + r] * s->ncd * s->hv_b[b];
        for (int c = 0; c < p->nx * p->ny; ++c)
            for (int b = 0; b < nb; ++b)
                ph += (s->ph[(size_t)c * nb + b] - s->n_pub[(size_t)rt_cell(s, c) * nb + b]) * s->hv_b[b];
    } else if (s->have_pulse) {
        int nb = s->pulse.n_bins;
        for (size_t q = 0; q < (size_t)p->ny * p->nx * nb; ++q) ph += s->ph[q] * s->hv_b[q % nb];
    }
    size_t ng = (size_t)p->ny * (p->nx + 1);
    for (size_t q = 0; q < 6 * ng; ++q) fe += s->f[q] * s->f[q];
    double E0 = ME_KG * C_SI / (Q_E * 1e-15);
    fe *= EPS0 * E0 * E0 / (2.0 * p->n_ref * 1e6 * Q_E);
    for (int q = 0; q < ORC_NT; ++q) t[q] = s->tally[q];
    t[ORC_T_KE_E] = kee; t[ORC_T_KE_I] = kei; t[ORC_T_PHOT] = ph; t[ORC_T_FIELD] = fe;
    for (int q = 0; q < ORC_NC; ++q) c[q] = s->cnt[q];
}

/* ---------------- decision trace ---------------- */
void orc_trace(orc_slab *s, double rel)
{
    s->trace_rel = rel;
    s->nnear = 0;
    s->ndraw = s->ndec = 0;
}
int orc_trace_count(const orc_slab *s) { return s->nnear; }
void orc_trace_decisions(const orc_slab *s, uint64_t out[2]) { out[0] = s->ndraw; out[1] = s->ndec; }
void orc_trace_get(const orc_slab *s, orc_near *out)
{
    if (s->nnear) memcpy(out, s->near, sizeof(orc_near) * s->nnear);
}

/* charge-state distribution (fractional charges split between Z and Z+1)
 * and the electron energy distribution on n_E log bins 0.1 eV .. E_max */
void orc_diag(const orc_slab *s, double *csd, int n_E, double E_max, double *eedf)
{
    for (int z = 0; z < ORC_NZ; ++z) csd[z] = 0.0;
    double tot = 0.0;
    for (int k = 0; k < s->ni; ++k) {
        const ionr *q = &s->ion[k];
        csd[q->Z] += 1.0 - q->zf;
        if (q->zf > 0.0 && q->Z < 13) csd[q->Z + 1] += q->zf;
        tot += 1.0;
    }
    for (int z = 0; z < ORC_NZ; ++z) csd[z] = tot > 0 ? csd[z] / tot : 0.0;
    for (int b = 0; b < n_E; ++b) eedf[b] = 0.0;
    double W = 0.0, lo = 0.1, lr = log(E_max / lo);
    for (int k = 0; k < s->ne; ++k) {
        double ke = kin(s->e[k].u, 1.0);
        int b = ke <= lo ? 0 : (int)floor(log(ke / lo) / lr * n_E);
        if (b < 0) b = 0;
        if (b >= n_E) b = n_E - 1;
        eedf[b] += s->e[k].w;
        W += s->e[k].w;
    }
    for (int b = 0; b < n_E; ++b) eedf[b] = W > 0 ? eedf[b] / W : 0.0;
}
