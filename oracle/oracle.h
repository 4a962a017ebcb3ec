/* FP64 CPU oracle for the collisional PIC step of Royle et al. (PICLS,
 * "Kinetic modeling of x-ray laser-driven solid Al plasmas via particle-in-
 * cell simulation").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Units: lengths nm (positions in cell units), times fs, energies eV,
 * momenta u = gamma*v/c, weights in units of n_ref*V_cell, fields
 * normalized by E0 = m_e c/(e*1fs) and B0 = m_e/(e*1fs).
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#define ORC_NS 5      /* subshells 1s 2s 2p 3s 3p */
#define ORC_NZ 14     /* charge states 0..13 of Al */

enum {
    ORC_F_COLL_EE = 1, ORC_F_COLL_EI = 2, ORC_F_IONIZE = 4, ORC_F_RECOMB = 8,
    ORC_F_PHOTO = 16, ORC_F_DECAY = 32, ORC_F_PUSH = 64, ORC_F_FIELD = 128,
    ORC_F_THERM = 256     /* forced thermalization on rad steps (Sec. VI C variant) */
};

typedef struct {
    int nx, ny;
    double dx, dy, dt;
    int rad_every;
    uint64_t seed;
    double cfl;
    double n_ref;        /* cm^-3 */
    double w_ion;        /* common ion weight */
    double m_ion;        /* ion mass / m_e */
    double E_bulk;       /* <= 0: all electrons are bulk */
    int ipd_model;       /* 0 none, 1 Ecker-Kroll, 2 Stewart-Pyatt */
    double coulomb_log;  /* <= 0: computed per cell */
    unsigned flags;
} orc_params;

typedef struct {
    double lotz_a[ORC_NS], lotz_b[ORC_NS], lotz_c[ORC_NS];
    double E_bind[ORC_NZ][ORC_NS];
    double tauK[ORC_NZ][2], omegaK[ORC_NZ][2], E_Ka[ORC_NZ];
    int n_hv;
    const double *hv_tab;     /* [n_hv] */
    const double *sigma;      /* [ORC_NS][n_hv] cm^2 per electron */
    int n_T, n_n;
    const double *eos_T, *eos_n, *eos_Z;   /* eos_Z[n_n][n_T] */
} orc_tables;

typedef struct {
    int shape;           /* 0 Gaussian, 1 flat-top */
    double I_peak, fwhm, t_peak, hv, bandwidth;
    int n_bins;
    double spot_sigma;   /* nm, <= 0 uniform */
} orc_pulse;

/* energy tallies (weighted eV, units n_ref*V_cell) and event counters */
enum { ORC_T_KE_E, ORC_T_KE_I, ORC_T_ION, ORC_T_PHOT, ORC_T_INC, ORC_T_TRANS,
       ORC_T_KA_ESC, ORC_T_ESC, ORC_T_FIELD,
       ORC_T_BACK,        /* radiation leaving through x = 0 (transport mode) */
       ORC_T_RT_NUM,      /* field energy the transport scheme itself gained (CIP is not conservative) */
       ORC_T_RT_PEND,     /* energy on its way from the radiation field to the bulk electrons */
       ORC_NT };
enum { ORC_C_ION, ORC_C_ION_REJ, ORC_C_REC, ORC_C_PH0, ORC_C_PH1, ORC_C_PH2,
       ORC_C_PH3, ORC_C_PH4, ORC_C_PART, ORC_C_AUG, ORC_C_KA, ORC_C_PGT1,
       ORC_C_ESC_E, ORC_C_ESC_I, ORC_C_EE, ORC_C_EI, ORC_NC };

typedef struct orc_slab orc_slab;

/* Decision trace (for classifying FP32-against-FP64 mismatches): every
 * comparison of a number x with a threshold thr that decides an integer
 * outcome of the step (r < P of a Monte-Carlo draw, a rounding of an event
 * count, an energy or photon budget, an edge) is counted, and recorded when
 * |x - thr| <= rel * |thr|.  Recording changes nothing in the step. */
enum { ORC_N_COLL_ACC = 1,   /* weighted acceptance r < w_other / w_max (particle) */
       ORC_N_ION_DRAW = 2,   /* impact ionization r < P_z (ion) */
       ORC_N_ION_PAY = 3,    /* payment budget: paid + w I > K (cell) */
       ORC_N_REC_K = 4,      /* recombination count rounding (cell) */
       ORC_N_REC_CAP = 5,    /* recombination electron-weight cap (cell) */
       ORC_N_PH_EDGE = 6,    /* photon energy against a lowered edge (ion) */
       ORC_N_PH_DRAW = 7,    /* photoionization r < P_s (ion) */
       ORC_N_PH_BIN = 8,     /* bin choice: cumulative > r P_s (ion) */
       ORC_N_PH_PART = 9,    /* photons left in the bin < w_i (cell) */
       ORC_N_PH_ZF = 10,     /* fractional charge reaching 1 (ion) */
       ORC_N_DECAY = 11,     /* K-vacancy decay r < dt_rad / tau (ion) */
       ORC_N_BRANCH = 12,    /* Auger / K-alpha branch r < 1 - omega (ion) */
       ORC_N_REC_TAKE = 13,  /* recombination weight reaching an electron's whole weight (cell) */
       ORC_N_EBULK = 14,     /* kinetic energy against E_bulk (electron) */
       ORC_N_BASIS = 15 };   /* azimuth frame of a collision: |n_xy|^2 against 1/4 (particle) */
typedef struct {
    uint32_t step;
    int32_t cell;        /* cell of the slab */
    int32_t kind;        /* ORC_N_* */
    int32_t species;     /* 0 electron, 1 ion, -1 the cell as a whole */
    uint64_t id;         /* particle id (0 for the cell) */
    double x, thr;
} orc_near;

orc_slab *orc_create(const orc_params *p, const orc_tables *t);
void orc_destroy(orc_slab *s);
void orc_set_pulse(orc_slab *s, const orc_pulse *pl);
void orc_set_step(orc_slab *s, uint32_t n);

/* Radiation transport mode (Sec. II, Eqs. 1a and 1b): the photon field is
 * the specific intensity on a rad grid `coarsen` times coarser than the PIC
 * grid, in discrete ordinates (the XFEL beam along +x and Gauss-Legendre
 * polar nodes x azimuths of the upper hemisphere, the lower one folded in
 * by symmetry), advected every rad step by the CIP scheme (scheme 0) or by
 * the conservative linear split of the ballistic march (scheme 1);
 * absorbed with the opacity of subshell photoionization, fed by K-alpha
 * emission; the energy the field loses to absorption beyond what the
 * Monte-Carlo photoionization events took heats (or cools) the bulk
 * electrons of the rad cell uniformly at the next rad step.  Set after
 * orc_set_pulse and before the first step; nx (and ny in 2D) must be
 * multiples of coarsen. */
typedef struct {
    int coarsen;       /* PIC cells per rad cell along x (and y) */
    int n_polar;       /* Gauss-Legendre nodes of mu = cos(theta) from +x (0: the beam only) */
    int n_azimuth;     /* azimuths in (0, pi) per polar node (2D; ignored in 1D) */
    int scheme;        /* 0 CIP, 1 linear split */
} orc_rt;
int orc_set_rt(orc_slab *s, const orc_rt *rt);   /* 0 on success */
int orc_rt_ordinates(const orc_slab *s, double *mu, double *vy, double *w);   /* returns the count */
/* rad field: photon density (n_ref units) per ordinate, bin and rad cell,
 * [nord][nb][nry][nrx]; the CIP derivatives along x and y the same */
void orc_rt_get(const orc_slab *s, double *F, double *Gx, double *Gy);
void orc_rt_set(orc_slab *s, const double *F, const double *Gx, const double *Gy);
/* one CIP (scheme 0) or linear (scheme 1) advection of a line of n nodes by
 * nu nodes: f, g in place; fin/gin: values of the inflow ghost nodes
 * j = -1, -2, ... (nu > 0) or n, n+1, ... (nu < 0), ng of them; outflow
 * ghosts repeat the edge value with zero slope.  in/out: content (node
 * units) that crossed the inflow and outflow faces.  periodic: wrap, no
 * ghosts. */
void orc_rt_line(double *f, double *g, double *gt, int n, double nu, int scheme, int periodic,
                 const double *fin, const double *gin, int ng, double *in, double *out);
/* per PIC cell after the last rad step (transport mode): opacity per bin
 * (cm^-1), photon energy taken by photoionization events, electron weight,
 * and the energy still to be given to the cell's bulk electrons */
void orc_rt_cells(const orc_slab *s, double *chi, double *emc, double *wcell, double *dEc);
uint32_t orc_get_step(const orc_slab *s);
void orc_load_electrons(orc_slab *s, int n, const double *X, const double *Y,
                        const double *u, const double *w, const uint64_t *id);
void orc_load_ions(orc_slab *s, int n, const double *X, const double *Y,
                   const double *u, const double *zf, const int32_t *Z,
                   const int32_t *nK, const uint32_t *id);
int orc_n_electrons(const orc_slab *s);
/* for each electron (orc_get_electrons order): the largest |u| among
 * itself and its e-e collision partners, taken before each collision of
 * the last step (0 if it did not collide): the momentum scale to which an
 * FP32 evaluation of those collisions rounds (test bookkeeping) */
void orc_get_electron_scales(const orc_slab *s, double *cs);
int orc_n_ions(const orc_slab *s);
void orc_get_electrons(const orc_slab *s, double *X, double *Y, double *u,
                       double *w, uint64_t *id);
void orc_get_ions(const orc_slab *s, double *X, double *Y, double *u,
                  double *zf, int32_t *Z, int32_t *nK, uint32_t *id);
void orc_set_fields(orc_slab *s, const double *f6);   /* [6][ny][nx+1] */
void orc_get_fields(const orc_slab *s, double *f6);
void orc_get_current(const orc_slab *s, double *j3);  /* [3][ny][nx+1] */
void orc_set_photons(orc_slab *s, const double *ph);  /* [ny][nx][nb] */
void orc_get_photons(const orc_slab *s, double *ph);
void orc_step(orc_slab *s, int nsteps, int nthreads);
void orc_tallies(orc_slab *s, double *t, uint64_t *c);
void orc_diag(const orc_slab *s, double *csd, int n_E, double E_max, double *eedf);
/* decision trace: rel <= 0 switches it off (the default); records of
 * earlier steps are kept until orc_trace is called again */
void orc_trace(orc_slab *s, double rel);
int orc_trace_count(const orc_slab *s);
/* decisions counted since orc_trace: [0] Monte-Carlo draws (r < P),
 * [1] every other threshold decision */
void orc_trace_decisions(const orc_slab *s, uint64_t out[2]);
void orc_trace_get(const orc_slab *s, orc_near *out);

/* building blocks exposed for the closed-form and invariant pins */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t x);
int orc_occ(int nb, int nk, int occ[ORC_NS]);
double orc_ipd(int model, int z, double n_e, double n_i, double T_e, double zbar);
double orc_lotz(const orc_tables *t, int z, double dE, double E);
double orc_coulomb_log(double n_e, double T_e, double zbar);
double orc_field_speed(const orc_params *p);   /* nm/fs, speed of the Yee update */
/* np2_out (may be NULL): squared in-plane part of the collision's
 * centre-of-momentum direction, which picks the azimuth frame */
int orc_collide(double ua[3], double ub[3], double ma, double mb, double qa,
                double qb, double wa, double wb, double n_l, double lnL,
                double dtc, const double r[4], double *np2_out);
void orc_boris(double u[3], const double e[3], const double b[3], double qm, double dt);
void orc_pair_order(int n, const uint64_t *id, uint32_t step, uint32_t purpose,
                    uint64_t seed, int *perm);
int orc_ee_pairs(int n, int *pa, int *pb, double *frac);
void orc_deposit(int nx, int ny, double dx, double dy, double dt, double X0,
                 double Y0, double X1, double Y1, double vz_nmfs, double vy_nmfs,
                 double qw, double *j3);
void orc_rho(int nx, int ny, double X, double Y, double qw, double *rho);
double orc_eos(const orc_tables *t, double n_i, double T_e);

#endif
