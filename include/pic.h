/* C ABI of the GB300 collisional-PIC step for XFEL-heated solid Al
 * (Royle, Sentoku, Mancini, Paraschiv, Johzaki: "Kinetic modeling of x-ray
 * laser-driven solid Al plasmas via particle-in-cell simulation", PICLS).
 *
 * One context owns one or more independent slabs ("batched" mode) on one
 * GPU.  Every step of the hot path runs in CUDA kernels: counting sort by
 * cell, per-cell random pairing and binary Coulomb scattering (Sec. IV),
 * Lotz impact ionization (Sec. IV, Eq. 3), EOS-clamped three-body
 * recombination (Sec. IV), subshell photoionization (Sec. III, Eq. 2) with
 * partial events, K-vacancy decay with KLL-Auger / K-alpha branching
 * (Sec. III), continuum lowering (Sec. V, Eqs. 4-5), ballistic march of the
 * XFEL photons (Sec. II, reduced to attenuation along x), Boris push,
 * charge-conserving deposit and one Yee field update per step at the
 * field speed the step resolves (light slowed where c dt exceeds the
 * Courant limit of the cells).
 *
 * Units: lengths nm, times fs, energies eV, momenta u = gamma v / c,
 * particle weights in units of n_ref * V_cell (n_ref = reference density),
 * fields normalized by E0 = m_e c / (e * 1 fs) and B0 = m_e / (e * 1 fs).
 * Positions passed across the ABI are absolute, in cell units
 * (X in [0, nx), Y in [0, ny)).
 *
 * Errors: every call returns a pic_status; nothing aborts.  Device-side
 * problems (cell overflow, capacity, numeric) latch an error word that the
 * next synchronizing call (pic_sync, pic_diagnostics, pic_get_*) returns;
 * pic_last_error gives a message.  A context is used by one host thread at
 * a time.  Where a declaration lists no errors of its own: PIC_ERR_ARG for
 * a NULL context or array, a negative count, a slot out of range or a value
 * out of its stated range (a per-slot batch call on a single-slab context
 * has no such slot: PIC_ERR_ARG too); PIC_ERR_STATE for a single-slab call
 * on a batch context; PIC_ERR_CUDA when a CUDA runtime call fails.
 *
 * Ownership: host arrays are read or written during the call only; the
 * library keeps no pointer to them (tables and pulses are copied).  The
 * device arena given to pic_init or pic_batch_init stays the caller's and
 * must outlive the context; with a NULL arena the context allocates its own
 * and pic_free releases it.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx;

typedef enum {
    PIC_OK = 0,
    PIC_ERR_ARG = 1,        /* invalid argument or size */
    PIC_ERR_OOM = 2,        /* device allocation failed / arena too small */
    PIC_ERR_TABLE = 3,      /* atomic table malformed */
    PIC_ERR_CUDA = 4,       /* a CUDA runtime call failed */
    PIC_ERR_TIMEOUT = 5,    /* a bounded device wait gave up */
    PIC_ERR_NUMERIC = 6,    /* NaN / negative energy detected on device */
    PIC_ERR_STATE = 7,      /* call out of order (e.g. step before load) */
    PIC_ERR_CAPACITY = 8    /* particle or per-cell capacity exceeded */
} pic_status;

/* process switches (bit flags) */
enum {
    PIC_F_COLL_EE = 1, PIC_F_COLL_EI = 2, PIC_F_IONIZE = 4, PIC_F_RECOMB = 8,
    PIC_F_PHOTO = 16, PIC_F_DECAY = 32, PIC_F_PUSH = 64, PIC_F_FIELD = 128,
    /* forced-thermalization variant (Sec. VI C): on rad steps each cell's
     * free electrons are redrawn from a Maxwellian at (2/3) E_ave, with the
     * cell's electron momentum and kinetic energy kept */
    PIC_F_THERM = 256
};
enum { PIC_IPD_NONE = 0, PIC_IPD_EK = 1, PIC_IPD_SP = 2 };

#define PIC_NSUB 5          /* subshells 1s 2s 2p 3s 3p */
#define PIC_NZ 14           /* Al charge states 0..13 */
#define PIC_MAX_BINS 8      /* photon energy bins */

/* Grid of one slab (Sec. VI: PIC grid, dt_PIC, dt_rad = rad_every dt_PIC).
 * ny == 1 is a 1D slab.  y is periodic; x boundaries absorb particles and
 * fields (first-order Mur).  Valid: 2 <= nx <= 8192, ny >= 1, (nx + 1) ny <= 2^27,
 * dx, dy, dt and cfl positive and finite. */
typedef struct {
    int nx, ny;
    double dx_nm, dy_nm;
    double dt_fs;
    int rad_every;          /* photon march / photoionization / decay period */
    uint64_t seed;          /* Philox key of the slab */
    double cfl;             /* Courant number of the field update: its speed is
                             * min(c, cfl / (dt sqrt(1/dx^2 + [ny>1]/dy^2))) */
} pic_grid;

/* Species and model switches of one slab.  Ions share one weight.  Valid:
 * n_ref, w_ion and m_ion positive and finite, coulomb_log finite, E_bulk
 * not NaN, ipd_model a PIC_IPD_* value. */
typedef struct {
    double n_ref_cm3;       /* density unit of the weights */
    double w_ion;           /* common ion weight */
    double m_ion_me;        /* ion mass / electron mass */
    double E_bulk_eV;       /* bulk threshold for T_e (Sec. II); <= 0: all */
    int ipd_model;          /* PIC_IPD_* (Sec. V) */
    double coulomb_log;     /* > 0: fixed; <= 0: computed per cell */
    unsigned flags;         /* PIC_F_* */
    int cap_e, cap_i;       /* particle capacity of the slab: > 0 with
                             * cap_e + 3 cap_i < 2^31 for pic_init (a step
                             * appends at most three electrons per ion, and
                             * particle indices are 32-bit); ignored by
                             * pic_batch_admit (the batch's own) */
} pic_species;

/* Atomic data (Sec. III-V).  Copied at pic_init; the caller keeps its
 * buffers.  E_bind[z][s]: binding of subshell s in charge state z (lowest-
 * energy configuration); tauK / omegaK indexed [N_b][nK-1]; E_Kalpha[z];
 * sigma_photo[s][n_hv] per electron in cm^2 on the grid hv_tab (eV);
 * eos_Zbar[n_n][n_T] on grids eos_n (cm^-3) and eos_T (eV). */
typedef struct {
    double lotz_a[PIC_NSUB], lotz_b[PIC_NSUB], lotz_c[PIC_NSUB];
    double E_bind[PIC_NZ][PIC_NSUB];
    double tauK[PIC_NZ][2], omegaK[PIC_NZ][2], E_Kalpha[PIC_NZ];
    int n_hv;
    const double *hv_tab;
    const double *sigma_photo;
    int n_T, n_n;
    const double *eos_T, *eos_n, *eos_Zbar;
} pic_tables;

/* XFEL pulse entering at x = 0 (Sec. VI): Gaussian (FWHM) or flat-top
 * intensity, n_bins photon-energy bins across the bandwidth.  Valid: shape
 * 0 or 1, hv > 0, I_peak, fwhm and bandwidth >= 0, all finite (spot_sigma
 * not NaN). */
typedef struct {
    int shape;              /* 0 Gaussian, 1 flat-top */
    double I_peak_Wcm2, fwhm_fs, t_peak_fs, hv_eV, bandwidth_eV;
    int n_bins;             /* 1..PIC_MAX_BINS */
    double spot_sigma_nm;   /* Gaussian in y (2D); <= 0 uniform */
} pic_pulse;

/* Diagnostics of one slab (Sec. VI: charge-state distribution, electron
 * energy distribution, transmission, T_e, Zbar, event counts).  Arrays
 * are caller-allocated. */
typedef struct {
    double *csd;            /* [PIC_NZ], weighted ion fraction per charge */
    double *eedf;           /* [n_E], electron weight fraction per log bin */
    int n_E;                /* bins on 0.1 eV .. E_max (log) */
    double E_max_eV;
    double t_fs;
    double transmission;    /* transmitted / incident photon energy so far */
    double T_e_eV, n_e_cm3, Zbar;
    /* energy bookkeeping, weighted eV (units n_ref V_cell) */
    double ke_e, ke_i, e_ion, e_phot, e_inc, e_trans, e_ka_esc, e_esc, e_field;
    /* event counters: impact ionization, rejected ionization, recombination,
     * photoionization per subshell, partial photoionization, Auger,
     * K-alpha, P > 1 warnings, escaped e / i, e-e and e-i collisions */
    uint64_t counts[16];
    int64_t n_e, n_i;
    /* radiation transport mode (pic_rt; 0 otherwise): radiation energy
     * that left through x = 0, field energy the transport scheme itself
     * gained (CIP is not conservative; the contents crossing the faces are
     * counted by the linear split), and energy owed between the field and
     * the electrons (photons taken by photoionization events before the
     * field's opacity removed them, absorption beyond the events not yet
     * given to the bulk electrons).  Conserved: ke_e + ke_i + e_ion +
     * e_phot + e_ka_esc + e_trans + e_back + e_esc + e_field - e_inc -
     * e_rt_num + e_rt_pend (up to the field solver's own drift). */
    double e_back, e_rt_num, e_rt_pend;
} pic_diag;

/* Bytes of device memory pic_init needs for this slab (n_e_cap / n_i_cap
 * > 0 override the species' capacities); 0 for an invalid grid or
 * capacities pic_init would refuse. */
size_t pic_required_bytes(const pic_grid *g, const pic_species *s, int n_e_cap, int n_i_cap);

/* Create a context for one slab.  arena/arena_bytes: caller-owned device
 * memory (e.g. a torch tensor) of at least pic_required_bytes, or NULL to
 * let the context allocate.  stream: cudaStream_t to run on (NULL: legacy
 * default).  The context never frees a caller arena. */
pic_status pic_init(pic_ctx **out, const pic_grid *g, const pic_species *s,
                    const pic_tables *t, void *arena, size_t arena_bytes, void *stream);

/* Set the XFEL pulse (Sec. III Eq. 2 inputs); may be called before any
 * step.  Without a pulse photoionization sees no photons. */
pic_status pic_source(pic_ctx *c, const pic_pulse *p);

/* Radiation transport (Sec. II, Eqs. 1a and 1b), instead of the ballistic
 * march of the pulse: the photon field is the photon density per discrete
 * ordinate and bin on a rad grid `coarsen` times coarser than the PIC grid
 * (the rad cell of the paper), advanced once per rad step: absorbed with
 * the opacity of subshell photoionization that the ions of each rad cell
 * present (Eq. 2's cross sections above the lowered edges), fed by the
 * K-alpha photons of the decays (isotropic, into the diffuse ordinates),
 * and advected by the CIP scheme (the intensity with its derivative,
 * cubic Hermite at the departure point; scheme 0) or by the march's linear
 * split (scheme 1).  The energy the field loses to its opacity beyond what
 * the Monte-Carlo photoionization events took (Eq. 1b's dE_ij) heats the
 * rad cell's bulk electrons uniformly at the next rad step (cools them when
 * negative), shared among its PIC cells by electron weight.  Ordinates:
 * the XFEL beam along +x, then n_polar Gauss-Legendre nodes of mu =
 * cos(theta) times n_azimuth azimuths in (0, pi) (2D; the lower hemisphere
 * is the mirror image).  Single-slab contexts only, after pic_source; nx
 * (and ny in 2D) multiples of coarsen, at most 4096 rad cells along each
 * axis, n_polar 0..16, n_azimuth 1..16, c dt_rad at most 61 rad cells
 * (the beam's inflow ghost nodes).  The context allocates the field
 * (cudaMalloc) and frees it in pic_free.  PIC_ERR_STATE without a pulse,
 * on a batch context or when already on; PIC_ERR_ARG for invalid sizes. */
typedef struct {
    int coarsen;       /* PIC cells per rad cell along x (and along y in 2D) */
    int n_polar;       /* diffuse polar nodes (0: the beam alone) */
    int n_azimuth;     /* azimuths per polar node (2D) */
    int scheme;        /* 0 CIP, 1 linear split */
} pic_rt_config;
pic_status pic_rt(pic_ctx *c, const pic_rt_config *rt);
/* The rad field and its CIP slopes along x and y, [nord][n_bins][nry][nrx]
 * (nord = 1 + n_polar * n_azimuth, n_azimuth = 1 in 1D), photon densities
 * in units of n_ref; caller-allocated.  Synchronizes. */
pic_status pic_rt_get(pic_ctx *c, double *F, double *Gx, double *Gy);
pic_status pic_rt_set(pic_ctx *c, const double *F, const double *Gx, const double *Gy);
/* What each PIC cell recorded at the last rad step for the transport:
 * opacity per bin (cm^-1, [ncell][n_bins]), photon energy its
 * photoionization events took, its electron weight, and the energy still
 * due to its bulk electrons ([ncell] each).  Synchronizes. */
pic_status pic_rt_cells(pic_ctx *c, double *chi, double *emc, double *w, double *dE);

/* Initial plasma of the slab (the solid Al target of Sec. VI, seeded on the
 * device): ppc_e electrons and ppc_i ions in every cell at uniform random
 * positions (y = 0.5 in 1D), ions at charge Z_init with full K shells,
 * Maxwellian momenta at T_i, electrons Maxwellian at T_e except a
 * beam_frac share (each electron drawn alone) at beam_E_eV with isotropic
 * directions.  Weights: ions the species' w_ion, electrons
 * Z_init ppc_i w_ion / ppc_e (the slab neutral).  Ids: cell-major
 * positions, 0 .. ncell ppc - 1 per species.  Random numbers: Philox4x32-10
 * keyed by (seed, id) on streams of their own.  Replaces any particles
 * (pic_load_* remain for states built elsewhere). */
typedef struct {
    int ppc_e, ppc_i;       /* macro-electrons and macro-ions per cell (>= 1) */
    int Z_init;             /* initial ion charge, 0 .. 12 */
    double T_e_eV, T_i_eV;  /* Maxwellian temperatures (>= 0, finite) */
    double beam_frac;       /* share of electrons in the beam, 0 .. 1 */
    double beam_E_eV;       /* beam kinetic energy (>= 0, finite) */
    uint64_t seed;          /* key of the seeding streams */
} pic_seed_spec;

/* PIC_ERR_ARG: spec out of range; PIC_ERR_CAPACITY: more particles than
 * the capacity; PIC_ERR_STATE: batch context.  Synchronizes. */
pic_status pic_seed(pic_ctx *c, const pic_seed_spec *s);

/* Load particles from host memory (absolute positions in cell units).
 * u is [n][3]; ids must be unique per species.  Replaces any particles.
 * Ions: Z 0..13, nK (K vacancies against the lowest configuration of the
 * 13 - Z bound electrons) 0..min(2, 13 - Z), zfrac (charge carried toward
 * Z + 1 by partial photoionization) in [0, 1).  The arrays are read during
 * the call only.  PIC_ERR_ARG for a position outside the slab or an ion
 * state out of range; PIC_ERR_CAPACITY for more particles than the
 * capacity; PIC_ERR_STATE on a batch context (which loads at admission). */
pic_status pic_load_electrons(pic_ctx *c, int64_t n, const double *X, const double *Y,
                              const float *u, const float *w, const uint64_t *id);
pic_status pic_load_ions(pic_ctx *c, int64_t n, const double *X, const double *Y,
                         const float *u, const float *zfrac, const int32_t *Z,
                         const int32_t *nK, const uint32_t *id);
/* Photon field (photon number per cell and bin, units n_ref V_cell),
 * [ny][nx][n_bins]; fields [6][ny][nx+1] (ex ey ez bx by bz). */
pic_status pic_set_photons(pic_ctx *c, const double *ph);
pic_status pic_set_fields(pic_ctx *c, const float *f6);

/* Checkpoint / restore of a single-slab context: a host image of the
 * sorted particles, the fields, the photon numbers, the tallies, the step
 * count and, in transport mode, the transport's state.  The random streams
 * are keyed by (seed, id, step, purpose), so nothing of the generator is
 * saved: a context restored from an image continues as the original would,
 * particle for particle (diagnostic sums agree to their atomic summation
 * order).  pic_checkpoint_bytes: the image size now (0 for a batch context
 * or before particles are loaded; synchronizes).  pic_checkpoint writes it
 * to host memory of at least that size (PIC_ERR_ARG if smaller;
 * synchronizes).  pic_restore loads an image into a context created with
 * the same grid, species, tables and pulse (and pic_rt setting), replacing
 * its particles and state; PIC_ERR_ARG for an image of another slab, build
 * or setting, a truncated one, or one whose cell starts or records are out
 * of range (offsets in the cell outside [0, 1), ion states beyond the
 * loaders' rules): a damaged image is refused, never read out of bounds on
 * the device; PIC_ERR_CAPACITY when its particles do not fit.  Launch-shape tuning and step graphs are not part of the image
 * (they change no result). */
size_t pic_checkpoint_bytes(pic_ctx *c);
pic_status pic_checkpoint(pic_ctx *c, void *host, size_t bytes);
pic_status pic_restore(pic_ctx *c, const void *host, size_t bytes);

/* Advance n PIC steps (asynchronous on the context stream; the call
 * synchronizes every 32 steps to re-size the cell tiers).  Device-side
 * problems are latched and reported by the next synchronizing call:
 * PIC_ERR_CAPACITY when the electrons created in a step would exceed the
 * context's capacity (or a cell outgrows the large-cell pass) and
 * PIC_ERR_NUMERIC on a non-finite move.  After PIC_ERR_CAPACITY the
 * electrons created in the failing cells are gone while their ions' charge
 * states, photon numbers and tallies moved on: the state is no longer
 * conserved and the context should be freed.  In a batch the error word is
 * shared, so it stops every slab; electron budgets
 * (pic_batch_set_budget) confine a capacity failure to its own slab. */
pic_status pic_step(pic_ctx *c, int n);

/* Wait for the stream; returns the latched device error, if any. */
pic_status pic_sync(pic_ctx *c);

/* Reductions on the device, small D2H copy; synchronizes. */
pic_status pic_diagnostics(pic_ctx *c, pic_diag *out);

/* Particle counts and copies back to host (synchronizes).  Arrays are
 * caller-allocated with at least the counted length. */
pic_status pic_counts(pic_ctx *c, int64_t *n_e, int64_t *n_i);
pic_status pic_get_electrons(pic_ctx *c, double *X, double *Y, float *u, float *w, uint64_t *id);
pic_status pic_get_ions(pic_ctx *c, double *X, double *Y, float *u, float *zfrac,
                        int32_t *Z, int32_t *nK, uint32_t *id);
/* The same read-back with momenta, weights and fractional charges in
 * double precision: the FP64 build's state without rounding to float (the
 * FP32 build returns its values widened).  Same layout and errors. */
pic_status pic_get_electrons64(pic_ctx *c, double *X, double *Y, double *u, double *w, uint64_t *id);
pic_status pic_get_ions64(pic_ctx *c, double *X, double *Y, double *u, double *zfrac,
                          int32_t *Z, int32_t *nK, uint32_t *id);
/* Bytes of the arithmetic type of the loaded build: 4 for the production
 * library (FP32 state and arithmetic), 8 for the FP64 build of the same
 * kernels (a check of the device logic free of single-precision rounding;
 * no counterpart in the paper, which runs in double precision). */
int pic_real_bytes(void);
pic_status pic_get_photons(pic_ctx *c, double *ph);
pic_status pic_get_fields(pic_ctx *c, float *f6);
/* Current density of the last step, [3][ny][nx+1], units e n_ref nm/fs. */
pic_status pic_get_current(pic_ctx *c, double *j3);

/* ---------------- batched slabs ----------------
 * A batch context steps many independent 1D slabs with one launch of each
 * kernel per step: slot k owns cells [k*slot_cells, (k+1)*slot_cells) of one
 * global numbering, its own grid points, photons, tallies and step counter.
 * A slab's random streams are keyed by its own seed, particle ids and its own
 * step count, and every cross-particle sum is fixed-point or in canonical
 * order, so a slab evolves bit-identically alone (pic_init) or in a batch,
 * whatever its neighbours.  Slabs are admitted and retired between steps;
 * admission copies the particles and re-sorts once, on the next step,
 * diagnostics or copy call.  pic_step, pic_sync and pic_timing work on batch
 * contexts; the single-slab calls above return PIC_ERR_STATE.
 * The paper runs one slab per job; batching is a throughput feature of
 * this implementation. */

/* Bytes of device memory pic_batch_init needs. 0 on invalid sizes. */
size_t pic_batch_required_bytes(int max_slabs, int slot_cells, int cap_e, int cap_i);

/* Create an empty batch context of max_slabs slots of slot_cells cells
 * (2..8192).  cap_e / cap_i: particle capacity summed over all slabs, > 0
 * with cap_e + 3 cap_i < 2^31 (as for pic_init; PIC_ERR_ARG otherwise).
 * arena / stream as in pic_init. */
pic_status pic_batch_init(pic_ctx **out, int max_slabs, int slot_cells, int cap_e, int cap_i,
                          const pic_tables *t, void *arena, size_t arena_bytes, void *stream);

/* Admit one 1D slab (g->ny == 1, g->nx <= slot_cells) with its species,
 * optional pulse (NULL: none) and particles (host arrays as in
 * pic_load_*).  The host arrays may be freed on return.  *slot_out gets the
 * slot; PIC_ERR_CAPACITY when no slot is free.  The slab starts at step 0
 * with zero fields and photons. */
pic_status pic_batch_admit(pic_ctx *c, const pic_grid *g, const pic_species *s, const pic_pulse *p,
                           int64_t n_e, const double *eX, const double *eY, const float *eu,
                           const float *ew, const uint64_t *eid,
                           int64_t n_i, const double *iX, const double *iY, const float *iu,
                           const float *izf, const int32_t *iZ, const int32_t *inK,
                           const uint32_t *iid, int *slot_out);

/* Retire an active slot: its particles are dropped by the next step, or
 * earlier by an admission that needs the slot or the space, after which the
 * slot is free again. */
pic_status pic_batch_retire(pic_ctx *c, int slot);

/* Electron budget of an active slot: the most electron slots the slab may
 * hold after any step (its particles plus those it created; 0: no budget of
 * its own, only the context's cap_e).  A step in which a cell would take
 * the slab beyond its budget drops the electrons that cell created and
 * fails that slab alone: it stops at the end of the step (its step count
 * no longer advances, its particles are dropped by the next step) and
 * pic_batch_slot reports state 3 once pic_step returns.  Retire a failed
 * slot to free it; its diagnostics and particles are no longer available.
 * With a budget on every active slot and the budgets summing to at most
 * cap_e, the shared capacity cannot run out: a capacity failure stays with
 * the slab that caused it (without budgets, running out of cap_e fails the
 * whole step with PIC_ERR_CAPACITY and leaves every slab's state
 * undefined).  Why a slab can outgrow a footprint bound: every partial
 * photoionization (Sec. III, Eq. 2, an absorption of fewer photons than
 * one ion weight) creates an electron macroparticle of fractional weight
 * while the ion's charge advances by that fraction only, up to one per
 * photon bin per cell per rad step.
 * PIC_ERR_ARG: max_e < 0 or above cap_e; PIC_ERR_STATE: slot not active. */
pic_status pic_batch_set_budget(pic_ctx *c, int slot, int64_t max_e);

/* Slot state (0 free, 1 active, 2 retired, not yet emptied, 3 failed: went
 * beyond its electron budget, stopped) and its step count (synchronizes
 * when step != NULL). */
pic_status pic_batch_slot(pic_ctx *c, int slot, int *state, uint32_t *step);

/* Per-slot versions of pic_diagnostics, pic_counts, pic_get_electrons and
 * pic_get_ions (positions in the slab's own cell units). */
pic_status pic_batch_diagnostics(pic_ctx *c, int slot, pic_diag *out);
pic_status pic_batch_counts(pic_ctx *c, int slot, int64_t *n_e, int64_t *n_i);
pic_status pic_batch_get_electrons(pic_ctx *c, int slot, double *X, double *Y, float *u, float *w,
                                   uint64_t *id);
pic_status pic_batch_get_ions(pic_ctx *c, int slot, double *X, double *Y, float *u, float *zfrac,
                              int32_t *Z, int32_t *nK, uint32_t *id);

/* Kernel launches issued by the last pic_step call (for accounting). */
int64_t pic_launch_count(const pic_ctx *c);

/* Step replay through CUDA graphs (default on).  pic_step(n) with n >= 2
 * and timing off launches a captured graph of two steps n/2 times (the
 * launch sequence of a step pair is the same as long as the cell staging
 * sizes, the active slabs' processes and the buffer parity are), capturing
 * it on a private stream at first use.  Results are identical either way. */
pic_status pic_use_graphs(pic_ctx *c, int enable);

/* Launch-shape autotuner (default off).  enable = 1: whenever a pic_step
 * call meets tier-0 staging sizes whose tuning is not finished, its first
 * steps run the cell kernel with 1, 2, 4 and 8 warps per CTA (as many as fit
 * in shared memory), each twice in the order 1 2 4 8 8 4 2 1, timing the
 * cell kernels with CUDA events; the fastest mean is kept for those sizes.
 * The context's first step is not timed.  These are steps of the
 * simulation: the launch shape changes no result.  enable = 0 stops tuning
 * (choices made are kept); -1 leaves it as is.  wpc_out (may be NULL) gets
 * the warps per CTA in use; ms_out (4 floats, may be NULL) the mean cell
 * kernel times measured for 1, 2, 4, 8 warps at the current sizes (0: not
 * tried). */
pic_status pic_autotune(pic_ctx *c, int enable, int *wpc_out, float *ms_out);

/* Device timing of kernel groups with CUDA events on the context stream.
 * enable = 1 starts recording (clearing earlier records), 0 stops; -1 keeps
 * the state.  With ms_out != NULL (6 doubles) the call synchronizes and
 * returns the summed device time of the steps recorded so far: [0] the
 * per-cell collision / atomic-process kernel (both passes), [1] photon march,
 * [2] push + deposit, [3] counting sort (scan + scatter), [4] field
 * update, [5] whole steps; *nsteps gets the number of steps. */
pic_status pic_timing(pic_ctx *c, int enable, double *ms_out, int64_t *nsteps);

pic_status pic_free(pic_ctx *c);
const char *pic_last_error(const pic_ctx *c);

/* Philox4x32-10 of the device path, for checking it against other
 * implementations: out[4*i..] = philox(ctr[4*i..], key) for i < n. */
pic_status pic_philox_check(const uint32_t *ctr, const uint32_t key[2], uint32_t *out, int n);

/* The sum of n <= 2^24 FP32 terms x (host array) as the cell kernel forms
 * its per-cell energy, weight and charge sums (Sec. IV's energy restore,
 * Sec. II's cell moments): double-float pairs (a float hi + lo, ~44-48 bit
 * significand; two doubles in the FP64 build) accumulated lane-strided by
 * one warp and reduced by its fixed tree; *out = hi + lo.  For bounding that
 * arithmetic against exact sums.  PIC_ERR_ARG on n out of range. */
pic_status pic_dd_sum_check(const float *x, int n, double *out);

/* The in-cell ordering of the device (ascending key, ties by id; the
 * canonical order every per-cell rule follows), run on n <= 4096 given
 * entries by one warp with the algorithm a cell of that size uses in the
 * cell-kernel instance rmax (128, 512 or 1024: the largest cell it sorts in
 * registers; the radix sort above 512, resp. 1024; rmax 128 takes n <= 128):
 * order[k] = index of the entry at position k.  For checking it against
 * other implementations.  PIC_ERR_ARG on other n or rmax. */
pic_status pic_order_check(const uint64_t *key, const uint64_t *id, int n, int rmax, uint16_t *order);

/* The same check without any device allocation.  The paper has no
 * counterpart: this serves callers that must not allocate, e.g. a host
 * thread of a serving loop whose device memory budget is fixed up front, or
 * code that is not allowed to enter the device allocator at all.
 * Scratch is a static device array of PIC_PHILOX_STATIC_MAX counters (four
 * words each, 128 KiB in all); n above that returns PIC_ERR_ARG.  Nothing in
 * the scratch needs to start at zero: every word is written before it is
 * read.  The scratch's address is looked up once per device (the first call
 * with that device current); make that first call before any stream
 * capture.  Calls run on the legacy default stream and return when the
 * result is on the host.  Two calls on the same device at the same time
 * (two host threads) race on the scratch: serialize them. */
#define PIC_PHILOX_STATIC_MAX 4096
pic_status pic_philox_check_static(const uint32_t *ctr, const uint32_t key[2], uint32_t *out, int n);

#ifdef __cplusplus
}
#endif
#endif
