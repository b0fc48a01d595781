/*
 * md.h -- C ABI of the GB300 laser-cluster molecular-dynamics hot path.
 *
 * Method: Holkundkar, "Parallel Implementation of 3D Molecular Dynamic
 * Simulation for Laser-Cluster Interaction", arXiv:1307.3711, Sec. II.
 * Each step advances every particle of every cluster under
 *   - the Coulomb field of all other charged particles (Sec. II, particle
 *     mover paragraph), a softened O(N^2) direct sum computed in FP32 with
 *     compensated (Kahan) accumulation per tile of sources,
 *   - the spatially uniform laser field of Eqs. 3-9 (dipole approximation,
 *     b0 = a0),
 *   - a relativistic Boris kick and an FP64 position update ("standard Boris
 *     leap frog", Sec. II).
 *
 * Units are the paper's (Sec. II): time in 1/omega, length in 1/k, velocity
 * in c, u = gamma*beta, fields a = eE/(m_e omega c), b = eB/(m_e omega),
 * charge in e, mass in m_e, energy in m_e c^2.  The Coulomb constant in these
 * units is K_C = 2 pi r_e / lambda (the field of charge Q at distance r is
 * K_C Q / r^2), computed from md_config.lambda_um.
 *
 * Conventions for every call:
 *   - Every call returns md_status; nothing is thrown across the ABI (a
 *     host allocation that fails inside a call returns MD_ERR_OOM).
 *     md_last_error() gives a thread-local message for the last failure.
 *   - The library owns the device memory of a context (allocated in md_init,
 *     freed in md_destroy).  Host pointers passed in are read or written only
 *     during the call.
 *   - Calls that launch work are asynchronous on the context's stream;
 *     md_diagnostics, md_get_particles, md_get_fields and md_sync
 *     synchronise that stream and report device-side errors (an mbarrier wait
 *     that ran out of its time budget: MD_ERR_TIMEOUT).
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef MD_H
#define MD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_ctx md_ctx;

typedef enum {
    MD_OK = 0,
    MD_ERR_ARG = -1,        /* invalid argument (message says which) */
    MD_ERR_OOM = -2,        /* device or pinned-host allocation failed */
    MD_ERR_CUDA = -3,       /* a CUDA runtime call failed */
    MD_ERR_TIMEOUT = -4,    /* a device-side wait exceeded its budget */
    MD_ERR_NONFINITE = -5,  /* diagnostics found NaN/Inf in the state */
    MD_ERR_STATE = -6,      /* call not valid in the current state */
    MD_ERR_UNSUPPORTED = -7 /* device or option this library does not support */
} md_status;

/* Temporal envelope of the laser (Eq. 3 and its readings). */
enum {
    MD_ENV_GAUSS = 0,       /* field exp[-2 ln2 (t-2tau)^2/tau^2]: intensity FWHM tau, peak at 2 tau */
    MD_ENV_SIN2 = 1,        /* field sin^2(pi t / tau) on [0, tau] (tau = total length T), 0 outside */
    MD_ENV_LITERAL_EQ3 = 2, /* field exp[-2.77 (t-2tau)^2/tau^2], Eq. 3 as printed */
    MD_ENV_FLAT = 3         /* constant amplitude (continuous wave) */
};

/* Boundary of the simulation box (Sec. II, first paragraph). */
enum {
    MD_BOUNDARY_OPEN = 0,
    MD_BOUNDARY_PERIODIC = 1, /* positions wrapped into the cube [-box/2, box/2)^3; image
                                 forces only with md_config.min_image */
    MD_BOUNDARY_MIXED = 2     /* periodic while t < t_switch, open afterwards */
};

/* Particle kinds. */
enum {
    MD_KIND_ION = 0,      /* ion or neutral atom (charge z >= 0) */
    MD_KIND_ELECTRON = 1, /* electron (z = -1) */
    MD_KIND_INACTIVE = 2  /* unused slot: no charge, never moves */
};

/* Physics of one cluster, all in the paper's units. */
typedef struct {
    double a0;          /* peak field amplitude (Eq. 2 gives it from I0, lambda); b0 = a0 */
    double tau;         /* envelope time: FWHM (GAUSS, LITERAL_EQ3) or total length T (SIN2) */
    double t0;          /* time of step 0 */
    double dt;          /* time step, > 0 */
    double softening;   /* Plummer softening length eps, > 0 */
    double box;         /* side of the periodic cube (PERIODIC / MIXED), e.g. 20 R0 */
    double t_switch;    /* MIXED: time at which the boundary becomes open */
    double lambda_um;   /* laser wavelength in micron (sets K_C); > 0 */
    int32_t polarization; /* 0 linear (E along x, B along y), 1 circular (Eqs. 4-9) */
    int32_t envelope;     /* MD_ENV_* */
    int32_t boundary;     /* MD_BOUNDARY_* */
    /* ---- Monte-Carlo ionization (Sec. II, ionization paragraph) ---- */
    int32_t rate_model;   /* MD_RATES_*: 0 none */
    int32_t ionize_every; /* k >= 1: one pass before every k-th step, dt_ion = k dt;
                             0: passes only through md_ionize (dt_ion = dt) */
    int32_t zmax;         /* highest charge state, 1..16 */
    int32_t n_ions;       /* records [0, n_ions) are the atoms/ions that can ionize */
    int32_t min_image;    /* 1: while the boundary is periodic (PERIODIC, or MIXED before
                             t_switch) every pair interacts through its nearest periodic
                             image (each displacement component reduced to
                             [-box/2, box/2]), in the step, the diagnostics and the
                             ionization pass (field and local moments); 0: no image
                             forces */
    int64_t slot_base;    /* records [slot_base, slot_base + zmax n_ions) are electron
                             slots (INACTIVE until used); freed electrons fill them
                             densely, after the last active one (see md_ionize) */
    uint64_t seed;        /* Philox key */
    double r_loc;         /* local electron moments from electrons within r_loc of the ion */
    double r_create;      /* new electron uniform in the ball of this radius around the ion */
    double ip_ev[16];     /* ionization energy of charge state z -> z+1 (eV), z < zmax */
    double q_outer[16];   /* electrons in the outermost subshell of charge state z (Lotz) */
} md_config;

/* Rate models of the ionization pass. */
enum {
    MD_RATES_NONE = 0,
    MD_RATES_PLAIN = 1, /* static ADK tunnelling + Lotz electron impact */
    MD_RATES_MLP = 2    /* learned surrogate of the plain total rate (md_set_rate_mlp) */
};

/* Host-side particle records of one cluster (structure of arrays, n records).
 * For md_init / md_set_particles the arrays are read; md_get_particles writes
 * the arrays whose pointer is non-NULL.  u is the momentum at the half step
 * before the current step (leap-frog), i.e. u^{n-1/2} at step n; the first
 * step uses the given u as u^{-1/2}. */
typedef struct {
    int64_t n;
    double *x;       /* [n][3] positions */
    double *u;       /* [n][3] u = gamma beta */
    int32_t *z;      /* [n] charge number (electron -1, neutral 0) */
    double *mass;    /* [n] mass of one real particle, m_e */
    double *w;       /* [n] macro weight (real particles per record) */
    uint8_t *kind;   /* [n] MD_KIND_* ; NULL on input: electron if z < 0, else ion */
} md_particles;

/* FP64 diagnostics at integer time t_n for the state (x^n, u^{n-1/2}):
 * u^n = (u^{n-1/2} + u^{n+1/2})/2 with u^{n+1/2} the kick of step n (not
 * applied to the state).  Energies in m_e c^2, momentum in m_e c. */
typedef struct {
    int64_t step;
    double t;
    double ke;            /* sum over active records of w m (gamma - 1) */
    double ke_ions;       /* kind ION */
    double ke_electrons;  /* kind ELECTRON */
    double pe;            /* 1/2 sum_i Q_i phi_i, softened */
    double total;         /* ke + pe */
    double p[3];          /* sum of w m u */
    int64_t n_active;
    int64_t n_nonfinite;  /* records with a NaN/Inf position or momentum */
    int64_t charge_count[16];   /* ION records by charge state z (z >= 15 in the last bin) */
    double charge_weight[16];   /* the same, weighted by w */
} md_diag;

/* Kernel configuration of the fused Coulomb/push kernel.  md_autotune picks
 * one by timing; md_set_tuning forces one (must be an entry of
 * md_tuning_list). */
typedef struct {
    int32_t threads;    /* threads per CTA */
    int32_t r;          /* i-particles per thread (register blocking) */
    int32_t tile;       /* sources per shared-memory stage */
    int32_t ctas_per_sm;/* persistent CTAs per SM (0: as many as fit) */
    int32_t jsplit;     /* how the sources of an i-block are split into pieces:
                           1..64: that many equal segments per i-block;
                           0: a segment count chosen for load balance;
                           -k (1 <= k <= 8): equal shares, the sources of all i-blocks
                           laid end to end in tiles and cut into k x the resident CTAs
                           equal shares of one or more pieces each (contexts with
                           ionizing clusters take 0 instead).
                           The partial fields of the pieces go to a library scratch
                           buffer and the last piece to finish adds them in source
                           order and pushes.  With jsplit > 0 a cluster's results do
                           not depend on the other clusters of the context; with 0 or
                           equal shares they may.  md_get_tuning reports -k for equal shares,
                           else the largest segment count of any cluster; md_autotune
                           tries 0 for every configuration and -2, -4 for the two
                           fastest. */
    int32_t packed;     /* 1: pair arithmetic in packed f32x2 (two i-particles per
                           instruction, bit-identical results), 0: scalar FP32 */
    int32_t min_blocks; /* register budget: 64K / (threads x min_blocks); 0 = left to the
                           compiler.  On input to md_set_tuning, -1 matches any value */
} md_tuning;

/* ---- context life cycle -------------------------------------------------
 * md_init: creates a context holding n_clusters independent clusters (a
 * batched parameter scan when > 1), uploads their particles and returns it
 * in *out.  A cluster is the system of Sec. II: macro-ions and macro-electrons
 * (weight w = N_atoms / N_macro, Eq. 1) in a sphere of radius R0, with the
 * laser, boundary and ionization settings of its md_config.  cfgs[c] and parts[c] describe cluster c.  stream: a cudaStream_t
 * to launch on (NULL: the library creates its own).  The device must be an
 * sm_103 GPU.  Errors: MD_ERR_ARG (n_clusters < 1, n < 1, dt/softening/
 * lambda <= 0, bad enum, kind/z mismatch), MD_ERR_OOM, MD_ERR_CUDA. */
md_status md_init(md_ctx **out, const md_config *cfgs, int32_t n_clusters,
                  const md_particles *parts, void *stream);
void md_destroy(md_ctx *ctx);
const char *md_last_error(void);

/* Seeded placement of one cluster's records (Sec. II: the atoms of a cluster
 * of radius R0 sit at random inside the sphere; Eq. 1: a macro-particle of
 * weight w stands for w atoms, w = N_atoms / N_macro).  Records in the order
 * ions [0, n_ions), electrons [n_ions, n_ions + n_electrons), then n_slots
 * INACTIVE electron slots (at the centre, at rest, z = 0, mass 1) for the
 * ionization pass.  Every ion and electron is uniform in the ball of radius
 * r0 about `center` (rejection from the cube, Philox4x32-10 keyed on seed,
 * counter (record, attempt, 0x67656E01)); its u is a non-relativistic
 * Maxwellian of temperature kt (eV): each component normal with variance
 * kt / (m m_e c^2), from Box-Muller on counter (record, 0, 0x67656E02).
 * Charges: ion_charge (ions), -1 (electrons); masses ion_mass and 1; weight w
 * for every record.  Positions are bit-identical to any IEEE FP64 evaluation
 * of these draws in the stated order; momenta go through the device's log,
 * sin and cos. */
typedef struct {
    double r0;            /* sphere radius (paper units), > 0 */
    double center[3];     /* sphere centre (paper units) */
    double ion_mass;      /* m_e, > 0 */
    double weight;        /* macro weight w, > 0 */
    double kt_e_ev;       /* electron temperature (eV), >= 0; 0: at rest */
    double kt_i_ev;       /* ion temperature (eV), >= 0; 0: at rest */
    int64_t n_ions;       /* >= 0 */
    int64_t n_electrons;  /* >= 0 */
    int64_t n_slots;      /* >= 0; n_ions + n_electrons + n_slots >= 1 */
    int32_t ion_charge;   /* z of every ion, >= 0 (0: neutral atoms) */
    int32_t reserved;     /* must be 0 */
    uint64_t seed;        /* Philox key */
} md_generate;

/* md_init_generate: as md_init, with cluster c's records generated on the
 * device from gens[c] (md_generate) instead of copied from host arrays;
 * cfgs[c] as in md_init (its ionization settings refer to the generated
 * record order, e.g. n_ions = gens[c].n_ions, slot_base = n_ions +
 * n_electrons).  md_get_particles reads the records back.  Errors: as md_init,
 * and MD_ERR_ARG for a bad md_generate (message says which field) or an
 * ionization setting the generated records do not fit. */
md_status md_init_generate(md_ctx **out, const md_config *cfgs, const md_generate *gens,
                           int32_t n_clusters, void *stream);

/* md_step: advances every cluster by nsteps full steps (Sec. II): softened
 * Coulomb field at x^n + laser at t_n, relativistic Boris kick, FP64 drift,
 * boundary.  One fused kernel per step; runs of steps are replayed from a
 * captured CUDA graph.  Asynchronous.  nsteps >= 0. */
md_status md_step(md_ctx *ctx, int32_t nsteps);

/* md_sync: waits for the context's stream and reports device-side errors
 * (runtime control; no counterpart in the paper). */
md_status md_sync(md_ctx *ctx);

/* md_diagnostics: FP64 energies, momentum and charge-state counts of cluster
 * `cluster` at the current step (synchronous; out is caller-owned): the
 * energy balance and the charge-state distribution that Sec. III reports, at
 * integer time as md_diag states.  Errors: MD_ERR_ARG (NULL, bad index),
 * MD_ERR_NONFINITE (a record with NaN/Inf; out is still filled). */
md_status md_diagnostics(md_ctx *ctx, int32_t cluster, md_diag *out);

/* md_step_diag: one step of every cluster (as md_step(ctx, 1)) that also
 * writes out[k], for every cluster k, the diagnostics md_diagnostics would
 * report at the start of the step (t_n).  The potential is summed inside the
 * step's Coulomb pass (one more FP32 add per pair) and the kinetic energy at
 * integer time comes from the step's own kick, so a diagnosed step costs
 * about one step instead of two N^2 passes.  Contexts with ionization or
 * detectors or minimum-image forces use md_diagnostics and md_step instead
 * (same results up to the order of the FP32 sums).
 * out: caller-owned md_diag[n_clusters].  Synchronous.  Errors: MD_ERR_ARG,
 * MD_ERR_NONFINITE (after the step) as md_diagnostics. */
md_status md_step_diag(md_ctx *ctx, md_diag *out);

/* md_count_active: the number of records of cluster `cluster` that are not
 * MD_KIND_INACTIVE (md_diag.n_active; the macro-particles in play once the
 * ionization pass of Sec. II has freed electrons) without the rest of the
 * diagnostics:
 * an O(n) count, where md_diagnostics also sums the potential over all pairs.
 * Synchronous; *out is caller-owned.  Errors: MD_ERR_ARG (NULL, bad index). */
md_status md_count_active(md_ctx *ctx, int32_t cluster, int64_t *out);

/* md_get_particles / md_set_particles: copy cluster `cluster`'s records to /
 * from host arrays (n must equal the cluster's record count).  get is
 * synchronous; set reads the host arrays before it returns (page-locked
 * arrays are copied directly, others staged through pinned memory).
 * set checks every record as md_init does (kind, positive mass if active,
 * charge sign of the kind, finite x, u, w): MD_ERR_ARG names the first bad
 * record and the state is left unchanged.  For a cluster without ionization
 * the checks run on the GPU on the copied block; with ionization they run
 * on the host, with the electron-slot capacity check. */
md_status md_get_particles(md_ctx *ctx, int32_t cluster, md_particles *out);
md_status md_set_particles(md_ctx *ctx, int32_t cluster, const md_particles *in);

/* md_get_fields: the Coulomb field of Sec. II's particle mover (without the
 * laser) and, if phi != NULL,
 * the potential K_C sum_{j!=i} Q_j / sqrt(r^2+eps^2) at the current positions
 * of cluster `cluster`, computed by the same FP32/Kahan sum as md_step.
 * In clusters with ionization, records in a block of 256 targets with no
 * active record get zero, and uncharged groups of 64 sources are skipped.
 * e: host [n][3], phi: host [n] or NULL.  Synchronous. */
md_status md_get_fields(md_ctx *ctx, int32_t cluster, double *e, double *phi);

/* md_ionize: one Monte-Carlo ionization pass (Sec. II) of every cluster with
 * rate_model != 0 at the current step, whatever ionize_every says (dt_ion =
 * ionize_every dt, or dt if it is 0).  For each ion/atom record i < n_ions of
 * charge z < zmax: the Coulomb field at x_i from all other particles plus the
 * laser at t_n, the weight, mean and spread of u of the electrons within
 * r_loc (density in cm^-3, temperature in eV), the total rate (static ADK +
 * Lotz, or the surrogate), P = 1 - exp(-nu dt_ion), alpha from
 * Philox4x32-10(counter = (i, step lo, step hi, 0), key = seed); if
 * alpha < P the ion's charge rises by one and it frees an electron at x_i + r
 * (r uniform in the ball of radius r_create, from Philox words 1-3) with the
 * ion's u and weight.  The electrons freed in one pass take the next free
 * slots in the order of their ions' indices: the first goes to the record
 * after the last active slot, so the active slots stay one dense block.
 * md_init and md_set_particles reject (MD_ERR_ARG) a state in which the
 * ionizations still possible (sum over ions of zmax - z) do not fit after its
 * last active slot.  Asynchronous. */
md_status md_ionize(md_ctx *ctx);

/* ---- ion energy detectors (Sec. III, Fig. 3) --------------------------------
 * The paper compares ion energy distributions seen along and across the laser
 * polarization.  Here they are read at a fixed radius: an ion (kind ION,
 * z >= 1) that crosses the sphere |x - center| = radius outward during a step,
 * |x^n - c| < radius <= |x^{n+1} - c| (x^{n+1} after the boundary), is
 * recorded once, with its kinetic energy (gamma - 1) m c^2 at u^{n+1/2} (eV),
 * in up to five histograms: 0 = +x, 1 = -x, 2 = +y, 3 = -y (direction
 * (x^{n+1} - c)/|x^{n+1} - c| within cone_half_angle_deg of the axis) and
 * 4 = all directions.  Bins: n_bins of width e_max_ev / n_bins over
 * [0, e_max_ev) plus an overflow bin n_bins.  Counts are macro-ions.  The
 * crossing, cone and bin are decided in FP64 with each operation rounded to
 * nearest in a fixed order (no fused multiply-add). */
typedef struct {
    double radius;              /* paper units (e.g. 9 R0) */
    double cone_half_angle_deg; /* 0..90 */
    double e_max_ev;            /* > 0 */
    int32_t n_bins;             /* 1..4096 */
    int32_t reserved;           /* must be 0 */
    double center[3];           /* sphere centre, paper units */
} md_detector_config;

/* md_set_detectors: configures (d != NULL) or switches off (d == NULL) the
 * detectors of cluster `cluster`; a new configuration starts with empty
 * histograms and no ion recorded.  The first call allocates the histograms
 * of all clusters (5 x 4097 x 8 B each) and one byte per record.
 * Synchronous.  Errors: MD_ERR_ARG (bad index or configuration). */
md_status md_set_detectors(md_ctx *ctx, int32_t cluster, const md_detector_config *d);

/* md_get_iedf: the detector histograms of cluster `cluster` (host
 * detected[5][n_bins + 1], or NULL) and, if inside != NULL (host
 * [n_bins + 1]), the histogram of the ions not yet recorded at their current
 * u (u^{n-1/2}); together they are the total ion energy distribution.
 * MD_ERR_STATE without detectors.  Allocates n_bins + 1 counters on the device
 * for `inside` during the call.  Synchronous. */
md_status md_get_iedf(md_ctx *ctx, int32_t cluster, uint64_t *detected, uint64_t *inside);

/* md_get_ionization: per-ion inputs and outcome of the last ionization pass
 * (Sec. II, ionization paragraph) of cluster `cluster`
 * (host arrays of n_ions entries, any may be NULL): field magnitude |E| (paper
 * units), local electron density (cm^-3) and temperature (eV), probability P
 * and whether the ion ionized.  Synchronous. */
md_status md_get_ionization(md_ctx *ctx, int32_t cluster, double *emag, double *ne, double *te,
                            double *prob, uint8_t *fired);

/* md_set_step: sets the step counter (with md_set_particles, a checkpoint is
 * restored exactly: the laser time t_n = t0 + n dt of Eqs. 3-9 and the Philox
 * counters derive from the step).  Synchronous.  Errors: MD_ERR_ARG (step < 0). */
md_status md_set_step(md_ctx *ctx, int64_t step);

/* ---- target slices: one cluster split over several GPUs ---------------------
 * The step's cost is the direct sum over all pairs (Sec. II, particle mover
 * paragraph; Sec. III: time grows as N_part^2).  The paper parallelises the
 * force and mover loops over target particles on the cores of one node; here
 * the same split spreads one cluster over GPUs.  Every GPU holds the whole
 * cluster, sums the field of all sources at its own slice of target records
 * and pushes only those; between steps the slices' new positions (the j-stream,
 * 16 bytes per record) are exchanged, e.g. by an all-gather, so every GPU
 * again holds every source.
 *
 * md_set_slice: from now on cluster `cluster` of this context pushes only its
 * records [i_begin, i_end).  i_begin and i_end are multiples of 1024 (a whole
 * number of i-blocks of every kernel configuration) or the record count n;
 * [0, n) undoes the slice, i_begin == i_end pushes nothing.
 * Records outside the slice keep their state (md_get_particles returns it as
 * it was: stale on this GPU); their j-stream entries are whatever the caller
 * writes through md_get_jstream.  md_get_fields writes e and phi for the
 * slice's records only; md_diagnostics and md_step_diag sum over the slice's
 * records (the field and potential at them from all sources), so the
 * cluster's totals are the sums over the GPUs' slices.
 * Errors: MD_ERR_ARG (bounds), MD_ERR_STATE (a context with ionization or
 * detectors).  Synchronous. */
md_status md_set_slice(md_ctx *ctx, int32_t cluster, int64_t i_begin, int64_t i_end);

/* md_get_jstream: device address of cluster `cluster`'s current j-stream,
 * the float4[n_pad] records (x, y, z, K_C w z) that the next step reads as
 * its sources (n_pad: the record count rounded up to a multiple of 16; the
 * padding records carry no charge).  After a step each GPU's slice of it holds
 * that GPU's new positions; the caller writes the other slices there (ordered
 * before the next md_step on the context's stream) from the GPUs that own
 * them.  The address changes from step to step (two buffers alternate).
 * Synchronises the context's stream. */
md_status md_get_jstream(md_ctx *ctx, int32_t cluster, void **posq, int64_t *n_pad);

/* md_wait_selftest (runtime check; no counterpart in the paper): exercises
 * the bounded device waits.  One CTA waits on an
 * mbarrier phase that nothing completes; after budget_ms (0 < budget_ms <=
 * 5000, converted with the nominal SM clock) the wait gives up, the kernel
 * sets the context's error word and returns.  Returns MD_ERR_TIMEOUT (the
 * expected outcome) and leaves the context usable. */
md_status md_wait_selftest(md_ctx *ctx, double budget_ms);

/* Step counter of the context (steps taken since md_init, or as set by
 * md_set_step): step n is at time t0 + n dt.  Synchronous. */
md_status md_get_step(md_ctx *ctx, int64_t *step);

/* ---- tuning (runtime control; no counterpart in the paper) ---------------
 * md_tuning_list: writes up to cap entries of the compiled kernel
 * configurations into list (may be NULL) and returns their number.
 * md_set_tuning: uses the given configuration from now on.
 * md_get_tuning: the configuration in use.
 * md_autotune: times every configuration over `steps` steps on the
 * context's own state (restored afterwards), with jsplit 0 and, for the two
 * fastest, jsplit -2 and -4 (no ionizing cluster), and keeps the fastest; the
 * per-configuration best mean step times in ms go to times_ms (cap entries,
 * may be NULL; -1 for a configuration not timed). */
int32_t md_tuning_list(md_tuning *list, int32_t cap);
md_status md_set_tuning(md_ctx *ctx, const md_tuning *t);
md_status md_get_tuning(md_ctx *ctx, md_tuning *t);
md_status md_autotune(md_ctx *ctx, int32_t steps, double *times_ms, int32_t cap);

/* md_plan_shares: the work units that equal shares (jsplit < 0) give the step
 * kernel, for clusters of n_pad[c] records (records with their zero-charge
 * padding, c < n_clusters) pushed in i-blocks of `per` targets (threads x r
 * of a configuration) with `tile`-record source tiles, when `shares` shares
 * are handed out (k x the resident CTAs).  The source tiles of every i-block,
 * laid end to end in cluster and i-block order (T tiles), are cut into
 * S = min(shares, T) shares of floor or ceil of T / S tiles; a share is one
 * or more pieces, a piece one i-block's tile range.  Host only: no device is
 * touched and the library's state is not changed.
 * units (may be NULL): caller-owned int32[6 x cap], per unit in share order
 * (cluster, i-block, piece of the i-block numbered in source order, pieces of
 * the i-block, first source record, source records); first (may be NULL):
 * caller-owned int32[shares + 1], the first unit of share s at first[s] and
 * the unit count at first[S].  *n_units and *n_shares receive the counts;
 * with units and first NULL the call only sizes them.  Errors: MD_ERR_ARG
 * (NULL n_pad/n_units/n_shares, n_clusters, per, tile or shares < 1, an
 * n_pad < 1, shares or T of 2^31 or more, units given with cap below the
 * unit count),
 * MD_ERR_OOM (host memory). */
md_status md_plan_shares(const int32_t *n_pad, int32_t n_clusters, int32_t per, int32_t tile,
                         int64_t shares, int32_t *units, int64_t cap, int32_t *first,
                         int64_t *n_units, int64_t *n_shares);

/* ---- stateless field evaluation on caller device buffers -----------------
 * md_coulomb_field_device: field (and potential) at nt targets from ns
 * sources, the FP32/Kahan direct sum of Sec. II on device memory the caller
 * owns.
 *   src:  device float4[ns] = (x, y, z, K_C * Q) per source (16-byte aligned)
 *   tgt:  device float4[nt] = (x, y, z, unused) per target
 *   eps2: softening squared
 *   self_offset: target i is source i + self_offset (its potential self term
 *         is removed), or -1 if targets are not sources
 *   e:    device double[nt][3] output field; phi: device double[nt] or NULL
 *   stream: cudaStream_t (NULL = legacy default stream).  Asynchronous.
 * When few targets would leave the GPU mostly idle, the sources are split
 * into segments whose partial fields are added in order (deterministic); the
 * partials are allocated and freed in stream order on `stream` (at most
 * 256 MB), so calls on different streams may overlap.
 * Errors: MD_ERR_ARG for NULL/unaligned pointers, ns < 0, nt < 0.  A
 * device-side wait that runs out of its budget (about 2 s) leaves e/phi not
 * (completely) written and is recorded in the device's sticky field error
 * word: md_field_device_status reports it. */
md_status md_coulomb_field_device(const void *src, int64_t ns, const void *tgt,
                                  int64_t nt, float eps2, int64_t self_offset,
                                  double *e, double *phi, void *stream);

/* md_coulomb_field_device_noalloc: the same field and potential as
 * md_coulomb_field_device, for callers that cannot allocate device memory
 * (code inside another framework's memory pool, a graph builder that must not
 * see cudaMalloc, a plugin whose host forbids allocation).  The paper has no
 * counterpart: this is a library-interface variant.  The sources are cut into
 * up to 8 segments whose partial fields go to a fixed scratch array compiled
 * into the library (about 8.6 MB of device memory on every GPU that loads it,
 * held until the process exits); the call itself allocates nothing.
 *   Arguments, layout and ownership: as md_coulomb_field_device.
 *   Limit: nt <= 32768 targets per call (MD_ERR_ARG beyond it, nothing is
 *   launched); ns is unbounded.
 *   The first call on a device looks up the scratch array's device address on
 *   that device; make that first call before any stream capture.
 *   Every call shares the one scratch array: calls that overlap on the GPU
 *   (other streams, other host threads) race and give wrong results, so
 *   serialise them.  Each call clears the counters it uses before its kernel.
 *   Asynchronous on `stream`. */
md_status md_coulomb_field_device_noalloc(const void *src, int64_t ns, const void *tgt,
                                          int64_t nt, float eps2, int64_t self_offset,
                                          double *e, double *phi, void *stream);

/* md_field_device_status (runtime control; no counterpart in the paper): the
 * outcome of the stateless field calls (md_coulomb_field_device and
 * md_coulomb_field_device_noalloc) on the current device.  Those calls are
 * asynchronous and return MD_OK once their kernels are launched; a device-side
 * wait that later runs out of its budget sets a per-device error word (a fixed
 * device array, no allocation) and the call's output is then not (completely)
 * written.  The word is sticky: it collects every such call on the device,
 * from any stream, until this call reads it.  md_field_device_status
 * synchronises `stream` (issue it on the stream of the calls to check, or
 * synchronise their streams first), reads the word and clears it.
 * Returns MD_ERR_TIMEOUT if a wait ran out, MD_ERR_STATE if a bounds check of
 * the checked build failed, else MD_OK.
 * The device addresses of the library's device arrays are looked up once per
 * device ordinal and kept for the life of the process: calling the stateless
 * entry points after cudaDeviceReset on that device is not supported. */
md_status md_field_device_status(void *stream);

/* md_field_wait_selftest (runtime check; no counterpart in the paper): one CTA
 * on `stream` waits on an mbarrier phase that nothing completes; after
 * budget_ms (0 < budget_ms <= 5000, converted with the nominal SM clock) it
 * gives up and sets the field error word of the current device, which the
 * next md_field_device_status reports as MD_ERR_TIMEOUT.  Asynchronous. */
md_status md_field_wait_selftest(double budget_ms, void *stream);

/* md_coulomb_field_fp64_device: the FP64 reference of the direct sum of
 * Sec. II (the precision study's reference, not on the hot path).  For each target i:
 *   E_i   = kc sum_j Q_j (x_i - x_j) / (|x_i - x_j|^2 + eps^2)^{3/2}
 *   phi_i = kc sum_j Q_j / sqrt(|x_i - x_j|^2 + eps^2)
 * over sources j in index order, skipping j == self_idx[i] and Q_j == 0, every
 * operation rounded to nearest in the order of this formula (no fused
 * multiply-add), so that a plain sequential program evaluating the same
 * formula in the same order gets the same bits.
 *   xs: device double[ns][3] source positions; qs: device double[ns] macro
 *   charges w z; xt: device double[nt][3] targets; self_idx: device
 *   int64[nt] (the source that is target i, or -1) or NULL; eps >= 0, kc > 0
 *   (paper units); e: device double[nt][3] out; phi: device double[nt] or NULL.
 * Caller-owned device buffers.  One thread per target: O(nt ns) FP64
 * operations, meant for subsets of targets.  Asynchronous on `stream`. */
md_status md_coulomb_field_fp64_device(const double *xs, const double *qs, int64_t ns,
                                       const double *xt, const int64_t *self_idx, int64_t nt,
                                       double eps, double kc, double *e, double *phi,
                                       void *stream);

/* ---- learned rate surrogate ------------------------------------------------
 * Not from the paper: a 4 -> 64 -> 64 -> 8 MLP (SiLU) standing in for the
 * per-ion rate evaluation of the ionization pass.  The hidden layers run on
 * the tensor cores with BF16 weights and activations and FP32 accumulation;
 * the output layer is an FP32 dot product.  Features of an ion of charge z:
 * ((log10(F/F0)+1.4)/1.5, z/8, (log10 max(n_e,1e15)-19.5)/4.5,
 * (log10(max(T_e,0.1)/Ip)+0.2)/3) with F = max(|E|,1e-6) in atomic units,
 * Ip = ip_ev[z], F0 = (2 Ip/E_h)^(3/2); output
 * y_k ~ (log10(nu_k + 1e-12)+6)/6 for the step k -> k+1, inverted as
 * nu = max(10^(6y-6) - 1e-12, 0) (rates below 1e-12 per unit time never
 * ionize: P < 1e-13 per pass).  Parameters:
 * 5000 FP32 values W1[64][4] b1[64] W2[64][64] b2[64] W3[8][64] b3[8]. */
typedef struct {
    double ip_ev[16];       /* species data as in md_config (z < zmax) */
    double q_outer[16];
    int32_t zmax;           /* 1..8 */
    int32_t epochs;
    double lambda_um;       /* laser wavelength of the unit conversion */
    int64_t n_samples;      /* training samples; a held-out set of max(4096, n/20) is added */
    int32_t batch;          /* minibatch size */
    int32_t reserved;       /* must be 0 */
    double lr;              /* Adam learning rate, cosine-decayed to 1 % */
    uint64_t seed;          /* Philox key of the samples and of the initial weights */
    double e_min, e_max;    /* training domain: |E| (paper units) */
    double ne_min, ne_max;  /* n_e (cm^-3) */
    double te_min, te_max;  /* T_e (eV) */
} md_mlp_train_config;

typedef struct {
    double loss_first, loss_last;  /* mean minibatch loss of the first and last step */
    double holdout_median_dlog10;  /* |log10 nu_surrogate - log10 nu_plain| on held-out samples */
    double holdout_p99_dlog10;
    double holdout_max_dlog10;
    double train_ms;               /* device time of sample generation + training */
    int64_t n_holdout;
    int64_t steps;
} md_mlp_report;

/* md_mlp_train: draws n_samples of (|E|, z, n_e, T_e) log-uniform over the
 * domain with Philox, labels them with the library's FP64 plain rate (static
 * ADK + Lotz), trains the surrogate on the GPU (its own forward/backward kernels,
 * deterministic gradient reduction, Adam) and writes the FP32 parameters to
 * params_out (host, 5000 floats).  Allocates and frees its own device
 * buffers.  Synchronous on `stream`. */
md_status md_mlp_train(const md_mlp_train_config *cfg, float *params_out, md_mlp_report *rep,
                       void *stream);

/* md_set_rate_mlp: installs surrogate parameters (host, 5000 floats) in the
 * context; clusters with rate_model MD_RATES_MLP then use it for ions inside
 * the domain of `domain` and the plain rates outside.  `domain` is the
 * training configuration: MD_ERR_ARG if its species table (ip_ev, q_outer
 * below zmax) or wavelength differs from such a cluster's. */
md_status md_set_rate_mlp(md_ctx *ctx, const float *params, const md_mlp_train_config *domain);

/* Device-buffer entry points of the surrogate (all pointers device memory):
 *   md_mlp_forward_device: y[n][8] from features feats[n][4].
 *   md_mlp_loss_grad_device: loss (mean squared error of y[z]) and its
 *     gradient grad[5000] for samples feats[n][4], z[n], target[n];
 *     allocates per-call scratch; synchronous.
 *   md_mlp_samples_device: the training samples of md_mlp_train (features,
 *     z, target, and raw[n][3] = |E|, n_e, T_e if raw != NULL).
 *   md_ion_rates_device: total rate per unit time nu[n] from |E|, z, n_e,
 *     T_e with model 1 (plain) or 2 (surrogate inside the domain of cfg,
 *     plain outside; params = device surrogate parameters). */
md_status md_mlp_forward_device(const float *params, const float *feats, int64_t n, float *y,
                                void *stream);
md_status md_mlp_loss_grad_device(const float *params, const float *feats, const int32_t *z,
                                  const float *target, int64_t n, float *grad, float *loss,
                                  void *stream);
md_status md_mlp_samples_device(const md_mlp_train_config *cfg, int64_t n, uint64_t seed,
                                float *feats, int32_t *z, float *target, double *raw,
                                void *stream);
md_status md_ion_rates_device(const md_mlp_train_config *cfg, int32_t model, const float *params,
                              const double *emag, const int32_t *z, const double *ne,
                              const double *te, int64_t n, double *nu, void *stream);

/* ---- helpers for SI inputs (Sec. II) ------------------------------------ */
double md_coulomb_constant(double lambda_um);                  /* K_C = 2 pi r_e / lambda */
double md_a0_from_intensity(double intensity_wcm2, double lambda_um); /* Eq. 2 */
double md_n_atoms(double r0, double r_wigner_seitz);           /* Eq. 1 */

/* Measurement helper (no counterpart in the paper): FP32 fused multiply-adds per second (lane operations)
 * of the current device, from kernels of 8 independent FMA chains per thread
 * on 8 x SMs CTAs of 256 threads: *ffma_per_s with scalar fma.rn.f32,
 * *packed_fma_per_s (may be NULL) with packed fma.rn.f32x2.  Synchronous on
 * `stream`.  The denominators of the FP32 roofline fraction. */
md_status md_measure_fp32_peak(double *ffma_per_s, double *packed_fma_per_s, void *stream);

/* Number of SMs and the device name of the current device (for reports; no
 * counterpart in the paper).  name: host buffer of name_cap bytes. */
md_status md_device_info(int32_t *sm_count, char *name, int32_t name_cap);

#ifdef __cplusplus
}
#endif

#endif /* MD_H */
