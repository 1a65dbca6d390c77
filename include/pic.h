/* pic.h -- C ABI of the GB300 (sm_103a) PIC-MCC positive-column library.
 *
 * The library advances the 1D3V electrostatic Particle-In-Cell Monte Carlo
 * Collisions model of a rare-gas positive column of Boeuf, "Ionization waves
 * (striations) in a low-current plasma column revisited with kinetic and
 * fluid models", Sec. II: electrons and ions move in the self-consistent
 * field E = -E0 + E_sp of a periodic column of length L; the field comes from
 * Poisson's equation on a uniform grid; collisions with the neutral gas are
 * Monte Carlo events drawn from cross sections; every ionization creates an
 * electron-ion pair and, in the paper's model, removes one randomly chosen
 * electron and one randomly chosen ion so that the particle number stays
 * constant.  Sec. V's alternative (an imposed loss frequency) is the RADIAL
 * loss mode.
 *
 * Every step runs in CUDA kernels on one GPU; there is no CPU fallback.  All
 * calls return 0 or a negative PIC_E* code; pic_last_error() gives a message.
 *
 * Conventions
 *  - Pointers in structs passed IN are caller-owned host memory, read during
 *    the call only; nothing is retained after the call returns.
 *  - Pointers in structs passed OUT are caller-owned host buffers of the
 *    documented length; a NULL pointer skips that output.
 *  - A handle owns its device memory and one CUDA stream; it is not
 *    thread-safe.  Errors raised on the device (capacity, non-finite field)
 *    latch in the handle and are returned by the call that detects them.
 *  - Units are SI except energies (eV) and pressure (Torr).
 */
#ifndef PIC_H
#define PIC_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_ABI_VERSION 1

/* error codes */
#define PIC_OK 0
#define PIC_EINVAL (-1)     /* bad argument */
#define PIC_ENOMEM (-2)     /* device or host allocation failed */
#define PIC_ECUDA (-3)      /* a CUDA runtime call failed */
#define PIC_ECAPACITY (-4)  /* particle capacity or per-step staging capacity exceeded */
#define PIC_ENONFINITE (-5) /* the field became non-finite */
#define PIC_ETIMEOUT (-6)   /* a bounded device wait gave up */
#define PIC_EPARAM (-7)     /* stability limit violated (nu* dt > 0.3) without PIC_FLAG_ALLOW_LARGE_NULL */

/* collision process kinds (Sec. II: electron-neutral elastic, excitation,
 * ionization; ion-neutral charge exchange ("backward") and isotropic) */
#define PIC_ELASTIC 0
#define PIC_EXCITATION 1
#define PIC_IONIZATION 2
#define PIC_ION_CX 3
#define PIC_ION_ISO 4

/* how the applied field E0 is set */
#define PIC_DRIVE_E0 0       /* E0 = E0_Vpm (the paper's control parameter) */
#define PIC_DRIVE_V 1        /* E0 = V_applied / L */
#define PIC_DRIVE_CIRCUIT 2  /* Sec. V: external circuit U_src = R_ext J + E0 L: E0 = (U_src - R_ext J) / L
                                after every step, J = e w (sum v_x,electrons - sum v_x,ions) / L the
                                discharge current density over the pushed particles (positive when the
                                electrons drift against the applied field -E0; ions at their last push;
                                velocities summed as round(256 v_x), exact) */
#define PIC_DRIVE_RI 3       /* tube radius R_m and current I_A (eq. 2): E0 and n0 from pic_drive_ri at
                                pic_init, then run as PIC_DRIVE_E0 (E0_Vpm and n0_m3 are ignored) */

/* field: self-consistent (Sec. II) or the applied field alone (uniform-field swarm) */
#define PIC_FIELD_POISSON 0
#define PIC_FIELD_APPLIED 1

/* particle losses */
#define PIC_LOSS_PAIR 0    /* Sec. II: one random electron and ion removed per ionization */
#define PIC_LOSS_RADIAL 1  /* Sec. V: every particle removed with probability 1 - exp(-nu_w dt) */
#define PIC_LOSS_NONE 2    /* births kept, nothing removed */
#define PIC_LOSS_SWARM 3   /* ionizations counted but no particle created or removed */

/* particle storage form */
#define PIC_FP64 0   /* FP64 offset and velocity */
#define PIC_MIXED 1  /* int32 cell + FP32 offset/velocity (float4); FP64 field */

/* flags */
#define PIC_FLAG_RECORD_CODES 1u        /* keep each particle's process code of the last step */
#define PIC_FLAG_NO_GRAPH 2u            /* launch kernels one by one instead of CUDA graphs */
#define PIC_FLAG_ALLOW_LARGE_NULL 4u    /* accept nu* dt > 0.3 */
#define PIC_FLAG_BOUNDED 8u             /* Sec. V: the bounded column instead of the periodic one.  The
                                           cathode (x = 0) and anode (x = L) take every particle that
                                           crosses them; the field solves Gauss's law between them
                                           with the potential V_D = E0 L across the gap (E0 from the
                                           drive: V_applied / L, E0_Vpm, or the circuit's
                                           (U_src - R_ext J) / L); the cathode emits J_emit_Am2 at
                                           T_emit_eV.  Node arrays get n_cells + 1 entries.  Needs
                                           PIC_LOSS_RADIAL (the fixed loss frequency nu_w of Sec. V)
                                           or PIC_LOSS_NONE; single columns only. */

/* One collision process (Sec. II: one member of a gas's cross-section set): sigma(eps)
 * on an ascending energy grid.  Electron processes use the electron energy;
 * ion processes use 0.5 M g^2 / e, g the ion-neutral relative speed.  Linear
 * interpolation between points, end values held outside; excitation and
 * ionization are zero below threshold_eV. */
typedef struct pic_xsec {
  int32_t kind;            /* PIC_ELASTIC .. PIC_ION_ISO */
  int32_t n;               /* number of points, >= 1 */
  double threshold_eV;     /* excitation / ionization threshold; ignored otherwise */
  const double *energy_eV; /* n ascending energies */
  const double *sigma_m2;  /* n cross sections */
} pic_xsec;

/* The problem statement of one periodic column (Sec. II). */
typedef struct pic_params {
  double gas_mass_amu;     /* neutral (= ion) mass */
  double pressure_torr;    /* gas pressure p */
  double T_gas_K;          /* gas temperature */
  double L_m;              /* column length L */
  double R_m;              /* column radius R (used by radius-based drives) */
  int32_t drive;           /* PIC_DRIVE_* */
  int32_t field_mode;      /* PIC_FIELD_* */
  double E0_Vpm;           /* |applied field| for PIC_DRIVE_E0; the applied field is -E0 */
  double V_applied;        /* voltage across L for PIC_DRIVE_V */
  double I_A, U_src, R_ext_ohm_m2;  /* discharge current (workload label); circuit source voltage (V) and
                                       resistor (Ohm m^2) of PIC_DRIVE_CIRCUIT */
  int32_t n_xsec, pad0;
  const pic_xsec *xsec;    /* n_xsec processes; at most 16 per species */
  int32_t n_cells;         /* grid cells = nodes (periodic), 3 <= n_cells <= 65536 */
  int32_t ion_subcycle;    /* ions advance every ion_subcycle steps with dt_i = ion_subcycle dt; 0 = frozen */
  double dt_s;             /* electron time step dt (Sec. II: dt < 0.2/w_pe) */
  int64_t n_e0, n_i0;      /* initial macroparticles per species */
  int64_t capacity;        /* particle slots per species; 0 = 1.25 max(n_e0, n_i0) + 1024 */
  double n0_m3;            /* initial density n0: macro weight w = n0 L / n_e0 (per m^2) */
  double Te0_eV, Ti0_eV;   /* initial Maxwellian temperatures */
  int32_t loss_mode;       /* PIC_LOSS_* */
  int32_t precision;       /* PIC_FP64 or PIC_MIXED */
  double nu_w;             /* loss frequency of PIC_LOSS_RADIAL (s^-1) */
  uint64_t seed;           /* Philox4x32-10 key */
  int32_t diag_every;      /* accumulate moments every diag_every steps (0 = never); must be a
                              multiple of ion_subcycle when ions move */
  int32_t sort_every;      /* counting sort of particles by cell every sort_every steps (0 = never) */
  int32_t n_table;         /* points of the uniform-energy collision-frequency tables, >= 3 */
  uint32_t flags;          /* PIC_FLAG_* */
  double eps_max_e_eV;     /* electron table range [0, eps_max_e]; higher energies hold the last value */
  double eps_max_i_eV;     /* ion table range */
  int32_t column, pad1;    /* column index mixed into the random-number counters (batched runs) */
  double J_emit_Am2;       /* PIC_FLAG_BOUNDED: electron current density emitted by the cathode: J dt / (e w)
                              macro-electrons per step (fraction carried over), velocities (s |g0|, s g1, s g2)
                              with s = (e T_emit / m)^(1/2), starting at x = u v_x dt */
  double T_emit_eV;        /* emission temperature */
} pic_params;

/* Particle state and field, host arrays.  pic_get_state fills the non-NULL
 * arrays (lengths >= n_e, n_i, and the node count: n_cells, or n_cells + 1 in a
 * bounded column); pic_set_state reads them.  For
 * PIC_MIXED the offsets/velocities are rounded to FP32 on set and widened on get.
 * Offsets lie in [0, 1): position x = (cell + off) L / n_cells. */
typedef struct pic_state {
  int64_t n_e, n_i;        /* live particles */
  int64_t step;            /* steps taken (the random-number counter of the next step) */
  int64_t next_id;         /* id of the next newborn particle */
  double E0;               /* current |applied field| */
  int32_t *cell_e; double *off_e, *vx_e, *vy_e, *vz_e; uint64_t *id_e;
  int32_t *cell_i; double *off_i, *vx_i, *vy_i, *vz_i; uint64_t *id_i;
  double *E;               /* node field E^n (V/m), one per node; set: NULL = recompute from the charges */
  int64_t *Q_e;            /* electron node charge, fixed point 2^32 per particle (get only) */
  int64_t *Q_i;            /* ion node charge, fixed point (set: NULL = re-deposit the ions) */
} pic_state;

/* The particle state with the offsets and velocities in FP32, the storage form of a PIC_MIXED
 * column (Sec. II's particles: cell, offset in the cell, three velocity components, id), for
 * pic_set_state_f32.  The other members mean what they mean in pic_state. */
typedef struct pic_state_f32 {
  int64_t n_e, n_i;
  int64_t step;
  int64_t next_id;
  double E0;
  int32_t *cell_e; float *off_e, *vx_e, *vy_e, *vz_e; uint64_t *id_e;
  int32_t *cell_i; float *off_i, *vx_i, *vy_i, *vz_i; uint64_t *id_i;
  double *E;               /* NULL = recompute from the charges */
  int64_t *Q_i;            /* NULL = re-deposit the ions */
} pic_state_f32;

/* Counters since pic_init. */
typedef struct pic_stats {
  int64_t step, n_e, n_i, next_id;
  int64_t n_coll_e[16];    /* real electron collisions per electron process (in xsec order) */
  int64_t n_coll_i[16];    /* real ion collisions per ion process */
  int64_t births;          /* ionization events (pairs created) */
  int64_t losses_e, losses_i;
  int64_t overflow_e, overflow_i;  /* collisions evaluated above the table range */
  double E0;
  int64_t n_diag;          /* diagnostic samples taken */
  int64_t absorbed_e[2], absorbed_i[2];   /* PIC_FLAG_BOUNDED: particles taken by [cathode, anode] */
  int64_t emitted;         /* electrons emitted by the cathode */
} pic_stats;

/* Time-averaged moments over the current window (the profiles of Fig. 4).
 * Every non-NULL array has one entry per node (n_cells, or n_cells + 1 in a bounded
 * column). */
typedef struct pic_moments_out {
  int64_t n_samples, n_steps;   /* diagnostic samples / steps in the window (out) */
  double *n_e, *n_i;            /* densities (m^-3) */
  double *gamma_e;              /* electron flux (m^-2 s^-1) */
  double *mean_eps_e;           /* electron mean energy (eV) */
  double *heat_e;               /* electron energy flux (eV m^-2 s^-1) */
  double *iz_rate;              /* ionizations (m^-3 s^-1), every step counted */
  double *gamma_i;              /* ion flux (m^-2 s^-1) */
  double *E;                    /* field (V/m) */
  double *phi;                  /* space-charge potential (V), phi_0 = 0 */
  int32_t reset, pad;           /* in: reset the window after reading */
} pic_moments_out;

typedef struct pic_handle pic_handle;

/* Create one column (Sec. II).  Validates params, builds the collision tables, allocates
 * device memory, places n_e0 electrons and n_i0 ions uniformly in x with Maxwellian
 * velocities at Te0 / Ti0, solves the initial field, and pulls the velocities back half a
 * step (the leapfrog start).  PIC_DRIVE_RI is first resolved into E0 and n0 by eq. 2
 * (pic_drive_ri).
 * params and its xsec arrays are read during the call only.  On success *out is a handle
 * owned by the caller until pic_free.  On failure *out = NULL and nothing stays allocated:
 * PIC_EINVAL for an invalid problem statement (checked before any device call; the message
 * names the offending field; also a capacity below the initial count), PIC_ENOMEM,
 * PIC_ECUDA (no device, or a failed launch). */
int pic_init(const pic_params *params, pic_handle **out);

/* Resolution limits of the explicit particle scheme (Sec. II): the time step must resolve the
 * electron plasma frequency, dt < 0.2 / w_pe, and the cell size the electron Debye length,
 * dx < lambda_De, with w_pe = (n0 e^2 / (eps0 m_e))^(1/2) and lambda_De = (eps0 Te0 / (n0 e))^(1/2)
 * (Te0 in eV) at the initial density and temperature (PIC_DRIVE_RI: the n0 of eq. 2).  Host
 * only: no device call.  These are warnings, not errors: pic_init does not enforce them.
 *   out    (may be NULL) out[0] = w_pe dt, out[1] = dx / lambda_De (HUGE_VAL when Te0 = 0)
 * Returns the PIC_WARN_* bits of the limits that fail (0 when both hold), or PIC_EINVAL for a
 * NULL, non-finite or non-positive statement. */
#define PIC_WARN_PLASMA_FREQ 1   /* w_pe dt >= 0.2 */
#define PIC_WARN_DEBYE 2         /* dx >= lambda_De */
int pic_check_stability(const pic_params *params, double out[2]);

/* Advance n >= 0 steps.  Each step: electron gather/push/collisions/deposit,
 * ion step on every ion_subcycle-th step, births and removals, periodic sort
 * every sort_every steps, field solve.  A plain ion cycle (ion_subcycle steps
 * with no sort and no diagnostic sample) is replayed from a CUDA graph captured
 * on first use (PIC_FLAG_NO_GRAPH or kernel timing: launched one by one); the
 * results are the same.  Stream-ordered; synchronises once at the end to read
 * the device status word.
 * Errors: PIC_EINVAL (n < 0, or a column of a batch); a device-side error of the step
 * (PIC_ECAPACITY: more births than free slots, or than particles to remove; PIC_ENONFINITE:
 * a non-finite field) is returned after the step and latched: every later call on the handle
 * returns it until pic_set_state installs a new state.  The births of the failing step are
 * not written. */
int pic_step(pic_handle *h, int64_t n);

/* Copy the moment window (Sec. III, the profiles of Fig. 4): time averages over the
 * diagnostic samples since the last reset (see pic_moments_out for units).  Every non-NULL
 * array is caller-owned host memory of one entry per node (n_cells, or n_cells + 1 in a
 * bounded column); NULL skips it.  Synchronises the handle's stream.  PIC_EINVAL for a NULL
 * argument. */
int pic_moments(pic_handle *h, pic_moments_out *out);

/* Electron energy probability function F(x, eps) (Sec. III.C, Fig. 8), sampled as a
 * histogram.  With n_x > 0, on every diagnostic step (diag_every) each live electron
 * adds 1 to bin (floor(cell n_x / n_cells), floor(eps n_eps / eps_max)) after its push
 * and collision; column n_eps collects the energies at or above eps_max (and non-finite
 * ones), so each sample adds exactly n_e counts.  eps = K (vx^2 + vy^2 + vz^2) and its
 * bin are computed in the storage precision, as in the collision test.  The host
 * normalises: F = counts / (sum eps^(1/2) counts deps) per spatial bin, so that
 * int eps^(1/2) F deps = 1.  pic_eepf_config allocates and clears the histogram
 * (n_x = 0 frees it); 1 <= n_x <= n_cells, 1 <= n_eps <= 65536, eps_max > 0.  Single
 * columns only: PIC_EINVAL on a batch or a column of one. */
int pic_eepf_config(pic_handle *h, int32_t n_x, int32_t n_eps, double eps_max_eV);
/* Copy the n_x (n_eps + 1) counts (x-major, host array) and the number of diagnostic
 * samples they hold; reset = 1 clears both afterwards. */
int pic_eepf_get(pic_handle *h, uint64_t *counts, int64_t *n_samples, int32_t reset);

/* Copy the state: counts, step counter, next id and E0 always; then every non-NULL array,
 * caller-owned host memory of at least n_e (electron arrays) or n_i (ion arrays) entries,
 * which pic_get_stats gives, or of the capacity; E, Q_e and Q_i hold one entry per node.  The
 * MIXED form's FP32 offsets and velocities are widened exactly to double.  Synchronises the
 * handle's stream; PIC_EINVAL for a NULL argument. */
int pic_get_state(pic_handle *h, pic_state *out);
/* Replace the state; the next step uses state->step as its counter.  The arrays are
 * uploaded as given (pinned host memory copies at full link speed) and checked on the
 * device: a particle outside the grid (cell not in [0, n_cells), offset not in [0, 1),
 * or, for PIC_MIXED, an offset that rounds to 1 in FP32) returns PIC_EINVAL naming the
 * lowest such particle and leaves the particles undefined until the next successful
 * call.  The first call allocates 32 bytes of device memory per particle of capacity. */
int pic_set_state(pic_handle *h, const pic_state *in);
/* pic_set_state with FP32 offsets and velocities (pic_state_f32).  A PIC_MIXED column stores
 * them as given, with no rounding on the way in, and the upload moves 28 bytes per particle
 * instead of 44.  A PIC_FP64 column widens them exactly.  Checks, errors, ownership (nothing is
 * kept after the call) and the first call's staging allocation are those of pic_set_state. */
int pic_set_state_f32(pic_handle *h, const pic_state_f32 *in);
/* Copy the counters (pic_stats) into *out.  Synchronises the handle's stream; PIC_EINVAL for a
 * NULL argument. */
int pic_get_stats(pic_handle *h, pic_stats *out);

/* Batched columns: n independent periodic columns (uneven lengths, cell counts,
 * pressures, particle counts, gases) advanced together, one kernel launch per
 * phase of the step for all columns, on a CTA schedule in proportion to each
 * column's particles, with the plain ion cycles replayed from a captured
 * CUDA graph.  The schedule has mult x SMs CTAs per species; the first steps
 * tune mult per species (1, 2, 3, 4, 6 or 8, each timed twice on that
 * species' push kernel, electrons first, then ions on their steps; no graph
 * replay meanwhile) and keep the fastest; the choice is cached for the life
 * of the process by batch shape (SMs, precision, and per column the cells and
 * particle counts rounded to powers of two).  The schedule never changes
 * results.  Column i keys its
 * random numbers with column index i (params[i].column is overridden), so
 * column i of a batch evolves bit for bit like a lone handle created with
 * column = i.  All columns need equal dt, ion_subcycle, precision,
 * diag_every, sort_every and field_mode (PIC_EINVAL otherwise). */
int pic_init_batch(const pic_params *params, int n, pic_handle **out);
/* Advance every column of the batch n steps (pic_step on a batch handle does the same). */
int pic_step_batch(pic_handle *batch, int64_t n);
/* Column i of a batch (owned by the batch: use it for get_state, stats,
 * moments; it cannot be stepped or freed on its own).  NULL if out of range. */
pic_handle *pic_batch_column(pic_handle *batch, int i);
/* Number of columns of a batch; 0 for NULL or a single column. */
int pic_batch_size(pic_handle *batch);
/* The batch's CTA multipliers (electrons, ions; either pointer may be NULL):
 * returns 1 once tuning has finished (or came from the cache), 0 while the
 * next steps still tune (the values are those in use), PIC_EINVAL for a
 * handle that is not a batch. */
int pic_batch_schedule(pic_handle *batch, int *mult_e, int *mult_i);

/* Per-particle process code of the last step (needs PIC_FLAG_RECORD_CODES):
 * -1 no collision, -2 removed by the radial loss, else the xsec index.
 * Indexed by the slot the particle had during that step; n <= capacity. */
int pic_last_codes(pic_handle *h, int species, int32_t *out, int64_t n);

/* Derived scalars: [n_g, nu*_e, P_null_e, nu*_i, P_null_i, w, dx]. */
int pic_derived(pic_handle *h, double out[7]);

/* Kernel classes of pic_kernel_times. */
#define PIC_K_PUSH_E 0   /* electron step (gather, push, collisions, deposit) */
#define PIC_K_PUSH_I 1   /* ion step */
#define PIC_K_BIRTHS 2   /* births and removals */
#define PIC_K_FIELD 3    /* field solve */
#define PIC_K_SORT 4     /* counting sort by cell */
#define PIC_K_OTHER 5
#define PIC_K_CLASSES 8

/* Per-kernel timing.  With timing on, pic_step records a CUDA event pair on
 * the handle's stream around every kernel it launches.  pic_kernel_times
 * returns, per class, the summed event milliseconds and the launch count
 * since the last call (launches are counted with timing off too), then
 * resets both.  ms and launches are host arrays of PIC_K_CLASSES. */
int pic_set_timing(pic_handle *h, int enable);
int pic_kernel_times(pic_handle *h, double *ms, int64_t *launches);

/* The CUDA stream the handle launches on (a cudaStream_t). */
void *pic_stream(pic_handle *h);

/* Release a column or a batch: waits for its stream, frees its device memory, graphs, events
 * and stream.  NULL is ignored, and so is a column of a batch (freed with its batch). */
void pic_free(pic_handle *h);

/* Message of the last error on this handle; with NULL, of the last error this thread met outside
 * a handle (pic_init, pic_init_batch, the standalone field solve).  Valid until the next call. */
const char *pic_last_error(pic_handle *h);

/* Periodic Poisson solve of Sec. II on caller device memory: the field step
 * that pic_step runs every step (the paper solves a pair of tridiagonal
 * systems; here the algebraically identical exact route).  From fixed-point node charges
 * (2^32 per particle) it computes the half-node space-charge field
 *   E_{j+1/2} = C (N S'_j - M) / N^2,  S'_j = N sum_{k<=j} D_k - (j+1) T,
 *   D = Q_i - Q_e, T = sum D, M = sum S'   (zero-mean field, uniform
 *   background T/N removed; integers exact, one rounding to double)
 * and the node field E_j = (E_{j-1/2} + E_{j+1/2}) / 2 - E0.
 *   Q_i, Q_e  device int64[n_cells], 3 <= n_cells <= 65536
 *   C         e w / (eps0 2^32): field of one fixed-point unit (V/m)
 *   E0        |applied field| (V/m)
 *   E, E_half device double[n_cells], written
 *   stream    cudaStream_t to run on (NULL: the legacy default stream)
 * Allocates its scratch with cudaMalloc, frees it, and synchronises the
 * stream before returning.  Errors: PIC_EINVAL (bad size or NULL pointer),
 * PIC_ENOMEM, PIC_ECUDA, PIC_ENONFINITE (a field value is not finite). */
int pic_field_periodic(const int64_t *Q_i, const int64_t *Q_e, int n_cells, double C, double E0, double *E,
                       double *E_half, void *stream);

/* pic_field_periodic for callers that must not allocate device memory during
 * a call.  (The paper has no counterpart: this is a deployment variant.)
 * pic_field_periodic gets its scratch with cudaMalloc and returns it with
 * cudaFree, and cudaFree waits for the whole device to go idle, stalling the
 * caller's other streams; callers that manage device memory through their own
 * pool may not allocate behind it at all.  This variant takes the same
 * arguments and computes the same result (bit for bit), but keeps its scratch
 * in a fixed array built into the library: 525 KiB that every GPU which
 * loads the library holds until the process exits.  It calls no allocator.
 *   n_cells    3 <= n_cells <= 65536; larger sizes return PIC_EINVAL
 *   every call looks up the array's device address on the current device (no
 *   allocation); the first call on a device also loads the library's device
 *   code there: make it before any stream capture
 *   every call shares and overwrites the one array: calls that overlap on the
 *   GPU (other streams, other host threads on the same device) race; order them
 * Synchronises the stream before returning.  Errors are returned as codes only
 * (PIC_EINVAL, PIC_ECUDA, PIC_ENONFINITE); pic_last_error does not see them. */
int pic_field_periodic_noalloc(const int64_t *Q_i, const int64_t *Q_e, int n_cells, double C, double E0, double *E,
                               double *E_half, void *stream);

/* ------------------------------------------------------------------------
 * Learned closure network (the extension that closes the paper's three-moment
 * quasi-neutral fluid model, Sec. IV.A): an MLP 15 -> 128 -> 128 -> 3 with
 * GELU (tanh form) on the hidden layers, trained by mean-squared error with
 * Adam (beta 0.9, 0.999, eps 1e-8).  BF16 operands on the tensor cores with
 * FP32 accumulation; FP32 master weights; deterministic gradient sums.
 * Inputs: 15 features per sample (5-point stencil of density, mean energy and
 * field, normalised by the caller); outputs: 3 (electron flux, energy flux,
 * ionization rate, normalised).  Parameter layout (FP32, flat, 18947 values):
 * W1[128][15], b1[128], W2[128][128], b2[128], W3[3][128], b3[3].
 * Sample arrays are row-major (n x 15, n x 3) FP32 in caller-owned device memory, read (or,
 * for Y, written) on the given stream (NULL: the default stream); nothing is retained after a
 * call.  Errors are returned as codes only (pic_last_error does not see them): PIC_EINVAL for
 * a NULL handle or array, n <= 0, or a parameter count other than pic_mlp_nparam();
 * PIC_ENOMEM; PIC_ECUDA; PIC_ETIMEOUT when a bounded wait of the kernels gave up (the
 * kernels then return without writing; the error latches until pic_mlp_set_params, see
 * pic_mlp_test_hook). */
typedef struct pic_mlp pic_mlp;
int pic_mlp_nparam(void);
/* weights and biases uniform in +-1/sqrt(fan_in) from a seeded generator */
int pic_mlp_create(uint64_t seed, pic_mlp **out);
/* release the network's device memory (NULL is ignored) */
void pic_mlp_free(pic_mlp *m);
/* host arrays of pic_mlp_nparam() floats; set resets the Adam state */
int pic_mlp_set_params(pic_mlp *m, const float *host, int n);
int pic_mlp_get_params(pic_mlp *m, float *host, int n);
/* Y (device, n x 3) = network(X (device, n x 15)); synchronises the stream */
int pic_mlp_forward(pic_mlp *m, const float *X, int n, float *Y, void *stream);
/* gradient of the loss mean((Y - T)^2) over the n samples (host array of nparam, may be NULL)
 * and the loss; X, T device arrays (n x 15, n x 3); no update */
int pic_mlp_grad(pic_mlp *m, const float *X, const float *T, int n, float *grad_host, double *loss, void *stream);
/* `steps` Adam steps on consecutive batches of `batch` samples cycling through the n samples;
 * last_loss receives the loss of the last batch (before its update) */
int pic_mlp_train(pic_mlp *m, const float *X, const float *T, int n, int batch, int steps, float lr,
                  double *last_loss, void *stream);

/* Test instrumentation of the bounded waits (not part of the method; the paper has no
 * counterpart).  Every wait of the network's kernels on an mbarrier gives up after `spin` polls
 * (each suspends for at most 10 us); a wait that gives up makes the call return PIC_ETIMEOUT,
 * leaves the parameters, the Adam state and the outputs unwritten, and latches: every later
 * call on the handle returns PIC_ETIMEOUT until pic_mlp_set_params.  hook selects waits that
 * are made to give up, with nothing ever arriving on their barrier (no copy or MMA is issued for
 * them, so nothing is left in flight):
 *   PIC_MLP_HOOK_NO_WEIGHT_COPY   the training kernel's copy of the BF16 weights
 *   PIC_MLP_HOOK_NO_FORWARD_MMA   the first layer-1 MMA of one group of the forward kernel
 * spin = 0 restores the default limit (200000 polls); hook = 0 ends the instrumentation.
 * Synchronises the device.  PIC_EINVAL for a NULL handle, spin < 0 or unknown hook bits. */
#define PIC_MLP_HOOK_NO_WEIGHT_COPY 1u
#define PIC_MLP_HOOK_NO_FORWARD_MMA 2u
int pic_mlp_test_hook(pic_mlp *m, unsigned hook, int spin);

/* ------------------------------------------------------------------------
 * Electron transport of a uniform-field swarm from the two-term Boltzmann
 * equation (steady state, homogeneous): the closure the paper tabulates for
 * its fluid model (Sec. IV.A, eqs. 6-9, "solutions of the 0D Boltzmann
 * equation").  Isotropic scattering for every process (momentum transfer =
 * sum of all electron cross sections), elastic recoil loss 2m/M with the gas
 * at rest, excitation loss u_k, ionization leaving the scattered electron a
 * uniform share of eps - u_iz and no new electron (population held fixed, as
 * in the particle model's swarm mode).  Host code, FP64.
 * All rates are per gas density N (multiply by N, or divide for mobility and
 * diffusion, to get SI values at a given pressure). */
typedef struct pic_transport {
  double EN_Td;       /* reduced field, Td (1e-21 V m^2) */
  double mean_eps_eV; /* mean energy; Te = 2/3 of it */
  double muN;         /* mobility x N, 1/(V m s) */
  double DN;          /* diffusion x N, 1/(m s) */
  double mueN;        /* energy mobility x N */
  double DeN;         /* energy diffusion x N */
  double nu_izN;      /* ionization frequency / N, m^3/s */
  double lossN;       /* energy loss frequency / N (elastic + sum of thresholds x rates), eV m^3/s */
  double powerN;      /* power gained from the field / N = muN (E/N)^2, eV m^3/s */
  double alphaN;      /* ionization coefficient / N = nu_izN / drift, m^2 */
} pic_transport;
/* xs: the cross sections of pic_params (ion processes are ignored); EN_Td: n_EN
 * reduced fields (> 0); eps_max_eV: top of the energy grid (F must be
 * negligible there); n_grid: energy cells (64 .. 8192).  out: n_EN records.
 * Errors: PIC_EINVAL (bad argument), PIC_ENOMEM. */
int pic_two_term(const pic_xsec *xs, int n_xsec, double gas_mass_amu, const double *EN_Td, int n_EN,
                 double eps_max_eV, int n_grid, pic_transport *out);

/* ------------------------------------------------------------------------
 * Quasi-neutral three-moment fluid model of the column (Sec. IV.A, eqs. 3-5,
 * 8-12, 17) for many independent periodic columns at once: the fast screen
 * of discharge conditions.  State per cell: electron density n (= ion
 * density) and temperature Te, FP32 on the device.  Closure: mu_e, D_e,
 * mu_eps, D_eps, nu_i and L_eps as functions of Te from transport records
 * (pic_two_term), optionally corrected per cell by the closure network.
 *
 * One step (dt, faces j+1/2 between cells j and j+1, face values averages of
 * the two cells, coefficients at the step's starting Te):
 *  0. nu_i + dnu at every cell; nu_w fixed, or <n (nu_i + dnu)>/<n> with pair losses;
 *  1. continuity, backward Euler in the ambipolar diffusion and the losses:
 *       n'_j (1 + dt nu_w) - dt/dx^2 [a_{j+1/2}((nD_e)'_{j+1} - (nD_e)'_j) - a_{j-1/2}((nD_e)'_j - (nD_e)'_{j-1})]
 *         + dt/dx (dG_{j+1/2} - dG_{j-1/2}) = n_j + dt/dx (b_{j+1/2} - b_{j-1/2}) Gamma_T + dt n_j (nu_i + dnu),
 *     a = mu_i/(mu_e + mu_i), b = 1 - a (eq. 11);
 *  2. Gamma_{j+1/2} (eq. 11, plus dG) and E_{j+1/2} from n', with
 *     E = -d_x(n D_e)/(n mu_e) + Gamma_T/(n (mu_e + mu_i)) (eq. 10 combined with eq. 12,
 *     the derivation of eq. 17; mu_e face-averaged);
 *  3. energy, backward Euler in Te' for conduction, energy drift and the
 *     linearised loss, with H = -3/2 mu_eps E n Te - d_x(3/2 n D_eps Te) + dH
 *     (eqs. 8-9 with beta = 3/2 Te mu_eps, G = 3/2 Te D_eps) and the heating
 *     P_j = -(Gamma E)_{j+1/2, j-1/2} averaged (eq. 5);
 *  4. Te' clamped to the table's range.
 * g, h, dnu: closure corrections at cells (flux per electron, energy flux per
 * electron, ionization frequency).  The flux corrections are implicit, as
 * first-order upwind advection by the face velocities gf = (g_j + g_{j+1})/2
 * and wf = (w_j + w_{j+1})/2, w = h/Te (the step's starting Te):
 * dG_{j+1/2} = max(gf,0) n'_j + min(gf,0) n'_{j+1} in the continuity matrix
 * and in Gamma, dH_{j+1/2} = max(wf,0) n'_j Te'_j + min(wf,0) n'_{j+1} Te'_{j+1}
 * in the energy matrix: n' stays positive at any dt.
 * Each tridiagonal system is cyclic and is solved by parallel cyclic
 * reduction in shared memory (one thread block per column). */
typedef struct pic_fluid_column {
  double L_m;      /* column length */
  double N_gas_m3; /* gas density */
  double mu_iN;    /* ion mobility x N, 1/(V m s) */
  double Gamma_T;  /* total particle flux J/e (ions minus electrons), 1/(m^2 s); > 0 gives E along +x */
  double nu_w;     /* wall-loss frequency (eq. 2), 1/s; unused with PIC_FLUID_LOSS_PAIR */
  int32_t n_cells; /* a power of two, 64 .. 4096 */
  int32_t loss;    /* PIC_FLUID_LOSS_FIXED: nu_w as given; PIC_FLUID_LOSS_PAIR: nu_w = <n nu_i>/<n>
                      each step (the continuum form of the particle model's pair losses: as many
                      electrons leave as are created, uniformly per electron) */
} pic_fluid_column;
#define PIC_FLUID_LOSS_FIXED 0
#define PIC_FLUID_LOSS_PAIR 1
typedef struct pic_fluid pic_fluid;
/* tr: n_tr >= 2 transport records in increasing Te = 2/3 mean energy, resampled
 * (linear in Te) onto n_T (2 .. 256) uniform Te points; dt_s > 0; the spectral
 * record c_m = (1/N) sum_j n_j exp(-2 pi i m j/N), m = 1..n_modes (0 .. 64),
 * and the mean density are taken after every diag_every-th step (0: never).
 * Errors: PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA. */
int pic_fluid_init(const pic_fluid_column *cols, int n_cols, const pic_transport *tr, int n_tr, int n_T,
                   double dt_s, int diag_every, int n_modes, pic_fluid **out);
/* host arrays of the column's n_cells values, n > 0 and finite (PIC_EINVAL otherwise, and for
 * a NULL handle or array or col out of range).  The state is kept in FP64 between launches; a
 * launch holds it in shared memory as FP32 (hi, lo) pairs */
int pic_fluid_set_state(pic_fluid *f, int col, const double *n_m3, const double *Te_eV);
/* the column's FP64 state into host arrays of n_cells; PIC_EINVAL for a NULL handle or array
 * or col out of range */
int pic_fluid_get_state(pic_fluid *f, int col, double *n_m3, double *Te_eV);
/* advance every column by n_steps; synchronises the handle's stream */
int pic_fluid_step(pic_fluid *f, int64_t n_steps);
/* copy out and clear the spectral record: out holds max_snaps x n_cols x
 * (n_modes + 1) complex values (re, im as floats), entry 0 of each = (mean n, 0);
 * *n_snaps receives the number written (PIC_ECAPACITY if more were recorded) */
int pic_fluid_modes(pic_fluid *f, float *out, int max_snaps, int *n_snaps);
/* attach (net != NULL) or detach the closure network: every `period` steps the
 * features of every cell j (15: n/<n>, 3/2 Te in eV and E/N in Td, with E at
 * cells the mean of its faces, at cells j + d stencil, d = -2..2; each divided
 * by feat_scale[k]) go through the network, whose 3 outputs times targ_scale
 * become dG, dH, dnu for the next `period` steps (a zero scale switches a
 * correction off).  nu_bound > 0 limits the learned ionization correction to
 * |dnu| <= nu_bound nu_i(Te) of the cell (a trust region for states unlike
 * the training data); <= 0: unbounded.  stencil: spacing of the stencil points in
 * cells, 1 <= 4 stencil <= n_cells of every column.  The network is not owned. */
int pic_fluid_set_closure(pic_fluid *f, pic_mlp *net, int period, const float *feat_scale, const float *targ_scale,
                          float nu_bound, int stencil);
/* fixed corrections (device array, total cells x 3, already scaled to SI; NULL clears) */
int pic_fluid_set_corrections(pic_fluid *f, const float *corr_dev);
/* features of the current state (device array, total cells x 15, divided by feat_scale and
 * spaced by the stencil of the attached closure, or unscaled at spacing 1 without one); cells are
 * numbered column after column */
int pic_fluid_features(pic_fluid *f, float *X_dev);
/* device time of the last pic_fluid_step and the kernels it launched */
int pic_fluid_elapsed(pic_fluid *f, double *ms, int64_t *launches);
/* the CUDA stream the screen launches on (a cudaStream_t) */
void *pic_fluid_stream(pic_fluid *f);
/* release the screen's device memory and stream (NULL is ignored) */
void pic_fluid_free(pic_fluid *f);

/* The (R, I) drive (Sec. II, eq. 2; the paper imposes E0 and recovers R from eq. 2): the field E0
 * of a homogeneous column of radius R whose ionization balances ambipolar diffusion to the wall,
 * nu_iz(E0/N) = D_a (2.405/R)^2 with D_a = mu_i D_e/mu_e, and the density carrying the current
 * I: J = I/(pi R^2) = e n0 (mu_e + mu_i) E0.  Electron transport from pic_two_term on the
 * params' electron cross sections (energy grid up to eps_max_e_eV); ion mobility from the ion
 * cross sections in the low-field Chapman-Enskog first approximation,
 * mu_i = 3e/(16 N Omega) sqrt(2 pi/(mu_r k T_gas)), mu_r = M/2, Omega = 2 sigma_cx + sigma_iso at
 * the mean thermal relative energy 8 k T_gas/(pi e) (charge exchange reverses the relative
 * velocity).  out: E0 (V/m), n0 (1/m^3), Te0 = 2/3 of the mean energy (eV), mu_i N (1/(V m s)).
 * Host code.  Errors: PIC_EINVAL (bad arguments, no ion process, no root in 1..2000 Td). */
int pic_drive_ri(const pic_params *p, double out[4]);

/* Self-test hook: int128 -> double conversion used by the field solve, run
 * on the device: v_k = hi[k] 2^64 + lo[k]; out[k] = double nearest to v_k
 * (ties to even).  Host arrays of n. */
int pic_test_i128_to_double(const int64_t *hi, const uint64_t *lo, double *out, int n);

/* Version of this interface: changes whenever a declaration or a struct layout in this header
 * changes, so a binding can refuse a library built from another header. */
int pic_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif
