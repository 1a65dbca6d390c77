/* CPU oracle of the 1D3V electrostatic PIC-MCC positive-column step.
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code with the CUDA library: every
 * declaration below is written for the oracle alone.
 *
 * The oracle follows the paper's Sec. II step by step, in FP64 (or, when
 * built with ORACLE_F32, with FP32 particle offsets/velocities and FP32
 * push/collision arithmetic; the field stays FP64).  It is single-threaded
 * and deliberately plain: no blocking, no fusion, particles visited in slot
 * order.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_ELASTIC = 0, ORA_EXCITATION = 1, ORA_IONIZATION = 2, ORA_ION_CX = 3, ORA_ION_ISO = 4 };
enum { ORA_DRIVE_E0 = 0, ORA_DRIVE_V = 1, ORA_DRIVE_CIRCUIT = 2 };
enum { ORA_FIELD_POISSON = 0, ORA_FIELD_APPLIED = 1 };
enum { ORA_LOSS_PAIR = 0, ORA_LOSS_RADIAL = 1, ORA_LOSS_NONE = 2, ORA_LOSS_SWARM = 3 };
/* flags: ORA_FLAG_BOUNDED = the bounded column of Sec. V (absorbing electrodes at x = 0, the
   cathode, and x = L, the anode; Dirichlet field; electron emission at the cathode) */
enum { ORA_FLAG_BOUNDED = 8 };
enum { ORA_OK = 0, ORA_EINVAL = -1, ORA_ENOMEM = -2, ORA_ECAPACITY = -4, ORA_ENONFINITE = -5,
       ORA_EPARAM = -7 };

typedef struct ora_xsec {
  int32_t kind;
  int32_t n;
  double threshold_eV;
  const double *energy_eV;
  const double *sigma_m2;
} ora_xsec;

typedef struct ora_params {
  double gas_mass_amu, pressure_torr, T_gas_K;
  double L_m, R_m;
  int32_t drive, field_mode;
  double E0_Vpm, V_applied, I_A, U_src, R_ext_ohm_m2;
  int32_t n_xsec, pad0;
  const ora_xsec *xsec;
  int32_t n_cells, ion_subcycle;
  double dt_s;
  int64_t n_e0, n_i0, capacity;
  double n0_m3, Te0_eV, Ti0_eV;
  int32_t loss_mode, precision;
  double nu_w;
  uint64_t seed;
  int32_t diag_every, sort_every, n_table, flags;
  double eps_max_e_eV, eps_max_i_eV;
  int32_t column, pad1;
  double J_emit_Am2, T_emit_eV;   /* bounded column: cathode emission current density, emission temperature */
} ora_params;

typedef struct ora_state {
  int64_t n_e, n_i, step, next_id;
  double E0;
  int32_t *cell_e; double *off_e, *vx_e, *vy_e, *vz_e; uint64_t *id_e;
  int32_t *cell_i; double *off_i, *vx_i, *vy_i, *vz_i; uint64_t *id_i;
  double *E;        /* node field E^n, n_cells values */
  int64_t *Q_e;     /* electron node charge, fixed point (2^32 per particle) */
  int64_t *Q_i;     /* ion node charge, fixed point */
} ora_state;

typedef struct ora_stats {
  int64_t step, n_e, n_i, next_id;
  int64_t n_coll_e[16], n_coll_i[16];
  int64_t births, losses_e, losses_i;
  int64_t overflow_e, overflow_i;
  double E0;
  int64_t n_diag;
  int64_t absorbed_e[2], absorbed_i[2];   /* bounded column: particles taken by [cathode, anode] */
  int64_t emitted;                        /* electrons emitted by the cathode */
} ora_stats;

typedef struct ora_moments {
  int64_t n_samples, n_steps;
  double *n_e, *n_i, *gamma_e, *mean_eps_e, *heat_e, *iz_rate, *gamma_i, *E, *phi;
  int32_t reset, pad;
} ora_moments;

typedef struct ora_t ora_t;

int  ora_create(const ora_params *p, ora_t **out);
void ora_destroy(ora_t *h);
int  ora_step(ora_t *h, int64_t n);
int  ora_get_state(ora_t *h, ora_state *s);
int  ora_set_state(ora_t *h, const ora_state *s);
int  ora_stats_get(ora_t *h, ora_stats *s);
int  ora_moments_get(ora_t *h, ora_moments *m);
/* electron energy histogram (Sec. III.C, the EEPF F(x, eps)): on each diagnostic step every
   live electron adds 1 to bin (cell n_x / n_cells, eps n_eps / eps_max), energies at or above
   eps_max in column n_eps; n_x = 0 switches it off */
int  ora_eepf_config(ora_t *h, int n_x, int n_eps, double eps_max_eV);
int  ora_eepf_get(ora_t *h, uint64_t *counts, int64_t *n_samples, int reset);
/* per-particle process code of the last step (-1 none, else xsec index), length n */
int  ora_last_codes(ora_t *h, int species, int32_t *out, int64_t n);
/* derived scalars: [n_g, nu_star_e, P_null_e, nu_star_i, P_null_i, w, dx] */
int  ora_derived(ora_t *h, double *out7);
/* electron/ion collision-frequency table of process j (index among that species' processes) */
int  ora_nu_table(ora_t *h, int species, int j, double *out, int n);

/* building blocks exposed for the pins */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void ora_gauss_table(float *out4097);
double ora_gauss_sample(const float *table, double u);
double ora_i128_to_double(int64_t hi, uint64_t lo);
/* E at half-nodes from node charges by the exact integer route (Gauss's law,
 * zero-mean field, uniform background removed); C = e w / (eps0 2^32) */
void ora_field_exact(int n_cells, const int64_t *Q_i, const int64_t *Q_e, double C, double *E_half);
/* bounded column: space-charge field at the n_cells faces from the charges of nodes 1..n_cells-1
   (the electrode nodes 0 and n_cells carry surface charge), with phi equal at both electrodes */
void ora_field_exact_bounded(int n_cells, const int64_t *Q_i, const int64_t *Q_e, double C, double *E_half);
/* phi at nodes (phi_0 = 0) from node charge density rho (C/m^3) by Thomas on the
 * gauge-pinned tridiagonal system; returns 0 or ORA_EINVAL */
int ora_poisson_thomas(int n_cells, double dx, const double *rho, double *phi);

#ifdef __cplusplus
}
#endif
#endif
