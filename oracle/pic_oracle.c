/* CPU oracle of the 1D3V electrostatic PIC-MCC positive-column step
 * (Boeuf, "Ionization waves (striations) in a low-current plasma column
 * revisited with kinetic and fluid models", Sec. II).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared [-DORACLE_F32].  Contraction
 * is off so that every a*b+c below is two roundings, as written.
 *
 * What it computes, in the paper's order (Sec. II):
 *   1. field gather at the particle (linear interpolation of the node field),
 *   2. leapfrog push (Birdsall's standard scheme) and periodic re-injection,
 *   3. null-collision Monte Carlo collisions with the neutral gas:
 *      electrons elastic / excitation / ionization, ions charge exchange /
 *      isotropic elastic,
 *   4. ionization births and the paired random removal of one electron and
 *      one ion per ionization (particle number constant), or a radial loss
 *      frequency,
 *   5. charge assignment to the grid and the periodic Poisson solve,
 *      E = -E0 + E_sp.
 * Readings where the paper is silent are listed beside each function.
 *
 * Parity pins live in tests/ (closed forms and invariants); see each
 * function's comment for which one pins it.  In brief:
 *   Philox, Gaussian table     known-answer vectors, quantiles, moments, KS
 *   push, subcycling           exact constant-field quadratics (electrons and
 *                              subcycled ions), the leapfrog plasma frequency
 *   deposit, field             Gauss's law, sinusoidal and uniform charge closed
 *                              forms, the paper's Thomas route (periodic and
 *                              Dirichlet), charge = N 2^32 exactly
 *   collisions                 counts against n_g sigma v, the majorant, the
 *                              table's end values with overflow counts,
 *                              elastic / inelastic / ionization kinematics,
 *                              charge exchange, centre-of-mass isotropic
 *                              scattering, the Maxwell-model swarm
 *   births, losses             pair counts and uniform victims, radial
 *                              binomials (electrons, subcycled ions),
 *                              compaction order, cathode emission
 *                              (half-Maxwellian, Child-Langmuir)
 *   moments, EEPF              column integrals, Poisson for the sampled
 *                              potential, mono-energetic and Maxwellian EEPFs
 *   the whole step             determinism, checkpoint/resume, the discharge
 *                              similarity laws bit for bit
 * Every function here has a pin.  What long runs produce (striation
 * wavelength and phase velocity under the synthetic cross sections) has no
 * value to compare against: parity unpinned there, compared statistically.
 */
#include "pic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORACLE_F32
typedef float real;
#define R_SQRT sqrtf
#define R_FLOOR floorf
#else
typedef double real;
#define R_SQRT sqrt
#define R_FLOOR floor
#endif

/* CODATA 2018 */
#define QE 1.602176634e-19
#define ME 9.1093837015e-31
#define AMU 1.66053906660e-27
#define KB 1.380649e-23
#define EPS0 8.8541878128e-12
#define TORR 133.32236842105263

#define TWO32 4294967296.0
#define NGAUSS 4096
#define MAXPROC 16

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its published
 * definition: ten rounds of two 32x32->64 multiplies with the S-box-free
 * permutation, Weyl-sequence key schedule.  Pinned by the known-answer
 * vectors of the Random123 distribution and, structurally, by the 64-bit
 * variant against numpy's Philox4x64-10 (tests/test_oracle_rng.py). */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    if (r < 9) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout: (id_lo, id_hi, step, stream<<28 | column<<16 | block). */
enum { ST_E = 0, ST_I = 1, ST_INIT_E = 2, ST_INIT_I = 3, ST_VIC_E = 4, ST_VIC_I = 5, ST_EMIT = 6 };

static void rng_block(uint64_t seed, uint64_t id, uint32_t step, uint32_t stream, uint32_t column,
                      uint32_t block, uint32_t w[4]) {
  uint32_t c[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, (stream << 28) | (column << 16) | block};
  uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  ora_philox4x32_10(c, k, w);
}

/* Uniforms: a 32-bit word w gives (w>>8) 2^-24 in FP32 storage mode; two words
 * (a, b) give ((a>>5) 2^26 + (b>>6)) 2^-53 in FP64 mode.  Both lie in [0,1). */
static inline float u_f32(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }
static inline double u_f64(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}
/* the 32-bit decision uniform of block 0 */
static real u_dec(uint32_t w) {
#ifdef ORACLE_F32
  return u_f32(w);
#else
  return (double)w * (1.0 / 4294967296.0);
#endif
}

/* On-demand uniform stream of one particle in one step: blocks 1, 2, ... */
typedef struct ustream {
  uint64_t seed, id; uint32_t step, stream, column, block;
  uint32_t w[4]; int pos;
} ustream;

static void us_init(ustream *s, uint64_t seed, uint64_t id, uint32_t step, uint32_t stream, uint32_t column) {
  s->seed = seed; s->id = id; s->step = step; s->stream = stream; s->column = column;
  s->block = 0; s->pos = 4;
}
static real us_next(ustream *s) {
#ifdef ORACLE_F32
  if (s->pos >= 4) { s->block++; rng_block(s->seed, s->id, s->step, s->stream, s->column, s->block, s->w); s->pos = 0; }
  return u_f32(s->w[s->pos++]);
#else
  if (s->pos >= 4) { s->block++; rng_block(s->seed, s->id, s->step, s->stream, s->column, s->block, s->w); s->pos = 0; }
  double u = u_f64(s->w[s->pos], s->w[s->pos + 1]);
  s->pos += 2;
  return u;
#endif
}

/* ------------------------------------------------------------------ */
/* Gaussian inverse-CDF table (reading: neutral and Maxwellian
 * velocities are sampled by table so that the step holds no
 * transcendental).  T[k] = Phi^-1(k/4096) for 1 <= k <= 4095, rounded to
 * FP32; the end entries are set so that the linear piece over the first
 * (last) interval has the exact conditional mean of the normal tail,
 * T[0] = 2 m0 - Phi^-1(1/4096), m0 = -4096 phi(Phi^-1(1/4096)).
 * Phi^-1 here is plain bisection on Phi(x) = erfc(-x/sqrt2)/2.
 * Pinned by the T9 tests (moments, KS against Phi, table values). */
static double phi_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }
static double inv_phi_bisect(double p) {
  double lo = -40.0, hi = 40.0;
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (phi_cdf(mid) < p) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}
void ora_gauss_table(float *T) {
  for (int k = 1; k <= NGAUSS / 2; ++k) {
    double z = inv_phi_bisect((double)k / NGAUSS);
    T[k] = (float)z;
    T[NGAUSS - k] = (float)(-z);
  }
  double z1 = inv_phi_bisect(1.0 / NGAUSS);
  double m0 = -(double)NGAUSS * exp(-0.5 * z1 * z1) / sqrt(2.0 * M_PI);
  T[0] = (float)(2.0 * m0 - z1);
  T[NGAUSS] = -T[0];
  T[NGAUSS / 2] = 0.0f;
}
static real gauss_sample(const float *T, real u) {
  real x = u * (real)NGAUSS;
  int i = (int)x;
  real fr = x - (real)i;
  real a = (real)T[i], b = (real)T[i + 1];
  return a + fr * (b - a);
}
double ora_gauss_sample(const float *T, double u) { return (double)gauss_sample(T, (real)u); }

/* Marsaglia (1972): isotropic unit vector from two uniforms on the unit disc. */
static void iso_dir(ustream *s, real *nx, real *ny, real *nz) {
  real a = 0, b = 0, q = 0;
  int ok = 0;
  for (int t = 0; t < 64; ++t) {
    a = (real)2 * us_next(s) - (real)1;
    b = (real)2 * us_next(s) - (real)1;
    q = a * a + b * b;
    if (q < (real)1) { ok = 1; break; }
  }
  if (!ok) { a = 0; b = 0; q = 0; }
  real t2 = (real)2 * R_SQRT((real)1 - q);
  *nx = a * t2; *ny = b * t2; *nz = (real)1 - (real)2 * q;
}

/* ------------------------------------------------------------------ */
/* int128 -> double, round to nearest even (libgcc's conversion). */
double ora_i128_to_double(int64_t hi, uint64_t lo) {
  __int128 v = ((__int128)hi << 64) | (__int128)lo;
  return (double)v;
}

/* Periodic Poisson by the exact integer route.  Gauss's law on the grid,
 * E_{j+1/2} - E_{j-1/2} = dx rho_j / eps0 (Sec. II: E_sp from Poisson's
 * equation; periodic potential => zero-mean E_sp).  With D_j = Q_i,j - Q_e,j
 * and the uniform background T/N removed (T = sum D):
 *   S'_j = N sum_{k<=j} D_k - (j+1) T,  M = sum_j S'_j,
 *   E_{j+1/2} = C (N S'_j - M) / N^2.
 * The integer numerator is exact; one rounding to double, one multiply.
 * Pinned against the Thomas solve and the discrete sinusoid closed form. */
void ora_field_exact(int N, const int64_t *Qi, const int64_t *Qe, double C, double *Eh) {
  __int128 T = 0;
  for (int j = 0; j < N; ++j) T += (__int128)(Qi[j] - Qe[j]);
  __int128 *Sp = (__int128 *)malloc(sizeof(__int128) * (size_t)N);
  __int128 run = 0, M = 0;
  for (int j = 0; j < N; ++j) {
    run += (__int128)(Qi[j] - Qe[j]);
    Sp[j] = (__int128)N * run - (__int128)(j + 1) * T;
    M += Sp[j];
  }
  double Cf = C / ((double)N * (double)N);
  for (int j = 0; j < N; ++j) {
    __int128 num = (__int128)N * Sp[j] - M;
    Eh[j] = (double)num * Cf;
  }
  free(Sp);
}

/* Bounded column (Sec. V): Gauss's law between the electrodes,
 * E_{j+1/2} - E_{j-1/2} = dx rho_j / eps0 for the interior nodes j = 1..N-1 (the
 * electrode nodes 0 and N hold surface charge), with the potential equal at both
 * electrodes (the applied voltage is added by the caller as -V/L).  With
 * P_j = sum_{k=1..j} D_k (P_0 = 0) and U = sum_{j<N} P_j:
 *   E_{j+1/2} = C (N P_j - U) / N  (zero mean over the N faces),
 * written as the periodic route's C (N S'_j - M) / N^2 with S'_j = N P_j, M = N U:
 * no uniform background, D_0 = 0. */
void ora_field_exact_bounded(int N, const int64_t *Qi, const int64_t *Qe, double C, double *Eh) {
  __int128 *Sp = (__int128 *)malloc(sizeof(__int128) * (size_t)N);
  __int128 run = 0, M = 0;
  for (int j = 0; j < N; ++j) {
    if (j > 0) run += (__int128)(Qi[j] - Qe[j]);
    Sp[j] = (__int128)N * run;
    M += Sp[j];
  }
  double Cf = C / ((double)N * (double)N);
  for (int j = 0; j < N; ++j) {
    __int128 num = (__int128)N * Sp[j] - M;
    Eh[j] = (double)num * Cf;
  }
  free(Sp);
}

/* The paper's route (Sec. II, Thomas algorithm): -phi_{j-1} + 2 phi_j - phi_{j+1}
 * = dx^2 rho_j / eps0 for j = 1..N-1 with the gauge phi_0 = 0 (periodic wrap
 * phi_N = phi_0); the j = 0 row is implied by neutrality (sum rho = 0). */
int ora_poisson_thomas(int N, double dx, const double *rho, double *phi) {
  if (N < 3) return ORA_EINVAL;
  int n = N - 1;
  double *cp = (double *)malloc(sizeof(double) * (size_t)n);
  double *dp = (double *)malloc(sizeof(double) * (size_t)n);
  for (int i = 0; i < n; ++i) {
    double a = (i > 0) ? -1.0 : 0.0, b = 2.0, c = (i < n - 1) ? -1.0 : 0.0;
    double d = dx * dx * rho[i + 1] / EPS0;
    if (i == 0) { cp[i] = c / b; dp[i] = d / b; }
    else {
      double m = b - a * cp[i - 1];
      cp[i] = c / m;
      dp[i] = (d - a * dp[i - 1]) / m;
    }
  }
  phi[0] = 0.0;
  phi[n] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) phi[i + 1] = dp[i] - cp[i] * phi[i + 2];
  free(cp); free(dp);
  return ORA_OK;
}

/* ------------------------------------------------------------------ */
typedef struct species {
  int64_t n, cap;
  int32_t *cell; real *off, *vx, *vy, *vz; uint64_t *id;
  int32_t *code;
  int64_t *Q;           /* node charge, fixed point */
} species;

typedef struct birth {
  int64_t parent; int32_t cell; real off;
  real ve[3], vi[3];
} birth;

struct ora_t {
  ora_params p;
  int N;
  /* derived (Sec. II) */
  double ng, dx, w, M, C_field, E0, Cj;
  double dt_i;
  real a_e, d_e, a_i, d_i, K_e, K_i, V_e, em, sig_n, sig_e0, sig_i0;
  real inv_de_e, inv_de_i;
  real P_e, P_i, nus_e, nus_i;
  uint32_t Pw_e, Pw_i;
  int ntab;
  int np_e, np_i;
  int kind_e[MAXPROC], kind_i[MAXPROC], xs_e[MAXPROC], xs_i[MAXPROC];
  real thr_e[MAXPROC];
  double *tab_e[MAXPROC], *tab_i[MAXPROC];   /* nu_k(eps_i), FP64 */
  real *rt_e[MAXPROC], *rt_i[MAXPROC];       /* tables in the storage precision */
  real *nub_e, *Pb_e;                        /* electrons: per-bin majorant and its null-collision probability */
  double nustar_e, nustar_i, Pnull_e, Pnull_i;
  float gauss[NGAUSS + 1];
  species e, i;
  double *E;      /* node field */
  double *Eh;     /* half-node space-charge field */
  real *Ef;       /* gather copy, N+1 */
  int64_t step, next_id;
  int64_t sumv[2];          /* circuit drive: sum of round(256 vx) over electrons (this step) and ions (last push) */
  birth *births; int64_t nb, bcap;
  int64_t *dead_e, *dead_i; int64_t nde, ndi;
  ora_stats st;
  /* moments window */
  double *m_ne, *m_ni, *m_ge, *m_ee, *m_he, *m_gi, *m_E, *m_phi;
  int64_t *m_iz;
  int64_t m_samples, m_steps;
  /* electron energy histogram: eepf_nx x (eepf_ne + 1) counts */
  uint64_t *eepf; int eepf_nx, eepf_ne; real eepf_scale; int64_t eepf_samples;
  /* bounded column (Sec. V) */
  int bounded, Nw;          /* Nw: nodes of the charge arrays = N (periodic, node N is node 0) or N + 1 */
  double emit_per_step, emit_acc;
  real sig_emit, emit_dtdx;
  int err;
};

static int is_electron_kind(int k) { return k == ORA_ELASTIC || k == ORA_EXCITATION || k == ORA_IONIZATION; }

/* cross section at eps by linear interpolation of the user's table; zero
 * below a process threshold; end values held outside the table. */
static double xs_eval(const ora_xsec *x, double eps) {
  if ((x->kind == ORA_EXCITATION || x->kind == ORA_IONIZATION) && eps < x->threshold_eV) return 0.0;
  const double *E = x->energy_eV, *S = x->sigma_m2;
  int n = x->n;
  if (eps <= E[0]) return S[0];
  if (eps >= E[n - 1]) return S[n - 1];
  int a = 0;
  while (a + 1 < n && E[a + 1] <= eps) ++a;
  double t = (eps - E[a]) / (E[a + 1] - E[a]);
  return S[a] + t * (S[a + 1] - S[a]);
}

/* nu_k(eps_i) = n_g sigma_k(eps_i) v(eps_i) on eps_i = i deps, deps = eps_max/(n-1);
 * v(eps) = sqrt(eps * 2e/m).  nu* = max_i sum_k nu_k(eps_i). */
static double build_table(const ora_xsec *x, double ng, double eps_max, int n, double Vq, double *out) {
  double de = eps_max / (double)(n - 1);
  for (int i = 0; i < n; ++i) {
    double eps = (double)i * de;
    double v = sqrt(eps * Vq);
    out[i] = ng * xs_eval(x, eps) * v;
  }
  return de;
}

/* cloud-in-cell charge of one particle; Nw = nodes (a periodic column wraps node N to 0) */
static void deposit(int64_t *Q, int Nw, int32_t cell, real off, int sign) {
  uint64_t k = (uint64_t)(off * (real)TWO32);
  int64_t a = (int64_t)(((uint64_t)1 << 32) - k), b = (int64_t)k;
  int c1 = (cell + 1 == Nw) ? 0 : cell + 1;
  Q[cell] += sign * a;
  Q[c1] += sign * b;
}

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

static int species_alloc(species *s, int64_t cap, int N) {
  s->cap = cap; s->n = 0;
  s->cell = (int32_t *)xcalloc((size_t)cap, sizeof(int32_t));
  s->off = (real *)xcalloc((size_t)cap, sizeof(real));
  s->vx = (real *)xcalloc((size_t)cap, sizeof(real));
  s->vy = (real *)xcalloc((size_t)cap, sizeof(real));
  s->vz = (real *)xcalloc((size_t)cap, sizeof(real));
  s->id = (uint64_t *)xcalloc((size_t)cap, sizeof(uint64_t));
  s->code = (int32_t *)xcalloc((size_t)cap, sizeof(int32_t));
  s->Q = (int64_t *)xcalloc((size_t)N, sizeof(int64_t));
  return (s->cell && s->off && s->vx && s->vy && s->vz && s->id && s->code && s->Q) ? 0 : -1;
}
static void species_free(species *s) {
  free(s->cell); free(s->off); free(s->vx); free(s->vy); free(s->vz); free(s->id); free(s->code); free(s->Q);
}

static void copy_particle(species *s, int64_t dst, int64_t src) {
  s->cell[dst] = s->cell[src]; s->off[dst] = s->off[src];
  s->vx[dst] = s->vx[src]; s->vy[dst] = s->vy[src]; s->vz[dst] = s->vz[src]; s->id[dst] = s->id[src];
}

/* Field: E_j = (E_{j-1/2} + E_{j+1/2})/2 - E0 (Sec. II, E = -E0 + E_sp). */
static void solve_field(ora_t *h) {
  int N = h->N;
  if (h->p.field_mode == ORA_FIELD_APPLIED) {
    for (int j = 0; j < h->Nw; ++j) { h->Eh[j < N ? j : N - 1] = 0.0; h->E[j] = -h->E0; }
  } else if (h->bounded) {
    /* Sec. V: E_0 = E_{1/2}, E_N = E_{N-1/2} at the electrodes; the applied -E0 = -V_D / L */
    ora_field_exact_bounded(N, h->i.Q, h->e.Q, h->C_field, h->Eh);
    double Eapp = -h->E0;
    h->E[0] = h->Eh[0] + Eapp;
    for (int j = 1; j < N; ++j) h->E[j] = 0.5 * (h->Eh[j - 1] + h->Eh[j]) + Eapp;
    h->E[N] = h->Eh[N - 1] + Eapp;
    for (int j = 0; j <= N; ++j)
      if (!isfinite(h->E[j])) h->err = ORA_ENONFINITE;
  } else {
    ora_field_exact(N, h->i.Q, h->e.Q, h->C_field, h->Eh);
    double Eapp = -h->E0;
    for (int j = 0; j < N; ++j) {
      double left = h->Eh[(j == 0) ? N - 1 : j - 1];
      h->E[j] = 0.5 * (left + h->Eh[j]) + Eapp;
      if (!isfinite(h->E[j])) h->err = ORA_ENONFINITE;
    }
  }
  for (int j = 0; j < N; ++j) h->Ef[j] = (real)h->E[j];
  h->Ef[N] = h->bounded ? (real)h->E[N] : h->Ef[0];
}

static real gather(const ora_t *h, int32_t cell, real off) {
  real a = h->Ef[cell], b = h->Ef[cell + 1];
  return a + off * (b - a);
}

/* leapfrog kick + drift with periodic re-injection (Sec. II: particles leaving
 * one end re-enter at the other with the same velocity).  Bounded column
 * (Sec. V): a particle leaving [0, L) is taken by the electrode it crossed;
 * returns -1 (cathode, x < 0) or +1 (anode, x >= L), else 0. */
static int push(const ora_t *h, real a, real d, real E, int32_t *cell, real *off, real *vx) {
  *vx = *vx + a * E;
  real f = *off + *vx * d;
  real c = R_FLOOR(f);
  f = f - c;
  int32_t cl = *cell + (int32_t)c;
  if (f >= (real)1) { f = (real)0; cl += 1; }
  if (h->bounded) {
    if (cl < 0) { *cell = 0; *off = 0; return -1; }
    if (cl >= h->N) { *cell = h->N - 1; *off = 0; return 1; }
    *cell = cl; *off = f;
    return 0;
  }
  cl %= h->N;
  if (cl < 0) cl += h->N;
  *cell = cl; *off = f;
  return 0;
}

/* table position of eps: i, fraction fr; above the table the last value is held */
static int tab_pos(real eps, real inv_de, int ntab, real *fr, int *ovf) {
  real x = eps * inv_de;
  if (!(x < (real)(ntab - 1))) { *fr = (real)1; *ovf = 1; return ntab - 2; }  /* also NaN */
  int i = (int)x;
  *fr = x - (real)i;
  *ovf = 0;
  return i;
}

static void moments_alloc(ora_t *h) {
  size_t N = (size_t)h->N + 1;
  h->m_ne = (double *)xcalloc(N, 8); h->m_ni = (double *)xcalloc(N, 8);
  h->m_ge = (double *)xcalloc(N, 8); h->m_ee = (double *)xcalloc(N, 8);
  h->m_he = (double *)xcalloc(N, 8); h->m_gi = (double *)xcalloc(N, 8);
  h->m_E = (double *)xcalloc(N, 8); h->m_phi = (double *)xcalloc(N, 8);
  h->m_iz = (int64_t *)xcalloc(N, 8);
}
static void moments_reset(ora_t *h) {
  size_t b = (size_t)(h->N + 1) * 8;
  memset(h->m_ne, 0, b); memset(h->m_ni, 0, b); memset(h->m_ge, 0, b); memset(h->m_ee, 0, b);
  memset(h->m_he, 0, b); memset(h->m_gi, 0, b); memset(h->m_E, 0, b); memset(h->m_phi, 0, b);
  memset(h->m_iz, 0, b);
  h->m_samples = 0; h->m_steps = 0;
}
static void moments_free(ora_t *h) {
  free(h->m_ne); free(h->m_ni); free(h->m_ge); free(h->m_ee); free(h->m_he); free(h->m_gi);
  free(h->m_E); free(h->m_phi); free(h->m_iz);
}
static void moment_add(double *acc, int N, int32_t cell, real off, double val) {
  uint64_t k = (uint64_t)(off * (real)TWO32);
  double w1 = (double)k * (1.0 / TWO32), w0 = 1.0 - w1;
  int c1 = (cell + 1 == N) ? 0 : cell + 1;
  acc[cell] += w0 * val;
  acc[c1] += w1 * val;
}

/* ------------------------------------------------------------------ */
static int stage_birth(ora_t *h, const birth *b) {
  if (h->nb >= h->bcap) {
    int64_t nc = h->bcap ? 2 * h->bcap : 1024;
    birth *nbf = (birth *)realloc(h->births, sizeof(birth) * (size_t)nc);
    if (!nbf) return ORA_ENOMEM;
    h->births = nbf; h->bcap = nc;
  }
  h->births[h->nb++] = *b;
  return 0;
}

/* Electron step of one particle (Sec. II): gather, kick, drift, wrap, then
 * the null-collision test against nu* and the process choice by the
 * cumulative collision frequencies at eps (elastic, excitation levels,
 * ionization in the order given).  Scattering is isotropic for every process
 * (reading); the elastic energy loss is eps (2m/M)(1 - cos chi); ionization
 * shares eps - eps_iz by a uniform fraction (reading of "as in Refs. [34,40]"). */
static void electron_step(ora_t *h, int64_t p, int diag) {
  species *s = &h->e;
  int32_t cell = s->cell[p]; real off = s->off[p];
  real vx = s->vx[p], vy = s->vy[p], vz = s->vz[p];
  uint64_t id = s->id[p];
  uint32_t stp = (uint32_t)h->step, col = (uint32_t)h->p.column;
  real Ep = gather(h, cell, off);
  int side = push(h, h->a_e, h->d_e, Ep, &cell, &off, &vx);
  uint32_t w[4];
  rng_block(h->p.seed, id, stp, ST_E, col, 0, w);
  ustream us; us_init(&us, h->p.seed, id, stp, ST_E, col);
  int32_t code = -1;
  int dead = 0;
  if (side) { dead = 1; h->st.absorbed_e[side > 0] += 1; }
  else if (h->p.loss_mode == ORA_LOSS_RADIAL && w[2] < h->Pw_e) dead = 1;
  if (!dead) {
    real u0 = u_dec(w[0]), u1 = u_dec(w[1]);
    real eps = h->K_e * (vx * vx + vy * vy + vz * vz);
    real fr; int ovf;
    int it = tab_pos(eps, h->inv_de_e, h->ntab, &fr, &ovf);
    if (u0 < h->Pb_e[it]) {
      if (ovf) h->st.overflow_e++;
      real r = u1 * h->nub_e[it], cum = 0;
      int sel = -1;
      for (int k = 0; k < h->np_e; ++k) {
        real nu;
        if (h->kind_e[k] != ORA_ELASTIC && eps < h->thr_e[k]) nu = 0;
        else { real a = h->rt_e[k][it], b = h->rt_e[k][it + 1]; nu = a + fr * (b - a); }
        cum = cum + nu;
        if (r < cum) { sel = k; break; }
      }
      if (sel >= 0) {
        int kind = h->kind_e[sel];
        code = h->xs_e[sel];
        h->st.n_coll_e[sel]++;
        real nx, ny, nz;
        if (kind == ORA_ELASTIC) {
          iso_dir(&us, &nx, &ny, &nz);
          real vm = R_SQRT(vx * vx + vy * vy + vz * vz);
          real cosx = (vm > (real)0) ? (nx * vx + ny * vy + nz * vz) / vm : (real)0;
          real e2 = eps * ((real)1 - h->em * ((real)1 - cosx));
          real sp = R_SQRT(e2 * h->V_e);
          vx = sp * nx; vy = sp * ny; vz = sp * nz;
        } else if (kind == ORA_EXCITATION) {
          real e2 = eps - h->thr_e[sel];
          iso_dir(&us, &nx, &ny, &nz);
          real sp = R_SQRT(e2 * h->V_e);
          vx = sp * nx; vy = sp * ny; vz = sp * nz;
        } else {
          real er = eps - h->thr_e[sel];
          real us_ = us_next(&us);
          real e_ej = us_ * er;
          real e_sc = er - e_ej;
          iso_dir(&us, &nx, &ny, &nz);
          real sp = R_SQRT(e_sc * h->V_e);
          vx = sp * nx; vy = sp * ny; vz = sp * nz;
          real mx, my, mz;
          iso_dir(&us, &mx, &my, &mz);
          real sq = R_SQRT(e_ej * h->V_e);
          birth b;
          b.parent = p; b.cell = cell; b.off = off;
          b.ve[0] = sq * mx; b.ve[1] = sq * my; b.ve[2] = sq * mz;
          real g0 = gauss_sample(h->gauss, us_next(&us));
          real g1 = gauss_sample(h->gauss, us_next(&us));
          real g2 = gauss_sample(h->gauss, us_next(&us));
          b.vi[0] = h->sig_n * g0; b.vi[1] = h->sig_n * g1; b.vi[2] = h->sig_n * g2;
          if (h->p.loss_mode != ORA_LOSS_SWARM) {
            if (stage_birth(h, &b)) h->err = ORA_ENOMEM;
          } else {
            h->st.births++;
          }
          if (h->m_iz) {
            uint64_t kk = (uint64_t)(off * (real)TWO32);
            int c1 = (cell + 1 == h->Nw) ? 0 : cell + 1;
            h->m_iz[cell] += (int64_t)(((uint64_t)1 << 32) - kk);
            h->m_iz[c1] += (int64_t)kk;
          }
        }
      }
    }
  } else {
    code = -2;
  }
  s->cell[p] = cell; s->off[p] = off; s->vx[p] = vx; s->vy[p] = vy; s->vz[p] = vz;
  s->code[p] = code;
  if (dead) { h->dead_e[h->nde++] = p; return; }
  deposit(s->Q, h->Nw, cell, off, +1);
  if (h->p.drive == ORA_DRIVE_CIRCUIT) h->sumv[0] += (int64_t)llrint((double)(vx * (real)256));
  if (diag) {
    real er = h->K_e * (vx * vx + vy * vy + vz * vz);
    double eps = (double)er;
    if (h->eepf) {   /* Sec. III.C: the electron's energy bin at its cell, after push and collision */
      real x = er * h->eepf_scale;
      int b = x < (real)h->eepf_ne ? (int)x : h->eepf_ne;
      int bx = (int)(((int64_t)cell * h->eepf_nx) / h->N);
      h->eepf[(size_t)bx * (size_t)(h->eepf_ne + 1) + (size_t)b] += 1;
    }
    moment_add(h->m_ge, h->Nw, cell, off, (double)vx);
    moment_add(h->m_ee, h->Nw, cell, off, eps);
    moment_add(h->m_he, h->Nw, cell, off, eps * (double)vx);
  }
}

/* Ion step of one particle on an ion push step (dt_i = subcycle dt): gather,
 * kick, drift, wrap; null collision against nu*_i with the relative speed g
 * to a neutral drawn from the gas Maxwellian; charge exchange gives the ion
 * the neutral's velocity; isotropic elastic scatters g in the centre-of-mass
 * frame (equal masses). */
static void ion_step(ora_t *h, int64_t p, int diag) {
  species *s = &h->i;
  int32_t cell = s->cell[p]; real off = s->off[p];
  real vx = s->vx[p], vy = s->vy[p], vz = s->vz[p];
  uint64_t id = s->id[p];
  uint32_t stp = (uint32_t)h->step, col = (uint32_t)h->p.column;
  real Ep = gather(h, cell, off);
  int side = push(h, h->a_i, h->d_i, Ep, &cell, &off, &vx);
  uint32_t w[4];
  rng_block(h->p.seed, id, stp, ST_I, col, 0, w);
  ustream us; us_init(&us, h->p.seed, id, stp, ST_I, col);
  int32_t code = -1;
  int dead = 0;
  if (side) { dead = 1; h->st.absorbed_i[side > 0] += 1; }
  else if (h->p.loss_mode == ORA_LOSS_RADIAL && w[2] < h->Pw_i) dead = 1;
  if (!dead) {
    real u0 = u_dec(w[0]), u1 = u_dec(w[1]);
    if (u0 < h->P_i) {
      real g0 = gauss_sample(h->gauss, us_next(&us));
      real g1 = gauss_sample(h->gauss, us_next(&us));
      real g2 = gauss_sample(h->gauss, us_next(&us));
      real nvx = h->sig_n * g0, nvy = h->sig_n * g1, nvz = h->sig_n * g2;
      real gx = vx - nvx, gy = vy - nvy, gz = vz - nvz;
      real eg = h->K_i * (gx * gx + gy * gy + gz * gz);
      real fr; int ovf;
      int it = tab_pos(eg, h->inv_de_i, h->ntab, &fr, &ovf);
      if (ovf) h->st.overflow_i++;
      real r = u1 * h->nus_i, cum = 0;
      int sel = -1;
      for (int k = 0; k < h->np_i; ++k) {
        real a = h->rt_i[k][it], b = h->rt_i[k][it + 1];
        cum = cum + (a + fr * (b - a));
        if (r < cum) { sel = k; break; }
      }
      if (sel >= 0) {
        code = h->xs_i[sel];
        h->st.n_coll_i[sel]++;
        if (h->kind_i[sel] == ORA_ION_CX) {
          vx = nvx; vy = nvy; vz = nvz;
        } else {
          real nx, ny, nz;
          iso_dir(&us, &nx, &ny, &nz);
          real gm = R_SQRT(gx * gx + gy * gy + gz * gz);
          real hg = (real)0.5 * gm;
          vx = (real)0.5 * (vx + nvx) + hg * nx;
          vy = (real)0.5 * (vy + nvy) + hg * ny;
          vz = (real)0.5 * (vz + nvz) + hg * nz;
        }
      }
    }
  } else {
    code = -2;
  }
  s->cell[p] = cell; s->off[p] = off; s->vx[p] = vx; s->vy[p] = vy; s->vz[p] = vz;
  s->code[p] = code;
  if (dead) { h->dead_i[h->ndi++] = p; return; }
  deposit(s->Q, h->Nw, cell, off, +1);
  if (h->p.drive == ORA_DRIVE_CIRCUIT) h->sumv[1] += (int64_t)llrint((double)(vx * (real)256));
  if (diag) moment_add(h->m_gi, h->Nw, cell, off, (double)vx);
}

/* uniform slot in [0, n) from a 64-bit word: floor(r n / 2^64) */
static int64_t slot_draw(uint64_t seed, int64_t k, uint32_t attempt, uint32_t step, uint32_t stream,
                         uint32_t col, int64_t n) {
  uint32_t c[4] = {(uint32_t)k, attempt, step, (stream << 28) | (col << 16)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  ora_philox4x32_10(c, key, w);
  uint64_t r = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
  return (int64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)n) >> 64);
}

/* Paired random removal (Sec. II: each ionization is balanced by removing one
 * electron and one ion, each picked at random anywhere in the column,
 * independently of each other).
 * Reading: victims are uniform over the pre-step slots, drawn without
 * replacement in rounds: every unsettled event k holds a candidate drawn
 * with its attempt counter; in one round an event settles iff no settled
 * event holds its candidate and no lower unsettled event has the same
 * candidate; the others redraw with attempt + 1. */
static int draw_victims(ora_t *h, int64_t nb, int64_t npre, uint32_t stream, int64_t *out) {
  if (nb == 0) return 0;
  if (nb > npre) return ORA_ECAPACITY;
  uint32_t *att = (uint32_t *)xcalloc((size_t)nb, 4);
  int64_t *cand = (int64_t *)xcalloc((size_t)nb, 8);
  char *settled = (char *)xcalloc((size_t)nb, 1), *mark = (char *)xcalloc((size_t)nb, 1);
  uint32_t stp = (uint32_t)h->step, col = (uint32_t)h->p.column;
  for (int64_t k = 0; k < nb; ++k) cand[k] = slot_draw(h->p.seed, k, 0, stp, stream, col, npre);
  int64_t left = nb;
  while (left > 0) {
    for (int64_t k = 0; k < nb; ++k) {
      mark[k] = 0;
      if (settled[k]) continue;
      int ok = 1;
      for (int64_t j = 0; j < nb && ok; ++j) {
        if (j == k) continue;
        if (settled[j] && out[j] == cand[k]) ok = 0;
        if (!settled[j] && j < k && cand[j] == cand[k]) ok = 0;
      }
      mark[k] = (char)ok;
    }
    for (int64_t k = 0; k < nb; ++k) {
      if (settled[k]) continue;
      if (mark[k]) { settled[k] = 1; out[k] = cand[k]; --left; }
      else { att[k]++; cand[k] = slot_draw(h->p.seed, k, att[k], stp, stream, col, npre); }
    }
  }
  free(att); free(cand); free(settled); free(mark);
  return 0;
}

static void write_newborn(species *s, int64_t slot, int32_t cell, real off, const real *v, uint64_t id) {
  s->cell[slot] = cell; s->off[slot] = off; s->vx[slot] = v[0]; s->vy[slot] = v[1]; s->vz[slot] = v[2];
  s->id[slot] = id;
}

/* RADIAL: births fill the dead slots in ascending order; extra births are
 * appended; extra holes are closed by moving the live particles of the tail
 * [N_new, N) into the holes below N_new, both in ascending order. */
static int fill_and_compact(ora_t *h, species *s, const int64_t *dead, int64_t nd, int is_ion) {
  int64_t nb = h->nb, N = s->n;
  int64_t m = nb < nd ? nb : nd;
  for (int64_t k = 0; k < m; ++k) {
    const birth *b = &h->births[k];
    uint64_t id = (uint64_t)h->next_id + 2 * (uint64_t)k + (uint64_t)is_ion;
    write_newborn(s, dead[k], b->cell, b->off, is_ion ? b->vi : b->ve, id);
    deposit(s->Q, h->Nw, b->cell, b->off, +1);
  }
  if (nb > nd) {
    if (N + (nb - nd) > s->cap) return ORA_ECAPACITY;
    for (int64_t k = m; k < nb; ++k) {
      const birth *b = &h->births[k];
      uint64_t id = (uint64_t)h->next_id + 2 * (uint64_t)k + (uint64_t)is_ion;
      write_newborn(s, N + (k - m), b->cell, b->off, is_ion ? b->vi : b->ve, id);
      deposit(s->Q, h->Nw, b->cell, b->off, +1);
    }
    s->n = N + (nb - nd);
  } else if (nd > nb) {
    int64_t Nn = N - (nd - nb);
    /* remaining holes dead[nb..nd) ascending: the first q lie below Nn */
    int64_t q = 0;
    while (nb + q < nd && dead[nb + q] < Nn) ++q;
    int64_t d = nb + q, t = Nn;
    for (int64_t c = 0; c < q; ++c) {
      while (d < nd && dead[d] == t) { ++t; ++d; }
      copy_particle(s, dead[nb + c], t);
      ++t;
    }
    s->n = Nn;
  }
  return 0;
}

static int births_and_losses(ora_t *h, int ion_pushed) {
  int64_t nb = h->nb;
  int lm = h->p.loss_mode;
  if (lm == ORA_LOSS_PAIR) {
    if (nb > 0) {
      int64_t *ve = (int64_t *)xcalloc((size_t)nb, 8), *vi = (int64_t *)xcalloc((size_t)nb, 8);
      int rc = draw_victims(h, nb, h->e.n, ST_VIC_E, ve);
      if (!rc) rc = draw_victims(h, nb, h->i.n, ST_VIC_I, vi);
      if (rc) { free(ve); free(vi); return rc; }
      for (int64_t k = 0; k < nb; ++k) {
        const birth *b = &h->births[k];
        deposit(h->e.Q, h->Nw, h->e.cell[ve[k]], h->e.off[ve[k]], -1);
        write_newborn(&h->e, ve[k], b->cell, b->off, b->ve, (uint64_t)h->next_id + 2 * (uint64_t)k);
        deposit(h->e.Q, h->Nw, b->cell, b->off, +1);
        deposit(h->i.Q, h->Nw, h->i.cell[vi[k]], h->i.off[vi[k]], -1);
        write_newborn(&h->i, vi[k], b->cell, b->off, b->vi, (uint64_t)h->next_id + 2 * (uint64_t)k + 1);
        deposit(h->i.Q, h->Nw, b->cell, b->off, +1);
      }
      free(ve); free(vi);
      h->st.losses_e += nb; h->st.losses_i += nb;
    }
  } else if (lm == ORA_LOSS_RADIAL || h->bounded) {
    /* removed particles (radial losses; in a bounded column also those the electrodes took) leave
       holes that the births fill, the rest compacted */
    int rc = fill_and_compact(h, &h->e, h->dead_e, h->nde, 0);
    if (!rc) rc = fill_and_compact(h, &h->i, h->dead_i, ion_pushed ? h->ndi : 0, 1);
    if (rc) return rc;
    h->st.losses_e += h->nde; h->st.losses_i += ion_pushed ? h->ndi : 0;
  } else if (lm == ORA_LOSS_NONE) {
    if (h->e.n + nb > h->e.cap || h->i.n + nb > h->i.cap) return ORA_ECAPACITY;
    for (int64_t k = 0; k < nb; ++k) {
      const birth *b = &h->births[k];
      write_newborn(&h->e, h->e.n + k, b->cell, b->off, b->ve, (uint64_t)h->next_id + 2 * (uint64_t)k);
      deposit(h->e.Q, h->Nw, b->cell, b->off, +1);
      write_newborn(&h->i, h->i.n + k, b->cell, b->off, b->vi, (uint64_t)h->next_id + 2 * (uint64_t)k + 1);
      deposit(h->i.Q, h->Nw, b->cell, b->off, +1);
    }
    h->e.n += nb; h->i.n += nb;
  }
  if (lm != ORA_LOSS_SWARM) {
    h->st.births += nb;
    h->next_id += 2 * nb;
  }
  h->nb = 0;
  if (h->bounded && h->emit_per_step > 0.0) {
    /* Sec. V: the cathode emits the current density J_emit: J_emit dt / (e w) macro-electrons per
       step (the fraction carried over).  Emitted electron k of step s draws (Philox counter k, s,
       emission stream) a half-Maxwellian velocity at T_emit, v_x = sig |g0|, v_y = sig g1,
       v_z = sig g2, and starts at x = u v_x dt (the part of the step it has already flown). */
    h->emit_acc += h->emit_per_step;
    int64_t ne = (int64_t)floor(h->emit_acc);
    h->emit_acc -= (double)ne;
    species *s = &h->e;
    if (s->n + ne > s->cap) return ORA_ECAPACITY;
    uint32_t stp = (uint32_t)h->step, col = (uint32_t)h->p.column;
    for (int64_t k = 0; k < ne; ++k) {
      ustream us; us_init(&us, h->p.seed, (uint64_t)k, stp, ST_EMIT, col);
      real g0 = gauss_sample(h->gauss, us_next(&us));
      real g1 = gauss_sample(h->gauss, us_next(&us));
      real g2 = gauss_sample(h->gauss, us_next(&us));
      real u = us_next(&us);
      real v[3];
      v[0] = h->sig_emit * (g0 < (real)0 ? -g0 : g0);
      v[1] = h->sig_emit * g1;
      v[2] = h->sig_emit * g2;
      real x = u * v[0] * h->emit_dtdx;
      int32_t cell = (int32_t)x;
      real off = x - (real)cell;
      if (cell >= h->N) { cell = h->N - 1; off = (real)0; }
      write_newborn(s, s->n + k, cell, off, v, (uint64_t)h->next_id + (uint64_t)k);
      deposit(s->Q, h->Nw, cell, off, +1);
    }
    s->n += ne;
    h->next_id += ne;
    h->st.emitted += ne;
  }
  return 0;
}

/* Stable counting sort of one species by cell (reading: particles are
 * reordered periodically so that each GPU thread block works on a narrow
 * cell window; slots, and hence victim draws, depend on the order, so the
 * sort is part of the step's definition).  Equal cells keep slot order. */
static void sort_species(ora_t *h, species *s) {
  int N = h->N;
  int64_t n = s->n;
  int64_t *start = (int64_t *)xcalloc((size_t)N + 1, 8);
  for (int64_t p = 0; p < n; ++p) start[s->cell[p] + 1]++;
  for (int c = 0; c < N; ++c) start[c + 1] += start[c];
  species t;
  t.cell = (int32_t *)xcalloc((size_t)n, 4); t.off = (real *)xcalloc((size_t)n, sizeof(real));
  t.vx = (real *)xcalloc((size_t)n, sizeof(real)); t.vy = (real *)xcalloc((size_t)n, sizeof(real));
  t.vz = (real *)xcalloc((size_t)n, sizeof(real)); t.id = (uint64_t *)xcalloc((size_t)n, 8);
  for (int64_t p = 0; p < n; ++p) {
    int64_t q = start[s->cell[p]]++;
    t.cell[q] = s->cell[p]; t.off[q] = s->off[p]; t.vx[q] = s->vx[p]; t.vy[q] = s->vy[p]; t.vz[q] = s->vz[p];
    t.id[q] = s->id[p];
  }
  memcpy(s->cell, t.cell, (size_t)n * 4); memcpy(s->off, t.off, (size_t)n * sizeof(real));
  memcpy(s->vx, t.vx, (size_t)n * sizeof(real)); memcpy(s->vy, t.vy, (size_t)n * sizeof(real));
  memcpy(s->vz, t.vz, (size_t)n * sizeof(real)); memcpy(s->id, t.id, (size_t)n * 8);
  free(t.cell); free(t.off); free(t.vx); free(t.vy); free(t.vz); free(t.id); free(start);
}

/* one full step s -> s+1 */
static int step_once(ora_t *h) {
  int sub = h->p.ion_subcycle;
  int ion_push = (sub > 0) && (h->step % sub == 0);
  int diag = (h->p.diag_every > 0) && (h->step % h->p.diag_every == 0);
  h->nde = 0; h->ndi = 0; h->nb = 0;
  /* electrons are sorted every sort_every steps, ions every sort_every * ion_subcycle steps */
  if (h->p.sort_every > 0 && h->step % h->p.sort_every == 0) {
    sort_species(h, &h->e);
    int64_t pi = (int64_t)h->p.sort_every * (sub > 0 ? sub : 1);
    if (h->step % pi == 0) sort_species(h, &h->i);
  }
  memset(h->e.Q, 0, sizeof(int64_t) * (size_t)h->Nw);
  h->sumv[0] = 0;
  for (int64_t p = 0; p < h->e.n; ++p) electron_step(h, p, diag);
  if (ion_push) {
    memset(h->i.Q, 0, sizeof(int64_t) * (size_t)h->Nw);
    h->sumv[1] = 0;
    for (int64_t p = 0; p < h->i.n; ++p) ion_step(h, p, diag);
  }
  if (h->err) return h->err;
  int rc = births_and_losses(h, ion_push);
  if (rc) return rc;
  h->step++;
  h->m_steps++;
  /* Sec. V: a source in series with a resistor sets the applied field,
   * U = R_ext J + V_D with V_D = E0 L, so E0 = (U - R_ext J) / L, where J is the
   * discharge current density e w (sum v_e - sum v_i) / L over the pushed particles
   * (ions at their last push): positive when the electrons drift against the
   * applied field -E0 -- a reading of the Sec. V circuit, whose resistor
   * adjusts E0. */
  if (h->p.drive == ORA_DRIVE_CIRCUIT) {
    double J = h->Cj * (double)(h->sumv[0] - h->sumv[1]);
    h->E0 = (h->p.U_src - h->p.R_ext_ohm_m2 * J) / h->p.L_m;
  }
  solve_field(h);
  if (diag) {
    double phi = 0.0;
    for (int j = 0; j < h->Nw; ++j) {
      h->m_ne[j] += (double)h->e.Q[j] * (1.0 / TWO32);
      h->m_ni[j] += (double)h->i.Q[j] * (1.0 / TWO32);
      h->m_E[j] += h->E[j];
      h->m_phi[j] += phi;
      if (j < h->N) phi = phi - h->dx * h->Eh[j];
    }
    h->m_samples++;
    h->st.n_diag++;
    if (h->eepf) h->eepf_samples++;
  }
  return h->err;
}

int ora_step(ora_t *h, int64_t n) {
  for (int64_t k = 0; k < n; ++k) {
    int rc = step_once(h);
    if (rc) return rc;
  }
  return 0;
}

/* initial half step of the leapfrog: v^{-1/2} = v^0 - (q dt / 2m) E^0(x^0) */
static void half_step_back(ora_t *h, species *s, real a) {
  real ha = (real)0.5 * a;
  for (int64_t p = 0; p < s->n; ++p) {
    real Ep = gather(h, s->cell[p], s->off[p]);
    s->vx[p] = s->vx[p] - ha * Ep;
  }
}

static void redeposit(ora_t *h, species *s) {
  memset(s->Q, 0, sizeof(int64_t) * (size_t)h->Nw);
  for (int64_t p = 0; p < s->n; ++p) deposit(s->Q, h->Nw, s->cell[p], s->off[p], +1);
}

/* Initial state (Sec. II: uniform, equal electron and ion densities;
 * Maxwellian velocities).  Electron p has id p, ion p has id n_e0 + p. */
static void init_species(ora_t *h, species *s, int64_t n, uint64_t id0, uint32_t stream, real sig) {
  uint32_t col = (uint32_t)h->p.column;
  for (int64_t p = 0; p < n; ++p) {
    uint64_t id = id0 + (uint64_t)p;
    uint32_t w[4], x[4];
    rng_block(h->p.seed, id, 0, stream, col, 0, w);
    rng_block(h->p.seed, id, 0, stream, col, 1, x);
    s->cell[p] = (int32_t)(((uint64_t)w[0] * (uint64_t)(uint32_t)h->N) >> 32);
    s->id[p] = id;
#ifdef ORACLE_F32
    s->off[p] = u_f32(w[1]);
    s->vx[p] = sig * gauss_sample(h->gauss, u_f32(w[2]));
    s->vy[p] = sig * gauss_sample(h->gauss, u_f32(w[3]));
    s->vz[p] = sig * gauss_sample(h->gauss, u_f32(x[0]));
#else
    uint32_t y[4];
    rng_block(h->p.seed, id, 0, stream, col, 2, y);
    s->off[p] = u_f64(w[1], w[2]);
    s->vx[p] = sig * gauss_sample(h->gauss, u_f64(x[0], x[1]));
    s->vy[p] = sig * gauss_sample(h->gauss, u_f64(x[2], x[3]));
    s->vz[p] = sig * gauss_sample(h->gauss, u_f64(y[0], y[1]));
#endif
  }
  s->n = n;
}

int ora_create(const ora_params *pp, ora_t **out) {
  *out = NULL;
  if (!pp || pp->n_cells < 3 || pp->dt_s <= 0 || pp->L_m <= 0 || pp->n_e0 < 0 || pp->n_i0 < 0 ||
      pp->n_table < 3 || pp->n_xsec < 0 || pp->n_xsec > 2 * MAXPROC)
    return ORA_EINVAL;
  ora_t *h = (ora_t *)calloc(1, sizeof(ora_t));
  if (!h) return ORA_ENOMEM;
  h->p = *pp;
  h->N = pp->n_cells;
  h->bounded = (pp->flags & ORA_FLAG_BOUNDED) != 0;
  h->Nw = h->N + h->bounded;
  if (h->bounded && ((pp->loss_mode != ORA_LOSS_RADIAL && pp->loss_mode != ORA_LOSS_NONE) ||
                     !(pp->J_emit_Am2 >= 0.0) || !(pp->T_emit_eV >= 0.0))) {
    free(h);
    return ORA_EINVAL;
  }
  h->ntab = pp->n_table;
  double M = pp->gas_mass_amu * AMU;
  h->M = M;
  h->ng = pp->pressure_torr * TORR / (KB * pp->T_gas_K);
  h->dx = pp->L_m / (double)pp->n_cells;
  h->w = (pp->n_e0 > 0) ? pp->n0_m3 * pp->L_m / (double)pp->n_e0 : 0.0;
  h->C_field = (QE * h->w) / (EPS0 * TWO32);
  h->E0 = (pp->drive == ORA_DRIVE_V) ? pp->V_applied / pp->L_m : pp->E0_Vpm;
  h->Cj = QE * h->w / (pp->L_m * 256.0);
  int sub = pp->ion_subcycle > 0 ? pp->ion_subcycle : 1;
  h->dt_i = (double)sub * pp->dt_s;
  h->a_e = (real)(-QE / ME * pp->dt_s);
  h->d_e = (real)(pp->dt_s / h->dx);
  h->a_i = (real)(QE / M * h->dt_i);
  h->d_i = (real)(h->dt_i / h->dx);
  h->K_e = (real)(0.5 * ME / QE);
  h->K_i = (real)(0.5 * M / QE);
  double Ve = 2.0 * QE / ME, Vi = 2.0 * QE / M;
  h->V_e = (real)Ve;
  h->em = (real)(2.0 * ME / M);
  h->sig_n = (real)sqrt(KB * pp->T_gas_K / M);
  h->sig_e0 = (real)sqrt(QE * pp->Te0_eV / ME);
  h->sig_i0 = (real)sqrt(QE * pp->Ti0_eV / M);
  h->sig_emit = (real)sqrt(QE * pp->T_emit_eV / ME);
  h->emit_dtdx = (real)(pp->dt_s / h->dx);
  h->emit_per_step = (h->bounded && h->w > 0.0) ? pp->J_emit_Am2 * pp->dt_s / (QE * h->w) : 0.0;
  /* collision-frequency tables */
  int n = h->ntab;
  double sum_e_max = 0.0, sum_i_max = 0.0;
  double *sum_e = (double *)xcalloc((size_t)n, 8), *sum_i = (double *)xcalloc((size_t)n, 8);
  double de_e = pp->eps_max_e_eV / (double)(n - 1), de_i = pp->eps_max_i_eV / (double)(n - 1);
  for (int k = 0; k < pp->n_xsec; ++k) {
    const ora_xsec *x = &pp->xsec[k];
    if (x->n < 1) { free(sum_e); free(sum_i); free(h); return ORA_EINVAL; }
    if (is_electron_kind(x->kind)) {
      if (h->np_e >= MAXPROC) { free(sum_e); free(sum_i); free(h); return ORA_EINVAL; }
      int j = h->np_e++;
      h->kind_e[j] = x->kind; h->xs_e[j] = k; h->thr_e[j] = (real)x->threshold_eV;
      h->tab_e[j] = (double *)xcalloc((size_t)n, 8);
      build_table(x, h->ng, pp->eps_max_e_eV, n, Ve, h->tab_e[j]);
      for (int i = 0; i < n; ++i) sum_e[i] = sum_e[i] + h->tab_e[j][i];
    } else {
      if (h->np_i >= MAXPROC) { free(sum_e); free(sum_i); free(h); return ORA_EINVAL; }
      int j = h->np_i++;
      h->kind_i[j] = x->kind; h->xs_i[j] = k;
      h->tab_i[j] = (double *)xcalloc((size_t)n, 8);
      build_table(x, h->ng, pp->eps_max_i_eV, n, Vi, h->tab_i[j]);
      for (int i = 0; i < n; ++i) sum_i[i] = sum_i[i] + h->tab_i[j][i];
    }
  }
  for (int i = 0; i < n; ++i) {
    if (sum_e[i] > sum_e_max) sum_e_max = sum_e[i];
    if (sum_i[i] > sum_i_max) sum_i_max = sum_i[i];
  }
  /* Electron majorant per energy bin [eps_i, eps_i+1]: the interpolated frequencies in a bin never
   * exceed the larger of the summed frequencies at its two ends (reading: an energy-binned
   * null-collision majorant; the electron energy is known before the collision test). */
  h->nub_e = (real *)xcalloc((size_t)n, sizeof(real));
  h->Pb_e = (real *)xcalloc((size_t)n, sizeof(real));
  for (int i = 0; i + 1 < n; ++i) {
    double mx = sum_e[i] > sum_e[i + 1] ? sum_e[i] : sum_e[i + 1];
    h->nub_e[i] = (real)mx;
    h->Pb_e[i] = (real)(-expm1(-mx * pp->dt_s));
  }
  free(sum_e); free(sum_i);
  h->nustar_e = sum_e_max; h->nustar_i = sum_i_max;
  h->Pnull_e = -expm1(-sum_e_max * pp->dt_s);
  h->Pnull_i = -expm1(-sum_i_max * h->dt_i);
  h->P_e = (real)h->Pnull_e; h->P_i = (real)h->Pnull_i;
  h->nus_e = (real)sum_e_max; h->nus_i = (real)sum_i_max;
  h->inv_de_e = (real)((double)(n - 1) / pp->eps_max_e_eV);
  h->inv_de_i = (real)((double)(n - 1) / pp->eps_max_i_eV);
  (void)de_e; (void)de_i;
  for (int j = 0; j < h->np_e; ++j) {
    h->rt_e[j] = (real *)xcalloc((size_t)n, sizeof(real));
    for (int i = 0; i < n; ++i) h->rt_e[j][i] = (real)h->tab_e[j][i];
  }
  for (int j = 0; j < h->np_i; ++j) {
    h->rt_i[j] = (real *)xcalloc((size_t)n, sizeof(real));
    for (int i = 0; i < n; ++i) h->rt_i[j][i] = (real)h->tab_i[j][i];
  }
  if (pp->loss_mode == ORA_LOSS_RADIAL) {
    double Pw = -expm1(-pp->nu_w * pp->dt_s), Pwi = -expm1(-pp->nu_w * h->dt_i);
    h->Pw_e = (uint32_t)(Pw * TWO32);
    h->Pw_i = (uint32_t)(Pwi * TWO32);
  }
  ora_gauss_table(h->gauss);
  int64_t cap = pp->capacity;
  int64_t nmax = pp->n_e0 > pp->n_i0 ? pp->n_e0 : pp->n_i0;
  if (cap <= 0) cap = nmax + nmax / 4 + 1024;
  if (cap < nmax) { ora_destroy(h); return ORA_EINVAL; }
  if (species_alloc(&h->e, cap, h->N + 1) || species_alloc(&h->i, cap, h->N + 1)) { ora_destroy(h); return ORA_ENOMEM; }
  h->E = (double *)xcalloc((size_t)h->N + 1, 8);
  h->Eh = (double *)xcalloc((size_t)h->N, 8);
  h->Ef = (real *)xcalloc((size_t)h->N + 1, sizeof(real));
  moments_alloc(h);
  h->dead_e = (int64_t *)xcalloc((size_t)cap, 8); h->dead_i = (int64_t *)xcalloc((size_t)cap, 8);
  init_species(h, &h->e, pp->n_e0, 0, ST_INIT_E, h->sig_e0);
  init_species(h, &h->i, pp->n_i0, (uint64_t)pp->n_e0, ST_INIT_I, h->sig_i0);
  h->next_id = pp->n_e0 + pp->n_i0;
  redeposit(h, &h->e);
  redeposit(h, &h->i);
  solve_field(h);
  half_step_back(h, &h->e, h->a_e);
  half_step_back(h, &h->i, h->a_i);
  for (int64_t p = 0; p < h->i.n; ++p) h->sumv[1] += (int64_t)llrint((double)(h->i.vx[p] * (real)256));
  *out = h;
  return 0;
}

void ora_destroy(ora_t *h) {
  if (!h) return;
  for (int j = 0; j < MAXPROC; ++j) { free(h->tab_e[j]); free(h->tab_i[j]); free(h->rt_e[j]); free(h->rt_i[j]); }
  free(h->nub_e); free(h->Pb_e);
  species_free(&h->e); species_free(&h->i);
  free(h->E); free(h->Eh); free(h->Ef); free(h->births); free(h->dead_e); free(h->dead_i);
  moments_free(h);
  free(h->eepf);
  free(h);
}

int ora_eepf_config(ora_t *h, int n_x, int n_eps, double eps_max_eV) {
  if (n_x < 0 || n_x > h->N || (n_x > 0 && (n_eps < 1 || n_eps > 65536 || !(eps_max_eV > 0.0)))) return ORA_EINVAL;
  free(h->eepf);
  h->eepf = NULL; h->eepf_nx = 0; h->eepf_ne = 0; h->eepf_samples = 0;
  if (n_x == 0) return 0;
  h->eepf = (uint64_t *)xcalloc((size_t)n_x * (size_t)(n_eps + 1), 8);
  h->eepf_nx = n_x; h->eepf_ne = n_eps;
  h->eepf_scale = (real)((double)n_eps / eps_max_eV);
  return 0;
}

int ora_eepf_get(ora_t *h, uint64_t *counts, int64_t *n_samples, int reset) {
  if (!h->eepf) return ORA_EINVAL;
  size_t n = (size_t)h->eepf_nx * (size_t)(h->eepf_ne + 1);
  if (counts) memcpy(counts, h->eepf, n * 8);
  if (n_samples) *n_samples = h->eepf_samples;
  if (reset) { memset(h->eepf, 0, n * 8); h->eepf_samples = 0; }
  return 0;
}

int ora_get_state(ora_t *h, ora_state *s) {
  s->n_e = h->e.n; s->n_i = h->i.n; s->step = h->step; s->next_id = h->next_id; s->E0 = h->E0;
  species *sp[2] = {&h->e, &h->i};
  int32_t *cells[2] = {s->cell_e, s->cell_i};
  double *offs[2] = {s->off_e, s->off_i}, *vxs[2] = {s->vx_e, s->vx_i}, *vys[2] = {s->vy_e, s->vy_i},
         *vzs[2] = {s->vz_e, s->vz_i};
  uint64_t *ids[2] = {s->id_e, s->id_i};
  for (int q = 0; q < 2; ++q) {
    for (int64_t p = 0; p < sp[q]->n; ++p) {
      if (cells[q]) cells[q][p] = sp[q]->cell[p];
      if (offs[q]) offs[q][p] = (double)sp[q]->off[p];
      if (vxs[q]) vxs[q][p] = (double)sp[q]->vx[p];
      if (vys[q]) vys[q][p] = (double)sp[q]->vy[p];
      if (vzs[q]) vzs[q][p] = (double)sp[q]->vz[p];
      if (ids[q]) ids[q][p] = sp[q]->id[p];
    }
  }
  /* node arrays: n_cells entries, n_cells + 1 in a bounded column */
  if (s->E) memcpy(s->E, h->E, sizeof(double) * (size_t)h->Nw);
  if (s->Q_e) memcpy(s->Q_e, h->e.Q, sizeof(int64_t) * (size_t)h->Nw);
  if (s->Q_i) memcpy(s->Q_i, h->i.Q, sizeof(int64_t) * (size_t)h->Nw);
  return 0;
}

/* Set the state.  E NULL -> recomputed from the charges; Q_i NULL -> ions re-deposited.
 * Electron charge is always re-deposited from the electrons. */
int ora_set_state(ora_t *h, const ora_state *s) {
  if (s->n_e < 0 || s->n_i < 0 || s->n_e > h->e.cap || s->n_i > h->i.cap) return ORA_EINVAL;
  species *sp[2] = {&h->e, &h->i};
  int32_t *cells[2] = {s->cell_e, s->cell_i};
  double *offs[2] = {s->off_e, s->off_i}, *vxs[2] = {s->vx_e, s->vx_i}, *vys[2] = {s->vy_e, s->vy_i},
         *vzs[2] = {s->vz_e, s->vz_i};
  uint64_t *ids[2] = {s->id_e, s->id_i};
  int64_t ns[2] = {s->n_e, s->n_i};
  for (int q = 0; q < 2; ++q) {
    for (int64_t p = 0; p < ns[q]; ++p) {
      int32_t c = cells[q][p];
      double o = offs[q][p];
      if (c < 0 || c >= h->N || !(o >= 0.0 && o < 1.0)) return ORA_EINVAL;
      sp[q]->cell[p] = c; sp[q]->off[p] = (real)o;
      if ((double)sp[q]->off[p] >= 1.0) return ORA_EINVAL;
      sp[q]->vx[p] = (real)vxs[q][p]; sp[q]->vy[p] = (real)vys[q][p]; sp[q]->vz[p] = (real)vzs[q][p];
      sp[q]->id[p] = ids[q][p];
    }
    sp[q]->n = ns[q];
  }
  h->step = s->step; h->next_id = s->next_id; h->E0 = s->E0;
  h->emit_acc = 0.0;
  h->sumv[1] = 0;
  for (int64_t p = 0; p < h->i.n; ++p) h->sumv[1] += (int64_t)llrint((double)(h->i.vx[p] * (real)256));
  redeposit(h, &h->e);
  if (s->Q_i) memcpy(h->i.Q, s->Q_i, sizeof(int64_t) * (size_t)h->Nw);
  else redeposit(h, &h->i);
  if (s->E) {
    memcpy(h->E, s->E, sizeof(double) * (size_t)h->Nw);
    for (int j = 0; j < h->N; ++j) h->Ef[j] = (real)h->E[j];
    h->Ef[h->N] = h->bounded ? (real)h->E[h->N] : h->Ef[0];
  } else {
    solve_field(h);
  }
  return 0;
}

int ora_stats_get(ora_t *h, ora_stats *s) {
  *s = h->st;
  s->step = h->step; s->n_e = h->e.n; s->n_i = h->i.n; s->next_id = h->next_id; s->E0 = h->E0;
  return 0;
}

int ora_moments_get(ora_t *h, ora_moments *m) {
  int N = h->Nw;
  double ns = h->m_samples > 0 ? (double)h->m_samples : 1.0;
  double dens = h->w / h->dx;
  double tsteps = (double)(h->m_steps > 0 ? h->m_steps : 1) * h->p.dt_s;
  m->n_samples = h->m_samples; m->n_steps = h->m_steps;
  for (int j = 0; j < N; ++j) {
    if (m->n_e) m->n_e[j] = h->m_ne[j] / ns * dens;
    if (m->n_i) m->n_i[j] = h->m_ni[j] / ns * dens;
    if (m->gamma_e) m->gamma_e[j] = h->m_ge[j] / ns * dens;
    if (m->mean_eps_e) m->mean_eps_e[j] = h->m_ne[j] > 0 ? h->m_ee[j] / h->m_ne[j] : 0.0;
    if (m->heat_e) m->heat_e[j] = h->m_he[j] / ns * dens;
    if (m->iz_rate) m->iz_rate[j] = (double)h->m_iz[j] * (1.0 / TWO32) * dens / tsteps;
    if (m->gamma_i) m->gamma_i[j] = h->m_gi[j] / ns * dens;
    if (m->E) m->E[j] = h->m_E[j] / ns;
    if (m->phi) m->phi[j] = h->m_phi[j] / ns;
  }
  if (m->reset) moments_reset(h);
  return 0;
}

int ora_last_codes(ora_t *h, int species_, int32_t *out, int64_t n) {
  species *s = species_ ? &h->i : &h->e;
  if (n > s->cap) return ORA_EINVAL;
  memcpy(out, s->code, sizeof(int32_t) * (size_t)n);
  return 0;
}

int ora_derived(ora_t *h, double *o) {
  o[0] = h->ng; o[1] = h->nustar_e; o[2] = h->Pnull_e; o[3] = h->nustar_i; o[4] = h->Pnull_i;
  o[5] = h->w; o[6] = h->dx;
  return 0;
}

int ora_nu_table(ora_t *h, int species_, int j, double *out, int n) {
  if (n != h->ntab) return ORA_EINVAL;
  if (species_ == 0) { if (j < 0 || j >= h->np_e) return ORA_EINVAL; memcpy(out, h->tab_e[j], 8 * (size_t)n); }
  else { if (j < 0 || j >= h->np_i) return ORA_EINVAL; memcpy(out, h->tab_i[j], 8 * (size_t)n); }
  return 0;
}
