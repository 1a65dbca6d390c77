// Host driver and C ABI (include/pic.h) of the PIC-MCC library.
//
// Owns the device memory of one periodic column, builds the uniform-energy
// collision-frequency tables from the caller's cross sections (Sec. II), and
// launches the step kernels on the handle's stream.  No step is computed on
// the host; the host only prepares tables, launches, and copies state.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pic_internal.cuh"

namespace {

// CODATA 2018
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kKb = 1.380649e-23;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kTorr = 133.32236842105263;
constexpr double kTwo32 = 4294967296.0;

thread_local std::string g_err;

}  // namespace

struct pic_handle {
  pic_params p{};
  int N = 0;
  int Nn = 0;                         // node-array entries: N, or N + 1 in a bounded column
  int ntab = 0;
  int nsm = 0;
  bool mixed = false;
  cudaStream_t stream = nullptr;
  // derived
  double ng = 0, dx = 0, w = 0, M = 0, Cfield = 0, E0 = 0, dt_i = 0;
  double nustar[2] = {0, 0}, Pnull[2] = {0, 0};
  // device memory
  pic::Ctl *ctl = nullptr;
  pic::SpeciesDev sp[2]{};
  double *E = nullptr, *Eh = nullptr;
  pic::FieldScan *fs = nullptr;       // exact prefix data between the two field kernels
  pic::SortBuf sb[2]{};               // sort buffers per species (sort_every > 0)
  void *Ef = nullptr;                 // R[N+1]
  void *tab[2] = {nullptr, nullptr};  // R[np * ntab]
  void *tabb = nullptr;               // electron per-bin majorant and null-collision probability, R[2 ntab]
  uint32_t *tabi = nullptr;           // FP32 form: the per-bin probabilities as 24-bit integer thresholds
  float *gauss = nullptr;
  void *bb_mem = nullptr;
  uint32_t *k3_mem = nullptr;
  double *mom = nullptr;              // 8 * N doubles
  unsigned long long *mom_iz = nullptr;
  long long eepf_base = 0;            // diagnostic samples (ctl n_diag) when the EEPF histogram was cleared
  double *stage = nullptr;            // pic_set_state: offsets and velocities uploaded as given (4 x cap doubles)
  unsigned long long *stage_bad = nullptr;   // first particle outside the grid (or ~0)
  // kernel parameter blocks
  pic::StepK<double> kd{};
  pic::StepK<float> kf{};
  pic::BirthBuf<double> bbd{};
  pic::BirthBuf<float> bbf{};
  pic::K3Scratch sc{};
  pic::Moments m{};
  pic::FieldK fk{};
  long long host_step = 0;
  std::string err;
  int latched = 0;
  // kernel timing
  bool timing = false;
  std::vector<cudaEvent_t> ev;        // event pool, used in pairs
  std::vector<int> ev_cls;            // class of each recorded pair
  size_t ev_used = 0;
  double kms[PIC_K_CLASSES] = {0};
  int64_t klaunch[PIC_K_CLASSES] = {0};
  // batch of columns (pic_init_batch): the columns are full handles sharing this handle's stream
  bool is_batch = false;
  pic_handle *owner = nullptr;        // set on the columns of a batch
  std::vector<pic_handle *> cols;
  void *coldev = nullptr;             // ColDev<R>[ncol] on the device
  int4 *sched = nullptr;              // CTA schedules: electrons at [0, nsched[0]), ions after
  pic::SortCol *scol[2] = {nullptr, nullptr};   // per species: the columns' sort table (sort_every > 0)
  int stiles[2] = {0, 0};             // sort tiles of all columns per species
  int spasses = 0;                    // radix passes of the largest column
  int nsched[2] = {0, 0};
  std::vector<int> mults;             // CTAs-per-SM multipliers the autotuner tries
  int mult[2] = {1, 1};               // chosen multiplier per species
  int tune_sp = 0;                    // species being tuned (2: done)
  int tune_i = 0, tune_round = 0;     // candidate and round of the species being tuned
  std::vector<float> tune_ms;         // best push time per candidate of that species
  int tune_mark = -1;                 // species whose push the next step brackets with tune_ev
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  std::string tune_key;               // shape of the batch (the autotuner's cache key)
  size_t push_smem = 0;
  int maxN = 0;
  cudaGraphExec_t cycle = nullptr;    // captured cycle of ion_subcycle steps (no sort, no diagnostics)
  int64_t cycle_launch[PIC_K_CLASSES] = {0};   // kernel launches per replay of the cycle
  cudaGraphExec_t dcycle = nullptr;   // the same with a diagnostic sample on its first step
  int64_t dcycle_launch[PIC_K_CLASSES] = {0};
};

namespace {

// pic_set_state: the uploaded offsets and velocities (FP64, as given) into the particle records,
// rounded once to the storage precision; *bad = the lowest index outside the grid
// (cell not in [0, N), offset not in [0, 1), or an offset that rounds to 1 in FP32 storage)
template <class R, class In>
__global__ void k_set_rec(const int32_t *__restrict__ cell, const In *__restrict__ st, long long n, int N,
                          void *rec, unsigned long long *bad) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    const double o = (double)st[p], vx = (double)st[n + p], vy = (double)st[2 * n + p], vz = (double)st[3 * n + p];
    const int32_t c = cell[p];
    bool ok = c >= 0 && c < N && o >= 0.0 && o < 1.0;
    if constexpr (std::is_same<R, float>::value) {
      ok = ok && (float)o < 1.0f;
      reinterpret_cast<float4 *>(rec)[p] = make_float4((float)o, (float)vx, (float)vy, (float)vz);
    } else {
      reinterpret_cast<pic::D4 *>(rec)[p] = pic::D4{o, vx, vy, vz};
    }
    if (!ok) atomicMin(bad, (unsigned long long)p);
  }
}

int set_err(pic_handle *h, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  if (h) h->err = buf;
  return code;
}

#define CU(h, x)                                                                                        \
  do {                                                                                                  \
    cudaError_t e_ = (x);                                                                               \
    if (e_ != cudaSuccess) return set_err(h, PIC_ECUDA, "%s: %s", #x, cudaGetErrorString(e_));       \
  } while (0)

bool is_e_kind(int k) { return k == PIC_ELASTIC || k == PIC_EXCITATION || k == PIC_IONIZATION; }

// sigma at eps: linear interpolation of the caller's table, end values held,
// zero below an excitation / ionization threshold
double xs_at(const pic_xsec &x, double eps) {
  if ((x.kind == PIC_EXCITATION || x.kind == PIC_IONIZATION) && eps < x.threshold_eV) return 0.0;
  const double *E = x.energy_eV, *S = x.sigma_m2;
  const int n = x.n;
  if (eps <= E[0]) return S[0];
  if (eps >= E[n - 1]) return S[n - 1];
  int lo = 0, hi = n - 1;  // largest a with E[a] <= eps: E[lo] <= eps < E[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (E[mid] <= eps) lo = mid; else hi = mid;
  }
  const double t = (eps - E[lo]) / (E[lo + 1] - E[lo]);
  return S[lo] + t * (S[lo + 1] - S[lo]);
}

// nu_k(eps_i) = n_g sigma_k(eps_i) sqrt(eps_i 2e/m), eps_i = i eps_max/(n-1)
void nu_table(const pic_xsec &x, double ng, double eps_max, int n, double Vq, double *out) {
  const double de = eps_max / (double)(n - 1);
  for (int i = 0; i < n; ++i) {
    const double eps = (double)i * de;
    const double v = std::sqrt(eps * Vq);
    out[i] = ng * xs_at(x, eps) * v;
  }
}

// Phi^-1(p) for p <= 1/2 by Newton's method from 0 on Phi(x) = erfc(-x/sqrt2)/2
// (Phi is convex for x < 0, so the iterates decrease monotonically to the root).
double inv_phi_newton(double p) {
  double x = 0.0;
  for (int it = 0; it < 200; ++it) {
    const double F = 0.5 * std::erfc(-x / std::sqrt(2.0));
    const double f = std::exp(-0.5 * x * x) / std::sqrt(2.0 * M_PI);
    const double dxn = (F - p) / f;
    const double xn = x - dxn;
    if (xn == x || std::fabs(dxn) <= 1e-17 * std::fabs(xn)) { x = xn; break; }
    x = xn;
  }
  return x;
}

// Gaussian inverse-CDF table, 4096 intervals, FP32 entries: T[k] = Phi^-1(k/4096),
// end entries with the exact conditional mean of the normal tail over the end interval.
void gauss_table(float *T) {
  const int n = pic::kGaussN;
  for (int k = 1; k <= n / 2; ++k) {
    const double z = inv_phi_newton((double)k / n);
    T[k] = (float)z;
    T[n - k] = (float)(-z);
  }
  T[n / 2] = 0.0f;
  const double z1 = inv_phi_newton(1.0 / n);
  const double m0 = -(double)n * std::exp(-0.5 * z1 * z1) / std::sqrt(2.0 * M_PI);
  T[0] = (float)(2.0 * m0 - z1);
  T[n] = -T[0];
}

template <class R> pic::StepK<R> &kparams(pic_handle *h);
template <> pic::StepK<double> &kparams<double>(pic_handle *h) { return h->kd; }
template <> pic::StepK<float> &kparams<float>(pic_handle *h) { return h->kf; }
template <class R> pic::BirthBuf<R> &bbuf(pic_handle *h);
template <> pic::BirthBuf<double> &bbuf<double>(pic_handle *h) { return h->bbd; }
template <> pic::BirthBuf<float> &bbuf<float>(pic_handle *h) { return h->bbf; }

// event pair around one launch (timing on), launch counting (always)
void t_begin(pic_handle *h) {
  if (!h->timing) return;
  if (h->ev_used + 2 > h->ev.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      h->ev.push_back(e);
    }
  }
  cudaEventRecord(h->ev[h->ev_used], h->stream);
}
void t_end(pic_handle *h, int cls, int nkernels = 1) {
  h->klaunch[cls] += nkernels;
  if (!h->timing) return;
  cudaEventRecord(h->ev[h->ev_used + 1], h->stream);
  h->ev_cls.push_back(cls);
  h->ev_used += 2;
}
// after a synchronisation: fold the recorded pairs into the per-class sums
void t_collect(pic_handle *h) {
  for (size_t i = 0; i < h->ev_cls.size(); ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]) == cudaSuccess) h->kms[h->ev_cls[i]] += ms;
  }
  h->ev_cls.clear();
  h->ev_used = 0;
}

int check_status(pic_handle *h) {
  pic::Ctl c;
  CU(h, cudaMemcpyAsync(&c, h->ctl, sizeof c, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  if (c.status) {
    if (c.status & pic::kStNonFinite) h->latched = set_err(h, PIC_ENONFINITE, "the field became non-finite");
    else if (c.status & pic::kStVictim) h->latched = set_err(h, PIC_ECAPACITY, "more births than particles to remove");
    else if (c.status & pic::kStTimeout) h->latched = set_err(h, PIC_ETIMEOUT, "a bounded wait of the particle step gave up");
    else h->latched = set_err(h, PIC_ECAPACITY, "capacity exceeded (status 0x%x)", c.status);
  }
  return h->latched;
}

template <class R> int setup_tables(pic_handle *h) {
  pic::StepK<R> &k = kparams<R>(h);
  const pic_params &p = h->p;
  const int n = h->ntab;
  k.N = h->N;
  k.bounded = (p.flags & PIC_FLAG_BOUNDED) ? 1 : 0;
  k.Nw = h->N + k.bounded;
  k.emit_per_step = (k.bounded && h->w > 0.0) ? p.J_emit_Am2 * p.dt_s / (kQe * h->w) : 0.0;
  k.sig_emit = (R)std::sqrt(kQe * p.T_emit_eV / kMe);
  k.emit_dtdx = (R)(p.dt_s / h->dx);
  k.ntab = n;
  k.loss_mode = p.loss_mode;
  k.field_mode = p.field_mode;
  k.drive = p.drive;
  k.flags = p.flags;
  k.diag_every = p.diag_every;
  k.sub = p.ion_subcycle;
  k.column = (uint32_t)p.column;
  k.seed = p.seed;
  for (int r = 0; r < 10; ++r) {
    k.rk[r][0] = (uint32_t)p.seed + (uint32_t)r * 0x9E3779B9u;
    k.rk[r][1] = (uint32_t)(p.seed >> 32) + (uint32_t)r * 0xBB67AE85u;
  }
  const double M = h->M;
  k.V_e = (R)(2.0 * kQe / kMe);
  k.em = (R)(2.0 * kMe / M);
  k.sig_n = (R)std::sqrt(kKb * p.T_gas_K / M);
  k.gauss = h->gauss;
  const double Vq[2] = {2.0 * kQe / kMe, 2.0 * kQe / M};
  const double emax[2] = {p.eps_max_e_eV, p.eps_max_i_eV};
  const double dts[2] = {p.dt_s, h->dt_i};
  std::vector<std::vector<double>> t64[2];
  std::vector<double> sum[2] = {std::vector<double>(n, 0.0), std::vector<double>(n, 0.0)};
  for (int q = 0; q < 2; ++q) { k.sp[q].np = 0; }
  for (int x = 0; x < p.n_xsec; ++x) {
    const pic_xsec &xs = p.xsec[x];
    const int q = is_e_kind(xs.kind) ? 0 : 1;
    pic::SpecK<R> &s = k.sp[q];
    const int j = s.np++;
    s.kind[j] = xs.kind;
    s.xs[j] = x;
    s.thr[j] = (R)xs.threshold_eV;
    t64[q].emplace_back(n);
    nu_table(xs, h->ng, emax[q], n, Vq[q], t64[q].back().data());
    for (int i = 0; i < n; ++i) sum[q][i] = sum[q][i] + t64[q].back()[i];
  }
  for (int q = 0; q < 2; ++q) {
    double mx = 0.0;
    for (int i = 0; i < n; ++i)
      if (sum[q][i] > mx) mx = sum[q][i];
    if (q == 0) {
      // majorant per energy bin [eps_i, eps_i+1]: the larger end value of the summed frequencies
      std::vector<R> bins(2 * (size_t)n, (R)0);
      for (int i = 0; i + 1 < n; ++i) {
        const double b = sum[0][i] > sum[0][i + 1] ? sum[0][i] : sum[0][i + 1];
        bins[i] = (R)b;
        bins[n + i] = (R)(-std::expm1(-b * dts[0]));
      }
      CU(h, cudaMalloc(&h->tabb, bins.size() * sizeof(R)));
      CU(h, cudaMemcpy(h->tabb, bins.data(), bins.size() * sizeof(R), cudaMemcpyHostToDevice));
      k.sp[0].nub = reinterpret_cast<const R *>(h->tabb);
      k.sp[0].Pb = reinterpret_cast<const R *>(h->tabb) + n;
      k.sp[0].Pbi = nullptr;
      if (std::is_same<R, float>::value) {
        std::vector<uint32_t> thr(n, 0u);
        for (int i = 0; i < n; ++i) thr[i] = (uint32_t)std::ceil((double)bins[n + i] * 16777216.0);
        CU(h, cudaMalloc(&h->tabi, thr.size() * 4));
        CU(h, cudaMemcpy(h->tabi, thr.data(), thr.size() * 4, cudaMemcpyHostToDevice));
        k.sp[0].Pbi = h->tabi;
      }
    }
    h->nustar[q] = mx;
    h->Pnull[q] = -std::expm1(-mx * dts[q]);
    pic::SpecK<R> &s = k.sp[q];
    s.P = (R)h->Pnull[q];
    s.Pi = (uint32_t)std::ceil((double)s.P * 16777216.0);
    s.nus = (R)mx;
    s.inv_de = (R)((double)(n - 1) / emax[q]);
    s.K = (R)(0.5 * (q == 0 ? kMe : M) / kQe);
    if (p.loss_mode == PIC_LOSS_RADIAL) {
      const double Pw = -std::expm1(-p.nu_w * dts[q]);
      s.Pw = (uint32_t)(Pw * kTwo32);
    } else {
      s.Pw = 0u;
    }
    std::vector<R> flat((size_t)s.np * n + 1);
    for (int j = 0; j < s.np; ++j)
      for (int i = 0; i < n; ++i) flat[(size_t)j * n + i] = (R)t64[q][j][i];
    CU(h, cudaMalloc(&h->tab[q], flat.size() * sizeof(R)));
    CU(h, cudaMemcpy(h->tab[q], flat.data(), flat.size() * sizeof(R), cudaMemcpyHostToDevice));
    s.tab = reinterpret_cast<const R *>(h->tab[q]);
  }
  k.sp[0].a = (R)(-kQe / kMe * p.dt_s);
  k.sp[0].d = (R)(p.dt_s / h->dx);
  k.sp[1].a = (R)(kQe / M * h->dt_i);
  k.sp[1].d = (R)(h->dt_i / h->dx);
  if (h->nustar[0] * p.dt_s > 0.3 && !(p.flags & PIC_FLAG_ALLOW_LARGE_NULL))
    return set_err(h, PIC_EPARAM, "nu*_e dt = %.3f > 0.3", h->nustar[0] * p.dt_s);
  return 0;
}

template <class R> int alloc_species(pic_handle *h) {
  const int64_t cap = h->sp[0].cap;
  for (int q = 0; q < 2; ++q) {
    pic::SpeciesDev &s = h->sp[q];
    CU(h, cudaMalloc(&s.cell, ((size_t)cap + pic::kPad) * 4));
    CU(h, cudaMalloc(&s.rec, ((size_t)cap + pic::kPad) * sizeof(typename pic::Rec<R>::T)));
    CU(h, cudaMalloc(&s.id, ((size_t)cap + pic::kPad) * 8));
    CU(h, cudaMalloc(&s.Q, (size_t)(h->N + 1) * 8));
    CU(h, cudaMalloc(&s.dead, (size_t)pic::kStageCap * 4));
    CU(h, cudaMemset(s.Q, 0, (size_t)(h->N + 1) * 8));
    if (h->p.flags & PIC_FLAG_RECORD_CODES) {
      CU(h, cudaMalloc(&s.code, (size_t)cap * 4));
      CU(h, cudaMemset(s.code, 0xff, (size_t)cap * 4));
    }
  }
  CU(h, cudaMalloc(&h->Ef, ((size_t)h->N + 1) * sizeof(R)));
  if (h->p.sort_every > 0) {
    for (int q = 0; q < 2; ++q) {
      pic::SortBuf &b = h->sb[q];
      CU(h, cudaMalloc(&b.cell, (size_t)cap * 4));
      CU(h, cudaMalloc(&b.rec, (size_t)cap * sizeof(typename pic::Rec<R>::T)));
      CU(h, cudaMalloc(&b.id, (size_t)cap * 8));
      CU(h, cudaMalloc(&b.hist, pic::sort_hist_words(cap) * 4));
    }
  }
  // birth staging: parent, cell (int32), off + 3 ve + 3 vi (R)
  const size_t sc = pic::kStageCap;
  CU(h, cudaMalloc(&h->bb_mem, sc * 8 + sc * 7 * sizeof(R)));
  pic::BirthBuf<R> &bb = bbuf<R>(h);
  char *b = reinterpret_cast<char *>(h->bb_mem);
  bb.parent = reinterpret_cast<int32_t *>(b);
  bb.cell = reinterpret_cast<int32_t *>(b + sc * 4);
  bb.off = reinterpret_cast<R *>(b + sc * 8);
  bb.ve = bb.off + sc;
  bb.vi = bb.ve + 3 * sc;
  return 0;
}

template <class R> int run_init(pic_handle *h) {
  pic::StepK<R> &k = kparams<R>(h);
  const pic_params &p = h->p;
  const R sig_e = (R)std::sqrt(kQe * p.Te0_eV / kMe);
  const R sig_i = (R)std::sqrt(kQe * p.Ti0_eV / h->M);
  pic::launch_init<R>(k, h->sp[0], 0, p.n_e0, 0, sig_e, h->stream);
  pic::launch_init<R>(k, h->sp[1], 1, p.n_i0, (uint64_t)p.n_e0, sig_i, h->stream);
  pic::launch_deposit<R>(k, h->sp[0], h->ctl, 0, h->stream);
  pic::launch_deposit<R>(k, h->sp[1], h->ctl, 1, h->stream);
  pic::launch_field<R>(h->fk, h->sp[0].Q, h->sp[1].Q, h->ctl, h->E, h->Eh, reinterpret_cast<R *>(h->Ef), h->m,
                       h->fs, false, false, h->stream);
  pic::launch_halfstep<R>(k, h->sp[0], h->ctl, reinterpret_cast<R *>(h->Ef), 0, h->stream);
  pic::launch_halfstep<R>(k, h->sp[1], h->ctl, reinterpret_cast<R *>(h->Ef), 1, h->stream);
  if (p.drive == PIC_DRIVE_CIRCUIT) pic::launch_sumv<R>(h->sp[1], h->ctl, 1, h->stream);
  CU(h, cudaGetLastError());
  return 0;
}

template <class R> int enqueue_step(pic_handle *h) {
  pic::StepK<R> &k = kparams<R>(h);
  const int sub = h->p.ion_subcycle;
  const bool ion_push = sub > 0 && (h->host_step % sub) == 0;
  const R *Ef = reinterpret_cast<const R *>(h->Ef);
  // electrons sorted every sort_every steps, ions every sort_every * ion_subcycle steps
  const int se = h->p.sort_every;
  const int sort_kernels = 3 * pic::sort_passes(h->N) + (pic::sort_passes(h->N) & 1);
  if (se > 0 && h->host_step % se == 0) {
    t_begin(h);
    int nk = sort_kernels;
    pic::launch_sort<R>(h->sp[0], h->sb[0], &h->ctl->n[0], h->sp[0].cap, h->N, h->nsm, h->stream);
    const long long pi = (long long)se * (sub > 0 ? sub : 1);
    if (h->host_step % pi == 0) {
      pic::launch_sort<R>(h->sp[1], h->sb[1], &h->ctl->n[1], h->sp[1].cap, h->N, h->nsm, h->stream);
      nk += sort_kernels;
    }
    t_end(h, PIC_K_SORT, nk);
  }
  const bool circuit = h->p.drive == PIC_DRIVE_CIRCUIT;
  if (circuit) CU(h, cudaMemsetAsync(&h->ctl->sumv[0], 0, 8, h->stream));
  CU(h, cudaMemsetAsync(h->sp[0].Q, 0, (size_t)h->Nn * 8, h->stream));
  const bool diag = h->p.diag_every > 0 && (h->host_step % h->p.diag_every) == 0;
  t_begin(h);
  pic::launch_push<R>(k, h->sp[0], h->ctl, Ef, bbuf<R>(h), h->m, 0, h->nsm, diag, h->stream);
  t_end(h, PIC_K_PUSH_E);
  if (ion_push) {
    CU(h, cudaMemsetAsync(h->sp[1].Q, 0, (size_t)h->Nn * 8, h->stream));
    if (circuit) CU(h, cudaMemsetAsync(&h->ctl->sumv[1], 0, 8, h->stream));
    t_begin(h);
    pic::launch_push<R>(k, h->sp[1], h->ctl, Ef, bbuf<R>(h), h->m, 1, h->nsm, diag, h->stream);
    t_end(h, PIC_K_PUSH_I);
  }
  t_begin(h);
  pic::launch_births<R>(k, h->sp[0], h->sp[1], h->ctl, bbuf<R>(h), h->sc, ion_push ? 1 : 0, h->stream);
  t_end(h, PIC_K_BIRTHS);
  t_begin(h);
  pic::launch_field<R>(h->fk, h->sp[0].Q, h->sp[1].Q, h->ctl, h->E, h->Eh, reinterpret_cast<R *>(h->Ef), h->m,
                       h->fs, diag, true, h->stream);
  t_end(h, PIC_K_FIELD, (h->p.field_mode == PIC_FIELD_POISSON ? 2 : 1) + (diag ? 1 : 0));
  CU(h, cudaGetLastError());
  h->host_step++;
  return 0;
}

void free_all(pic_handle *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (pic_handle *c : h->cols) {
    c->stream = nullptr;  // shared with the batch
    free_all(c);
    delete c;
  }
  h->cols.clear();
  cudaFree(h->coldev);
  cudaFree(h->sched);
  cudaFree(h->scol[0]);
  cudaFree(h->scol[1]);
  for (cudaEvent_t &e : h->tune_ev)
    if (e) cudaEventDestroy(e);
  if (h->cycle) cudaGraphExecDestroy(h->cycle);
  if (h->dcycle) cudaGraphExecDestroy(h->dcycle);
  for (int q = 0; q < 2; ++q) {
    cudaFree(h->sp[q].cell); cudaFree(h->sp[q].rec); cudaFree(h->sp[q].id); cudaFree(h->sp[q].code);
    cudaFree(h->sp[q].Q); cudaFree(h->sp[q].dead); cudaFree(h->tab[q]);
    cudaFree(h->sb[q].cell); cudaFree(h->sb[q].rec); cudaFree(h->sb[q].id); cudaFree(h->sb[q].hist);
  }
  cudaFree(h->tabb);
  cudaFree(h->tabi);
  cudaFree(h->ctl); cudaFree(h->E); cudaFree(h->Eh); cudaFree(h->fs); cudaFree(h->Ef); cudaFree(h->gauss);
  cudaFree(h->bb_mem); cudaFree(h->k3_mem); cudaFree(h->mom); cudaFree(h->mom_iz);
  cudaFree(h->stage); cudaFree(h->stage_bad); cudaFree(h->m.eepf);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  if (h->stream) cudaStreamDestroy(h->stream);
}

// (R, I) drive: the E0-drive parameters of the same column (E0 and n0 from pic_drive_ri)
int resolve_ri(const pic_params *p, pic_params *q) {
  double v[4];
  const int rc = pic_drive_ri(p, v);
  if (rc) return rc;
  *q = *p;
  q->drive = PIC_DRIVE_E0;
  q->E0_Vpm = v[0];
  q->n0_m3 = v[1];
  return 0;
}

// every floating-point input finite (a non-finite field or rate would reach the particle step)
static int check_finite(const pic_params *p) {
  const struct {
    const char *name;
    double v;
  } f[] = {{"gas_mass_amu", p->gas_mass_amu}, {"pressure_torr", p->pressure_torr}, {"T_gas_K", p->T_gas_K},
           {"L_m", p->L_m}, {"R_m", p->R_m}, {"E0_Vpm", p->E0_Vpm}, {"V_applied", p->V_applied}, {"I_A", p->I_A},
           {"U_src", p->U_src}, {"R_ext_ohm_m2", p->R_ext_ohm_m2}, {"dt_s", p->dt_s}, {"n0_m3", p->n0_m3},
           {"Te0_eV", p->Te0_eV}, {"Ti0_eV", p->Ti0_eV}, {"nu_w", p->nu_w}, {"eps_max_e_eV", p->eps_max_e_eV},
           {"eps_max_i_eV", p->eps_max_i_eV}, {"J_emit_Am2", p->J_emit_Am2}, {"T_emit_eV", p->T_emit_eV}};
  for (const auto &x : f)
    if (!std::isfinite(x.v)) return set_err(nullptr, PIC_EINVAL, "%s is not finite", x.name);
  return 0;
}

int validate(const pic_params *p) {
  if (!p) return set_err(nullptr, PIC_EINVAL, "params is NULL");
  if (int rc = check_finite(p)) return rc;
  if (!(p->gas_mass_amu > 0) || !(p->T_gas_K > 0)) return set_err(nullptr, PIC_EINVAL, "gas mass and temperature must be > 0");
  if (p->pressure_torr < 0) return set_err(nullptr, PIC_EINVAL, "pressure must be >= 0");
  if (p->Te0_eV < 0 || p->Ti0_eV < 0) return set_err(nullptr, PIC_EINVAL, "initial temperatures must be >= 0");
  if (p->nu_w < 0) return set_err(nullptr, PIC_EINVAL, "nu_w must be >= 0");
  if (p->n_cells < 3 || p->n_cells > 65536) return set_err(nullptr, PIC_EINVAL, "n_cells must be in [3, 65536]");
  if (!(p->dt_s > 0) || !(p->L_m > 0)) return set_err(nullptr, PIC_EINVAL, "dt and L must be > 0");
  if (p->n_e0 < 0 || p->n_i0 < 0) return set_err(nullptr, PIC_EINVAL, "negative particle count");
  if (p->n_table < 3) return set_err(nullptr, PIC_EINVAL, "n_table must be >= 3");
  if (p->precision != PIC_FP64 && p->precision != PIC_MIXED) return set_err(nullptr, PIC_EINVAL, "bad precision");
  if (p->loss_mode < PIC_LOSS_PAIR || p->loss_mode > PIC_LOSS_SWARM) return set_err(nullptr, PIC_EINVAL, "bad loss mode");
  if (p->drive != PIC_DRIVE_E0 && p->drive != PIC_DRIVE_V && p->drive != PIC_DRIVE_CIRCUIT)
    return set_err(nullptr, PIC_EINVAL, "drive %d not supported", p->drive);
  if (p->drive == PIC_DRIVE_CIRCUIT && p->field_mode != PIC_FIELD_POISSON)
    return set_err(nullptr, PIC_EINVAL, "the circuit drive needs the self-consistent field");
  if (p->field_mode != PIC_FIELD_POISSON && p->field_mode != PIC_FIELD_APPLIED)
    return set_err(nullptr, PIC_EINVAL, "bad field mode");
  if (p->ion_subcycle < 0) return set_err(nullptr, PIC_EINVAL, "ion_subcycle < 0");
  if (p->flags & PIC_FLAG_BOUNDED) {
    if (p->loss_mode != PIC_LOSS_RADIAL && p->loss_mode != PIC_LOSS_NONE)
      return set_err(nullptr, PIC_EINVAL, "a bounded column needs PIC_LOSS_RADIAL or PIC_LOSS_NONE");
    if (!(p->J_emit_Am2 >= 0.0) || !(p->T_emit_eV >= 0.0))
      return set_err(nullptr, PIC_EINVAL, "emission current and temperature must be >= 0");
  }
  if (p->diag_every < 0) return set_err(nullptr, PIC_EINVAL, "diag_every < 0");
  if (p->diag_every > 0 && p->ion_subcycle > 0 && p->diag_every % p->ion_subcycle != 0)
    return set_err(nullptr, PIC_EINVAL, "diag_every must be a multiple of ion_subcycle");
  if (p->n_xsec < 0 || (p->n_xsec > 0 && !p->xsec)) return set_err(nullptr, PIC_EINVAL, "bad xsec list");
  int ne = 0, ni = 0;
  for (int x = 0; x < p->n_xsec; ++x) {
    const pic_xsec &xs = p->xsec[x];
    if (xs.kind < PIC_ELASTIC || xs.kind > PIC_ION_ISO || xs.n < 1 || !xs.energy_eV || !xs.sigma_m2)
      return set_err(nullptr, PIC_EINVAL, "bad cross section %d", x);
    for (int i = 1; i < xs.n; ++i)
      if (!(xs.energy_eV[i] >= xs.energy_eV[i - 1])) return set_err(nullptr, PIC_EINVAL, "xsec %d not ascending", x);
    if (!std::isfinite(xs.threshold_eV) || xs.threshold_eV < 0)
      return set_err(nullptr, PIC_EINVAL, "xsec %d: bad threshold", x);
    for (int i = 0; i < xs.n; ++i)
      if (!std::isfinite(xs.energy_eV[i]) || !std::isfinite(xs.sigma_m2[i]) || xs.sigma_m2[i] < 0)
        return set_err(nullptr, PIC_EINVAL, "xsec %d has a negative or non-finite value", x);
    (is_e_kind(xs.kind) ? ne : ni)++;
  }
  if (ne > pic::kMaxProc || ni > pic::kMaxProc) return set_err(nullptr, PIC_EINVAL, "at most %d processes per species", pic::kMaxProc);
  if (p->n_e0 > 0 && !(p->n0_m3 > 0) && p->field_mode == PIC_FIELD_POISSON)
    return set_err(nullptr, PIC_EINVAL, "n0 must be > 0");
  if (!(p->eps_max_e_eV > 0) || !(p->eps_max_i_eV > 0)) return set_err(nullptr, PIC_EINVAL, "eps_max must be > 0");
  if (p->column < 0 || p->column > 4095) return set_err(nullptr, PIC_EINVAL, "column must be in [0, 4095]");
  return 0;
}

template <class R> int init_typed(pic_handle *h) {
  int rc = setup_tables<R>(h);
  if (rc) return rc;
  rc = alloc_species<R>(h);
  if (rc) return rc;
  const size_t ms = (size_t)h->N + 1;   // moment arrays: one entry per node (N + 1 in a bounded column)
  h->m.ge = h->mom; h->m.ee = h->mom + ms; h->m.he = h->mom + 2 * ms; h->m.gi = h->mom + 3 * ms;
  h->m.ne = h->mom + 4 * ms; h->m.ni = h->mom + 5 * ms; h->m.E = h->mom + 6 * ms; h->m.phi = h->mom + 7 * ms;
  h->m.iz = h->mom_iz;
  return run_init<R>(h);
}

// ---------------------------------------------------------------------------
// batches

template <class R> pic::ColDev<R> coldev_of(pic_handle *c) {
  pic::ColDev<R> d{};
  d.k = kparams<R>(c);
  d.sp[0] = c->sp[0];
  d.sp[1] = c->sp[1];
  d.ctl = c->ctl;
  d.Ef = c->Ef;
  d.E = c->E;
  d.Eh = c->Eh;
  d.bb = bbuf<R>(c);
  d.sc = c->sc;
  d.m = c->m;
  d.fk = c->fk;
  d.fs = c->fs;
  d.N = c->N;
  pic::push_layout<R>(c->N, d.W, d.smemE, d.mofs, d.Wm);
  return d;
}

// CTA schedule of one species: mult x SMs CTAs, given to the columns in proportion to their
// particles (at least one each, and at least 1024 particles per CTA)
void build_schedule(pic_handle *b, int species, int mult, std::vector<int4> &out) {
  long long tot = 0;
  std::vector<long long> n(b->cols.size());
  for (size_t c = 0; c < b->cols.size(); ++c) {
    const pic_params &p = b->cols[c]->p;
    n[c] = species == 0 ? p.n_e0 : p.n_i0;
    tot += n[c];
  }
  const long long G = (long long)b->nsm * mult;
  for (size_t c = 0; c < b->cols.size(); ++c) {
    if (n[c] == 0) continue;
    long long k = tot > 0 ? (G * n[c] + tot - 1) / tot : 1;
    if (k < 1) k = 1;
    const long long per = (n[c] + k - 1) / k;
    if (per < 1024) k = (n[c] + 1023) / 1024;  // at least a full CTA of particles each
    for (long long i = 0; i < k; ++i) out.push_back(make_int4((int)c, (int)i, (int)k, 0));
  }
}

template <class R> int batch_schedules(pic_handle *b, int mult_e, int mult_i) {
  std::vector<int4> se, si;
  build_schedule(b, 0, mult_e, se);
  build_schedule(b, 1, mult_i, si);
  b->nsched[0] = (int)se.size();
  b->nsched[1] = (int)si.size();
  cudaFree(b->sched);
  b->sched = nullptr;
  std::vector<int4> all(se);
  all.insert(all.end(), si.begin(), si.end());
  if (all.empty()) all.push_back(make_int4(0, 0, 1, 0));
  CU(b, cudaMalloc(&b->sched, all.size() * sizeof(int4)));
  CU(b, cudaMemcpy(b->sched, all.data(), all.size() * sizeof(int4), cudaMemcpyHostToDevice));
  if (b->cycle) { cudaGraphExecDestroy(b->cycle); b->cycle = nullptr; }
  if (b->dcycle) { cudaGraphExecDestroy(b->dcycle); b->dcycle = nullptr; }
  return 0;
}

constexpr int kTuneRounds = 2;

// the autotuner's choices by batch shape, for the life of the process
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune_cache;

// shape of a batch: SMs, precision, columns, and per column its cells and particle counts
// rounded to powers of two
std::string tune_key(const pic_handle *b) {
  auto lg = [](long long v) { int k = 0; while ((1ll << k) < v) ++k; return k; };
  std::string k = std::to_string(b->nsm) + (b->mixed ? "m" : "d") + std::to_string(b->cols.size());
  for (const pic_handle *c : b->cols)
    k += ":" + std::to_string(lg(c->N)) + "," + std::to_string(lg(c->p.n_e0)) + "," + std::to_string(lg(c->p.n_i0));
  return k;
}
bool tune_lookup(pic_handle *b) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tune_cache.find(b->tune_key);
  if (it == g_tune_cache.end()) return false;
  b->mult[0] = it->second.first;
  b->mult[1] = it->second.second;
  return true;
}
void tune_store(pic_handle *b) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune_cache[b->tune_key] = {b->mult[0], b->mult[1]};
}

template <class R> int enqueue_batch_step(pic_handle *b) {
  pic_handle *c0 = b->cols[0];
  const int ncol = (int)b->cols.size();
  const int sub = c0->p.ion_subcycle;
  const bool ion_push = sub > 0 && (b->host_step % sub) == 0;
  const pic::ColDev<R> *cd = reinterpret_cast<const pic::ColDev<R> *>(b->coldev);
  const int se = c0->p.sort_every;
  if (se > 0 && b->host_step % se == 0) {
    t_begin(b);
    const long long pi = (long long)se * (sub > 0 ? sub : 1);
    // all columns of a species at once: one launch per phase of each radix pass
    const int sk = 3 * b->spasses + (b->spasses & 1);
    int nk = 0;
    for (int q = 0; q < 2; ++q) {
      if (q == 1 && b->host_step % pi != 0) break;
      if (b->stiles[q] == 0) continue;
      pic::launch_sort_batch<R>(b->scol[q], ncol, b->stiles[q], b->spasses, b->nsm, b->stream);
      nk += sk;
    }
    t_end(b, PIC_K_SORT, nk);
  }
  const bool diag = c0->p.diag_every > 0 && (b->host_step % c0->p.diag_every) == 0;
  // the kernel without the optional work when no column needs it on this step
  bool plain = !diag;
  for (pic_handle *c : b->cols)
    plain = plain && !(c->p.flags & PIC_FLAG_RECORD_CODES) && c->p.drive != PIC_DRIVE_CIRCUIT &&
            c->p.loss_mode != PIC_LOSS_RADIAL;
  t_begin(b);
  pic::launch_zero_q_batch<R>(cd, ncol, 0, b->maxN, b->stream);
  if (b->tune_mark == 0) cudaEventRecord(b->tune_ev[0], b->stream);
  pic::launch_push_batch<R>(cd, b->sched, b->nsched[0], 0, b->push_smem, plain, b->stream);
  if (b->tune_mark == 0) cudaEventRecord(b->tune_ev[1], b->stream);
  t_end(b, PIC_K_PUSH_E, 2);
  if (ion_push && b->nsched[1] > 0) {
    t_begin(b);
    pic::launch_zero_q_batch<R>(cd, ncol, 1, b->maxN, b->stream);
    if (b->tune_mark == 1) cudaEventRecord(b->tune_ev[0], b->stream);
    pic::launch_push_batch<R>(cd, b->sched + b->nsched[0], b->nsched[1], 1, b->push_smem, plain, b->stream);
    if (b->tune_mark == 1) cudaEventRecord(b->tune_ev[1], b->stream);
    t_end(b, PIC_K_PUSH_I, 2);
  }
  t_begin(b);
  pic::launch_births_batch<R>(cd, ncol, ion_push ? 1 : 0, b->stream);
  t_end(b, PIC_K_BIRTHS);
  t_begin(b);
  pic::launch_field_batch<R>(cd, ncol, b->maxN, c0->p.field_mode == PIC_FIELD_POISSON, diag, b->stream);
  t_end(b, PIC_K_FIELD, (c0->p.field_mode == PIC_FIELD_POISSON ? 2 : 1) + (diag ? 1 : 0));
  CU(b, cudaGetLastError());
  b->host_step++;
  for (pic_handle *c : b->cols) c->host_step = b->host_step;
  return 0;
}

// the ion cycle of steps s .. s+sub-1 as a captured graph replays it: 0 not replayed (it holds a
// sort, or a diagnostic sample after its first step), 1 plain, 2 a diagnostic sample on its first
// step only (diag_every is a multiple of ion_subcycle, so a sample falls on a cycle's first step)
static int cycle_kind(const pic_params &p, long long s, int sub) {
  int kind = 1;
  for (long long q = s; q < s + sub; ++q) {
    if (p.sort_every > 0 && q % p.sort_every == 0) return 0;
    if (p.diag_every > 0 && q % p.diag_every == 0) {
      if (q != s) return 0;
      kind = 2;
    }
  }
  return kind;
}

template <class R> int step_batch(pic_handle *b, int64_t n) {
  const int sub = b->cols[0]->p.ion_subcycle > 0 ? b->cols[0]->p.ion_subcycle : 1;
  const bool graphs = !(b->p.flags & PIC_FLAG_NO_GRAPH) && !b->timing;
  int64_t done = 0;
  while (done < n) {
    // autotuner (the schedule does not change results): each candidate multiplier of a species
    // is timed on that species' push kernel, kRounds times (the shortest counts); electrons
    // first, then ions on the steps that push them
    if (b->tune_sp < 2) {
      const int q = b->tune_sp;
      const bool ion_step = sub > 0 && b->host_step % sub == 0;
      if (b->nsched[q] == 0 || (q == 1 && b->cols[0]->p.ion_subcycle <= 0)) {
        b->tune_sp = q + 1;   // nothing to tune for this species
        if (b->tune_sp == 2) {
          tune_store(b);
          const int rc = batch_schedules<R>(b, b->mult[0], b->mult[1]);
          if (rc) return rc;
        }
        continue;
      }
      if (q == 1 && !ion_step) {
        const int rc = enqueue_batch_step<R>(b);
        if (rc) return rc;
        ++done;
        continue;
      }
      int m[2] = {b->mult[0], b->mult[1]};
      m[q] = b->mults[b->tune_i];
      int rc = batch_schedules<R>(b, m[0], m[1]);
      if (rc) return rc;
      b->tune_mark = q;
      rc = enqueue_batch_step<R>(b);
      b->tune_mark = -1;
      if (rc) return rc;
      CU(b, cudaEventSynchronize(b->tune_ev[1]));
      float ms = 0.f;
      CU(b, cudaEventElapsedTime(&ms, b->tune_ev[0], b->tune_ev[1]));
      if (b->tune_round == 0) b->tune_ms.push_back(ms);
      else b->tune_ms[b->tune_i] = std::min(b->tune_ms[b->tune_i], ms);
      if (++b->tune_i == (int)b->mults.size()) {
        b->tune_i = 0;
        if (++b->tune_round == kTuneRounds) {
          size_t best = 0;
          for (size_t i = 1; i < b->tune_ms.size(); ++i)
            if (b->tune_ms[i] < b->tune_ms[best]) best = i;
          b->mult[q] = b->mults[best];
          b->tune_ms.clear();
          b->tune_round = 0;
          b->tune_sp = q + 1;
          if (b->tune_sp == 2) tune_store(b);
        }
      }
      if (b->tune_sp == 2 || b->tune_sp != q) {
        rc = batch_schedules<R>(b, b->mult[0], b->mult[1]);
        if (rc) return rc;
      }
      ++done;
      continue;
    }
    const int kind =
        graphs && n - done >= sub && b->host_step % sub == 0 ? cycle_kind(b->cols[0]->p, b->host_step, sub) : 0;
    if (kind) {
      cudaGraphExec_t &gx = kind == 1 ? b->cycle : b->dcycle;
      int64_t *gl = kind == 1 ? b->cycle_launch : b->dcycle_launch;
      if (!gx) {
        // capture one ion cycle; the kernels read the step counter on the device, so it replays
        const long long s0 = b->host_step;
        int64_t before[PIC_K_CLASSES];
        for (int q = 0; q < PIC_K_CLASSES; ++q) before[q] = b->klaunch[q];
        cudaGraph_t g;
        CU(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int rc = 0;
        for (int q = 0; q < sub && !rc; ++q) rc = enqueue_batch_step<R>(b);
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        b->host_step = s0;
        for (pic_handle *c : b->cols) c->host_step = s0;
        if (rc) {
          if (e == cudaSuccess) cudaGraphDestroy(g);
          return rc;
        }
        if (e != cudaSuccess) return set_err(b, PIC_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&gx, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return set_err(b, PIC_ECUDA, "graph instantiation: %s", cudaGetErrorString(e));
        for (int q = 0; q < PIC_K_CLASSES; ++q) {   // the capture only recorded the launches
          gl[q] = b->klaunch[q] - before[q];
          b->klaunch[q] = before[q];
        }
      }
      CU(b, cudaGraphLaunch(gx, b->stream));
      for (int q = 0; q < PIC_K_CLASSES; ++q) b->klaunch[q] += gl[q];
      b->host_step += sub;
      for (pic_handle *c : b->cols) c->host_step = b->host_step;
      done += sub;
      continue;
    }
    const int rc = enqueue_batch_step<R>(b);
    if (rc) return rc;
    ++done;
    if (b->timing && b->ev_cls.size() > 1024) {
      CU(b, cudaStreamSynchronize(b->stream));
      t_collect(b);
    }
  }
  return 0;
}

template <class R> int init_batch_typed(pic_handle *b) {
  std::vector<pic::ColDev<R>> d;
  size_t smem = 0;
  for (pic_handle *c : b->cols) {
    d.push_back(coldev_of<R>(c));
    int W = 0, se = 0, mo = -1, wm = 0;
    const size_t by = pic::push_layout<R>(c->N, W, se, mo, wm);
    if (by > smem) smem = by;
    if (c->N > b->maxN) b->maxN = c->N;
  }
  b->push_smem = smem;
  // the batched field scan stages nodes in shared memory only when the largest column fits
  for (auto &x : d)
    if (b->maxN > pic::kFieldSmemMax) x.fk.smem = 0;
  CU(b, cudaMalloc(&b->coldev, d.size() * sizeof(pic::ColDev<R>)));
  CU(b, cudaMemcpy(b->coldev, d.data(), d.size() * sizeof(pic::ColDev<R>), cudaMemcpyHostToDevice));
  if (b->cols[0]->p.sort_every > 0) {
    // the batched sort's column tables (the arrays of a column do not move after pic_init)
    for (pic_handle *c : b->cols) b->spasses = std::max(b->spasses, pic::sort_passes(c->N));
    for (int q = 0; q < 2; ++q) {
      std::vector<pic::SortCol> t;
      int tile0 = 0;
      for (pic_handle *c : b->cols) {
        pic::SortCol e{};
        e.cell[0] = c->sp[q].cell; e.rec[0] = c->sp[q].rec; e.id[0] = c->sp[q].id;
        e.cell[1] = c->sb[q].cell; e.rec[1] = c->sb[q].rec; e.id[1] = c->sb[q].id;
        e.hist = c->sb[q].hist;
        e.n = &c->ctl->n[q];
        e.tile0 = tile0;
        e.ntiles = c->sp[q].cap > 0 && c->sb[q].hist ? pic::sort_tiles(c->sp[q].cap) : 0;
        tile0 += e.ntiles;
        t.push_back(e);
      }
      b->stiles[q] = tile0;
      CU(b, cudaMalloc(&b->scol[q], t.size() * sizeof(pic::SortCol)));
      CU(b, cudaMemcpy(b->scol[q], t.data(), t.size() * sizeof(pic::SortCol), cudaMemcpyHostToDevice));
    }
  }
  b->tune_key = tune_key(b);
  if (tune_lookup(b)) b->tune_sp = 2;
  CU(b, cudaEventCreate(&b->tune_ev[0]));
  CU(b, cudaEventCreate(&b->tune_ev[1]));
  return batch_schedules<R>(b, b->mult[0], b->mult[1]);
}

}  // namespace

extern "C" {

int pic_abi_version(void) { return PIC_ABI_VERSION; }

const char *pic_last_error(pic_handle *h) { return h ? h->err.c_str() : g_err.c_str(); }

int pic_check_stability(const pic_params *params, double out[2]) {
  if (!params) return set_err(nullptr, PIC_EINVAL, "params is NULL");
  if (int rc = check_finite(params)) return rc;
  pic_params ri;
  if (params->drive == PIC_DRIVE_RI) {   // the density of the column is the one eq. 2 gives
    if (resolve_ri(params, &ri)) return set_err(nullptr, PIC_EINVAL, "the (R, I) drive has no solution");
    params = &ri;
  }
  const pic_params &p = *params;
  if (!(p.dt_s > 0) || !(p.L_m > 0) || p.n_cells < 1 || !(p.n0_m3 >= 0) || !(p.Te0_eV >= 0))
    return set_err(nullptr, PIC_EINVAL, "dt, L, n_cells, n0 and Te0 must be positive");
  // Sec. II: dt < 0.2 / w_pe and dx < lambda_De at the initial density and electron temperature
  const double wpe = std::sqrt(p.n0_m3 * kQe * kQe / (kEps0 * kMe));
  const double lde = p.n0_m3 > 0 ? std::sqrt(kEps0 * p.Te0_eV / (p.n0_m3 * kQe)) : HUGE_VAL;
  const double dx = p.L_m / (double)p.n_cells;
  const double r0 = wpe * p.dt_s, r1 = lde > 0 ? dx / lde : HUGE_VAL;
  if (out) { out[0] = r0; out[1] = r1; }
  return (r0 < 0.2 ? 0 : (int)PIC_WARN_PLASMA_FREQ) | (r1 < 1.0 ? 0 : (int)PIC_WARN_DEBYE);
}

int pic_init(const pic_params *params, pic_handle **out) {
  if (!out) return set_err(nullptr, PIC_EINVAL, "out is NULL");
  *out = nullptr;
  pic_params ri;
  if (params && params->drive == PIC_DRIVE_RI) {   // resolve (R, I) -> (E0, n0), then run as the E0 drive
    if (int rc = check_finite(params)) return rc;
    if (resolve_ri(params, &ri)) return set_err(nullptr, PIC_EINVAL, "the (R, I) drive has no solution");
    params = &ri;
  }
  int rc = validate(params);
  if (rc) return rc;
  pic_handle *h = new (std::nothrow) pic_handle();
  if (!h) return set_err(nullptr, PIC_ENOMEM, "host allocation failed");
  h->p = *params;  // p.xsec is caller-owned: used during pic_init only, cleared below
  const pic_params &p = *params;
  h->N = p.n_cells;
  h->Nn = p.n_cells + ((p.flags & PIC_FLAG_BOUNDED) ? 1 : 0);
  h->ntab = p.n_table;
  h->mixed = p.precision == PIC_MIXED;
  h->M = p.gas_mass_amu * kAmu;
  h->ng = p.pressure_torr * kTorr / (kKb * p.T_gas_K);
  h->dx = p.L_m / (double)p.n_cells;
  h->w = p.n_e0 > 0 ? p.n0_m3 * p.L_m / (double)p.n_e0 : 0.0;
  h->Cfield = (kQe * h->w) / (kEps0 * kTwo32);
  h->E0 = p.drive == PIC_DRIVE_V ? p.V_applied / p.L_m : p.E0_Vpm;
  h->dt_i = (double)(p.ion_subcycle > 0 ? p.ion_subcycle : 1) * p.dt_s;
  const int64_t nmax = p.n_e0 > p.n_i0 ? p.n_e0 : p.n_i0;
  int64_t cap = p.capacity > 0 ? p.capacity : nmax + nmax / 4 + 1024;
  if (cap < nmax || cap > (int64_t)INT32_MAX) {
    delete h;
    return set_err(nullptr, PIC_EINVAL, "capacity out of range");
  }
  h->sp[0].cap = h->sp[1].cap = cap;
  int dev = 0;
  auto fail = [&](int code) {
    free_all(h);
    g_err = h->err.empty() ? g_err : h->err;
    delete h;
    return code;
  };
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(set_err(h, PIC_ECUDA, "no CUDA device"));
  if (cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(set_err(h, PIC_ECUDA, "device query failed"));
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(set_err(h, PIC_ECUDA, "stream creation failed"));
  if (cudaMalloc(&h->ctl, sizeof(pic::Ctl)) != cudaSuccess || cudaMalloc(&h->E, (size_t)(h->N + 1) * 8) != cudaSuccess ||
      cudaMalloc(&h->Eh, (size_t)h->N * 8) != cudaSuccess ||
      cudaMalloc(&h->fs, sizeof(pic::FieldScan)) != cudaSuccess ||
      cudaMalloc(&h->gauss, (pic::kGaussN + 1) * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&h->k3_mem, (size_t)pic::kStageCap * 7 * 4) != cudaSuccess ||
      cudaMalloc(&h->mom, (size_t)(h->N + 1) * 8 * 8) != cudaSuccess ||
      cudaMalloc(&h->mom_iz, (size_t)(h->N + 1) * 8) != cudaSuccess)
    return fail(set_err(h, PIC_ENOMEM, "device allocation failed"));
  cudaMemset(h->mom, 0, (size_t)(h->N + 1) * 8 * 8);
  cudaMemset(h->fs, 0, sizeof(pic::FieldScan));
  cudaMemset(h->mom_iz, 0, (size_t)(h->N + 1) * 8);
  h->sc.order = h->k3_mem;
  h->sc.cand = h->k3_mem + pic::kStageCap;
  h->sc.att = h->k3_mem + 2 * pic::kStageCap;
  h->sc.settled = h->k3_mem + 3 * pic::kStageCap;
  h->sc.win = h->k3_mem + 4 * pic::kStageCap;
  h->sc.vic = h->k3_mem + 5 * pic::kStageCap;
  std::vector<float> T(pic::kGaussN + 1);
  gauss_table(T.data());
  cudaMemcpy(h->gauss, T.data(), T.size() * sizeof(float), cudaMemcpyHostToDevice);
  pic::Ctl c{};
  c.n[0] = p.n_e0;
  c.n[1] = p.n_i0;
  c.step = 0;
  c.next_id = p.n_e0 + p.n_i0;
  c.E0 = h->E0;
  if (cudaMemcpy(h->ctl, &c, sizeof c, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(set_err(h, PIC_ECUDA, "control block upload failed"));
  h->fk.N = h->N;
  h->fk.bounded = (p.flags & PIC_FLAG_BOUNDED) ? 1 : 0;
  h->fk.field_mode = p.field_mode;
  h->fk.sub = p.ion_subcycle;
  h->fk.diag_every = 0;  // the initial solve takes no diagnostic sample
  h->fk.Cf = h->Cfield / ((double)h->N * (double)h->N);
  h->fk.dx = h->dx;
  h->fk.smem = h->N <= pic::kFieldSmemMax ? 1 : 0;
  h->fk.seg = (h->N + pic::kFieldThreads - 1) / pic::kFieldThreads;
  h->fk.circuit = p.drive == PIC_DRIVE_CIRCUIT ? 1 : 0;
  h->fk.Cj = kQe * h->w / (p.L_m * 256.0);
  h->fk.U = p.U_src;
  h->fk.Rext = p.R_ext_ohm_m2;
  h->fk.L = p.L_m;
  int rc2 = h->mixed ? init_typed<float>(h) : init_typed<double>(h);
  h->p.xsec = nullptr;
  h->p.n_xsec = 0;
  if (rc2) return fail(rc2);
  h->fk.diag_every = p.diag_every;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(set_err(h, PIC_ECUDA, "init failed"));
  if (check_status(h)) return fail(h->latched);
  *out = h;
  return 0;
}


int pic_step(pic_handle *h, int64_t n) {
  if (!h || n < 0) return set_err(h, PIC_EINVAL, "bad arguments");
  if (h->is_batch) return pic_step_batch(h, n);
  if (h->owner) return set_err(h, PIC_EINVAL, "a column of a batch advances with pic_step_batch");
  if (h->latched) return h->latched;
  const int sub = h->p.ion_subcycle > 0 ? h->p.ion_subcycle : 1;
  const bool graphs = !(h->p.flags & PIC_FLAG_NO_GRAPH) && !h->timing;
  int64_t done = 0;
  while (done < n) {
    const int kind = graphs && n - done >= sub && h->host_step % sub == 0 ? cycle_kind(h->p, h->host_step, sub) : 0;
    if (kind) {
      cudaGraphExec_t &gx = kind == 1 ? h->cycle : h->dcycle;
      int64_t *gl = kind == 1 ? h->cycle_launch : h->dcycle_launch;
      if (!gx) {
        // capture one ion cycle; the kernels read the step counter on the device, so it replays
        const long long s0 = h->host_step;
        int64_t before[PIC_K_CLASSES];
        for (int q = 0; q < PIC_K_CLASSES; ++q) before[q] = h->klaunch[q];
        cudaGraph_t g;
        CU(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        int rc = 0;
        for (int q = 0; q < sub && !rc; ++q) rc = h->mixed ? enqueue_step<float>(h) : enqueue_step<double>(h);
        cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        h->host_step = s0;
        if (rc) {
          if (e == cudaSuccess) cudaGraphDestroy(g);
          return rc;
        }
        if (e != cudaSuccess) return set_err(h, PIC_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&gx, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return set_err(h, PIC_ECUDA, "graph instantiation: %s", cudaGetErrorString(e));
        for (int q = 0; q < PIC_K_CLASSES; ++q) {   // the capture only recorded the launches
          gl[q] = h->klaunch[q] - before[q];
          h->klaunch[q] = before[q];
        }
      }
      CU(h, cudaGraphLaunch(gx, h->stream));
      for (int q = 0; q < PIC_K_CLASSES; ++q) h->klaunch[q] += gl[q];
      h->host_step += sub;
      done += sub;
      continue;
    }
    const int rc = h->mixed ? enqueue_step<float>(h) : enqueue_step<double>(h);
    if (rc) return rc;
    ++done;
    // keep the event pool bounded: fold recorded pairs every 256 steps
    if (h->timing && h->ev_cls.size() > 1024) {
      CU(h, cudaStreamSynchronize(h->stream));
      t_collect(h);
    }
  }
  const int rc = check_status(h);
  t_collect(h);
  return rc;
}

int pic_set_timing(pic_handle *h, int enable) {
  if (!h) return set_err(h, PIC_EINVAL, "bad arguments");
  CU(h, cudaStreamSynchronize(h->stream));
  t_collect(h);
  h->timing = enable != 0;
  return 0;
}

int pic_kernel_times(pic_handle *h, double *ms, int64_t *launches) {
  if (!h) return set_err(h, PIC_EINVAL, "bad arguments");
  CU(h, cudaStreamSynchronize(h->stream));
  t_collect(h);
  for (int c = 0; c < PIC_K_CLASSES; ++c) {
    if (ms) ms[c] = h->kms[c];
    if (launches) launches[c] = h->klaunch[c];
    h->kms[c] = 0.0;
    h->klaunch[c] = 0;
  }
  return 0;
}

int pic_init_batch(const pic_params *params, int n, pic_handle **out) {
  if (!out || !params || n < 1 || n > 4096) return set_err(nullptr, PIC_EINVAL, "bad arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (params[i].flags & PIC_FLAG_BOUNDED)
      return set_err(nullptr, PIC_EINVAL, "bounded columns run alone (column %d)", i);
  std::vector<pic_params> resolved;
  for (int i = 0; i < n; ++i)
    if (params[i].drive == PIC_DRIVE_RI) {
      resolved.assign(params, params + n);
      for (int k = 0; k < n; ++k)
        if (resolved[k].drive == PIC_DRIVE_RI && resolve_ri(&params[k], &resolved[k]))
          return set_err(nullptr, PIC_EINVAL, "the (R, I) drive of column %d has no solution", k);
      params = resolved.data();
      break;
    }
  for (int i = 0; i < n; ++i) {
    const int rc = validate(&params[i]);
    if (rc) return rc;
    if (params[i].dt_s != params[0].dt_s || params[i].ion_subcycle != params[0].ion_subcycle ||
        params[i].precision != params[0].precision || params[i].diag_every != params[0].diag_every ||
        params[i].sort_every != params[0].sort_every || params[i].field_mode != params[0].field_mode)
      return set_err(nullptr, PIC_EINVAL, "batched columns need equal dt, ion_subcycle, precision, diag_every, "
                                          "sort_every and field_mode");
  }
  pic_handle *b = new (std::nothrow) pic_handle();
  if (!b) return set_err(nullptr, PIC_ENOMEM, "host allocation failed");
  b->is_batch = true;
  b->p = params[0];
  b->p.xsec = nullptr;
  b->mixed = params[0].precision == PIC_MIXED;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return set_err(nullptr, PIC_ECUDA, "stream creation failed");
  }
  for (int i = 0; i < n; ++i) {
    pic_params pi = params[i];
    pi.column = i;  // the column index keys the column's random numbers
    pic_handle *c = nullptr;
    const int rc = pic_init(&pi, &c);
    if (rc) {
      free_all(b);
      delete b;
      return rc;
    }
    cudaStreamDestroy(c->stream);
    c->stream = b->stream;
    c->owner = b;
    b->cols.push_back(c);
  }
  b->mults = {1, 2, 3, 4, 6, 8};
  const int rc = b->mixed ? init_batch_typed<float>(b) : init_batch_typed<double>(b);
  if (rc) {
    free_all(b);
    delete b;
    return rc;
  }
  *out = b;
  return 0;
}

int pic_batch_schedule(pic_handle *b, int *mult_e, int *mult_i) {
  if (!b || !b->is_batch) return set_err(b, PIC_EINVAL, "not a batch handle");
  if (mult_e) *mult_e = b->mult[0];
  if (mult_i) *mult_i = b->mult[1];
  return b->tune_sp >= 2 ? 1 : 0;
}

int pic_step_batch(pic_handle *b, int64_t n) {
  if (!b || !b->is_batch || n < 0) return set_err(b, PIC_EINVAL, "not a batch handle");
  if (b->latched) return b->latched;
  const int rc = b->mixed ? step_batch<float>(b, n) : step_batch<double>(b, n);
  if (rc) return rc;
  int worst = 0;
  for (pic_handle *c : b->cols) {
    const int r = check_status(c);
    if (r && !worst) {
      worst = r;
      b->err = c->err;
    }
  }
  t_collect(b);
  b->latched = worst;
  return worst;
}

pic_handle *pic_batch_column(pic_handle *b, int i) {
  if (!b || !b->is_batch || i < 0 || i >= (int)b->cols.size()) return nullptr;
  return b->cols[i];
}

int pic_batch_size(pic_handle *b) { return (b && b->is_batch) ? (int)b->cols.size() : 0; }

int pic_get_stats(pic_handle *h, pic_stats *out) {
  if (!h || !out) return set_err(h, PIC_EINVAL, "bad arguments");
  pic::Ctl c;
  CU(h, cudaMemcpyAsync(&c, h->ctl, sizeof c, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  memset(out, 0, sizeof *out);
  out->step = c.step; out->n_e = c.n[0]; out->n_i = c.n[1]; out->next_id = c.next_id;
  for (int j = 0; j < pic::kMaxProc; ++j) { out->n_coll_e[j] = (int64_t)c.n_coll[0][j]; out->n_coll_i[j] = (int64_t)c.n_coll[1][j]; }
  out->births = (int64_t)c.births;
  out->losses_e = (int64_t)c.losses[0]; out->losses_i = (int64_t)c.losses[1];
  out->overflow_e = (int64_t)c.overflow[0]; out->overflow_i = (int64_t)c.overflow[1];
  out->E0 = c.E0;
  out->n_diag = c.n_diag;
  for (int q = 0; q < 2; ++q) {
    out->absorbed_e[q] = (int64_t)c.absorbed[0][q];
    out->absorbed_i[q] = (int64_t)c.absorbed[1][q];
  }
  out->emitted = (int64_t)c.emitted;
  return 0;
}

int pic_get_state(pic_handle *h, pic_state *o) {
  if (!h || !o) return set_err(h, PIC_EINVAL, "bad arguments");
  pic::Ctl c;
  CU(h, cudaMemcpyAsync(&c, h->ctl, sizeof c, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  o->n_e = c.n[0]; o->n_i = c.n[1]; o->step = c.step; o->next_id = c.next_id; o->E0 = c.E0;
  int32_t *cells[2] = {o->cell_e, o->cell_i};
  double *offs[2] = {o->off_e, o->off_i}, *vxs[2] = {o->vx_e, o->vx_i}, *vys[2] = {o->vy_e, o->vy_i},
         *vzs[2] = {o->vz_e, o->vz_i};
  uint64_t *ids[2] = {o->id_e, o->id_i};
  for (int q = 0; q < 2; ++q) {
    const int64_t n = c.n[q];
    if (n == 0) continue;
    if (cells[q]) CU(h, cudaMemcpy(cells[q], h->sp[q].cell, (size_t)n * 4, cudaMemcpyDeviceToHost));
    if (ids[q]) CU(h, cudaMemcpy(ids[q], h->sp[q].id, (size_t)n * 8, cudaMemcpyDeviceToHost));
    if (offs[q] || vxs[q] || vys[q] || vzs[q]) {
      if (h->mixed) {
        std::vector<float4> r((size_t)n);
        CU(h, cudaMemcpy(r.data(), h->sp[q].rec, (size_t)n * 16, cudaMemcpyDeviceToHost));
        for (int64_t p = 0; p < n; ++p) {
          if (offs[q]) offs[q][p] = r[p].x;
          if (vxs[q]) vxs[q][p] = r[p].y;
          if (vys[q]) vys[q][p] = r[p].z;
          if (vzs[q]) vzs[q][p] = r[p].w;
        }
      } else {
        std::vector<pic::D4> r((size_t)n);
        CU(h, cudaMemcpy(r.data(), h->sp[q].rec, (size_t)n * 32, cudaMemcpyDeviceToHost));
        for (int64_t p = 0; p < n; ++p) {
          if (offs[q]) offs[q][p] = r[p].off;
          if (vxs[q]) vxs[q][p] = r[p].vx;
          if (vys[q]) vys[q][p] = r[p].vy;
          if (vzs[q]) vzs[q][p] = r[p].vz;
        }
      }
    }
  }
  if (o->E) CU(h, cudaMemcpy(o->E, h->E, (size_t)h->Nn * 8, cudaMemcpyDeviceToHost));
  if (o->Q_e) CU(h, cudaMemcpy(o->Q_e, h->sp[0].Q, (size_t)h->Nn * 8, cudaMemcpyDeviceToHost));
  if (o->Q_i) CU(h, cudaMemcpy(o->Q_i, h->sp[1].Q, (size_t)h->Nn * 8, cudaMemcpyDeviceToHost));
  return 0;
}

}  // extern "C"

// pic_set_state's arrays, with the offsets and velocities in FP64 or FP32 (In)
template <class In> struct StateIn {
  int64_t n_e, n_i, step, next_id;
  double E0;
  const int32_t *cell[2];
  const In *off[2], *vx[2], *vy[2], *vz[2];
  const uint64_t *id[2];
  const double *E;
  const int64_t *Q_i;
};

template <class In> static int set_state_in(pic_handle *h, const StateIn<In> &st) {
  const StateIn<In> *in = &st;
  if (in->n_e < 0 || in->n_i < 0 || in->n_e > h->sp[0].cap || in->n_i > h->sp[1].cap)
    return set_err(h, PIC_EINVAL, "particle count out of range");
  if (in->step < 0) return set_err(h, PIC_EINVAL, "step < 0");
  if (h->is_batch) return set_err(h, PIC_EINVAL, "set the state of the batch's columns");
  if (h->owner && in->step != h->owner->host_step)
    return set_err(h, PIC_EINVAL, "a column of a batch keeps the batch's step counter");
  CU(h, cudaStreamSynchronize(h->stream));
  const int32_t *const *cells = in->cell;
  const In *const *offs = in->off, *const *vxs = in->vx, *const *vys = in->vy, *const *vzs = in->vz;
  const uint64_t *const *ids = in->id;
  const int64_t ns[2] = {in->n_e, in->n_i};
  // the arrays go to the device as given (cells and ids to their places, offsets and velocities
  // to a staging area), then one kernel per species checks the grid and writes the records
  for (int q = 0; q < 2; ++q)
    if (ns[q] > 0 && (!cells[q] || !offs[q] || !vxs[q] || !vys[q] || !vzs[q] || !ids[q]))
      return set_err(h, PIC_EINVAL, "missing state array");
  if (!h->stage && (ns[0] > 0 || ns[1] > 0)) {
    const int64_t cap = std::max(h->sp[0].cap, h->sp[1].cap);
    if (cudaMalloc(&h->stage, (size_t)cap * 4 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->stage_bad, 2 * sizeof(unsigned long long)) != cudaSuccess) {
      cudaFree(h->stage);
      h->stage = nullptr;
      return set_err(h, PIC_ENOMEM, "no device memory for the state upload");
    }
  }
  unsigned long long bad[2] = {~0ull, ~0ull};
  for (int q = 0; q < 2; ++q) {
    const int64_t n = ns[q];
    if (n == 0) continue;
    const size_t b8 = (size_t)n * 8, bv = (size_t)n * sizeof(In);
    In *stg = reinterpret_cast<In *>(h->stage);   // 4n values of In fit the 4 cap doubles
    CU(h, cudaMemcpyAsync(h->sp[q].cell, cells[q], (size_t)n * 4, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(h->sp[q].id, ids[q], b8, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(stg, offs[q], bv, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(stg + n, vxs[q], bv, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(stg + 2 * n, vys[q], bv, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(stg + 3 * n, vzs[q], bv, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(h->stage_bad + q, &bad[q], 8, cudaMemcpyHostToDevice, h->stream));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)h->nsm * 8);
    if (h->mixed)
      k_set_rec<float, In><<<blocks, 256, 0, h->stream>>>(h->sp[q].cell, stg, n, h->N, h->sp[q].rec,
                                                           h->stage_bad + q);
    else
      k_set_rec<double, In><<<blocks, 256, 0, h->stream>>>(h->sp[q].cell, stg, n, h->N, h->sp[q].rec,
                                                            h->stage_bad + q);
    CU(h, cudaGetLastError());
    CU(h, cudaMemcpyAsync(&bad[q], h->stage_bad + q, 8, cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));   // the staging area is reused by the next species
  }
  for (int q = 0; q < 2; ++q)
    if (bad[q] != ~0ull)
      return set_err(h, PIC_EINVAL, "particle %lld of species %d outside the grid", (long long)bad[q], q);
  pic::Ctl c;
  CU(h, cudaMemcpy(&c, h->ctl, sizeof c, cudaMemcpyDeviceToHost));
  c.n[0] = in->n_e; c.n[1] = in->n_i; c.step = in->step; c.next_id = in->next_id; c.E0 = in->E0;
  c.emit_acc = 0.0;
  c.status = 0; c.n_birth = 0; c.n_dead[0] = c.n_dead[1] = 0;
  c.sumv[0] = c.sumv[1] = 0;
  CU(h, cudaMemcpy(h->ctl, &c, sizeof c, cudaMemcpyHostToDevice));
  if (h->p.drive == PIC_DRIVE_CIRCUIT) {
    if (h->mixed) pic::launch_sumv<float>(h->sp[1], h->ctl, 1, h->stream);
    else pic::launch_sumv<double>(h->sp[1], h->ctl, 1, h->stream);
  }
  h->latched = 0;
  h->host_step = in->step;
  CU(h, cudaMemset(h->sp[0].Q, 0, (size_t)h->Nn * 8));
  if (h->mixed) pic::launch_deposit<float>(h->kf, h->sp[0], h->ctl, 0, h->stream);
  else pic::launch_deposit<double>(h->kd, h->sp[0], h->ctl, 0, h->stream);
  if (in->Q_i) {
    CU(h, cudaMemcpyAsync(h->sp[1].Q, in->Q_i, (size_t)h->Nn * 8, cudaMemcpyHostToDevice, h->stream));
  } else {
    CU(h, cudaMemsetAsync(h->sp[1].Q, 0, (size_t)h->Nn * 8, h->stream));
    if (h->mixed) pic::launch_deposit<float>(h->kf, h->sp[1], h->ctl, 1, h->stream);
    else pic::launch_deposit<double>(h->kd, h->sp[1], h->ctl, 1, h->stream);
  }
  if (in->E) {
    CU(h, cudaMemcpyAsync(h->E, in->E, (size_t)h->Nn * 8, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    const bool bounded = h->Nn > h->N;   // the gather copy's node N: the anode node, or node 0 again
    if (h->mixed) {
      std::vector<float> f((size_t)h->N + 1);
      for (int j = 0; j < h->N; ++j) f[j] = (float)in->E[j];
      f[h->N] = bounded ? (float)in->E[h->N] : f[0];
      CU(h, cudaMemcpy(h->Ef, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
    } else {
      std::vector<double> f((size_t)h->N + 1);
      for (int j = 0; j < h->N; ++j) f[j] = in->E[j];
      f[h->N] = bounded ? in->E[h->N] : f[0];
      CU(h, cudaMemcpy(h->Ef, f.data(), f.size() * 8, cudaMemcpyHostToDevice));
    }
  } else {
    // solve the field of the new charges without advancing the step counter
    if (h->mixed)
      pic::launch_field<float>(h->fk, h->sp[0].Q, h->sp[1].Q, h->ctl, h->E, h->Eh, reinterpret_cast<float *>(h->Ef),
                               h->m, h->fs, false, false, h->stream);
    else
      pic::launch_field<double>(h->fk, h->sp[0].Q, h->sp[1].Q, h->ctl, h->E, h->Eh,
                                reinterpret_cast<double *>(h->Ef), h->m, h->fs, false, false, h->stream);
  }
  CU(h, cudaStreamSynchronize(h->stream));
  CU(h, cudaGetLastError());
  return check_status(h);
}

template <class In, class S> static StateIn<In> state_view(const S *in) {
  StateIn<In> v;
  v.n_e = in->n_e;
  v.n_i = in->n_i;
  v.step = in->step;
  v.next_id = in->next_id;
  v.E0 = in->E0;
  v.cell[0] = in->cell_e; v.cell[1] = in->cell_i;
  v.off[0] = in->off_e; v.off[1] = in->off_i;
  v.vx[0] = in->vx_e; v.vx[1] = in->vx_i;
  v.vy[0] = in->vy_e; v.vy[1] = in->vy_i;
  v.vz[0] = in->vz_e; v.vz[1] = in->vz_i;
  v.id[0] = in->id_e; v.id[1] = in->id_i;
  v.E = in->E;
  v.Q_i = in->Q_i;
  return v;
}

extern "C" {

int pic_set_state(pic_handle *h, const pic_state *in) {
  if (!h || !in) return set_err(h, PIC_EINVAL, "bad arguments");
  return set_state_in<double>(h, state_view<double>(in));
}

int pic_set_state_f32(pic_handle *h, const pic_state_f32 *in) {
  if (!h || !in) return set_err(h, PIC_EINVAL, "bad arguments");
  return set_state_in<float>(h, state_view<float>(in));
}

int pic_eepf_config(pic_handle *h, int32_t n_x, int32_t n_eps, double eps_max_eV) {
  if (!h) return set_err(h, PIC_EINVAL, "bad arguments");
  if (h->is_batch || h->owner) return set_err(h, PIC_EINVAL, "the EEPF histogram is for single columns");
  if (n_x < 0 || n_x > h->N || (n_x > 0 && (n_eps < 1 || n_eps > 65536 || !(eps_max_eV > 0.0))))
    return set_err(h, PIC_EINVAL, "bad EEPF histogram shape");
  CU(h, cudaStreamSynchronize(h->stream));
  cudaFree(h->m.eepf);
  h->m.eepf = nullptr;
  h->m.eepf_nx = 0;
  h->m.eepf_ne = 0;
  if (n_x == 0) return 0;
  const size_t bytes = (size_t)n_x * (size_t)(n_eps + 1) * 8;
  if (cudaMalloc(&h->m.eepf, bytes) != cudaSuccess) {
    h->m.eepf = nullptr;
    return set_err(h, PIC_ENOMEM, "no device memory for the EEPF histogram");
  }
  CU(h, cudaMemset(h->m.eepf, 0, bytes));
  h->m.eepf_nx = n_x;
  h->m.eepf_ne = n_eps;
  h->m.eepf_scale = (double)n_eps / eps_max_eV;
  pic::Ctl c;
  CU(h, cudaMemcpy(&c, h->ctl, sizeof c, cudaMemcpyDeviceToHost));
  h->eepf_base = c.n_diag;
  // the captured ion cycles hold the old histogram in their kernel parameters
  if (h->cycle) {
    cudaGraphExecDestroy(h->cycle);
    h->cycle = nullptr;
  }
  if (h->dcycle) {
    cudaGraphExecDestroy(h->dcycle);
    h->dcycle = nullptr;
  }
  return 0;
}

int pic_eepf_get(pic_handle *h, uint64_t *counts, int64_t *n_samples, int32_t reset) {
  if (!h || !h->m.eepf) return set_err(h, PIC_EINVAL, "no EEPF histogram (pic_eepf_config)");
  const size_t n = (size_t)h->m.eepf_nx * (size_t)(h->m.eepf_ne + 1);
  pic::Ctl c;
  CU(h, cudaMemcpyAsync(&c, h->ctl, sizeof c, cudaMemcpyDeviceToHost, h->stream));
  if (counts) CU(h, cudaMemcpyAsync(counts, h->m.eepf, n * 8, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  if (n_samples) *n_samples = c.n_diag - h->eepf_base;
  if (reset) {
    CU(h, cudaMemset(h->m.eepf, 0, n * 8));
    h->eepf_base = c.n_diag;
  }
  return 0;
}

int pic_moments(pic_handle *h, pic_moments_out *o) {
  if (!h || !o) return set_err(h, PIC_EINVAL, "bad arguments");
  const int N = h->Nn;                       // nodes
  const size_t ms = (size_t)h->N + 1;        // stride of the device moment arrays
  std::vector<double> acc(ms * 8);
  std::vector<unsigned long long> iz(ms);
  pic::Ctl c;
  CU(h, cudaMemcpyAsync(&c, h->ctl, sizeof c, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaMemcpyAsync(acc.data(), h->mom, acc.size() * 8, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaMemcpyAsync(iz.data(), h->mom_iz, iz.size() * 8, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  const double *ge = acc.data(), *ee = ge + ms, *he = ge + 2 * ms, *gi = ge + 3 * ms, *ne = ge + 4 * ms,
               *ni = ge + 5 * ms, *E = ge + 6 * ms, *phi = ge + 7 * ms;
  const double ns = c.m_samples > 0 ? (double)c.m_samples : 1.0;
  const double dens = h->w / h->dx;
  const double tsteps = (double)(c.m_steps > 0 ? c.m_steps : 1) * h->p.dt_s;
  o->n_samples = c.m_samples;
  o->n_steps = c.m_steps;
  for (int j = 0; j < N; ++j) {
    if (o->n_e) o->n_e[j] = ne[j] / ns * dens;
    if (o->n_i) o->n_i[j] = ni[j] / ns * dens;
    if (o->gamma_e) o->gamma_e[j] = ge[j] / ns * dens;
    if (o->mean_eps_e) o->mean_eps_e[j] = ne[j] > 0 ? ee[j] / ne[j] : 0.0;
    if (o->heat_e) o->heat_e[j] = he[j] / ns * dens;
    if (o->iz_rate) o->iz_rate[j] = (double)(long long)iz[j] * (1.0 / kTwo32) * dens / tsteps;
    if (o->gamma_i) o->gamma_i[j] = gi[j] / ns * dens;
    if (o->E) o->E[j] = E[j] / ns;
    if (o->phi) o->phi[j] = phi[j] / ns;
  }
  if (o->reset) {
    CU(h, cudaMemsetAsync(h->mom, 0, ms * 8 * 8, h->stream));
    CU(h, cudaMemsetAsync(h->mom_iz, 0, ms * 8, h->stream));
    long long z[3] = {0, 0, 0};  // m_samples, m_steps (n_diag kept)
    CU(h, cudaMemcpyAsync(&h->ctl->m_samples, &z[0], 8, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(&h->ctl->m_steps, &z[1], 8, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
  }
  return 0;
}

int pic_last_codes(pic_handle *h, int species, int32_t *out, int64_t n) {
  if (!h || !out || species < 0 || species > 1 || n < 0 || n > h->sp[species].cap)
    return set_err(h, PIC_EINVAL, "bad arguments");
  if (!h->sp[species].code) return set_err(h, PIC_EINVAL, "codes need PIC_FLAG_RECORD_CODES");
  CU(h, cudaStreamSynchronize(h->stream));
  CU(h, cudaMemcpy(out, h->sp[species].code, (size_t)n * 4, cudaMemcpyDeviceToHost));
  return 0;
}

int pic_derived(pic_handle *h, double out[7]) {
  if (!h || !out) return set_err(h, PIC_EINVAL, "bad arguments");
  out[0] = h->ng; out[1] = h->nustar[0]; out[2] = h->Pnull[0]; out[3] = h->nustar[1]; out[4] = h->Pnull[1];
  out[5] = h->w; out[6] = h->dx;
  return 0;
}

void *pic_stream(pic_handle *h) { return h ? (void *)h->stream : nullptr; }

void pic_free(pic_handle *h) {
  if (!h || h->owner) return;  // columns of a batch are freed with the batch
  free_all(h);
  delete h;
}

int pic_field_periodic(const int64_t *Q_i, const int64_t *Q_e, int n_cells, double C, double E0, double *E,
                       double *E_half, void *stream) {
  if (!Q_i || !Q_e || !E || !E_half || n_cells < 3 || n_cells > 65536)
    return set_err(nullptr, PIC_EINVAL, "bad arguments");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int N = n_cells;
  pic::Ctl *ctl = nullptr;
  pic::FieldScan *fs = nullptr;
  double *Ef = nullptr;
  int rc = 0;
  if (cudaMalloc(&ctl, sizeof(pic::Ctl)) != cudaSuccess || cudaMalloc(&fs, sizeof(pic::FieldScan)) != cudaSuccess ||
      cudaMalloc(&Ef, ((size_t)N + 1) * 8) != cudaSuccess) {
    rc = set_err(nullptr, PIC_ENOMEM, "device allocation failed");
  } else {
    pic::Ctl c{};
    c.E0 = E0;
    cudaMemsetAsync(fs, 0, sizeof(pic::FieldScan), st);
    pic::FieldK f{};
    f.N = N;
    f.field_mode = PIC_FIELD_POISSON;
    f.smem = N <= pic::kFieldSmemMax ? 1 : 0;
    f.seg = (N + pic::kFieldThreads - 1) / pic::kFieldThreads;
    f.Cf = C / ((double)N * (double)N);
    if (cudaMemcpyAsync(ctl, &c, sizeof c, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = set_err(nullptr, PIC_ECUDA, "upload failed");
    } else {
      pic::launch_field<double>(f, reinterpret_cast<const unsigned long long *>(Q_e),
                                reinterpret_cast<const unsigned long long *>(Q_i), ctl, E, E_half, Ef, pic::Moments{},
                                fs, false, false, st);
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaMemcpyAsync(&c, ctl, sizeof c, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = set_err(nullptr, PIC_ECUDA, "%s", cudaGetErrorString(e));
      else if (c.status & pic::kStNonFinite) rc = set_err(nullptr, PIC_ENONFINITE, "the field became non-finite");
    }
  }
  cudaFree(ctl); cudaFree(fs); cudaFree(Ef);
  return rc;
}

int pic_test_i128_to_double(const int64_t *hi, const uint64_t *lo, double *out, int n) {
  if (!hi || !lo || !out || n < 0) return set_err(nullptr, PIC_EINVAL, "bad arguments");
  if (n == 0) return 0;
  int64_t *dh = nullptr;
  uint64_t *dl = nullptr;
  double *dout = nullptr;
  if (cudaMalloc(&dh, (size_t)n * 8) != cudaSuccess || cudaMalloc(&dl, (size_t)n * 8) != cudaSuccess ||
      cudaMalloc(&dout, (size_t)n * 8) != cudaSuccess) {
    cudaFree(dh); cudaFree(dl); cudaFree(dout);
    return set_err(nullptr, PIC_ENOMEM, "device allocation failed");
  }
  cudaMemcpy(dh, hi, (size_t)n * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dl, lo, (size_t)n * 8, cudaMemcpyHostToDevice);
  pic::launch_i128_test(dh, dl, dout, n, nullptr);
  const cudaError_t e = cudaMemcpy(out, dout, (size_t)n * 8, cudaMemcpyDeviceToHost);
  cudaFree(dh); cudaFree(dl); cudaFree(dout);
  if (e != cudaSuccess) return set_err(nullptr, PIC_ECUDA, "%s", cudaGetErrorString(e));
  return 0;
}

}  // extern "C"
