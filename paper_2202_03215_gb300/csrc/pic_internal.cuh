// Internal types shared by the host driver (pic_host.cu) and the kernels
// (pic_kernels.cu) of the PIC-MCC library.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pic.h"

namespace pic {

constexpr int kMaxProc = 16;   // collision processes per species
constexpr int kGaussN = 4096;          // Gaussian inverse-CDF intervals
constexpr int kStageCap = 8192;        // births / radial losses staged per step and species
constexpr int kFieldThreads = 1024;
constexpr int kStepThreads = 1024;
constexpr int kFieldSmemMax = 24576;   // nodes whose int64 charges fit in shared memory

// device status bits
constexpr unsigned kStBirthOverflow = 1u;
constexpr unsigned kStCapacity = 2u;
constexpr unsigned kStNonFinite = 4u;
constexpr unsigned kStDeadOverflow = 8u;
constexpr unsigned kStVictim = 16u;
constexpr unsigned kStTimeout = 32u;    // a bounded wait of the particle step gave up
// particle arrays hold this many slots past their capacity: the bulk copies of a tile round its
// length up to a multiple of 4 slots
constexpr int kPad = 64;

// random-number streams (counter word 3 = stream<<28 | column<<16 | block)
enum Stream : uint32_t { kStE = 0, kStI = 1, kStInitE = 2, kStInitI = 3, kStVicE = 4, kStVicI = 5, kStEmit = 6 };

// FP64 particle record (offset in cell, velocity); MIXED uses float4 with the same order
struct alignas(32) D4 { double off, vx, vy, vz; };

template <class R> struct Rec;
template <> struct Rec<double> { using T = D4; };
template <> struct Rec<float> { using T = float4; };

// device control block
struct Ctl {
  long long n[2];          // live particles per species
  long long step;          // steps taken
  long long next_id;
  double E0;
  unsigned int status;
  int n_birth;             // staged births of the current step
  int n_dead[2];           // staged radial losses
  int pad;
  unsigned long long n_coll[2][kMaxProc];
  unsigned long long births, losses[2], overflow[2];
  long long n_diag, m_samples, m_steps;
  long long sumv[2];       // circuit drive: sum of round(256 vx), electrons of this step, ions of their last push
  unsigned long long absorbed[2][2];   // bounded column: particles taken by [species][cathode, anode]
  unsigned long long emitted;          // bounded column: electrons emitted by the cathode
  double emit_acc;                     // bounded column: fraction of a macro-electron carried to the next step
};

struct SpeciesDev {
  int32_t *cell;
  void *rec;               // D4 or float4 records
  uint64_t *id;
  int32_t *code;           // optional per-particle process code
  unsigned long long *Q;   // node charge (fixed point, two's complement)
  int32_t *dead;           // staged radial losses (kStageCap)
  int64_t cap;
};

template <class R> struct SpecK {
  R a, d, K, inv_de, P, nus;      // kick q dt/m, drift dt/dx, energy m/2e, 1/deps, P_null, nu*
  uint32_t Pw;                    // radial loss threshold on a 32-bit word
  int np;
  int kind[kMaxProc];
  int xs[kMaxProc];               // index of the process in the caller's xsec list
  R thr[kMaxProc];
  const R *tab;                   // np x ntab collision frequencies
  const R *nub, *Pb;              // electrons: per energy bin majorant and its null-collision probability
  // FP32 form: the null-collision tests as integer compares on the top 24 bits of the decision
  // word, (w >> 8) < ceil(P 2^24), the same decision as the FP32 compare (w >> 8) 2^-24 < P
  const uint32_t *Pbi;            // electrons, per energy bin
  uint32_t Pi;                    // the species' global P_null
};

template <class R> struct StepK {
  int N, ntab, loss_mode, field_mode;
  int drive, pad_;
  unsigned flags;
  int diag_every, sub;
  uint32_t column;
  uint64_t seed;
  uint32_t rk[10][2];             // Philox round keys of seed: key + r (0x9E3779B9, 0xBB67AE85)
  int bounded, Nw;                // bounded column (Sec. V); nodes of the charge arrays (N, or N + 1)
  double emit_per_step;           // bounded column: J_emit dt / (e w) macro-electrons per step
  R sig_emit, emit_dtdx;          // (e T_emit / m)^(1/2); dt / dx
  R V_e, em, sig_n;               // 2e/m, 2m/M, sqrt(kT_g/M)
  const float *gauss;             // kGaussN+1 entries
  SpecK<R> sp[2];
};

template <class R> struct BirthBuf {
  int32_t *parent, *cell;
  R *off, *ve, *vi;               // ve, vi: 3 * kStageCap (component-major)
};

struct Moments {
  double *ge, *ee, *he, *gi, *ne, *ni, *E, *phi;
  unsigned long long *iz;
  unsigned long long *eepf;   // electron energy histogram, eepf_nx x (eepf_ne + 1), or null
  int eepf_nx, eepf_ne;
  double eepf_scale;          // eepf_ne / eps_max (rounded to the storage precision at the use)
};

struct K3Scratch {
  uint32_t *order;   // births sorted by parent slot -> staging index
  uint32_t *cand, *att, *settled, *win;
  uint32_t *vic;     // 2 * kStageCap victim slots (electrons, ions)
};

// exact integer data handed from the reduction kernel to the evaluation kernel
constexpr int kEvalThreads = 256;                         // nodes per block of the field kernels
constexpr int kFieldBlocksMax = 65536 / kEvalThreads;     // n_cells <= 65536
struct FieldScan {
  __int128 R[kFieldBlocksMax];     // per node block: sum of D
  __int128 U[kFieldBlocksMax];     // per node block: sum of (N - k) D_k
  __int128 Sp0[kFieldBlocksMax];   // S'_{j0 - 1} at the start of each node block
  __int128 T, M;
  unsigned int ticket;             // blocks done (the last one finishes, then resets it)
};

struct FieldK {
  int N, field_mode, sub, diag_every;
  int bounded, pad_;  // bounded column (Sec. V): Dirichlet field, node arrays of N + 1
  int smem;           // node arrays staged in shared memory (N <= kFieldSmemMax)
  int seg;            // nodes per thread segment: ceil(N / kFieldThreads)
  int circuit;        // E0 = (U - R_ext J) / L after every step (Sec. V)
  double Cj, U, Rext, L;   // J = Cj (sum_i - sum_e); source voltage; resistor (Ohm m^2); length
  double Cf;          // e w / (eps0 2^32 N^2)
  double dx;
};

// device descriptor of one column of a batch (everything the step kernels need)
template <class R> struct ColDev {
  StepK<R> k;
  SpeciesDev sp[2];
  Ctl *ctl;
  void *Ef;
  double *E, *Eh;
  BirthBuf<R> bb;
  K3Scratch sc;
  Moments m;
  FieldK fk;
  FieldScan *fs;
  int W, smemE;   // shared-memory layout of the particle step for this column
  int mofs, Wm;   // byte offset of its diagnostic moment bins (-1: none) and their window
  int N;
};

// second set of particle buffers and digit histograms for the sort
struct SortBuf {
  int32_t *cell;
  void *rec;
  uint64_t *id;
  unsigned *hist;
};

// one column's sort of one species in a batch: buffers 0 are the species arrays, buffers 1 the
// sort buffers; hist holds ntiles * 128 + 128 words (sort_hist_words(cap))
struct SortCol {
  int32_t *cell[2];
  void *rec[2];
  uint64_t *id[2];
  unsigned *hist;
  const long long *n;   // live particles (device)
  int tile0, ntiles;
};

// sort (pic_sort.cu)
int sort_passes(int n_cells);
int sort_tiles(int64_t cap);
size_t sort_hist_words(int64_t cap);
template <class R>
void launch_sort_batch(const SortCol *cols, int ncols, int total_tiles, int passes, int nsm, cudaStream_t st);
template <class R>
void launch_sort(SpeciesDev s, SortBuf alt, const long long *n_dev, long long cap, int n_cells, int nsm,
                 cudaStream_t st);

// launchers (pic_kernels.cu)
template <class R>
void launch_init(const StepK<R> &k, SpeciesDev s, int species, int64_t n, uint64_t id0, R sig, cudaStream_t st);
template <class R>
void launch_deposit(const StepK<R> &k, SpeciesDev s, const Ctl *ctl, int species, cudaStream_t st);
template <class R>
void launch_halfstep(const StepK<R> &k, SpeciesDev s, const Ctl *ctl, const R *Ef, int species, cudaStream_t st);
// ctl->sumv[species] += sum of round(256 vx) over the species (circuit drive start)
template <class R> void launch_sumv(SpeciesDev s, Ctl *ctl, int species, cudaStream_t st);
template <class R>
void launch_push(const StepK<R> &k, SpeciesDev s, Ctl *ctl, const R *Ef, BirthBuf<R> bb, Moments m,
                 int species, int nsm, bool diag_step, cudaStream_t st);
template <class R>
void launch_births(const StepK<R> &k, SpeciesDev e, SpeciesDev i, Ctl *ctl, BirthBuf<R> bb, K3Scratch sc,
                   int ion_pushed, cudaStream_t st);
// field solve; diag: take a diagnostic sample; advance: count the step
template <class R>
void launch_field(const FieldK &f, const unsigned long long *Qe, const unsigned long long *Qi, Ctl *ctl,
                  double *E, double *Eh, R *Ef, Moments m, FieldScan *fs, bool diag, bool advance, cudaStream_t st);
void launch_i128_test(const int64_t *hi, const uint64_t *lo, double *out, int n, cudaStream_t st);
template <class R> int push_smem_bytes(int N);
// shared-memory layout of the particle step for n_cells: bin window W, node field in shared memory
template <class R> size_t push_layout(int n_cells, int &W, int &smemE, int &mofs, int &Wm);

// batched columns (one launch per phase for all columns)
template <class R> void launch_zero_q_batch(const ColDev<R> *cols, int ncol, int species, int maxN, cudaStream_t st);
template <class R>
void launch_push_batch(const ColDev<R> *cols, const int4 *sched, int nblocks, int species, size_t smem, bool plain,
                       cudaStream_t st);
template <class R> void launch_births_batch(const ColDev<R> *cols, int ncol, int ion_pushed, cudaStream_t st);
template <class R>
void launch_field_batch(const ColDev<R> *cols, int ncol, int maxN, bool poisson, bool diag, cudaStream_t st);

}  // namespace pic
