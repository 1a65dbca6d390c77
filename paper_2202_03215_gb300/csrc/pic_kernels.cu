// CUDA kernels of the 1D3V electrostatic PIC-MCC positive-column step
// (Boeuf, Sec. II; the bounded column of Sec. V), written for sm_103a.
//
//   k_push      field gather, leapfrog push, periodic wrap (or absorption at the
//               electrodes of a bounded column), null-collision MCC, radial-loss
//               flag, birth staging, cloud-in-cell deposit into shared-memory
//               64-bit fixed-point bins (one persistent CTA per SM)
//   k_births    ionization births and the paired random removal (or radial
//               losses and absorbed particles with compaction; cathode emission
//               of a bounded column); one CTA
//   k_field_reduce / k_field_eval   Poisson solve by the exact integer route
//               (periodic, or Dirichlet between two electrodes), blocks of
//               nodes, the last block to finish forms the totals
//   k_init / k_deposit / k_halfstep   initial state
#include <cstdint>

#include "pic_device.cuh"

namespace pic {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kDirectMax = 1024;   // births handled by O(n^2) ranking instead of a sort
constexpr int kBirthThreads = 512;

template <class R> __device__ __forceinline__ void rec_load(const void *base, long long p, R &off, R &vx, R &vy, R &vz) {
  if constexpr (std::is_same<R, float>::value) {
    const float4 r = __ldcs(reinterpret_cast<const float4 *>(base) + p);
    off = r.x; vx = r.y; vy = r.z; vz = r.w;
  } else {
    const double2 *q = reinterpret_cast<const double2 *>(reinterpret_cast<const D4 *>(base) + p);
    const double2 a = __ldcs(q), b = __ldcs(q + 1);
    off = a.x; vx = a.y; vy = b.x; vz = b.y;
  }
}
template <class R> __device__ __forceinline__ void rec_store(void *base, long long p, R off, R vx, R vy, R vz) {
  if constexpr (std::is_same<R, float>::value) {
    __stcs(reinterpret_cast<float4 *>(base) + p, make_float4(off, vx, vy, vz));
  } else {
    double2 *q = reinterpret_cast<double2 *>(reinterpret_cast<D4 *>(base) + p);
    __stcs(q, make_double2(off, vx));
    __stcs(q + 1, make_double2(vy, vz));
  }
}
// a record written earlier in the same kernel, read from L2 (not through L1)
template <class R> __device__ __forceinline__ void rec_load_l2(const void *base, long long p, R &off, R &vx, R &vy, R &vz) {
  if constexpr (std::is_same<R, float>::value) {
    const float4 r = __ldcg(reinterpret_cast<const float4 *>(base) + p);
    off = r.x; vx = r.y; vy = r.z; vz = r.w;
  } else {
    const double2 *q = reinterpret_cast<const double2 *>(reinterpret_cast<const D4 *>(base) + p);
    const double2 a = __ldcg(q), b = __ldcg(q + 1);
    off = a.x; vx = a.y; vy = b.x; vz = b.y;
  }
}
template <class R> __device__ __forceinline__ R rec_get_off(const void *base, long long p) {
  if constexpr (std::is_same<R, float>::value) return reinterpret_cast<const float4 *>(base)[p].x;
  else return reinterpret_cast<const D4 *>(base)[p].off;
}

// signed fixed-point deposit straight to global memory (births, removals, init)
template <class R>
__device__ __forceinline__ void dep_global(unsigned long long *Q, int N, int32_t cell, R off, bool add) {
  // N: nodes of Q (node N wraps to 0 in a periodic column; a bounded column passes N + 1)
  const unsigned long long k = wfix(off);
  unsigned long long a = (1ull << 32) - k, b = k;
  if (!add) { a = 0ull - a; b = 0ull - b; }
  const int c1 = (cell + 1 == N) ? 0 : cell + 1;
  atomicAdd(Q + cell, a);
  atomicAdd(Q + c1, b);
}

template <class R> __device__ __forceinline__ int64_t pow2ceil(int64_t n) {
  int64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

__device__ void bitonic_sort(unsigned long long *a, int n2) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const unsigned long long x = a[i], y = a[ixj];
          if ((x > y) == up) { a[i] = y; a[ixj] = x; }
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Particle step.  One persistent CTA per SM walks a contiguous slot range in
// tiles of particles.
//   phase A (every particle): gather, leapfrog push, wrap, the Philox block
//     that decides collision candidacy (u0 < P_null) and radial loss, the
//     cloud-in-cell deposit (into fixed-point bins in shared memory over a
//     cell window: three 32-bit additions per particle whose results are not
//     read), and the store of every non-candidate; candidates go to a
//     shared-memory queue;
//   phase B (whenever a warp has queued 32 candidates, and at the end): the
//     collision path for 32 queued candidates, one per lane, so that a warp
//     runs it densely instead of whenever any of its lanes collides.
// Every compute warp owns its queue (64 entries).  The only block-wide
// barriers of the loop are the rare bin flushes (every flush_tiles tiles), so
// the warps' memory latencies overlap freely.  Collisions change velocities
// only, so the deposit in phase A is final.
//
// MIXED form: the particles of the next kStages tiles are staged in shared
// memory while a tile is processed.  Two ways are built (PIC_STAGING):
//   1  every thread copies its own particle of each tile with asynchronous
//      copies (cp.async of 4, 16 and 8 bytes, one commit group per tile and
//      thread) and reads back only what it copied, so no warp waits for another;
//   2  the last warp of the CTA is a copy warp: one of its threads stages each
//      tile as three contiguous ranges (int32 cells, float4 records, ids) with
//      bulk asynchronous copies (the TMA engine) that complete on the stage's
//      "full" mbarrier; the compute warps wait on it, read their particle and
//      release the stage through its "empty" mbarrier.
// FP64 form: every warp computes and the next tile's particle is prefetched in
// registers.
#ifndef PIC_STAGING
#define PIC_STAGING 1
#endif
#ifndef PIC_STAGES
#define PIC_STAGES 2
#endif

constexpr int kWarpQ = 64;           // queue entries per compute warp
constexpr int kStages = PIC_STAGES;  // tiles in flight (MIXED form)
constexpr int kStageSpin = 1 << 18;  // polls of a stage barrier (each suspends up to 10 us) before giving up

template <class R> __host__ __device__ constexpr bool staged() { return std::is_same<R, float>::value; }
// 0: register prefetch (FP64 form), 1: per-thread asynchronous copies, 2: copy warp + bulk copies
template <class R> __host__ __device__ constexpr int stage_mode() { return staged<R>() ? PIC_STAGING : 0; }
template <class R> __host__ __device__ constexpr int compute_warps() {
  return kStepThreads / 32 - (stage_mode<R>() == 2 ? 1 : 0);
}
template <class R> __host__ __device__ constexpr int tile_of() { return compute_warps<R>() * 32; }
// tiles between two flushes of the shared-memory bins: a cell of the window then receives fewer
// than 2^16 particles in between, so the 16-bit halves of the weights sum without overflow
template <class R> __host__ __device__ constexpr int flush_tiles() { return 65535 / tile_of<R>(); }

// queued candidates: the slot and the raw 32-bit word of the process-choice uniform, 8 bytes; the
// candidate's cell, record and id were written to (or stay in) the particle arrays in phase A and
// are read back from L2 when its warp runs the collision path
template <class R> __host__ __device__ constexpr int queue_cap() { return compute_warps<R>() * kWarpQ; }
template <class R> __host__ __device__ constexpr size_t queue_bytes() { return (size_t)queue_cap<R>() * 8; }

// MIXED form: the first kPbHot per-bin null-collision thresholds of the electrons (the energies
// where nearly every electron is: 50 eV on a 200 eV table of 8193 points) are read from shared
// memory, the rest through L1
constexpr int kPbHot = 2048;
template <class R> __host__ __device__ constexpr size_t pbhot_bytes() { return staged<R>() ? (size_t)kPbHot * 4 : 0; }

// MIXED form: kStages stages of one tile each: int32 cells, float4 records, ids
template <class R> __host__ __device__ constexpr size_t stage_bytes() {
  return staged<R>() ? (size_t)kStages * tile_of<R>() * (4 + 16 + 8) : 0;
}
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int G> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(G) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, unsigned bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
// bounded wait for the completion of the barrier's phase of the given parity: false if the polls ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned parity, int limit) {
  for (int i = 0; i < limit; ++i) {
    unsigned ok;
    asm volatile("{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, 10000;\nselp.b32 %0, 1, 0, P;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(b)), "r"(parity)
                 : "memory");
    if (ok) return true;
  }
  return false;
}
// bulk copy global -> shared (16-byte aligned addresses, a multiple of 16 bytes), completing on bar
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void named_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// round(256 vx) to nearest even, as an integer (exact, order independent sums)
__device__ __forceinline__ long long vfix(float v) { return __float2ll_rn(v * 256.0f); }
__device__ __forceinline__ long long vfix(double v) { return __double2ll_rn(v * 256.0); }

// diagnostic moments of one particle (FP64, cloud-in-cell weights)
// EEPF sample (Sec. III.C): the energy bin decided in the storage precision
template <class R>
__device__ __forceinline__ void eepf_count(const Moments &m, int N, int32_t cell, R epsr) {
  const R x = epsr * (R)m.eepf_scale;
  const int b = x < (R)m.eepf_ne ? (int)x : m.eepf_ne;
  const int bx = (int)(((long long)cell * m.eepf_nx) / N);
  atomicAdd(m.eepf + (size_t)bx * (m.eepf_ne + 1) + b, 1ull);
}

template <class R, int SP>
__device__ __forceinline__ void add_moments(const SpecK<R> &sp, const Moments &m, int N, int Nw, int32_t cell, R off,
                                            R vx, R vy, R vz) {
  const unsigned long long kk = wfix(off);
  const int c1 = (cell + 1 == Nw) ? 0 : cell + 1;
  const double w1 = (double)kk * (1.0 / 4294967296.0), w0 = 1.0 - w1;
  const double vxd = (double)vx;
  if constexpr (SP == 0) {
    const R epsr = sp.K * (vx * vx + vy * vy + vz * vz);
    const double eps = (double)epsr;
    if (m.eepf) eepf_count<R>(m, N, cell, epsr);
    atomicAdd(m.ge + cell, w0 * vxd); atomicAdd(m.ge + c1, w1 * vxd);
    atomicAdd(m.ee + cell, w0 * eps); atomicAdd(m.ee + c1, w1 * eps);
    const double h = eps * vxd;
    atomicAdd(m.he + cell, w0 * h); atomicAdd(m.he + c1, w1 * h);
  } else {
    atomicAdd(m.gi + cell, w0 * vxd); atomicAdd(m.gi + c1, w1 * vxd);
  }
}

// Collision of one candidate (u0 < P_null already drawn): process choice by
// u1 nu* against the cumulative collision frequencies, then the scattering.
// Returns the process index within the species, or -1 for a null collision.
template <class R, int SP, bool BD>
__device__ __forceinline__ int collide(const StepK<R> &k, const SpecK<R> &sp, Ctl *ctl, const BirthBuf<R> &bb,
                                       const Moments &m, uint64_t id, uint32_t step, uint32_t c3, int32_t p,
                                       int32_t cell, R off, R u1, R &vx, R &vy, R &vz, bool &ovf) {
  const int N = k.N;
  UStream<R> us(seed_key(k.seed), id, step, c3);
  int sel = -1;
  if constexpr (SP == 0) {
    // electron-neutral: elastic, excitation levels, ionization (Sec. II)
    const R eps = sp.K * (vx * vx + vy * vy + vz * vz);
    R fr;
    const int it = tab_pos(eps, sp.inv_de, k.ntab, fr, ovf);
    const R r = u1 * __ldg(sp.nub + it);
    R cum = 0;
    for (int q = 0; q < sp.np; ++q) {
      R nu;
      if (sp.kind[q] != PIC_ELASTIC && eps < sp.thr[q]) nu = 0;
      else nu = tab_at(sp.tab + (size_t)q * k.ntab, it, fr);
      cum = cum + nu;
      if (r < cum) { sel = q; break; }
    }
    if (sel >= 0) {
      const int kind = sp.kind[sel];
      R nx, ny, nz;
      if (kind == PIC_ELASTIC) {
        iso_dir(us, nx, ny, nz);
        const R vm = sqrt(vx * vx + vy * vy + vz * vz);
        const R cosx = (vm > (R)0) ? (nx * vx + ny * vy + nz * vz) / vm : (R)0;
        const R e2 = eps * ((R)1 - k.em * ((R)1 - cosx));
        const R spd = sqrt(e2 * k.V_e);
        vx = spd * nx; vy = spd * ny; vz = spd * nz;
      } else if (kind == PIC_EXCITATION) {
        const R e2 = eps - sp.thr[sel];
        iso_dir(us, nx, ny, nz);
        const R spd = sqrt(e2 * k.V_e);
        vx = spd * nx; vy = spd * ny; vz = spd * nz;
      } else {
        const R er = eps - sp.thr[sel];
        const R ush = us.next();
        const R e_ej = ush * er;
        const R e_sc = er - e_ej;
        iso_dir(us, nx, ny, nz);
        const R spd = sqrt(e_sc * k.V_e);
        vx = spd * nx; vy = spd * ny; vz = spd * nz;
        R mx, my, mz;
        iso_dir(us, mx, my, mz);
        const R sq = sqrt(e_ej * k.V_e);
        const R g0 = gauss<R>(k.gauss, us.next());
        const R g1 = gauss<R>(k.gauss, us.next());
        const R g2 = gauss<R>(k.gauss, us.next());
        if (k.loss_mode != PIC_LOSS_SWARM) {
          const int idx = atomicAdd(&ctl->n_birth, 1);
          if (idx < kStageCap) {
            bb.parent[idx] = p;
            bb.cell[idx] = cell;
            bb.off[idx] = off;
            bb.ve[idx] = sq * mx; bb.ve[kStageCap + idx] = sq * my; bb.ve[2 * kStageCap + idx] = sq * mz;
            bb.vi[idx] = k.sig_n * g0; bb.vi[kStageCap + idx] = k.sig_n * g1; bb.vi[2 * kStageCap + idx] = k.sig_n * g2;
          } else {
            atomicOr(&ctl->status, kStBirthOverflow);
          }
        } else {
          atomicAdd(&ctl->births, 1ull);
        }
        const unsigned long long kk = wfix(off);
        const int c1 = (cell + 1 == N + (BD ? 1 : 0)) ? 0 : cell + 1;   // nodes: N, or N + 1 bounded
        atomicAdd(m.iz + cell, (1ull << 32) - kk);
        atomicAdd(m.iz + c1, kk);
      }
    }
  } else {
    // ion-neutral: neutral velocity from the gas Maxwellian, relative speed g,
    // charge exchange or isotropic elastic in the centre-of-mass frame
    const R g0 = gauss<R>(k.gauss, us.next());
    const R g1 = gauss<R>(k.gauss, us.next());
    const R g2 = gauss<R>(k.gauss, us.next());
    const R nvx = k.sig_n * g0, nvy = k.sig_n * g1, nvz = k.sig_n * g2;
    const R gx = vx - nvx, gy = vy - nvy, gz = vz - nvz;
    const R eg = sp.K * (gx * gx + gy * gy + gz * gz);
    R fr;
    const int it = tab_pos(eg, sp.inv_de, k.ntab, fr, ovf);
    const R r = u1 * sp.nus;
    R cum = 0;
    for (int q = 0; q < sp.np; ++q) {
      cum = cum + tab_at(sp.tab + (size_t)q * k.ntab, it, fr);
      if (r < cum) { sel = q; break; }
    }
    if (sel >= 0) {
      if (sp.kind[sel] == PIC_ION_CX) {
        vx = nvx; vy = nvy; vz = nvz;
      } else {
        R nx, ny, nz;
        iso_dir(us, nx, ny, nz);
        const R gm = sqrt(gx * gx + gy * gy + gz * gz);
        const R hg = (R)0.5 * gm;
        vx = (R)0.5 * (vx + nvx) + hg * nx;
        vy = (R)0.5 * (vy + nvy) + hg * ny;
        vz = (R)0.5 * (vz + nvz) + hg * nz;
      }
    }
  }
  return sel;
}

// bytes of the shared-memory bins of W cells, rounded so that what follows stays 16-byte aligned
__host__ __device__ constexpr size_t bins_bytes(int W) { return ((size_t)W * 12 + 15) & ~(size_t)15; }

// Shared-memory charge bins per cell of a window [c0, c0 + W): the particle count and the sums
// of the low and high 16-bit halves of the cloud-in-cell weights k.  Cell c's n particles give
// node c: n 2^32 - sum k and node c+1: sum k, added at a flush.  Between two flushes a cell
// receives fewer than 2^16 particles, so no 32-bit sum overflows.
struct CellBins {
  unsigned *cnt, *klo, *khi;
  int W, c0;
};

// one particle of cell `cell` with weight k into the window's bins (three additions whose
// results are not read), or, outside the window, straight into the node charges
__device__ __forceinline__ void deposit_one(const CellBins &b, int N, int Nw, int32_t cell, uint32_t k,
                                            unsigned long long *Q) {
  int li = cell;
  if (b.W < N) {
    li = cell - b.c0;
    if (li < 0) li += N;
  }
  if (li < b.W) {
    atomicAdd(b.cnt + li, 1u);
    atomicAdd(b.klo + li, k & 0xffffu);
    atomicAdd(b.khi + li, k >> 16);
  } else {
    const int c1 = (cell + 1 == Nw) ? 0 : cell + 1;
    atomicAdd(Q + cell, (1ull << 32) - (unsigned long long)k);
    atomicAdd(Q + c1, (unsigned long long)k);
  }
}

// add the bins to the node charges and clear them (threads t0, t0 + nt, ... of the CTA)
__device__ __forceinline__ void bins_flush(const CellBins &b, int N, int Nw, unsigned long long *Q, int t0, int nt) {
  for (int j = t0; j < b.W; j += nt) {
    const unsigned nq = b.cnt[j];
    if (nq) {
      const unsigned long long sk = ((unsigned long long)b.khi[j] << 16) + (unsigned long long)b.klo[j];
      int cell = j;
      if (b.W < N) { cell = b.c0 + j; if (cell >= N) cell -= N; }
      const int c1 = (cell + 1 == Nw) ? 0 : cell + 1;
      atomicAdd(Q + cell, ((unsigned long long)nq << 32) - sk);
      if (sk) atomicAdd(Q + c1, sk);
      b.cnt[j] = 0u;
      b.klo[j] = 0u;
      b.khi[j] = 0u;
    }
  }
}

// Diagnostic moment bins, per node of the moment window [c0, c0 + Wm] (Wm + 1 nodes, Wm <= W,
// the same origin as the charge window).  The electron flux and energy flux (and the ion flux)
// are cancelling sums of thermal velocities of both signs: they are summed exactly as fixed point
// (mom_scale_v, kMomScaleH per unit), each value split into a low 16-bit and a signed high part
// added to two 32-bit words, like the charge bins; between two flushes a node receives fewer than
// 2^16 values, so no word overflows.  The energy, a sum of positive terms, is summed in FP32.  The
// w0 parts go to the left node, the w1 parts to the right one; a particle outside the moment
// window, or with a value beyond the fixed-point range, goes straight to the FP64 node sums.
// Flushed into the FP64 sums with the charge bins.  Words per node: electrons flux lo, hi, energy
// flux lo, hi, energy; ions flux lo, hi.
constexpr int kMomWords = 5;
__host__ __device__ constexpr size_t mbins_bytes(int Wm) {
  return ((size_t)(Wm + 1) * kMomWords * 4 + 15) & ~(size_t)15;
}
// fixed-point scales (powers of two, so the scaling is exact): flux in m/s (electrons 2^6, range
// 3.3e7 m/s; ions 2^14, range 1.3e5 m/s) and energy flux in eV m/s (2^-1, range 4.2e9)
template <int SP> __device__ __forceinline__ float mom_scale_v() { return SP == 0 ? 64.0f : 16384.0f; }
constexpr float kMomScaleH = 0.5f;
constexpr float kMomRange = 2147483520.0f;   // largest float below 2^31

__device__ __forceinline__ void fix_add(uint32_t *lo, uint32_t *hi, int i, float v) {
  const int q = __float2int_rn(v);
  atomicAdd(lo + i, (uint32_t)q & 0xffffu);
  atomicAdd(hi + i, (uint32_t)(q >> 16));
}
__device__ __forceinline__ long long fix_sum(uint32_t lo, uint32_t hi) {
  return (long long)(int32_t)hi * 65536ll + (long long)lo;
}

template <class R, int SP>
__device__ __forceinline__ void add_moments_win(const SpecK<R> &sp, const Moments &m, const CellBins &b, uint32_t *sM,
                                                int Wm, int N, int Nw, int32_t cell, R off, R vx, R vy, R vz) {
  int li = cell;
  if (b.W < N) {
    li = cell - b.c0;
    if (li < 0) li += N;
  }
  const float fx = (float)vx;
  const float sv = mom_scale_v<SP>();
  if (li >= Wm || !(fabsf(fx) * sv < kMomRange)) {
    add_moments<R, SP>(sp, m, N, Nw, cell, off, vx, vy, vz);
    return;
  }
  const float w1 = (float)wfix32(off) * 2.3283064365386963e-10f, w0 = 1.0f - w1;
  const int W1 = Wm + 1;
  if constexpr (SP == 0) {
    const R epsr = sp.K * (vx * vx + vy * vy + vz * vz);
    const float fe = (float)epsr, fh = fe * fx;
    if (!(fabsf(fh) * kMomScaleH < kMomRange)) {
      add_moments<R, SP>(sp, m, N, Nw, cell, off, vx, vy, vz);
      return;
    }
    if (m.eepf) eepf_count<R>(m, N, cell, epsr);
    fix_add(sM, sM + W1, li, (w0 * fx) * sv);
    fix_add(sM, sM + W1, li + 1, (w1 * fx) * sv);
    fix_add(sM + 2 * W1, sM + 3 * W1, li, (w0 * fh) * kMomScaleH);
    fix_add(sM + 2 * W1, sM + 3 * W1, li + 1, (w1 * fh) * kMomScaleH);
    float *se = reinterpret_cast<float *>(sM + 4 * W1);
    atomicAdd(se + li, w0 * fe);
    atomicAdd(se + li + 1, w1 * fe);
  } else {
    fix_add(sM, sM + W1, li, (w0 * fx) * sv);
    fix_add(sM, sM + W1, li + 1, (w1 * fx) * sv);
  }
}

// add the moment bins to the FP64 node sums and clear them (threads t0, t0 + nt, ... of the CTA)
template <int SP>
__device__ __forceinline__ void mbins_flush(const CellBins &b, uint32_t *sM, int Wm, const Moments &m, int N, int Nw,
                                            int t0, int nt) {
  const int W1 = Wm + 1;
  for (int j = t0; j < W1; j += nt) {
    // node j: the left node of window cell j, or for j = Wm the right node of cell Wm - 1
    int c = j < Wm ? j : Wm - 1;
    if (b.W < N) { c = b.c0 + c; if (c >= N) c -= N; }
    const int node = j < Wm ? c : ((c + 1 == Nw) ? 0 : c + 1);
    const long long g = fix_sum(sM[j], sM[W1 + j]);
    if (g) atomicAdd((SP == 0 ? m.ge : m.gi) + node, (double)g * (1.0 / (double)mom_scale_v<SP>()));
    sM[j] = 0u;
    sM[W1 + j] = 0u;
    if constexpr (SP == 0) {
      const long long h = fix_sum(sM[2 * W1 + j], sM[3 * W1 + j]);
      if (h) atomicAdd(m.he + node, (double)h * (1.0 / (double)kMomScaleH));
      float *se = reinterpret_cast<float *>(sM + 4 * W1);
      if (se[j] != 0.0f) atomicAdd(m.ee + node, (double)se[j]);
      sM[2 * W1 + j] = 0u;
      sM[3 * W1 + j] = 0u;
      se[j] = 0.0f;
    }
  }
}

// one CTA's share (cta of ncta) of the particle step of one column; PK: k is a launch
// parameter (the Philox round keys are read from it as constants); PL: a plain step (no
// process codes, no diagnostic sample, no circuit sums, no radial losses), compiled without
// those branches
template <class R, int SP, bool PK, bool BD, bool PL = false>
__device__ __forceinline__ void push_body(const StepK<R> &k, SpeciesDev s, Ctl *ctl, const R *__restrict__ Ef,
                                          BirthBuf<R> bb, Moments m, int W, int smemE, int mofs, int Wm,
                                          int cta, int ncta, unsigned char *smem) {
  __shared__ unsigned int s_cnt[kMaxProc + 1];
  __shared__ __align__(8) uint64_t s_full[kStages], s_empty[kStages];
  constexpr int kMode = stage_mode<R>();
  constexpr bool kStg = kMode == 2;        // copy warp and bulk copies
  constexpr int CW = compute_warps<R>();   // compute warps (with a copy warp: all but the last)
  constexpr int TILE = tile_of<R>();
  constexpr int FT = flush_tiles<R>();
  const int N = k.N, Nw = N + (BD ? 1 : 0);
  constexpr bool bounded = BD;   // a bounded column (Sec. V), a separate instantiation
  const SpecK<R> &sp = k.sp[SP];
  const size_t eb = (smemE ? ((((size_t)N + 1) * sizeof(R) + 15) & ~(size_t)15) : 0) + pbhot_bytes<R>();
  R *sE = reinterpret_cast<R *>(smem + pbhot_bytes<R>());
  uint32_t *sPb = reinterpret_cast<uint32_t *>(smem);   // MIXED form: hot null-collision thresholds
  CellBins bins;
  bins.cnt = reinterpret_cast<unsigned *>(smem + eb);
  bins.klo = bins.cnt + W;
  bins.khi = bins.klo + W;
  bins.W = W;
  uint2 *Qd = reinterpret_cast<uint2 *>(smem + eb + bins_bytes(W));
  unsigned char *stg = smem + eb + bins_bytes(W) + queue_bytes<R>();
  const long long n = ctl->n[SP];
  const long long stepll = ctl->step;
  const uint32_t step = (uint32_t)stepll;
  const bool diag = !PL && k.diag_every > 0 && (stepll % k.diag_every) == 0;
  // this step's moments go to shared-memory bins (mofs >= 0: the layout has room for them); when
  // they take the field's place, the field is gathered from global memory on this step
  const bool mb = diag && mofs >= 0;
  const bool eSmem = smemE && !(mb && mofs == (int)pbhot_bytes<R>());
  uint32_t *sM = reinterpret_cast<uint32_t *>(smem + (mofs >= 0 ? mofs : 0));
  // bin flushes every FT tiles; on a sampled step every FT / 2, so that with the candidates whose
  // collision (and moments) come after a flush a node still receives fewer than 2^16 values
  const int ftiles = mb ? FT / 2 : FT;
  const uint2 key = seed_key(k.seed);
  const uint32_t c3 = ((SP == 0 ? (uint32_t)kStE : (uint32_t)kStI) << 28) | (k.column << 16);
  // slot range of this CTA; the chunk is a multiple of 4 slots, so that every tile starts on a
  // 16-byte boundary of the int32 and uint64 arrays
  const long long chunk = (((n + ncta - 1) / ncta) + 3) & ~3ll;
  const long long p0 = min(n, (long long)cta * chunk);
  const long long p1 = min(n, p0 + chunk);
  int c0 = 0;
  if (W < N && p0 < p1) {
    // the window is centred on the median of five cells in the middle of the slot range, taken as
    // offsets on the periodic grid from the first of them: particles out of cell order (newborns
    // in victims' slots since the last sort) cannot pull the window away from the rest
    const long long pm = min(p1 - 5, max(p0, p0 + (p1 - p0) / 2 - 2));
    int d[5];
    const int ref = s.cell[max(p0, pm)];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const long long pq = min(p1 - 1, max(p0, pm + q));
      int x = s.cell[pq] - ref;
      if (x > N / 2) x -= N;
      else if (x <= -(N / 2)) x += N;
      d[q] = x;
    }
    int med = 0;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      int below = 0;
#pragma unroll
      for (int r = 0; r < 5; ++r) below += (d[r] < d[q]) || (d[r] == d[q] && r < q);
      if (below == 2) med = d[q];
    }
    c0 = ref + med - W / 2;
    c0 %= N;
    if (c0 < 0) c0 += N;
  }
  bins.c0 = c0;
  // slots fit in 32 bits (the capacity is at most INT32_MAX)
  const int ip0 = (int)p0, ip1 = (int)p1;
  const int ntiles = ip1 > ip0 ? (ip1 - ip0 + TILE - 1) / TILE : 0;
  // per-thread asynchronous copies: this thread's particle of tile tt into stage tt % kStages
  auto stage_in = [&](int tt) {
    const int p = ip0 + tt * TILE + (int)threadIdx.x;
    if (tt < ntiles && p < ip1) {
      unsigned char *sb = stg + (size_t)(tt % kStages) * TILE * 28;
      cp_async4(reinterpret_cast<int32_t *>(sb) + threadIdx.x, s.cell + p);
      cp_async16(reinterpret_cast<float4 *>(sb + (size_t)TILE * 4) + threadIdx.x,
                 reinterpret_cast<const float4 *>(s.rec) + p);
      cp_async8(reinterpret_cast<uint64_t *>(sb + (size_t)TILE * 20) + threadIdx.x, s.id + p);
    }
    cp_async_commit();
  };
  // the first tiles are in flight while the field and the tables are staged
  if constexpr (kMode == 1)
    for (int tt = 0; tt < kStages; ++tt) stage_in(tt);
  if constexpr (staged<R>() && SP == 0)
    for (int j = threadIdx.x; j < kPbHot && j < k.ntab; j += blockDim.x) sPb[j] = __ldg(sp.Pbi + j);
  if (eSmem)
    for (int j = threadIdx.x; j <= N; j += blockDim.x) sE[j] = Ef[j];
  for (int j = threadIdx.x; j < W; j += blockDim.x) { bins.cnt[j] = 0u; bins.klo[j] = 0u; bins.khi[j] = 0u; }
  if (mb)
    for (int j = threadIdx.x; j < kMomWords * (Wm + 1); j += blockDim.x) sM[j] = 0u;
  if (threadIdx.x <= kMaxProc) s_cnt[threadIdx.x] = 0u;
  if (kStg && threadIdx.x == 0) {
    for (int q = 0; q < kStages; ++q) {
      mbar_init(&s_full[q], 1);
      mbar_init(&s_empty[q], CW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const R *E = eSmem ? sE : Ef;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;

  if (kStg && warp == CW) {
    // copy warp: one thread stages tile t in stage t % kStages once the compute warps have
    // released that stage's previous tile
    if (lane == 0) {
      int t = 0;
      for (; t < ntiles; ++t) {
        const int st = t % kStages;
        if (t >= kStages && !mbar_wait(&s_empty[st], (unsigned)((t / kStages - 1) & 1), kStageSpin)) {
          atomicOr(&ctl->status, kStTimeout);
          break;
        }
        const int base = ip0 + t * TILE;
        const int cnt = min(TILE, ip1 - base);
        const unsigned c4 = (unsigned)((cnt + 3) & ~3);   // the arrays are padded past the capacity
        unsigned char *sb = stg + (size_t)st * TILE * 28;
        mbar_expect_tx(&s_full[st], c4 * 28u);
        bulk_g2s(sb, s.cell + base, c4 * 4u, &s_full[st]);
        bulk_g2s(sb + (size_t)TILE * 4, reinterpret_cast<const float4 *>(s.rec) + base, c4 * 16u, &s_full[st]);
        bulk_g2s(sb + (size_t)TILE * 20, s.id + base, c4 * 8u, &s_full[st]);
      }
      // no copy may still be landing when the CTA exits: wait for the last tiles issued (they
      // have landed already unless a compute warp gave up)
      for (int u = t - kStages; u < t; ++u)
        if (u >= 0 && !mbar_wait(&s_full[u % kStages], (unsigned)((u / kStages) & 1), kStageSpin))
          atomicOr(&ctl->status, kStTimeout);
    }
  } else {
    const unsigned lt = (1u << lane) - 1u;
    const bool radial = !PL && k.loss_mode == PIC_LOSS_RADIAL;
    const bool record = !PL && (k.flags & PIC_FLAG_RECORD_CODES) != 0;
    const int qoff = warp * kWarpQ;   // this warp's queue slice
    int wq = 0;                       // its length (warp-uniform)
    const bool circuit = !PL && k.drive == PIC_DRIVE_CIRCUIT;
    long long vsum = 0;               // circuit drive: this thread's sum of round(256 vx)

    // collision path for the warp's first nq (<= 32) queued candidates, one per lane
    auto flush = [&](int nq) {
      int sel = -1;
      bool ovf = false;
      if (lane < nq) {
        const uint2 e = Qd[qoff + lane];
        const int32_t qp = (int32_t)e.x;
        const R qu1 = u_dec<R>(e.y);
        // the candidate as phase A stored it (L2 reads: written by this warp, not through L1)
        const int32_t qcell = __ldcg(s.cell + qp);
        const uint64_t qid = __ldcg(reinterpret_cast<const unsigned long long *>(s.id) + qp);
        R qoff_, qx, qy, qz;
        rec_load_l2<R>(s.rec, qp, qoff_, qx, qy, qz);
        sel = collide<R, SP, BD>(k, sp, ctl, bb, m, qid, step, c3, qp, qcell, qoff_, qu1, qx, qy, qz, ovf);
        rec_store<R>(s.rec, qp, qoff_, qx, qy, qz);
        if (record) s.code[qp] = sel >= 0 ? sp.xs[sel] : -1;
        if (mb) add_moments_win<R, SP>(sp, m, bins, sM, Wm, N, Nw, qcell, qoff_, qx, qy, qz);
        else if (diag) add_moments<R, SP>(sp, m, N, Nw, qcell, qoff_, qx, qy, qz);
        if (circuit) vsum += vfix(qx);
      }
      for (int q = 0; q < sp.np; ++q) {
        const unsigned b = __ballot_sync(kFull, sel == q);
        if (lane == 0 && b) atomicAdd(&s_cnt[q], (unsigned)__popc(b));
      }
      const unsigned bo = __ballot_sync(kFull, ovf);
      if (lane == 0 && bo) atomicAdd(&s_cnt[kMaxProc], (unsigned)__popc(bo));
      __syncwarp();
    };

    // FP64 form: the next tile's particle in registers while this one is processed
    int32_t n_cell = 0;
    R n_off = 0, n_vx = 0, n_vy = 0, n_vz = 0;
    uint64_t n_id = 0;
    if constexpr (kMode == 0) {
      const int p = ip0 + (int)threadIdx.x;
      if (p < ip1) {
        n_cell = s.cell[p];
        rec_load<R>(s.rec, p, n_off, n_vx, n_vy, n_vz);
        n_id = s.id[p];
      }
    }
    bool live = true;   // warp-uniform: false once a stage wait gave up
    int until = ftiles; // tiles left before the next bin flush (a countdown: no division per tile)
    for (int t = 0; t < ntiles; ++t) {
      const int base = ip0 + t * TILE;
      const int p = base + warp * 32 + lane;
      const bool valid = p < ip1;
      bool cand = false, dead = false;
      int32_t cell = n_cell;
      R off = n_off, vx = n_vx, vy = n_vy, vz = n_vz;
      uint32_t w1 = 0;   // raw word of the process-choice uniform (converted for candidates only)
      uint64_t id = n_id;
      if constexpr (kStg) {
        const int st = t % kStages;
        if (live) {
          live = __all_sync(kFull, mbar_wait(&s_full[st], (unsigned)((t / kStages) & 1), kStageSpin));
          if (!live && lane == 0) atomicOr(&ctl->status, kStTimeout);
        }
        if (live) {
          if (valid) {
            const unsigned char *sb = stg + (size_t)st * TILE * 28;
            const int q = warp * 32 + lane;
            cell = reinterpret_cast<const int32_t *>(sb)[q];
            const float4 r = reinterpret_cast<const float4 *>(sb + (size_t)TILE * 4)[q];
            off = r.x; vx = r.y; vy = r.z; vz = r.w;
            id = reinterpret_cast<const uint64_t *>(sb + (size_t)TILE * 20)[q];
          }
        }
      } else if constexpr (kMode == 1) {
        cp_async_wait<kStages - 1>();   // this thread's copies of the tile have landed
        if (valid) {
          const unsigned char *sb = stg + (size_t)(t % kStages) * TILE * 28;
          cell = reinterpret_cast<const int32_t *>(sb)[threadIdx.x];
          const float4 r = reinterpret_cast<const float4 *>(sb + (size_t)TILE * 4)[threadIdx.x];
          off = r.x; vx = r.y; vy = r.z; vz = r.w;
          id = reinterpret_cast<const uint64_t *>(sb + (size_t)TILE * 20)[threadIdx.x];
        }
      } else {
        const int pn = p + TILE;
        if (pn < ip1) {
          n_cell = s.cell[pn];
          rec_load<R>(s.rec, pn, n_off, n_vx, n_vy, n_vz);
          n_id = s.id[pn];
        }
      }
      if (valid && live) {
        const R Ep = gather(E, cell, off);
        const int side = push<R>(N, bounded, sp.a, sp.d, Ep, cell, off, vx);
        const uint4 ctr = make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, c3);
        const uint4 w0 = PK ? philox10_rk(ctr, k.rk) : philox10(ctr, key);
        dead = side != 0 || (radial && (w0.z < sp.Pw));
        if (side != 0) atomicAdd(&ctl->absorbed[SP][side > 0 ? 1 : 0], 1ull);
        if (!dead) {
          w1 = w0.y;
          if constexpr (SP == 0) {
            // electrons: null-collision probability of the energy bin of the particle
            const R eps = sp.K * (vx * vx + vy * vy + vz * vz);
            R fr;
            bool ovf;
            const int it = tab_pos(eps, sp.inv_de, k.ntab, fr, ovf);
            if constexpr (std::is_same<R, float>::value) cand = (w0.x >> 8) < (it < kPbHot ? sPb[it] : __ldg(sp.Pbi + it));
            else cand = u_dec<R>(w0.x) < __ldg(sp.Pb + it);
          } else {
            if constexpr (std::is_same<R, float>::value) cand = (w0.x >> 8) < sp.Pi;
            else cand = u_dec<R>(w0.x) < sp.P;
          }
        }
        s.cell[p] = cell;
        rec_store<R>(s.rec, p, off, vx, vy, vz);   // a candidate's record is rewritten after its collision
        if (!cand) {
          if (record) s.code[p] = dead ? -2 : -1;
          if (!dead && mb) add_moments_win<R, SP>(sp, m, bins, sM, Wm, N, Nw, cell, off, vx, vy, vz);
          else if (!dead && diag) add_moments<R, SP>(sp, m, N, Nw, cell, off, vx, vy, vz);
          if (!dead && circuit) vsum += vfix(vx);
        }
        if (dead) {
          const int idx = atomicAdd(&ctl->n_dead[SP], 1);
          if (idx < kStageCap) s.dead[idx] = p;
          else atomicOr(&ctl->status, kStDeadOverflow);
        }
        // charge deposit into the window bins
        if (!dead) deposit_one(bins, N, Nw, cell, wfix32(off), s.Q);
      }
      if constexpr (kStg) {
        // this warp is done with the stage: every value it read from it has been used above (so
        // the loads have returned) before the copy warp may refill it
        if (live) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&s_empty[t % kStages]);
        }
      }
      if constexpr (kMode == 1) stage_in(t + kStages);   // this thread's slot of the stage is free again
      // queue the candidates in this warp's slice
      const unsigned bal = __ballot_sync(kFull, cand);
      if (cand) Qd[qoff + wq + __popc(bal & lt)] = make_uint2((uint32_t)p, w1);
      wq += __popc(bal);
      __syncwarp();
      if (wq >= 32) {
        // the collision path reads the candidates' records back from L2: make this warp's
        // stores of phase A (all tiles so far) visible to its lanes first
        __threadfence_block();
        __syncwarp();
        flush(32);
        // move the remaining entries to the front of the slice
        const int rest = wq - 32;
        if (lane < rest) Qd[qoff + lane] = Qd[qoff + 32 + lane];
        __syncwarp();
        wq = rest;
      }
      // keep every cell of the window below 2^16 particles between flushes
      if (--until == 0 && t + 1 < ntiles) {
        until = ftiles;
        named_sync(1, CW * 32);
        bins_flush(bins, N, Nw, s.Q, threadIdx.x, CW * 32);
        if (mb) mbins_flush<SP>(bins, sM, Wm, m, N, Nw, threadIdx.x, CW * 32);
        named_sync(1, CW * 32);
      }
    }
    if (wq > 0) {
      __threadfence_block();
      __syncwarp();
      flush(wq);
    }
    if constexpr (kMode == 1) cp_async_wait<0>();
    if (circuit) {
      unsigned long long u = (unsigned long long)vsum;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(kFull, u, o);
      if (lane == 0 && u) atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->sumv[SP]), u);
    }
  }
  __syncthreads();
  bins_flush(bins, N, Nw, s.Q, threadIdx.x, blockDim.x);
  if (mb) mbins_flush<SP>(bins, sM, Wm, m, N, Nw, threadIdx.x, blockDim.x);
  if (threadIdx.x < sp.np && s_cnt[threadIdx.x])
    atomicAdd(&ctl->n_coll[SP][threadIdx.x], (unsigned long long)s_cnt[threadIdx.x]);
  if (threadIdx.x == 0 && s_cnt[kMaxProc]) atomicAdd(&ctl->overflow[SP], (unsigned long long)s_cnt[kMaxProc]);
}

template <class R, int SP, bool BD, bool PL>
__global__ void __launch_bounds__(kStepThreads, 1)
k_push(const __grid_constant__ StepK<R> k, SpeciesDev s, Ctl *ctl, const R *__restrict__ Ef, BirthBuf<R> bb,
       Moments m, int W, int smemE, int mofs, int Wm) {
  extern __shared__ __align__(16) unsigned char smem[];
  push_body<R, SP, true, BD, PL>(k, s, ctl, Ef, bb, m, W, smemE, mofs, Wm, blockIdx.x, gridDim.x, smem);
}

// batched columns: CTA b runs share sched[b].y of sched[b].z of column sched[b].x
template <class R, int SP, bool PL>
__global__ void __launch_bounds__(kStepThreads, 1) k_push_batch(const ColDev<R> *cols, const int4 *sched) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) StepK<R> sk;
  const int4 sc = sched[blockIdx.x];
  const ColDev<R> *cd = cols + sc.x;
  {
    const int *src = reinterpret_cast<const int *>(&cd->k);
    int *dst = reinterpret_cast<int *>(&sk);
    for (int q = threadIdx.x; q < (int)(sizeof(StepK<R>) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
  }
  __syncthreads();
  push_body<R, SP, false, false, PL>(sk, cd->sp[SP], cd->ctl, reinterpret_cast<const R *>(cd->Ef), cd->bb, cd->m, cd->W, cd->smemE,
                   cd->mofs, cd->Wm, sc.y, sc.z, smem);
}

template <class R> int push_smem_bytes(int N) {
  const size_t e = (((size_t)N + 1) * sizeof(R) + 15) & ~(size_t)15;
  return (int)e;
}

template <class R> size_t push_layout(int n_cells, int &W, int &smemE, int &mofs, int &Wm) {
  const size_t budget = 226 * 1024;   // of 227 KB: room for the batched kernel's static StepK
  const size_t qb = queue_bytes<R>() + stage_bytes<R>() + pbhot_bytes<R>();
  size_t eb = (((size_t)n_cells + 1) * sizeof(R) + 15) & ~(size_t)15;
  // the node field goes to shared memory when it leaves room for a 2048-cell bin window
  smemE = eb + qb + bins_bytes(2048) <= budget ? 1 : 0;
  if (!smemE) eb = 0;
  const size_t wmax = (budget - eb - qb) / 12;
  W = (int)((size_t)n_cells < wmax ? (size_t)n_cells : wmax);
  if (W < n_cells) W = W < 4096 ? (W & ~63) : 4096;
  const size_t base = eb + bins_bytes(W) + qb;
  // diagnostic moment bins: after everything for the whole charge window when they fit; else in
  // the field's place (the field is then gathered from global memory on sampled steps) for as many
  // nodes as fit there; else none (the moments then go straight to the FP64 node sums)
  mofs = -1;
  Wm = 0;
  if (base + mbins_bytes(W) <= budget) {
    mofs = (int)base;
    Wm = W;
    return base + mbins_bytes(W);
  }
  if (smemE) {
    int wm = (int)(eb / (kMomWords * 4)) - 1;
    if (wm >= W) wm = W;
    else wm &= ~63;
    if (wm >= 64) {
      mofs = (int)pbhot_bytes<R>();
      Wm = wm;
    }
  }
  return base;
}

template <class R>
void launch_push(const StepK<R> &k, SpeciesDev s, Ctl *ctl, const R *Ef, BirthBuf<R> bb, Moments m, int species,
                 int nsm, bool diag_step, cudaStream_t st) {
  int W = 0, smemE = 0, mofs = -1, Wm = 0;
  // a step with none of the optional work runs the kernel compiled without it
  const bool plain = !diag_step && !(k.flags & PIC_FLAG_RECORD_CODES) && k.drive != PIC_DRIVE_CIRCUIT &&
                     k.loss_mode != PIC_LOSS_RADIAL;
  const size_t bytes = push_layout<R>(k.N, W, smemE, mofs, Wm);
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    kern<<<nsm, kStepThreads, bytes, st>>>(k, s, ctl, Ef, bb, m, W, smemE, mofs, Wm);
  };
  if (species == 0) {
    if (k.bounded) go(k_push<R, 0, true, false>);
    else if (plain) go(k_push<R, 0, false, true>);
    else go(k_push<R, 0, false, false>);
  } else {
    if (k.bounded) go(k_push<R, 1, true, false>);
    else if (plain) go(k_push<R, 1, false, true>);
    else go(k_push<R, 1, false, false>);
  }
}

template <class R>
void launch_push_batch(const ColDev<R> *cols, const int4 *sched, int nblocks, int species, size_t smem, bool plain,
                       cudaStream_t st) {
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<nblocks, kStepThreads, smem, st>>>(cols, sched);
  };
  if (species == 0) {
    if (plain) go(k_push_batch<R, 0, true>); else go(k_push_batch<R, 0, false>);
  } else {
    if (plain) go(k_push_batch<R, 1, true>); else go(k_push_batch<R, 1, false>);
  }
}

template <class R> __global__ void k_zero_q_batch(const ColDev<R> *cols, int species) {
  const ColDev<R> *cd = cols + blockIdx.y;
  unsigned long long *Q = cd->sp[species].Q;
  if (blockIdx.x == 0 && threadIdx.x == 0) cd->ctl->sumv[species] = 0;   // circuit-drive sum of this push
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cd->N; j += gridDim.x * blockDim.x) Q[j] = 0ull;
}

template <class R> void launch_zero_q_batch(const ColDev<R> *cols, int ncol, int species, int maxN, cudaStream_t st) {
  const int bx = (maxN + 255) / 256 < 16 ? (maxN + 255) / 256 : 16;
  k_zero_q_batch<R><<<dim3(bx, ncol), 256, 0, st>>>(cols, species);
}

// ---------------------------------------------------------------------------
// Births and losses (one CTA).  Births are ordered by parent slot; event k
// gets ids next_id + 2k (electron) and next_id + 2k + 1 (ion).

__device__ __forceinline__ uint32_t victim_draw(uint2 key, uint32_t k, uint32_t att, uint32_t step, uint32_t c3,
                                                unsigned long long npre) {
  const uint4 w = philox10(make_uint4(k, att, step, c3), key);
  const unsigned long long r = ((unsigned long long)w.y << 32) | (unsigned long long)w.x;
  return (uint32_t)__umul64hi(r, npre);
}

// Victims without replacement, in rounds: an unsettled event settles iff no
// settled event holds its candidate and no lower unsettled event shares it.
__device__ bool draw_victims(uint2 key, uint32_t step, uint32_t c3, int nb, long long npre, unsigned long long *keys,
                             K3Scratch sc, uint32_t *out) {
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    sc.att[t] = 0u;
    sc.settled[t] = 0u;
    sc.cand[t] = victim_draw(key, (uint32_t)t, 0u, step, c3, (unsigned long long)npre);
  }
  __syncthreads();
  const int n2 = (int)pow2ceil<float>(nb);
  const bool direct = nb <= kDirectMax;
  for (int round = 0; round < 64; ++round) {
    if (direct) {
      // O(nb^2) conflict test: no sort for the usual few hundred events; the scan over the
      // shared-memory candidates has no early exit, so its loads pipeline
      for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        if (sc.settled[t]) continue;
        const uint32_t c = sc.cand[t];
        uint32_t clash = 0u;
#pragma unroll 8
        for (int j = 0; j < nb; ++j)
          clash |= (uint32_t)(sc.cand[j] == c) & (uint32_t)(j != t) & (uint32_t)((sc.settled[j] != 0u) | (j < t));
        sc.win[t] = clash ? 0u : 1u;
      }
    } else {
      for (int t = threadIdx.x; t < n2; t += blockDim.x)
        keys[t] = t < nb ? (((unsigned long long)sc.cand[t] << 32) | ((sc.settled[t] ? 0ull : 1ull) << 31) |
                            (unsigned long long)t)
                         : ~0ull;
      __syncthreads();
      bitonic_sort(keys, n2);
      for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const unsigned long long kk = keys[i];
        if ((kk >> 31) & 1ull) {
          const uint32_t ev = (uint32_t)(kk & 0x7fffffffull);
          sc.win[ev] = (i == 0 || (keys[i - 1] >> 32) != (kk >> 32)) ? 1u : 0u;
        }
      }
    }
    __syncthreads();
    int any = 0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
      if (!sc.settled[t]) {
        if (sc.win[t]) sc.settled[t] = 1u;
        else {
          sc.att[t] += 1u;
          sc.cand[t] = victim_draw(key, (uint32_t)t, sc.att[t], step, c3, (unsigned long long)npre);
          any = 1;
        }
      }
    }
    if (!__syncthreads_or(any)) {
      for (int t = threadIdx.x; t < nb; t += blockDim.x) out[t] = sc.cand[t];
      __syncthreads();
      return true;
    }
  }
  return false;
}

template <class R>
__device__ void write_newborn(SpeciesDev s, long long slot, int32_t cell, R off, R vx, R vy, R vz, uint64_t id, int N) {
  s.cell[slot] = cell;
  rec_store<R>(s.rec, slot, off, vx, vy, vz);
  s.id[slot] = id;
  dep_global<R>(s.Q, N, cell, off, true);
}

template <class R>
__device__ void copy_particle(SpeciesDev s, long long dst, long long src) {
  s.cell[dst] = s.cell[src];
  using T = typename Rec<R>::T;
  reinterpret_cast<T *>(s.rec)[dst] = reinterpret_cast<const T *>(s.rec)[src];
  s.id[dst] = s.id[src];
}

// radial mode: births fill the dead slots (ascending); extra births are
// appended; extra holes below N_new take the live tail particles in order
template <class R>
__device__ void fill_compact(const StepK<R> &k, SpeciesDev s, Ctl *ctl, int SP, BirthBuf<R> bb, K3Scratch sc, int nb,
                             int nd, long long next_id, unsigned long long *keys, int *s_scan) {
  const int N = k.N;
  const long long Nold = ctl->n[SP];
  const int n2 = (int)pow2ceil<float>(nd);
  for (int t = threadIdx.x; t < n2; t += blockDim.x)
    keys[t] = t < nd ? (unsigned long long)(uint32_t)s.dead[t] : ~0ull;
  __syncthreads();
  if (nd > 1) bitonic_sort(keys, n2);
  const int m = nb < nd ? nb : nd;
  const R *bv = SP == 0 ? bb.ve : bb.vi;
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    const uint32_t b = sc.order[t];
    write_newborn<R>(s, (long long)keys[t], bb.cell[b], bb.off[b], bv[b], bv[kStageCap + b], bv[2 * kStageCap + b],
                     (uint64_t)next_id + 2ull * (uint64_t)t + (uint64_t)SP, k.Nw);
  }
  long long Nnew = Nold;
  if (nb > nd) {
    Nnew = Nold + (nb - nd);
    if (Nnew > s.cap) {
      if (threadIdx.x == 0) atomicOr(&ctl->status, kStCapacity);
      Nnew = Nold;
    } else {
      for (int t = m + threadIdx.x; t < nb; t += blockDim.x) {
        const uint32_t b = sc.order[t];
        write_newborn<R>(s, Nold + (t - m), bb.cell[b], bb.off[b], bv[b], bv[kStageCap + b], bv[2 * kStageCap + b],
                         (uint64_t)next_id + 2ull * (uint64_t)t + (uint64_t)SP, k.Nw);
      }
    }
  } else if (nd > nb) {
    Nnew = Nold - (nd - nb);
    // q = number of remaining holes below Nnew (keys[nb..nd) ascending)
    __shared__ int s_q;
    if (threadIdx.x == 0) {
      int lo = nb, hi = nd;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((long long)keys[mid] < Nnew) lo = mid + 1; else hi = mid;
      }
      s_q = lo - nb;
    }
    __syncthreads();
    const int q = s_q;
    const int T = nd - nb;
    int carry = 0;
    for (int c0 = 0; c0 < T; c0 += blockDim.x) {
      const int i = c0 + threadIdx.x;
      int live = 0;
      long long t = Nnew + i;
      if (i < T) {
        int lo = nb + q, hi = nd;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if ((long long)keys[mid] < t) lo = mid + 1; else hi = mid;
        }
        live = !(lo < nd && (long long)keys[lo] == t);
      }
      s_scan[threadIdx.x] = live;
      __syncthreads();
      for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const int v = threadIdx.x >= (unsigned)off ? s_scan[threadIdx.x - off] : 0;
        __syncthreads();
        s_scan[threadIdx.x] += v;
        __syncthreads();
      }
      const int incl = s_scan[threadIdx.x];
      if (live) copy_particle<R>(s, (long long)keys[nb + carry + incl - 1], t);
      const int tot = s_scan[blockDim.x - 1];
      __syncthreads();
      carry += tot;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) ctl->n[SP] = Nnew;
}

template <class R>
__device__ __forceinline__ void births_body(const StepK<R> &k, SpeciesDev e, SpeciesDev ion, Ctl *ctl,
                                            BirthBuf<R> bb, K3Scratch sc, int ion_pushed, unsigned long long *keys) {
  __shared__ int s_scan[kBirthThreads];
  __shared__ uint32_t s_scr[7 * kDirectMax];
  const int N = k.N;
  int nb = ctl->n_birth;
  if (nb > kStageCap) nb = kStageCap;
  if (nb <= kDirectMax) {
    // the usual few hundred events: scratch in shared memory instead of global memory
    sc.order = s_scr;
    sc.cand = s_scr + kDirectMax;
    sc.att = s_scr + 2 * kDirectMax;
    sc.settled = s_scr + 3 * kDirectMax;
    sc.win = s_scr + 4 * kDirectMax;
    sc.vic = s_scr + 5 * kDirectMax;
  }
  int nde = ctl->n_dead[0], ndi = ion_pushed ? ctl->n_dead[1] : 0;
  if (nde > kStageCap) nde = kStageCap;
  if (ndi > kStageCap) ndi = kStageCap;
  const long long next_id = ctl->next_id;
  const uint32_t step = (uint32_t)ctl->step;
  const uint2 key = seed_key(k.seed);
  // births in parent-slot order
  if (nb > 0 && nb <= kDirectMax) {
    // rank of each birth by parent slot (parents are distinct), from a shared-memory copy of the
    // parents (the candidate array, unused until the victims are drawn)
    int32_t *s_par = reinterpret_cast<int32_t *>(sc.cand);
    for (int t = threadIdx.x; t < nb; t += blockDim.x) s_par[t] = bb.parent[t];
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
      const int32_t pt = s_par[t];
      int r = 0;
#pragma unroll 8
      for (int j = 0; j < nb; ++j) r += s_par[j] < pt;
      sc.order[r] = (uint32_t)t;
    }
    __syncthreads();
  } else if (nb > 0) {
    const int n2 = (int)pow2ceil<float>(nb);
    for (int t = threadIdx.x; t < n2; t += blockDim.x)
      keys[t] = t < nb ? (((unsigned long long)(uint32_t)bb.parent[t] << 32) | (unsigned long long)t) : ~0ull;
    __syncthreads();
    bitonic_sort(keys, n2);
    for (int t = threadIdx.x; t < nb; t += blockDim.x) sc.order[t] = (uint32_t)keys[t];
    __syncthreads();
  }
  const int vstride = nb <= kDirectMax ? kDirectMax : kStageCap;
  if (k.loss_mode == PIC_LOSS_PAIR) {
    if (nb > 0) {
      const long long npe = ctl->n[0], npi = ctl->n[1];
      bool ok = nb <= npe && nb <= npi;
      if (ok) ok = draw_victims(key, step, ((uint32_t)kStVicE << 28) | (k.column << 16), nb, npe, keys, sc, sc.vic);
      if (ok)
        ok = draw_victims(key, step, ((uint32_t)kStVicI << 28) | (k.column << 16), nb, npi, keys, sc,
                          sc.vic + vstride);
      if (!ok) {
        if (threadIdx.x == 0) atomicOr(&ctl->status, kStVictim);
      } else {
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
          const uint32_t b = sc.order[t];
          const long long ve = sc.vic[t], vi = sc.vic[vstride + t];
          dep_global<R>(e.Q, k.Nw, e.cell[ve], rec_get_off<R>(e.rec, ve), false);
          write_newborn<R>(e, ve, bb.cell[b], bb.off[b], bb.ve[b], bb.ve[kStageCap + b], bb.ve[2 * kStageCap + b],
                           (uint64_t)next_id + 2ull * (uint64_t)t, k.Nw);
          dep_global<R>(ion.Q, k.Nw, ion.cell[vi], rec_get_off<R>(ion.rec, vi), false);
          write_newborn<R>(ion, vi, bb.cell[b], bb.off[b], bb.vi[b], bb.vi[kStageCap + b], bb.vi[2 * kStageCap + b],
                           (uint64_t)next_id + 2ull * (uint64_t)t + 1ull, k.Nw);
        }
        if (threadIdx.x == 0) { ctl->losses[0] += nb; ctl->losses[1] += nb; }
      }
    }
  } else if (k.loss_mode == PIC_LOSS_RADIAL || k.bounded) {
    // removed particles (radial losses; in a bounded column also those the electrodes took)
    // leave holes that the births fill, the rest compacted
    fill_compact<R>(k, e, ctl, 0, bb, sc, nb, nde, next_id, keys, s_scan);
    __syncthreads();
    fill_compact<R>(k, ion, ctl, 1, bb, sc, nb, ndi, next_id, keys, s_scan);
    if (threadIdx.x == 0) { ctl->losses[0] += nde; ctl->losses[1] += ndi; }
  } else if (k.loss_mode == PIC_LOSS_NONE) {
    const long long ne = ctl->n[0], ni = ctl->n[1];
    if (ne + nb > e.cap || ni + nb > ion.cap) {
      if (threadIdx.x == 0) atomicOr(&ctl->status, kStCapacity);
    } else {
      for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        const uint32_t b = sc.order[t];
        write_newborn<R>(e, ne + t, bb.cell[b], bb.off[b], bb.ve[b], bb.ve[kStageCap + b], bb.ve[2 * kStageCap + b],
                         (uint64_t)next_id + 2ull * (uint64_t)t, k.Nw);
        write_newborn<R>(ion, ni + t, bb.cell[b], bb.off[b], bb.vi[b], bb.vi[kStageCap + b], bb.vi[2 * kStageCap + b],
                         (uint64_t)next_id + 2ull * (uint64_t)t + 1ull, k.Nw);
      }
      __syncthreads();
      if (threadIdx.x == 0) { ctl->n[0] = ne + nb; ctl->n[1] = ni + nb; }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (k.loss_mode != PIC_LOSS_SWARM) {
      ctl->next_id = next_id + 2 * (long long)nb;
      ctl->births += (unsigned long long)nb;
    }
    ctl->n_birth = 0;
    ctl->n_dead[0] = 0;
    ctl->n_dead[1] = 0;
  }
  if (k.bounded && k.emit_per_step > 0.0) {
    // Sec. V: the cathode emits J_emit dt / (e w) macro-electrons per step (the fraction carried
    // over).  Emitted electron q of step s draws (Philox counter q, s, emission stream) a
    // half-Maxwellian velocity at T_emit, (s |g0|, s g1, s g2), and starts at x = u v_x dt.
    __shared__ long long s_em[3];   // count, first slot, first id
    __syncthreads();
    if (threadIdx.x == 0) {
      double acc = ctl->emit_acc + k.emit_per_step;
      long long ne = (long long)floor(acc);
      acc -= (double)ne;
      const long long n0 = ctl->n[0];
      if (n0 + ne > e.cap) {
        atomicOr(&ctl->status, kStCapacity);
        ne = 0;
      }
      ctl->emit_acc = acc;
      s_em[0] = ne;
      s_em[1] = n0;
      s_em[2] = ctl->next_id;
      ctl->n[0] = n0 + ne;
      ctl->next_id += ne;
      ctl->emitted += (unsigned long long)ne;
    }
    __syncthreads();
    const long long ne = s_em[0], n0 = s_em[1], id0 = s_em[2];
    const uint32_t c3 = ((uint32_t)kStEmit << 28) | (k.column << 16);
    for (long long q = threadIdx.x; q < ne; q += blockDim.x) {
      UStream<R> us(key, (uint64_t)q, step, c3);
      const R g0 = gauss<R>(k.gauss, us.next());
      const R g1 = gauss<R>(k.gauss, us.next());
      const R g2 = gauss<R>(k.gauss, us.next());
      const R u = us.next();
      const R vx = k.sig_emit * (g0 < (R)0 ? -g0 : g0), vy = k.sig_emit * g1, vz = k.sig_emit * g2;
      const R x = u * vx * k.emit_dtdx;
      int32_t cell = (int32_t)x;
      R off = x - (R)cell;
      if (cell >= N) { cell = N - 1; off = (R)0; }
      write_newborn<R>(e, n0 + q, cell, off, vx, vy, vz, (uint64_t)(id0 + q), k.Nw);
    }
  }
}

template <class R>
__global__ void __launch_bounds__(kBirthThreads, 1)
k_births(const __grid_constant__ StepK<R> k, SpeciesDev e, SpeciesDev ion, Ctl *ctl, BirthBuf<R> bb, K3Scratch sc,
         int ion_pushed) {
  extern __shared__ __align__(16) unsigned long long keys[];   // kStageCap
  births_body<R>(k, e, ion, ctl, bb, sc, ion_pushed, keys);
}

// batched columns: one CTA per column
template <class R>
__global__ void __launch_bounds__(kBirthThreads, 1) k_births_batch(const ColDev<R> *cols, int ion_pushed) {
  extern __shared__ __align__(16) unsigned long long keys[];
  __shared__ __align__(16) StepK<R> sk;
  const ColDev<R> *cd = cols + blockIdx.x;
  {
    const int *src = reinterpret_cast<const int *>(&cd->k);
    int *dst = reinterpret_cast<int *>(&sk);
    for (int q = threadIdx.x; q < (int)(sizeof(StepK<R>) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
  }
  __syncthreads();
  births_body<R>(sk, cd->sp[0], cd->sp[1], cd->ctl, cd->bb, cd->sc, ion_pushed, keys);
}

template <class R>
void launch_births(const StepK<R> &k, SpeciesDev e, SpeciesDev i, Ctl *ctl, BirthBuf<R> bb, K3Scratch sc,
                   int ion_pushed, cudaStream_t st) {
  const int bytes = kStageCap * 8;
  cudaFuncSetAttribute(k_births<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  k_births<R><<<1, kBirthThreads, bytes, st>>>(k, e, i, ctl, bb, sc, ion_pushed);
}

template <class R> void launch_births_batch(const ColDev<R> *cols, int ncol, int ion_pushed, cudaStream_t st) {
  const int bytes = kStageCap * 8;
  cudaFuncSetAttribute(k_births_batch<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  k_births_batch<R><<<ncol, kBirthThreads, bytes, st>>>(cols, ion_pushed);
}

// ---------------------------------------------------------------------------
// Field (one CTA).  Gauss's law on the grid with zero-mean space-charge field
// and the uniform background removed (Sec. II, E = -E0 + E_sp):
//   D_j = Q_i,j - Q_e,j,  T = sum D,  S'_j = N sum_{k<=j} D_k - (j+1) T,
//   M = sum S'_j,  E_{j+1/2} = (N S'_j - M) Cf,  Cf = e w / (eps0 2^32 N^2),
//   E_j = (E_{j-1/2} + E_{j+1/2}) / 2 - E0.
// The numerator is an exact 128-bit integer, rounded once to double.

__device__ double i128_to_double(__int128 v) {
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  const unsigned __int128 u = neg ? (unsigned __int128)0 - (unsigned __int128)v : (unsigned __int128)v;
  const unsigned long long hi = (unsigned long long)(u >> 64);
  double d;
  if (hi == 0) {
    d = __ull2double_rn((unsigned long long)u);
  } else {
    const int sh = 64 - __clzll((long long)hi);          // bits dropped below the top 64
    const unsigned long long top = (unsigned long long)(u >> sh);
    const unsigned __int128 rest = u - ((unsigned __int128)top << sh);
    const unsigned long long t = top | (rest != 0 ? 1ull : 0ull);   // sticky bit below the rounding point
    d = __ull2double_rn(t) * __longlong_as_double((long long)(1023 + sh) << 52);
  }
  return neg ? -d : d;
}

// x * n modulo 2^128 (two's complement), n < 2^32
__device__ __forceinline__ __int128 mul_u32(__int128 x, uint32_t n) {
  const unsigned __int128 ux = (unsigned __int128)x;
  const unsigned long long lo = (unsigned long long)ux, hi = (unsigned long long)(ux >> 64);
  const unsigned long long plo = lo * (unsigned long long)n;
  const unsigned long long phi = hi * (unsigned long long)n + __umul64hi(lo, (unsigned long long)n);
  return (__int128)(((unsigned __int128)phi << 64) | (unsigned __int128)plo);
}

__device__ __forceinline__ __int128 shfl_up_i128(__int128 v, int o) {
  const unsigned __int128 u = (unsigned __int128)v;
  const unsigned long long lo = __shfl_up_sync(0xffffffffu, (unsigned long long)u, o);
  const unsigned long long hi = __shfl_up_sync(0xffffffffu, (unsigned long long)(u >> 64), o);
  return (__int128)(((unsigned __int128)hi << 64) | (unsigned __int128)lo);
}
__device__ __forceinline__ __int128 shfl_i128(__int128 v, int src) {
  const unsigned __int128 u = (unsigned __int128)v;
  const unsigned long long lo = __shfl_sync(0xffffffffu, (unsigned long long)u, src);
  const unsigned long long hi = __shfl_sync(0xffffffffu, (unsigned long long)(u >> 64), src);
  return (__int128)(((unsigned __int128)hi << 64) | (unsigned __int128)lo);
}

__device__ __forceinline__ __int128 shfl_i128_down(__int128 v, int o) {
  const unsigned __int128 u = (unsigned __int128)v;
  const unsigned long long lo = __shfl_down_sync(0xffffffffu, (unsigned long long)u, o);
  const unsigned long long hi = __shfl_down_sync(0xffffffffu, (unsigned long long)(u >> 64), o);
  return (__int128)(((unsigned __int128)hi << 64) | (unsigned __int128)lo);
}

// exclusive block scan of 128-bit integers (warp shuffles, one pass through
// shared memory for the warp totals); total receives the block sum
__device__ __int128 block_excl_scan_i128(__int128 v, __int128 *sh, __int128 &total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __int128 incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const __int128 t = shfl_up_i128(incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) sh[w] = incl;
  __syncthreads();
  if (w == 0) {
    __int128 x = lane < nw ? sh[lane] : (__int128)0;
    __int128 xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const __int128 t = shfl_up_i128(xi, o);
      if (lane >= o) xi += t;
    }
    sh[32 + lane] = xi - x;                      // exclusive prefix of warp totals
    if (lane == 31) sh[64] = xi;                 // block total
  }
  __syncthreads();
  const __int128 res = sh[32 + w] + incl - v;
  total = sh[64];
  __syncthreads();
  return res;
}

__device__ double block_excl_scan_f64(double v, double *sh, double &total) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    const double x = t >= off ? sh[t - off] : 0.0;
    __syncthreads();
    sh[t] += x;
    __syncthreads();
  }
  const double incl = sh[t];
  total = sh[blockDim.x - 1];
  __syncthreads();
  return incl - v;
}


// Field solve in two launches over blocks of kEvalThreads nodes.
// Reduction: each block sums R_b = sum D_k and U_b = sum (N - k) D_k over its
// nodes (D = Q_i - Q_e); the last block to finish (atomic ticket, no waiting)
// forms T = sum R_b, M = N U - T N (N+1)/2 (U = sum U_b) and the exact
// block-start values S'_{jb-1} = N (R_0 + .. + R_{b-1}) - jb T.
__device__ __forceinline__ void field_reduce_body(const FieldK &f, const unsigned long long *__restrict__ Qe,
                                                  const unsigned long long *__restrict__ Qi, FieldScan *fs, Ctl *ctl,
                                                  int blk, int nblk, int advance) {
  __shared__ __int128 sh[2 * 32 + 2];   // also the block scans of the last block (65 entries)
  __shared__ bool last;
  const int N = f.N;
  const int j = blk * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __int128 r = 0, u = 0;
  if (j < N && !(f.bounded && j == 0)) {   // bounded column: node 0 is the cathode (surface charge)
    const long long d = (long long)__ldcg(Qi + j) - (long long)__ldcg(Qe + j);
    r = (__int128)d;
    u = mul_u32(r, (uint32_t)(N - j));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r += shfl_i128_down(r, o);
    u += shfl_i128_down(u, o);
  }
  if (lane == 0) { sh[w] = r; sh[32 + w] = u; }
  __syncthreads();
  if (threadIdx.x == 0) {
    __int128 R = 0, U = 0;
    for (int q = 0; q < nw; ++q) { R += sh[q]; U += sh[32 + q]; }
    fs->R[blk] = R;
    fs->U[blk] = U;
    __threadfence();
    last = atomicAdd(&fs->ticket, 1u) == (unsigned)(nblk - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block: one thread per node block (nblk <= blockDim)
  const uint32_t Nu = (uint32_t)N;
  __int128 Rb = 0, Ub = 0;
  if ((int)threadIdx.x < nblk) {
    // L2 reads (the other blocks' writes are not in this SM's L1)
    const longlong2 r2 = __ldcg(reinterpret_cast<const longlong2 *>(&fs->R[threadIdx.x]));
    const longlong2 u2 = __ldcg(reinterpret_cast<const longlong2 *>(&fs->U[threadIdx.x]));
    Rb = (__int128)(((unsigned __int128)(unsigned long long)r2.y << 64) | (unsigned __int128)(unsigned long long)r2.x);
    Ub = (__int128)(((unsigned __int128)(unsigned long long)u2.y << 64) | (unsigned __int128)(unsigned long long)u2.x);
  }
  __int128 T, U;
  const __int128 run = block_excl_scan_i128(Rb, sh, T);    // sum of D before this thread's block
  (void)block_excl_scan_i128(Ub, sh, U);
  if (f.bounded) T = 0;   // between electrodes: no uniform background, the electrodes hold the image charge
  if ((int)threadIdx.x < nblk) fs->Sp0[threadIdx.x] = mul_u32(run, Nu) - (__int128)(threadIdx.x * blockDim.x) * T;
  if (threadIdx.x == 0) {
    const __int128 half = (__int128)((unsigned long long)N * (unsigned long long)(N + 1) / 2ull);
    fs->T = T;
    fs->M = mul_u32(U, Nu) - half * T;
    fs->ticket = 0u;
    if (f.circuit && advance) {
      // Sec. V: the external circuit sets the applied field for the next step
      const double J = f.Cj * (double)(ctl->sumv[0] - ctl->sumv[1]);   // discharge current density
      ctl->E0 = (f.U - f.Rext * J) / f.L;
    }
  }
}

template <class R>
__global__ void __launch_bounds__(kEvalThreads) k_field_reduce(FieldK f, const unsigned long long *__restrict__ Qe,
                                                               const unsigned long long *__restrict__ Qi,
                                                               FieldScan *fs, Ctl *ctl, int advance) {
  field_reduce_body(f, Qe, Qi, fs, ctl, blockIdx.x, gridDim.x, advance);
}

template <class R>
__global__ void __launch_bounds__(kEvalThreads) k_field_reduce_batch(const ColDev<R> *cols) {
  const ColDev<R> *cd = cols + blockIdx.y;
  const FieldK f = cd->fk;
  const int nblk = (f.N + kEvalThreads - 1) / kEvalThreads;
  if ((int)blockIdx.x >= nblk || f.field_mode != PIC_FIELD_POISSON) return;
  field_reduce_body(f, cd->sp[0].Q, cd->sp[1].Q, cd->fs, cd->ctl, blockIdx.x, nblk, 1);
}

// Evaluation (one thread per node): S'_j = S'_{jb-1} + sum over the block up
// to j of (N D_k - T) by a block scan;
//   E_{j+1/2} = (N S'_j - M) Cf,  E_j = (E_{j-1/2} + E_{j+1/2}) / 2 - E0.
// S'_{-1} = 0 = S'_{N-1}, so node 0 gets E_{-1/2} = E_{N-1/2} from the same formula.
template <class R>
__device__ __forceinline__ void field_eval_body(const FieldK &f, const unsigned long long *__restrict__ Qe,
                                                const unsigned long long *__restrict__ Qi, Ctl *ctl,
                                                const FieldScan *fs, double *E, double *Eh, R *Ef, int advance,
                                                int blk) {
  __shared__ __int128 sh[32 + 32 + 1];
  __shared__ double sEh[kEvalThreads + 1];
  const int N = f.N;
  const int j = blk * blockDim.x + threadIdx.x;
  const double E0 = ctl->E0;
  const bool poisson = f.field_mode == PIC_FIELD_POISSON;
  double eh = 0.0;
  if (poisson) {
    const uint32_t Nu = (uint32_t)N;
    const __int128 T = fs->T, M = fs->M;
    __int128 v = 0;
    if (j < N && !(f.bounded && j == 0)) v = mul_u32((__int128)((long long)Qi[j] - (long long)Qe[j]), Nu) - T;
    __int128 tot;
    const __int128 ex = block_excl_scan_i128(v, sh, tot);
    const __int128 Sp0 = fs->Sp0[blk];
    const __int128 Sp = Sp0 + ex + v;                                         // S'_j
    eh = i128_to_double(mul_u32(Sp, Nu) - M) * f.Cf;                          // E_{j+1/2}
    if (threadIdx.x == 0) sEh[0] = i128_to_double(mul_u32(Sp0, Nu) - M) * f.Cf;   // E_{jb-1/2}
  }
  sEh[threadIdx.x + 1] = eh;
  __syncthreads();
  bool bad = false;
  if (j < N) {
    double e;
    if (poisson) {
      Eh[j] = eh;
      // bounded column: the cathode node takes the field of the first half cell
      e = (f.bounded && j == 0) ? eh + (-E0) : 0.5 * (sEh[threadIdx.x] + eh) + (-E0);
    } else {
      Eh[j] = 0.0;
      e = -E0;
    }
    E[j] = e;
    Ef[j] = (R)e;
    if (f.bounded) {
      if (j == N - 1) {   // the anode node: the field of the last half cell
        const double ea = poisson ? eh + (-E0) : -E0;
        E[N] = ea;
        Ef[N] = (R)ea;
        if (!isfinite(ea)) bad = true;
      }
    } else if (j == 0) {
      Ef[N] = (R)e;
    }
    if (!isfinite(e)) bad = true;
  }
  if (bad) atomicOr(&ctl->status, kStNonFinite);
  if (advance && j == 0) {
    ctl->step += 1;
    ctl->m_steps += 1;
  }
}

template <class R>
__global__ void __launch_bounds__(kEvalThreads)
k_field_eval(FieldK f, const unsigned long long *__restrict__ Qe, const unsigned long long *__restrict__ Qi, Ctl *ctl,
             const FieldScan *fs, double *E, double *Eh, R *Ef, int advance) {
  field_eval_body<R>(f, Qe, Qi, ctl, fs, E, Eh, Ef, advance, blockIdx.x);
}

// batched columns: blockIdx.y = column, blockIdx.x = block of nodes
template <class R>
__global__ void __launch_bounds__(kEvalThreads) k_field_eval_batch(const ColDev<R> *cols, int advance) {
  const ColDev<R> *cd = cols + blockIdx.y;
  const FieldK f = cd->fk;
  if ((int)(blockIdx.x * blockDim.x) >= f.N) return;
  field_eval_body<R>(f, cd->sp[0].Q, cd->sp[1].Q, cd->ctl, cd->fs, cd->E, cd->Eh, reinterpret_cast<R *>(cd->Ef),
                     advance, blockIdx.x);
}

// Diagnostic sample of the field step (one CTA, diagnostic steps only):
// phi_j = -dx sum_{k<j} E_{k+1/2} (space-charge potential, phi_0 = 0), densities, E.
__device__ __forceinline__ void field_diag_body(const FieldK &f, const unsigned long long *__restrict__ Qe,
                                                const unsigned long long *__restrict__ Qi, Ctl *ctl, const double *E,
                                                const double *Eh, const Moments &m) {
  __shared__ double shd[kFieldThreads];
  const int N = f.N;
  const int t = threadIdx.x;
  const int seg = f.seg;
  const int j0 = min(N, t * seg), j1 = min(N, j0 + seg);
  double loc = 0.0;
  for (int j = j0; j < j1; ++j) loc += Eh[j];
  double tot;
  const double pre = block_excl_scan_f64(loc, shd, tot);
  double run = pre;
  for (int j = j0; j < j1; ++j) {
    m.phi[j] += -f.dx * run;
    run += Eh[j];
  }
  const int nodes = N + (f.bounded ? 1 : 0);   // a bounded column's anode node N
  for (int j = t; j < nodes; j += blockDim.x) {
    m.ne[j] += (double)(long long)Qe[j] * (1.0 / 4294967296.0);
    m.ni[j] += (double)(long long)Qi[j] * (1.0 / 4294967296.0);
    m.E[j] += E[j];
  }
  if (f.bounded && t == 0) m.phi[N] += -f.dx * tot;
  __syncthreads();
  if (t == 0) {
    ctl->m_samples += 1;
    ctl->n_diag += 1;
  }
}

template <class R>
__global__ void __launch_bounds__(kFieldThreads, 1)
k_field_diag(FieldK f, const unsigned long long *__restrict__ Qe, const unsigned long long *__restrict__ Qi,
             Ctl *ctl, const double *E, const double *Eh, Moments m) {
  field_diag_body(f, Qe, Qi, ctl, E, Eh, m);
}

template <class R>
__global__ void __launch_bounds__(kFieldThreads, 1) k_field_diag_batch(const ColDev<R> *cols) {
  const ColDev<R> *cd = cols + blockIdx.x;
  const FieldK f = cd->fk;
  field_diag_body(f, cd->sp[0].Q, cd->sp[1].Q, cd->ctl, cd->E, cd->Eh, cd->m);
}

template <class R>
void launch_field(const FieldK &f, const unsigned long long *Qe, const unsigned long long *Qi, Ctl *ctl, double *E,
                  double *Eh, R *Ef, Moments m, FieldScan *fs, bool diag, bool advance, cudaStream_t st) {
  const int nblk = (f.N + kEvalThreads - 1) / kEvalThreads;
  if (f.field_mode == PIC_FIELD_POISSON)
    k_field_reduce<R><<<nblk, kEvalThreads, 0, st>>>(f, Qe, Qi, fs, ctl, advance ? 1 : 0);
  k_field_eval<R><<<nblk, kEvalThreads, 0, st>>>(f, Qe, Qi, ctl, fs, E, Eh, Ef, advance ? 1 : 0);
  if (diag) k_field_diag<R><<<1, kFieldThreads, 0, st>>>(f, Qe, Qi, ctl, E, Eh, m);
}

template <class R>
void launch_field_batch(const ColDev<R> *cols, int ncol, int maxN, bool poisson, bool diag, cudaStream_t st) {
  const dim3 grid((maxN + kEvalThreads - 1) / kEvalThreads, ncol);
  if (poisson) k_field_reduce_batch<R><<<grid, kEvalThreads, 0, st>>>(cols);
  k_field_eval_batch<R><<<grid, kEvalThreads, 0, st>>>(cols, 1);
  if (diag) k_field_diag_batch<R><<<ncol, kFieldThreads, 0, st>>>(cols);
}

__global__ void k_i128_test(const int64_t *hi, const uint64_t *lo, double *out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const __int128 v = (__int128)(((unsigned __int128)(uint64_t)hi[i] << 64) | (unsigned __int128)lo[i]);
    out[i] = i128_to_double(v);
  }
}

void launch_i128_test(const int64_t *hi, const uint64_t *lo, double *out, int n, cudaStream_t st) {
  k_i128_test<<<(n + 255) / 256, 256, 0, st>>>(hi, lo, out, n);
}

// ---------------------------------------------------------------------------
// Initial state: uniform positions, Maxwellian velocities (Sec. II).
template <class R>
__global__ void k_init(const __grid_constant__ StepK<R> k, SpeciesDev s, int species, long long n, uint64_t id0, R sig) {
  const uint2 key = seed_key(k.seed);
  const uint32_t c3 = ((species == 0 ? (uint32_t)kStInitE : (uint32_t)kStInitI) << 28) | (k.column << 16);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    const uint64_t id = id0 + (uint64_t)p;
    const uint32_t a = (uint32_t)id, b = (uint32_t)(id >> 32);
    const uint4 w = philox10(make_uint4(a, b, 0u, c3 | 0u), key);
    const uint4 x = philox10(make_uint4(a, b, 0u, c3 | 1u), key);
    const int32_t cell = (int32_t)(((unsigned long long)w.x * (unsigned long long)(uint32_t)k.N) >> 32);
    R off, vx, vy, vz;
    if constexpr (std::is_same<R, float>::value) {
      off = u24(w.y);
      vx = sig * gauss<float>(k.gauss, u24(w.z));
      vy = sig * gauss<float>(k.gauss, u24(w.w));
      vz = sig * gauss<float>(k.gauss, u24(x.x));
    } else {
      const uint4 y = philox10(make_uint4(a, b, 0u, c3 | 2u), key);
      off = u53(w.y, w.z);
      vx = sig * gauss<double>(k.gauss, u53(x.x, x.y));
      vy = sig * gauss<double>(k.gauss, u53(x.z, x.w));
      vz = sig * gauss<double>(k.gauss, u53(y.x, y.y));
    }
    s.cell[p] = cell;
    rec_store<R>(s.rec, p, off, vx, vy, vz);
    s.id[p] = id;
  }
}

template <class R>
void launch_init(const StepK<R> &k, SpeciesDev s, int species, int64_t n, uint64_t id0, R sig, cudaStream_t st) {
  if (n <= 0) return;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_init<R><<<blocks, 256, 0, st>>>(k, s, species, (long long)n, id0, sig);
}

template <class R>
__global__ void k_deposit(SpeciesDev s, const Ctl *ctl, int species, int N) {
  const long long n = ctl->n[species];
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
    dep_global<R>(s.Q, N, s.cell[p], rec_get_off<R>(s.rec, p), true);
}

template <class R>
void launch_deposit(const StepK<R> &k, SpeciesDev s, const Ctl *ctl, int species, cudaStream_t st) {
  k_deposit<R><<<152 * 8, 256, 0, st>>>(s, ctl, species, k.Nw);
}

// leapfrog start: v^{-1/2} = v^0 - (q dt / 2m) E^0(x^0)
template <class R>
__global__ void k_halfstep(SpeciesDev s, const Ctl *ctl, const R *Ef, int species, R a) {
  const long long n = ctl->n[species];
  const R ha = (R)0.5 * a;
  using T = typename Rec<R>::T;
  T *rec = reinterpret_cast<T *>(s.rec);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    R off, vx, vy, vz;
    rec_load<R>(s.rec, p, off, vx, vy, vz);
    const R Ep = gather(Ef, s.cell[p], off);
    vx = vx - ha * Ep;
    rec_store<R>(s.rec, p, off, vx, vy, vz);
  }
  (void)rec;
}

template <class R>
void launch_halfstep(const StepK<R> &k, SpeciesDev s, const Ctl *ctl, const R *Ef, int species, cudaStream_t st) {
  k_halfstep<R><<<152 * 8, 256, 0, st>>>(s, ctl, Ef, species, k.sp[species].a);
}

template <class R> __global__ void k_sumv(SpeciesDev s, Ctl *ctl, int species) {
  const long long n = ctl->n[species];
  long long acc = 0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    R off, vx, vy, vz;
    rec_load<R>(s.rec, p, off, vx, vy, vz);
    acc += vfix(vx);
  }
  unsigned long long u = (unsigned long long)acc;
  for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
  if ((threadIdx.x & 31) == 0 && u) atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->sumv[species]), u);
}

template <class R> void launch_sumv(SpeciesDev s, Ctl *ctl, int species, cudaStream_t st) {
  k_sumv<R><<<152 * 4, 256, 0, st>>>(s, ctl, species);
}

// explicit instantiations
#define PIC_INST(R)                                                                                                  \
  template void launch_init<R>(const StepK<R> &, SpeciesDev, int, int64_t, uint64_t, R, cudaStream_t);              \
  template void launch_deposit<R>(const StepK<R> &, SpeciesDev, const Ctl *, int, cudaStream_t);                    \
  template void launch_halfstep<R>(const StepK<R> &, SpeciesDev, const Ctl *, const R *, int, cudaStream_t);        \
  template void launch_push<R>(const StepK<R> &, SpeciesDev, Ctl *, const R *, BirthBuf<R>, Moments, int, int, bool, \
                               cudaStream_t);                                                                        \
  template void launch_births<R>(const StepK<R> &, SpeciesDev, SpeciesDev, Ctl *, BirthBuf<R>, K3Scratch, int,      \
                                 cudaStream_t);                                                                      \
  template void launch_field<R>(const FieldK &, const unsigned long long *, const unsigned long long *, Ctl *,       \
                                double *, double *, R *, Moments, FieldScan *, bool, bool, cudaStream_t);            \
  template int push_smem_bytes<R>(int);                                                                             \
  template void launch_sumv<R>(SpeciesDev, Ctl *, int, cudaStream_t);                                               \
  template size_t push_layout<R>(int, int &, int &, int &, int &);                                                                \
  template void launch_zero_q_batch<R>(const ColDev<R> *, int, int, int, cudaStream_t);                             \
  template void launch_push_batch<R>(const ColDev<R> *, const int4 *, int, int, size_t, bool, cudaStream_t);              \
  template void launch_births_batch<R>(const ColDev<R> *, int, int, cudaStream_t);                                  \
  template void launch_field_batch<R>(const ColDev<R> *, int, int, bool, bool, cudaStream_t);
PIC_INST(double)
PIC_INST(float)

}  // namespace pic
