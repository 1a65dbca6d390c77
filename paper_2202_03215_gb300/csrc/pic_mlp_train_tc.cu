// Closure-network training on the 5th-generation tensor cores (tcgen05): forward,
// backward and weight gradients of one tile of 128 samples per CTA.
//
// Every product is a tcgen05.mma of kind::f16 (BF16 operands in shared memory, FP32
// accumulators in tensor memory), issued by one thread; the CTA's 512 threads run the
// epilogues between them (tcgen05.ld of the accumulator rows, bias, GELU and its
// derivative, BF16 conversion).  Operands use the canonical no-swizzle layouts: a tile
// stored K-major for one product is read MN-major (transpose bit of the instruction
// descriptor) by the next, so no transposed copy is made:
//   forward   Z1 = X W1^T, A1 = gelu(Z1 + b1); Z2 = A1 W2^T, A2 = gelu(Z2 + b2);
//             Y = A2 W3^T + b3
//   backward  dY = 2 (Y - T) / (3 n); dA2 = dY W3; dZ2 = dA2 gelu'(Z2 + b2);
//             dA1 = dZ2 W2; dZ1 = dA1 gelu'(Z1 + b1)
//   gradients dW3^T = A2^T dY, dW2 = dZ2^T A1, dW1 = dZ1^T X; the bias gradients are the
//             column sums of dZ (dZ^T times a tile of ones; dz is split into a BF16 high
//             part and a BF16 low part so that the sums keep FP32 accuracy) and of dY
//             (warp sums in FP32)
// Tensor-memory columns: Z1 [0,128), Z2 [128,256) then dA1, Y [256,272), dA2 [272,400)
// then dW2, dW3^T [400,416), gb2 [416,432), dW1 [432,448), gb1 [448,464).
// The CTA writes its tile's partial gradient (the parameter layout, FP32) and its summed
// squared error; the reduction kernel of pic_mlp.cu sums the tiles in a fixed order and
// applies Adam.  Every wait is bounded: a wait that gives up sets *status, and the CTA
// frees its tensor memory once no MMA it issued can still be running.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pic.h"
#include "pic_mlp_layout.cuh"

namespace {

using bf = __nv_bfloat16;
using namespace mlpl;

constexpr int TM = 128;              // samples per tile (MMA rows)
constexpr int THREADS = 512;         // four threads per sample row in the epilogues (32 columns each)
constexpr int CW = NH / (THREADS / TM);   // columns per thread in the epilogues
constexpr uint32_t kCols = 512;      // tensor-memory columns of the CTA
constexpr uint32_t cZ1 = 0, cZ2 = 128, cY = 256, cA2d = 272, cW3t = 400, cGb2 = 416, cW1 = 432, cGb1 = 448;

struct __align__(1024) TrSmem {
  TrainW w;               // BF16 weights (canonical K-major)
  bf X[TM * K1];          // inputs, K-major (K = 16 inputs, column 15 zero)
  bf dY[TM * N3];         // dL/dy, K-major (K = 16 outputs, columns 3..15 zero)
  bf ones[N3 * TM];       // B operand of the bias sums: N = 16, K = 128 samples, all ones
  bf A1[TM * NH];         // activations of layer 1 (K-major, K = hidden)
  bf A2[TM * NH];         // activations of layer 2, then dZ1
  bf dZ2[TM * NH];        // dL/dz2 (BF16 high part)
  bf dZlo[TM * NH];       // low BF16 parts of dz2, then of dz1
  float b1[NH], b2[NH], b3[N3];
  float red[4][4];        // per-warp sums: dy of the three outputs, squared error
  unsigned long long mbar_w, mbar_mma;
  uint32_t tmem_slot;
  int ok;
};

__device__ __forceinline__ uint32_t su(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (no swizzle): start >> 4, leading offset >> 4 (bits 16..29),
// stride offset >> 4 (bits 32..45), fixed 0b001 at bits 46..48
__device__ __forceinline__ uint64_t sdesc(const void *p, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((su(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// K-major operand with K elements per row: core matrices 128 B apart along K, 8-row groups K x 16 B apart
__device__ __forceinline__ uint64_t dk(const void *p, int K) { return sdesc(p, 128, (uint32_t)K * 16); }
// MN-major operand (no swizzle) read from a tile stored K-major for another product: core
// matrices of 8 K-rows x 16 bytes along M (or N), 8-element groups along M mn_stride bytes apart,
// 8-row groups along K k_stride bytes apart.  The leading byte offset holds the K stride and the
// stride byte offset the M stride (checked on the GPU against a reference product).
__device__ __forceinline__ uint64_t dmn(const void *p, uint32_t mn_stride, uint32_t k_stride) {
  return sdesc(p, k_stride, mn_stride);
}
// instruction descriptor of kind::f16: D FP32, A and B BF16, transpose (MN-major) bits 15 (A) and
// 16 (B), N >> 3 at bits 17..22, M >> 4 at bits 24..28
__host__ __device__ constexpr uint32_t idesc(uint32_t M, uint32_t N, uint32_t ta, uint32_t tb) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (ta << 15) | (tb << 16) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit(unsigned long long *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su(mbar))
               : "memory");
}
__device__ __forceinline__ bool wait_phase(unsigned long long *mbar, uint32_t parity, int spin) {
  for (int it = 0; it < spin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, 10000;\nselp.b32 %0, 1, 0, P;\n}\n"
        : "=r"(done)
        : "r"(su(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
    __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// operands written by the threads become visible to the tensor core; tensor-memory reads before
// the barrier are ordered before the MMAs after it
__device__ __forceinline__ void handoff() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_before();
  __syncthreads();
  tc_after();
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// GELU (tanh form) and its derivative with the hardware tanh (relative error about 2^-11):
// gelu = z (1 + th)/2, gelu' = (1 + th)/2 + z (1 - th^2) du/dz / 2, u = sqrt(2/pi)(z + 0.044715 z^3)
__device__ __forceinline__ float gelu(float z) {
  const float u = 0.7978845608028654f * z * (1.0f + 0.044715f * z * z);
  float th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(u));
  const float h = 0.5f * z;
  return h + h * th;
}
__device__ __forceinline__ float gelu_d(float z) {
  const float c = 0.7978845608028654f, z2 = z * z;
  float th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(c * z * (1.0f + 0.044715f * z2)));
  const float h = 0.5f * (1.0f + th);
  return h + 0.5f * z * (1.0f - th * th) * c * (1.0f + 3.0f * 0.044715f * z2);
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}
// eight values -> row r, columns c..c+7 of a K-major tile with K columns (16 bytes)
__device__ __forceinline__ void put8(bf *tile, int r, int c, int K, const float *v) {
  uint4 q;
  q.x = pack2(v[0], v[1]); q.y = pack2(v[2], v[3]); q.z = pack2(v[4], v[5]); q.w = pack2(v[6], v[7]);
  *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(tile) + cm_off(r, c, K)) = q;
}

// forward epilogue: CW columns (c0..) of accumulator row r -> gelu(z + b) in BF16
__device__ __forceinline__ void epi_act(bf *A, uint32_t tz, const float *b, int r, int c0) {
#pragma unroll 1
  for (int c = c0; c < c0 + CW; c += 16) {
    float v[16];
    ld16(tz + (uint32_t)c, v);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = gelu(v[i] + b[c + i]);
    put8(A, r, c, NH, v);
    put8(A, r, c + 8, NH, v + 8);
  }
}
// backward epilogue: dz = dA gelu'(z + b), stored as BF16 high and low parts
__device__ __forceinline__ void epi_dz(bf *D, bf *Dlo, uint32_t tda, uint32_t tz, const float *b, int r, int c0) {
#pragma unroll 1
  for (int c = c0; c < c0 + CW; c += 16) {
    float a[16], z[16], hi[16], lo[16];
    ld16(tda + (uint32_t)c, a);
    ld16(tz + (uint32_t)c, z);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float dz = a[i] * gelu_d(z[i] + b[c + i]);
      hi[i] = __bfloat162float(__float2bfloat16_rn(dz));
      lo[i] = dz - hi[i];
    }
    put8(D, r, c, NH, hi);
    put8(D, r, c + 8, NH, hi + 8);
    put8(Dlo, r, c, NH, lo);
    put8(Dlo, r, c + 8, NH, lo + 8);
  }
}

__global__ void __launch_bounds__(THREADS, 1)
k_mlp_tile_tc(const float *__restrict__ P, const TrainW *__restrict__ Wb, const float *__restrict__ X,
              const float *__restrict__ T, int n, float inv_n3, float *__restrict__ gpart, float *__restrict__ lpart,
              int *__restrict__ status, int spin, unsigned hook) {
  extern __shared__ __align__(1024) unsigned char raw[];
  TrSmem &S = *reinterpret_cast<TrSmem *>(raw);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int q = w & 3, part = w >> 2;            // lane quadrant of the warp, column part
  const int r = 32 * q + lane;                   // accumulator row (sample, or hidden unit)
  const int c0 = CW * part;
  const int tile = blockIdx.x, s0 = tile * TM;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su(&S.tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the tile's inputs (the caller's, ready before the launch) while the previous kernel of the
  // stream may still run; the weights come from its Adam update: wait for it before reading them
  const int rows = min(TM, n - s0);
  for (int e = tid; e < TM * K1; e += THREADS) {
    const int rr = e / K1, i = e % K1;
    *reinterpret_cast<bf *>(reinterpret_cast<unsigned char *>(S.X) + cm_off(rr, i, K1)) =
        __float2bfloat16_rn((rr < rows && i < NI) ? X[(size_t)(s0 + rr) * NI + i] : 0.0f);
    *reinterpret_cast<bf *>(reinterpret_cast<unsigned char *>(S.dY) + cm_off(rr, i, N3)) = __float2bfloat16_rn(0.0f);
    S.ones[e] = __float2bfloat16_rn(1.0f);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su(&S.mbar_w)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su(&S.mbar_mma)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!(hook & PIC_MLP_HOOK_NO_WEIGHT_COPY)) {   // the hook leaves this barrier without an arrival
      asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                       su(&S.mbar_w)),
                   "r"((unsigned)sizeof(TrainW))
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       su(&S.w)),
                   "l"(Wb), "r"((unsigned)sizeof(TrainW)), "r"(su(&S.mbar_w))
                   : "memory");
    }
  }
  for (int e = tid; e < NH; e += THREADS) { S.b1[e] = P[ob1 + e]; S.b2[e] = P[ob2 + e]; }
  if (tid < N3) S.b3[tid] = tid < NO ? P[ob3 + tid] : 0.0f;
  if (tid == 0) {
    const bool ok = wait_phase(&S.mbar_w, 0, spin);
    S.ok = ok ? 1 : 0;
    if (!ok) atomicExch(status, 1);   // nothing was issued on the barrier: nothing is in flight
  }
  handoff();
  const uint32_t tm = S.tmem_slot;
  const uint32_t trow = tm + ((uint32_t)(32 * q) << 16);   // this warp's lanes
  uint32_t ph = 0;
  bool pending = false;   // an MMA batch was committed whose completion was not seen
  // thread 0 issues, commits and waits; the barrier passes the outcome on
  auto run = [&](auto issue) -> bool {
    if (tid == 0) {
      issue();
      commit(&S.mbar_mma);
      S.ok = wait_phase(&S.mbar_mma, ph, spin) ? 1 : 0;
      if (!S.ok) atomicExch(status, 1);
    }
    ph ^= 1u;
    __syncthreads();
    const bool ok = S.ok != 0;
    pending = !ok;
    tc_after();
    return ok;
  };
  bool ok = S.ok != 0;
  constexpr uint32_t kM = 4096, kX = 512;   // bytes per K step of 16 samples: 128-wide and 16-wide tiles
  if (ok) ok = run([&] { mma(tm + cZ1, dk(S.X, K1), dk(S.w.W1, K1), idesc(TM, NH, 0, 0), 0u); });
  if (ok) {
    epi_act(S.A1, trow + cZ1, S.b1, r, c0);
    handoff();
    ok = run([&] {
      for (uint32_t k = 0; k < NH / 16; ++k)
        mma(tm + cZ2, dk(S.A1, NH) + k * 16u, dk(S.w.W2, NH) + k * 16u, idesc(TM, NH, 0, 0), k);
    });
  }
  if (ok) {
    epi_act(S.A2, trow + cZ2, S.b2, r, c0);
    handoff();
    ok = run([&] {
      for (uint32_t k = 0; k < NH / 16; ++k)
        mma(tm + cY, dk(S.A2, NH) + k * 16u, dk(S.w.W3, NH) + k * 16u, idesc(TM, N3, 0, 0), k);
    });
  }
  if (ok) {
    // outputs, loss and dL/dy (rows of samples past n contribute nothing)
    if (part == 0) {
      float v[16];
      ld16(trow + cY, v);
      const bool valid = r < rows;
      float dy[NO], sq = 0.0f;
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        const float d = valid ? v[o] + S.b3[o] - T[(size_t)(s0 + r) * NO + o] : 0.0f;
        sq += d * d;
        dy[o] = 2.0f * d * inv_n3;
        *reinterpret_cast<bf *>(reinterpret_cast<unsigned char *>(S.dY) + cm_off(r, o, N3)) = __float2bfloat16_rn(dy[o]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dy[0] += __shfl_xor_sync(0xffffffffu, dy[0], o);
        dy[1] += __shfl_xor_sync(0xffffffffu, dy[1], o);
        dy[2] += __shfl_xor_sync(0xffffffffu, dy[2], o);
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
      }
      if (lane == 0) { S.red[q][0] = dy[0]; S.red[q][1] = dy[1]; S.red[q][2] = dy[2]; S.red[q][3] = sq; }
    }
    handoff();
    ok = run([&] {
      // dA2 = dY W3 (W3 read MN-major: N = hidden, K = outputs)
      mma(tm + cA2d, dk(S.dY, N3), dmn(S.w.W3, 128, 2048), idesc(TM, NH, 0, 1), 0u);
      // dW3^T = A2^T dY (both MN-major, K = samples)
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cW3t, dmn(S.A2, 128, 2048) + k * (kM >> 4), dmn(S.dY, 128, 256) + k * (kX >> 4),
            idesc(TM, N3, 1, 1), k);
    });
  }
  if (ok) {
    epi_dz(S.dZ2, S.dZlo, trow + cA2d, trow + cZ2, S.b2, r, c0);
    handoff();
    ok = run([&] {
      // dA1 = dZ2 W2 (W2 read MN-major: N = hidden in, K = hidden out), into Z2's columns
      for (uint32_t k = 0; k < NH / 16; ++k)
        mma(tm + cZ2, dk(S.dZ2, NH) + k * 16u, dmn(S.w.W2, 128, 2048) + k * (kM >> 4), idesc(TM, NH, 0, 1), k);
      // dW2 = dZ2^T A1 (both MN-major, K = samples), into dA2's columns
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cA2d, dmn(S.dZ2, 128, 2048) + k * (kM >> 4), dmn(S.A1, 128, 2048) + k * (kM >> 4),
            idesc(NH, NH, 1, 1), k);
      // gb2 = column sums of dz2 (high and low parts) against a tile of ones
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cGb2, dmn(S.dZ2, 128, 2048) + k * (kM >> 4), dk(S.ones, TM) + k * 16u, idesc(NH, N3, 1, 0), k);
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cGb2, dmn(S.dZlo, 128, 2048) + k * (kM >> 4), dk(S.ones, TM) + k * 16u, idesc(NH, N3, 1, 0), 1u);
    });
  }
  if (ok) {
    bf *dZ1 = S.A2;   // A2 was last read by the dW3 product, which has completed
    epi_dz(dZ1, S.dZlo, trow + cZ2, trow + cZ1, S.b1, r, c0);
    handoff();
    ok = run([&] {
      // dW1 = dZ1^T X (both MN-major, K = samples); gb1 as gb2
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cW1, dmn(dZ1, 128, 2048) + k * (kM >> 4), dmn(S.X, 128, 256) + k * (kX >> 4), idesc(NH, N3, 1, 1), k);
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cGb1, dmn(dZ1, 128, 2048) + k * (kM >> 4), dk(S.ones, TM) + k * 16u, idesc(NH, N3, 1, 0), k);
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cGb1, dmn(S.dZlo, 128, 2048) + k * (kM >> 4), dk(S.ones, TM) + k * 16u, idesc(NH, N3, 1, 0), 1u);
    });
  }
  if (ok) {
    // the tile's partial gradient: accumulator row r is hidden unit r
    float *gp = gpart + (size_t)tile * GSTRIDE;
#pragma unroll 1
    for (int c = c0; c < c0 + CW; c += 16) {
      float v[16];
      ld16(trow + cA2d + (uint32_t)c, v);
      float4 *dst = reinterpret_cast<float4 *>(gp + oW2 + r * NH + c);   // oW2 and the row stride are multiples of 4
#pragma unroll
      for (int i = 0; i < 4; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
    if (part == 0) {
      float v[16];
      ld16(trow + cW1, v);
#pragma unroll
      for (int i = 0; i < NI; ++i) gp[oW1 + r * NI + i] = v[i];
      ld16(trow + cGb1, v);
      gp[ob1 + r] = v[0];
      ld16(trow + cGb2, v);
      gp[ob2 + r] = v[0];
      ld16(trow + cW3t, v);
#pragma unroll
      for (int o = 0; o < NO; ++o) gp[oW3 + o * NH + r] = v[o];
    }
    if (tid == 0) {
      float gb3[NO] = {0.0f, 0.0f, 0.0f}, sq = 0.0f;
      for (int k = 0; k < 4; ++k) {
        for (int o = 0; o < NO; ++o) gb3[o] += S.red[k][o];
        sq += S.red[k][3];
      }
      for (int o = 0; o < NO; ++o) gp[ob3 + o] = gb3[o];
      lpart[tile] = sq;
    }
  }
  // a batch whose wait gave up: wait once more (bounded) before the tensor memory is freed
  if (pending && tid == 0) wait_phase(&S.mbar_mma, ph ^ 1u, spin);
  tc_before();
  __syncthreads();
  tc_after();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kCols) : "memory");
}

}  // namespace

// one training tile kernel per 128 samples, with programmatic stream serialization (the next
// kernel of the stream may be scheduled while this one drains)
int mlp_train_tiles_tc(const float *P, const void *Wb, const float *X, const float *T, int n, float inv_n3,
                       float *gpart, float *lpart, int *status, int spin, unsigned hook, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_mlp_tile_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrSmem)) !=
        cudaSuccess)
      return PIC_ECUDA;
    attr = true;
  }
  cudaLaunchAttribute pdl;
  pdl.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl.val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.stream = st;
  cfg.attrs = &pdl;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((n + TM - 1) / TM);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = sizeof(TrSmem);
  return cudaLaunchKernelEx(&cfg, k_mlp_tile_tc, P, reinterpret_cast<const TrainW *>(Wb), X, T, n, inv_n3, gpart,
                            lpart, status, spin, hook) == cudaSuccess
             ? 0
             : PIC_ECUDA;
}
