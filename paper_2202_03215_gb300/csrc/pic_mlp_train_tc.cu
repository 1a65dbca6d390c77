// Closure-network training on the 5th-generation tensor cores (tcgen05): forward,
// backward and weight gradients of tiles of 128 samples, one persistent CTA per SM.
//
// Every product is a tcgen05.mma of kind::f16 (BF16 operands in shared memory, FP32
// accumulators in tensor memory), issued by one thread; the CTA's 512 threads run the
// epilogues between them (tcgen05.ld of the accumulator rows, bias, GELU, BF16 conversion).
// Operands use the canonical no-swizzle layouts: a tile stored K-major for one product is
// read MN-major (transpose bit of the instruction descriptor) by the next, so no transposed
// copy is made.  Per tile:
//   R1  Z1 = X W1^T;          epilogue A1 = gelu(Z1 + b1), gelu'(Z1 + b1) stored over Z1
//   R2  Z2 = A1 W2^T;         epilogue A2 = gelu(Z2 + b2), gelu'(Z2 + b2) stored over Z2, and
//                             Y = A2 W3^T (three outputs: on the CUDA cores from the BF16 A2 and W3
//                             an MMA would take); then dY = 2 (Y + b3 - T) / (3 n),
//                             dA2 = dY W3 (CUDA cores, BF16-rounded dY and W3), dZ2 = dA2 gelu'
//   R3  dW3^T += A2^T dY, gb2 += dZ2lo^T 1, dA1 = dZ2 W2 (waited for); dW2^T += A1^T dZ2 and
//       gb2 += dZ2hi^T 1 run on under the epilogue dZ1 = dA1 gelu'
//   R4  [dW1 | gb1] += dZ1^T [X 1] (X carries a column of ones, so column 15 is gb1); issued after
//       the next tile's R1 (committed on its own), so that it runs under that tile's layer-1
//       epilogue; the next tile's R2 commit covers it (and the unwaited half of R3)
// dZ is stored as a BF16 high part and a BF16 low part: the weight gradients take the high
// part (BF16 operands, like every product), the bias gradients (gb2, gb1) take both, so that
// the sums keep FP32 accuracy.  gb3 and the squared error are warp sums in FP32.  The weight
// gradients accumulate in tensor memory over the CTA's tiles (tiles b, b + G, b + 2G, .. of a
// grid of G CTAs); the CTA writes them once as its partial, and the reduction kernel of
// pic_mlp.cu sums the G partials in a fixed order and applies Adam.
// Tensor-memory columns: Z1 then gelu'(Z1) [0,128), Z2 then gelu'(Z2) then dA1 [128,256),
// dW2^T [272,400), dW3^T [400,416), gb2 [416,432), dW1 | gb1 [432,448), the low
// part's [X 1] product (its column 15 completes gb1) [448,464).
// Every wait is bounded: a wait that gives up sets *status, and the CTA frees its tensor
// memory once no MMA it issued can still be running.
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
constexpr int ISSUER = 0;            // the thread that also issues, commits and waits for the MMAs
constexpr int CW = NH / (THREADS / TM);   // columns per thread in the epilogues
constexpr int XPT = (TM * NI + THREADS - 1) / THREADS;   // input values per thread per tile
constexpr uint32_t kCols = 512;      // tensor-memory columns of the CTA
constexpr uint32_t cZ1 = 0, cZ2 = 128, cW2 = 272, cW3t = 400, cGb2 = 416, cW1 = 432, cW1lo = 448;

struct __align__(1024) TrSmem {
  TrainW w;               // BF16 weights (canonical K-major)
  bf X[2][TM * K1];       // inputs of this tile and the next, K-major (K = 16: 15 inputs, then 1)
  bf dY[TM * N3];         // dL/dy, K-major (K = 16 outputs, columns 3..15 zero)
  bf ones[N3 * TM];       // B operand of the bias sums: N = 16, K = 128 samples, all ones
  bf A1[TM * NH];         // activations of layer 1 (K-major, K = hidden)
  bf A2[TM * NH];         // activations of layer 2, then dZ1
  bf dZ2[TM * NH];        // dL/dz2 (BF16 high part)
  bf dZlo[TM * NH];       // low BF16 parts of dz2, then of dz1
  float b1[NH], b2[NH], b3[N3];
  float W3[NO][NH];       // output weights rounded to BF16 (Y = A2 W3^T and dA2 = dY W3)
  float yp[THREADS / TM][NO][TM];   // partial outputs of each column part
  float red[4][4];        // per-warp sums over the CTA's tiles: dy of the three outputs, squared error
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

// 16 consecutive FP32 columns into this thread's tensor-memory lane
__device__ __forceinline__ void st16(uint32_t taddr, const float v[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Pairs of FP32 values in one 64-bit register, operated on by the packed FP32 instructions
// (.f32x2): half the instructions of the scalar form in the epilogues.
using f2 = unsigned long long;
__device__ __forceinline__ f2 pk(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(f2 v, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ f2 dup(float a) { return pk(a, a); }
// the pair rounded to BF16, packed (first value in the low half: the lower address)
__device__ __forceinline__ uint32_t bf2(f2 v) {
  float a, b;
  upk(v, a, b);
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}
// the packed BF16 pair back to FP32 (exact)
__device__ __forceinline__ f2 unbf2(uint32_t w) { return pk(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u)); }
__device__ __forceinline__ f2 tanh2(f2 u) {
  float a, b;
  upk(u, a, b);
  asm("tanh.approx.f32 %0, %0;" : "+f"(a));
  asm("tanh.approx.f32 %0, %0;" : "+f"(b));
  return pk(a, b);
}

// GELU (tanh form) and its derivative from one hardware tanh (relative error about 2^-11), on a
// pair: u = sqrt(2/pi)(z + 0.044715 z^3), th = tanh u, h = (1 + th)/2,
// gelu = z h, gelu' = h + z (1 - th^2) du/dz / 2
__device__ __forceinline__ void gelu2(f2 z, f2 &g, f2 &d) {
  const float c = 0.7978845608028654f, a = 0.044715f;
  const f2 z2 = mul2(z, z);
  const f2 th = tanh2(mul2(z, fma2(z2, dup(c * a), dup(c))));
  const f2 h = fma2(th, dup(0.5f), dup(0.5f));
  g = mul2(z, h);
  const f2 q = mul2(z, fma2(z2, dup(1.5f * c * a), dup(0.5f * c)));
  d = fma2(q, sub2(dup(1.0f), mul2(th, th)), h);
}
// four packed BF16 pairs -> row r, columns c..c+7 of a K-major tile with K columns (16 bytes)
__device__ __forceinline__ void put8w(bf *tile, int r, int c, int K, uint32_t w0, uint32_t w1, uint32_t w2,
                                      uint32_t w3) {
  *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(tile) + cm_off(r, c, K)) = make_uint4(w0, w1, w2, w3);
}
__device__ __forceinline__ void put1(bf *tile, int r, int c, int K, float v) {
  *reinterpret_cast<bf *>(reinterpret_cast<unsigned char *>(tile) + cm_off(r, c, K)) = __float2bfloat16_rn(v);
}
// 16 values (8 pairs) as BF16 high parts into H and the BF16-rounded rests into L, row r, columns c..c+15
__device__ __forceinline__ void put16_split(bf *H, bf *L, int r, int c, const f2 v[8]) {
  uint32_t hw[8], lw[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    hw[i] = bf2(v[i]);
    lw[i] = bf2(sub2(v[i], unbf2(hw[i])));
  }
  put8w(H, r, c, NH, hw[0], hw[1], hw[2], hw[3]);
  put8w(H, r, c + 8, NH, hw[4], hw[5], hw[6], hw[7]);
  put8w(L, r, c, NH, lw[0], lw[1], lw[2], lw[3]);
  put8w(L, r, c + 8, NH, lw[4], lw[5], lw[6], lw[7]);
}

// forward epilogue: CW columns (c0..) of accumulator row r -> gelu(z + b) in BF16 into A,
// gelu'(z + b) in FP32 back into the accumulator's columns; with OUT, also this part's share
// of the outputs y_o = sum_c a_c W3[o][c] (the BF16 a_c and W3 an MMA would take, FP32 sums)
template <bool OUT>
__device__ __forceinline__ void epi_act(bf *A, uint32_t tz, const float *b, int r, int c0, const float (*W3)[NH],
                                        float (*yp)[TM]) {
  f2 y0 = 0ull, y1 = 0ull, y2 = 0ull;   // (+0, +0) pairs
#pragma unroll 1
  for (int c = c0; c < c0 + CW; c += 16) {
    float v[16];
    uint32_t w[8];
    ld16(tz + (uint32_t)c, v);
    const float2 *b2 = reinterpret_cast<const float2 *>(b + c);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 bb = b2[i];
      f2 g, d;
      gelu2(add2(pk(v[2 * i], v[2 * i + 1]), pk(bb.x, bb.y)), g, d);
      w[i] = bf2(g);
      upk(d, v[2 * i], v[2 * i + 1]);
      if (OUT) {
        const f2 a = unbf2(w[i]);
        y0 = fma2(a, reinterpret_cast<const f2 *>(&W3[0][c])[i], y0);
        y1 = fma2(a, reinterpret_cast<const f2 *>(&W3[1][c])[i], y1);
        y2 = fma2(a, reinterpret_cast<const f2 *>(&W3[2][c])[i], y2);
      }
    }
    put8w(A, r, c, NH, w[0], w[1], w[2], w[3]);
    put8w(A, r, c + 8, NH, w[4], w[5], w[6], w[7]);
    st16(tz + (uint32_t)c, v);
  }
  if (OUT) {
    float a, b2;
    upk(y0, a, b2); yp[0][r] = a + b2;
    upk(y1, a, b2); yp[1][r] = a + b2;
    upk(y2, a, b2); yp[2][r] = a + b2;
  }
}

// the tile's inputs: XPT values per thread (row-major X, NI per sample), in registers until stored
__device__ __forceinline__ void load_x(const float *__restrict__ X, int s0, int rows, int tid, float xv[XPT]) {
#pragma unroll
  for (int j = 0; j < XPT; ++j) {
    const int e = tid + THREADS * j;
    xv[j] = (e < rows * NI) ? __ldg(X + (size_t)s0 * NI + e) : 0.0f;
  }
}
__device__ __forceinline__ void put_x(bf *Xt, int rows, int tid, const float xv[XPT]) {
#pragma unroll
  for (int j = 0; j < XPT; ++j) {
    const int e = tid + THREADS * j;
    if (e < TM * NI) put1(Xt, e / NI, e % NI, K1, xv[j]);
  }
  if (tid < TM) put1(Xt, tid, NI, K1, tid < rows ? 1.0f : 0.0f);   // the ones column (W1's is zero)
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
  const int ntiles = (n + TM - 1) / TM, G = gridDim.x;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su(&S.tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the first tile's inputs (the caller's, ready before the launch) while the previous kernel of
  // the stream may still run; the weights come from its Adam update: wait for it before reading them
  float xv[XPT];
  {
    const int s0 = blockIdx.x * TM;
    load_x(X, s0, min(TM, n - s0), tid, xv);
    put_x(S.X[0], min(TM, n - s0), tid, xv);
  }
  for (int e = tid; e < TM * N3; e += THREADS) {
    S.ones[e] = __float2bfloat16_rn(1.0f);
    S.dY[e] = __float2bfloat16_rn(0.0f);
  }
  if (tid < 16) S.red[tid >> 2][tid & 3] = 0.0f;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (tid == ISSUER) {
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
  for (int e = tid; e < NH; e += THREADS) {
    S.b1[e] = P[ob1 + e];
    S.b2[e] = P[ob2 + e];
  }
  for (int e = tid; e < NO * NH; e += THREADS) S.W3[e / NH][e % NH] = __bfloat162float(__float2bfloat16_rn(P[oW3 + e]));
  if (tid < N3) S.b3[tid] = tid < NO ? P[ob3 + tid] : 0.0f;
  if (tid == ISSUER) {
    const bool ok = wait_phase(&S.mbar_w, 0, spin);
    S.ok = ok ? 1 : 0;
    if (!ok) atomicExch(status, 1);   // nothing was issued on the barrier: nothing is in flight
  }
  handoff();
  const uint32_t tm = S.tmem_slot;
  const uint32_t trow = tm + ((uint32_t)(32 * q) << 16);   // this warp's lanes
  uint32_t ph = 0;
  bool pending = false;   // an MMA batch was committed whose completion was not seen
  // the issuing thread issues and commits (submit), then waits for that commit (await_); the
  // barrier passes the outcome on
  auto submit = [&](auto issue) {
    if (tid == ISSUER) {
      issue();
      commit(&S.mbar_mma);
    }
  };
  auto await_ = [&]() -> bool {
    if (tid == ISSUER) {
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
  auto run = [&](auto issue) -> bool {
    submit(issue);
    return await_();
  };
  bool ok = S.ok != 0;
  constexpr uint32_t kM = 4096 >> 4, kX = 512 >> 4;   // descriptor steps of 16 samples: 128-wide, 16-wide tiles
  int it = 0;
  for (int tile = blockIdx.x; ok && tile < ntiles; tile += G, ++it) {
    const int s0 = tile * TM, rows = min(TM, n - s0), buf = it & 1;
    const uint32_t fresh = it == 0 ? 0u : 1u;   // accumulate into the gradients after the first tile
    bf *Xt = S.X[buf];
    // targets of this thread's row and the next tile's inputs, in flight during the products
    float tg[NO];
    const int nt = tile + G, ns0 = nt * TM, nrows = nt < ntiles ? min(TM, n - ns0) : 0;
    {
#pragma unroll
      for (int o = 0; o < NO; ++o) tg[o] = r < rows ? __ldg(T + (size_t)(s0 + r) * NO + o) : 0.0f;
      load_x(X, ns0, nrows, tid, xv);
    }
    // R1 (after the first tile it was submitted at the end of the previous tile, ahead of that
    // tile's dW1 products)
    if (it == 0) submit([&] { mma(tm + cZ1, dk(Xt, K1), dk(S.w.W1, K1), idesc(TM, NH, 0, 0), 0u); });
    ok = await_();
    if (!ok) break;
    epi_act<false>(S.A1, trow + cZ1, S.b1, r, c0, S.W3, S.yp[part]);
    handoff();
    ok = run([&] {
      for (uint32_t k = 0; k < NH / 16; ++k)
        mma(tm + cZ2, dk(S.A1, NH) + k * 16u, dk(S.w.W2, NH) + k * 16u, idesc(TM, NH, 0, 0), k);
    });
    if (!ok) break;
    epi_act<true>(S.A2, trow + cZ2, S.b2, r, c0, S.W3, S.yp[part]);
    handoff();
    {
      // outputs (the column parts' shares summed in a fixed order), loss and dL/dy of row r
      // (rows of samples past n contribute nothing); every thread of the row computes them, the
      // first column part stores them
      float dy[NO], sq = 0.0f;
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        float y = S.yp[0][o][r];
#pragma unroll
        for (int p = 1; p < THREADS / TM; ++p) y += S.yp[p][o][r];
        const float d = r < rows ? y + S.b3[o] - tg[o] : 0.0f;
        sq += d * d;
        dy[o] = 2.0f * d * inv_n3;
      }
      if (part == 0) {
        put8w(S.dY, r, 0, N3, bf2(pk(dy[0], dy[1])), bf2(pk(dy[2], 0.0f)), 0u, 0u);
        float s0v = dy[0], s1v = dy[1], s2v = dy[2];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          s0v += __shfl_xor_sync(0xffffffffu, s0v, o);
          s1v += __shfl_xor_sync(0xffffffffu, s1v, o);
          s2v += __shfl_xor_sync(0xffffffffu, s2v, o);
          sq += __shfl_xor_sync(0xffffffffu, sq, o);
        }
        if (lane == 0) { S.red[q][0] += s0v; S.red[q][1] += s1v; S.red[q][2] += s2v; S.red[q][3] += sq; }
      }
      // dZ2 = (dY W3) gelu'(Z2 + b2), as BF16 high and low parts
      const f2 dy0 = dup(__bfloat162float(__float2bfloat16_rn(dy[0]))),
               dy1 = dup(__bfloat162float(__float2bfloat16_rn(dy[1]))),
               dy2 = dup(__bfloat162float(__float2bfloat16_rn(dy[2])));
#pragma unroll 1
      for (int c = c0; c < c0 + CW; c += 16) {
        float d[16];
        f2 dz[8];
        ld16(trow + cZ2 + (uint32_t)c, d);
        const f2 *w0 = reinterpret_cast<const f2 *>(&S.W3[0][c]), *w1 = reinterpret_cast<const f2 *>(&S.W3[1][c]),
                 *w2 = reinterpret_cast<const f2 *>(&S.W3[2][c]);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          dz[i] = mul2(fma2(dy2, w2[i], fma2(dy1, w1[i], mul2(dy0, w0[i]))), pk(d[2 * i], d[2 * i + 1]));
        put16_split(S.dZ2, S.dZlo, r, c, dz);
      }
      // the next tile's inputs: its buffer was last read by the previous tile's products
      put_x(S.X[buf ^ 1], nrows, tid, xv);
    }
    handoff();
    // R3, first the products whose operands the dZ1 epilogue overwrites (A2's buffer, dZlo) and
    // dA1, which it reads; waited for
    ok = run([&] {
      // dW3^T += A2^T dY (both MN-major, K = samples)
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cW3t, dmn(S.A2, 128, 2048) + k * kM, dmn(S.dY, 128, 256) + k * kX, idesc(TM, N3, 1, 1), k | fresh);
      // gb2 += column sums of dz2 (low parts here, high parts below) against a tile of ones
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cGb2, dmn(S.dZlo, 128, 2048) + k * kM, dk(S.ones, TM) + k * 16u, idesc(NH, N3, 1, 0), k | fresh);
      // dA1 = dZ2 W2 (W2 read MN-major: N = hidden in, K = hidden out), over gelu'(Z2)
      for (uint32_t k = 0; k < NH / 16; ++k)
        mma(tm + cZ2, dk(S.dZ2, NH) + k * 16u, dmn(S.w.W2, 128, 2048) + k * kM, idesc(TM, NH, 0, 1), k);
    });
    if (!ok) break;
    // then the products that read only A1 and dZ2 (untouched until the next tile's epilogues,
    // which follow the next commit): they run under the dZ1 epilogue
    if (tid == ISSUER) {
      // dW2^T += A1^T dZ2 (both MN-major, K = samples): accumulator row = hidden unit in, so that
      // the partial's rows of W2 are written by consecutive lanes
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cW2, dmn(S.A1, 128, 2048) + k * kM, dmn(S.dZ2, 128, 2048) + k * kM, idesc(NH, NH, 1, 1), k | fresh);
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cGb2, dmn(S.dZ2, 128, 2048) + k * kM, dk(S.ones, TM) + k * 16u, idesc(NH, N3, 1, 0), 1u);
    }
    {
      // dZ1 = dA1 gelu'(Z1 + b1) into A2's buffer (last read by the dW3 products, completed)
      // and dZlo (last read by the gb2 products of the low parts, completed)
      bf *dZ1 = S.A2;
#pragma unroll 1
      for (int c = c0; c < c0 + CW; c += 16) {
        float a[16], d[16];
        f2 dz[8];
        ld16(trow + cZ2 + (uint32_t)c, a);
        ld16(trow + cZ1 + (uint32_t)c, d);
#pragma unroll
        for (int i = 0; i < 8; ++i) dz[i] = mul2(pk(a[2 * i], a[2 * i + 1]), pk(d[2 * i], d[2 * i + 1]));
        put16_split(dZ1, S.dZlo, r, c, dz);
      }
    }
    handoff();
    // the next tile's R1 first, committed on its own (its inputs were written in the dY/dZ2
    // epilogue; Z1's columns were last read just above), so that its wait does not take in R4
    if (nt < ntiles)
      submit([&] { mma(tm + cZ1, dk(S.X[buf ^ 1], K1), dk(S.w.W1, K1), idesc(TM, NH, 0, 0), 0u); });
    // R4: [dW1 | gb1] += dZ1^T [X 1] (both MN-major, K = samples), high and low parts apart; it
    // runs under the next tile's layer-1 epilogue, and the next commit covers it
    if (tid == ISSUER) {
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cW1, dmn(S.A2, 128, 2048) + k * kM, dmn(Xt, 128, 256) + k * kX, idesc(NH, N3, 1, 1), k | fresh);
      for (uint32_t k = 0; k < TM / 16; ++k)
        mma(tm + cW1lo, dmn(S.dZlo, 128, 2048) + k * kM, dmn(Xt, 128, 256) + k * kX, idesc(NH, N3, 1, 1),
            k | fresh);
    }
  }
  // the last tile's dW1 products
  if (ok) ok = run([] {});
  if (ok) {
    // the CTA's partial gradient: accumulator row r is hidden unit r (the input unit of W2)
    float *gp = gpart + (size_t)blockIdx.x * GSTRIDE;
#pragma unroll 1
    for (int c = c0; c < c0 + CW; c += 16) {
      float v[16];
      ld16(trow + cW2 + (uint32_t)c, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) gp[oW2 + (c + i) * NH + r] = v[i];
    }
    if (part == 0) {
      float v[16];
      ld16(trow + cW1, v);
#pragma unroll
      for (int i = 0; i < NI; ++i) gp[oW1 + r * NI + i] = v[i];
      const float gb1 = v[NI];
      ld16(trow + cW1lo, v);
      gp[ob1 + r] = gb1 + v[NI];
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
      lpart[blockIdx.x] = sq;
    }
  }
  // a batch whose wait gave up: wait once more (bounded), then commit whatever was issued after
  // it (the dW1 products follow the next tile's R1 commit) and wait for that, before the tensor
  // memory is freed
  if (pending && tid == ISSUER && wait_phase(&S.mbar_mma, ph ^ 1u, spin)) {
    commit(&S.mbar_mma);
    wait_phase(&S.mbar_mma, ph, spin);
  }
  tc_before();
  __syncthreads();
  tc_after();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kCols) : "memory");
}

}  // namespace

// the training tiles of n samples on `ctas` persistent CTAs (each writes one partial), with
// programmatic stream serialization (the next kernel of the stream may be scheduled while this
// one drains)
int mlp_train_tiles_tc(const float *P, const void *Wb, const float *X, const float *T, int n, float inv_n3,
                       float *gpart, float *lpart, int ctas, int *status, int spin, unsigned hook, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_mlp_tile_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrSmem)) !=
        cudaSuccess)
      return PIC_ECUDA;
    attr = true;
  }
  if (n <= 0 || ctas <= 0 || ctas > (n + TM - 1) / TM) return PIC_EINVAL;
  cudaLaunchAttribute pdl;
  pdl.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl.val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.stream = st;
  cfg.attrs = &pdl;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = sizeof(TrSmem);
  return cudaLaunchKernelEx(&cfg, k_mlp_tile_tc, P, reinterpret_cast<const TrainW *>(Wb), X, T, n, inv_n3, gpart,
                            lpart, status, spin, hook) == cudaSuccess
             ? 0
             : PIC_ECUDA;
}
