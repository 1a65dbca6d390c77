// Closure-network inference on the 5th-generation tensor cores (tcgen05).
//
// A block runs G = 4 independent groups of 128 threads; a group takes 128 samples
// at a time (a persistent loop over tiles) and its thread t owns sample row t.
// The groups share the weights (loaded once per block) and overlap: while one
// waits for its MMAs, the others run their epilogues.  Each layer is one or eight
// tcgen05.mma (kind::f16: BF16 operands, FP32 accumulation) of M = 128 rows,
// issued by thread 0, with A (activations) and B (weights, [out][in] = N x K,
// K-major) in shared memory and the accumulator D in tensor memory (128
// columns of the block's allocation, reused by the three layers).  Operands
// are laid out in the canonical K-major form without swizzle: 8-row x 16-byte
// core matrices, consecutive along K (leading offset 128 B), row groups of 8
// one full K-row of core matrices apart (stride offset K x 16 B).  Completion
// comes through an mbarrier (tcgen05.commit); each warp then reads its 32 rows
// of D (tcgen05.ld, one lane per row), adds the bias, applies GELU and writes
// the BF16 activations back as the next layer's A operand.
//
// One thread of each group waits on its mbarrier (a suspending try_wait with a
// back-off); a named barrier of the group then hands completion to the other threads (which
// order their tensor-memory reads after it with tcgen05.fence::after_thread_sync).
// Every wait is bounded: a wait that gives up sets *status and the block
// stops after freeing its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pic.h"

namespace {

constexpr int NI = 15, NH = 128, NO = 3;
constexpr int oW1 = 0, ob1 = NH * NI, oW2 = ob1 + NH, ob2 = oW2 + NH * NH, oW3 = ob2 + NH, ob3 = oW3 + NO * NH;
constexpr int TM = 128;            // samples per tile = MMA rows = threads per block
constexpr int K1 = 16;             // input width padded to one MMA K step
constexpr int N3 = 16;             // output width padded to the smallest N of an M = 128 MMA
constexpr int G = 4;               // groups of TM threads per block
constexpr uint32_t kCols = 128 * G;   // tensor-memory columns of a block: 128 per group

using bf = __nv_bfloat16;

// byte offset of element (r, k) of an R x K BF16 matrix in the canonical K-major, no-swizzle layout
__host__ __device__ constexpr int cm_off(int r, int k, int K) {
  return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

struct TcGroup {
  bf X[TM * K1];    // A of layer 1
  bf H[TM * NH];    // A of layers 2 and 3
};

struct __align__(128) TcSmem {
  bf W1[NH * K1];   // N = 128 x K = 16
  bf W2[NH * NH];   // 128 x 128
  bf W3[N3 * NH];   // 16 x 128 (rows 3..15 zero)
  TcGroup g[G];
  float b1[NH], b2[NH], b3[N3];
  unsigned long long mbar[G];
  int ok[G];
  uint32_t tmem_slot;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start >> 4, leading offset >> 4 (bits 16..29), stride
// offset >> 4 (bits 32..45), fixed 0b001 at bits 46..48, no swizzle
__device__ __forceinline__ uint64_t sdesc(const void *p, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32 (bits 4..5 = 1), A and B BF16 (bits 7..9, 10..12 = 1),
// both K-major, N >> 3 at bits 17..22, M >> 4 at bits 24..28
__host__ __device__ constexpr uint32_t idesc(uint32_t M, uint32_t N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity, int spin) {
  for (int it = 0; it < spin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, 10000;\nselp.b32 %0, 1, 0, P;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

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

// gelu(z) = z/2 (1 + tanh u), u = sqrt(2/pi) z (1 + 0.044715 z^2), with the hardware tanh
// (tanh.approx.f32, relative error about 2^-11: below half a BF16 ulp of the stored activation)
__device__ __forceinline__ float gelu(float z) {
  const float u = 0.7978845608028654f * z * (1.0f + 0.044715f * z * z);
  float th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(u));
  const float h = 0.5f * z;
  return h + h * th;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

// D row t (128 columns) + bias -> GELU -> BF16 -> row t of H (canonical layout)
__device__ __forceinline__ void epilogue(bf *Hs, uint32_t taddr, const float *b, int t) {
  unsigned char *H = reinterpret_cast<unsigned char *>(Hs);
#pragma unroll 1
  for (int c = 0; c < NH; c += 16) {
    float v[16];
    ld16(taddr + (uint32_t)c, v);
    uint4 q0, q1;
    q0.x = pack2(gelu(v[0] + b[c + 0]), gelu(v[1] + b[c + 1]));
    q0.y = pack2(gelu(v[2] + b[c + 2]), gelu(v[3] + b[c + 3]));
    q0.z = pack2(gelu(v[4] + b[c + 4]), gelu(v[5] + b[c + 5]));
    q0.w = pack2(gelu(v[6] + b[c + 6]), gelu(v[7] + b[c + 7]));
    q1.x = pack2(gelu(v[8] + b[c + 8]), gelu(v[9] + b[c + 9]));
    q1.y = pack2(gelu(v[10] + b[c + 10]), gelu(v[11] + b[c + 11]));
    q1.z = pack2(gelu(v[12] + b[c + 12]), gelu(v[13] + b[c + 13]));
    q1.w = pack2(gelu(v[14] + b[c + 14]), gelu(v[15] + b[c + 15]));
    *reinterpret_cast<uint4 *>(H + cm_off(t, c, NH)) = q0;
    *reinterpret_cast<uint4 *>(H + cm_off(t, c + 8, NH)) = q1;
  }
}

__device__ __forceinline__ void group_bar(int g) { asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(TM) : "memory"); }

// the threads of group g: operands written by the group become visible to the tensor core, and
// tensor-memory reads before the barrier are ordered before MMAs after it
__device__ __forceinline__ void group_handoff(int g) {
  fence_async_smem();
  tc_before_sync();
  group_bar(g);
  tc_after_sync();
}

// one thread of the group waits for the group's MMAs (thread 32 (g % 4): the four groups' waiters
// sit in warps of four different schedulers); the barrier passes the outcome to the group
__device__ __forceinline__ bool group_wait(TcSmem &S, int g, int lt, uint32_t mbar, uint32_t parity, int spin) {
  if (lt == 32 * (g & 3)) S.ok[g] = wait_phase(mbar, parity, spin) ? 1 : 0;
  group_bar(g);
  const bool ok = S.ok[g] != 0;
  group_bar(g);   // the flag is read before thread 0 can rewrite it
  return ok;
}

__global__ void __launch_bounds__(TM * G) k_mlp_fwd_tc(const float *__restrict__ P, const float *__restrict__ X,
                                                       int n, float *__restrict__ Y, int *status, int spin,
                                                       unsigned hook) {
  extern __shared__ __align__(128) unsigned char raw[];
  TcSmem &S = *reinterpret_cast<TcSmem *>(raw);
  const int tid = threadIdx.x, w = tid >> 5, g = tid / TM, lt = tid % TM;
  unsigned char *W1 = reinterpret_cast<unsigned char *>(S.W1);
  unsigned char *W2 = reinterpret_cast<unsigned char *>(S.W2);
  unsigned char *W3 = reinterpret_cast<unsigned char *>(S.W3);
  for (int q = tid; q < NH * K1; q += TM * G) {
    const int h = q / K1, i = q % K1;
    *reinterpret_cast<bf *>(W1 + cm_off(h, i, K1)) = __float2bfloat16_rn(i < NI ? P[oW1 + h * NI + i] : 0.0f);
  }
  for (int q = tid; q < NH * NH; q += TM * G) {
    const int h = q / NH, k = q % NH;
    *reinterpret_cast<bf *>(W2 + cm_off(h, k, NH)) = __float2bfloat16_rn(P[oW2 + q]);
  }
  for (int q = tid; q < N3 * NH; q += TM * G) {
    const int o = q / NH, k = q % NH;
    *reinterpret_cast<bf *>(W3 + cm_off(o, k, NH)) = __float2bfloat16_rn(o < NO ? P[oW3 + o * NH + k] : 0.0f);
  }
  if (tid < NH) { S.b1[tid] = P[ob1 + tid]; S.b2[tid] = P[ob2 + tid]; }
  if (tid < N3) S.b3[tid] = tid < NO ? P[ob3 + tid] : 0.0f;
  if (lt == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar[g])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  // group g: tensor-memory columns [128 g, 128 g + 128); warp w reads lanes 32 (w % 4) .. + 31
  const uint32_t tmem = S.tmem_slot + (uint32_t)(128 * g);
  const uint32_t row = tmem + ((uint32_t)((w & 3) * 32) << 16);
  const uint32_t mbar = smem_u32(&S.mbar[g]);
  TcGroup &Gs = S.g[g];
  unsigned char *Xs = reinterpret_cast<unsigned char *>(Gs.X);
  const uint64_t dW1 = sdesc(S.W1, 128, K1 * 16), dW2 = sdesc(S.W2, 128, NH * 16), dW3 = sdesc(S.W3, 128, NH * 16);
  const uint64_t dX = sdesc(Gs.X, 128, K1 * 16), dH = sdesc(Gs.H, 128, NH * 16);
  constexpr uint32_t id12 = idesc(TM, NH), id3 = idesc(TM, N3);
  uint32_t parity = 0;
  bool ok = true;
  bool pending = false;   // an MMA was committed whose completion the group has not seen
  // test hook: block 0's group 0 issues no MMA for its first tile, so its wait runs out
  bool skip = (hook & PIC_MLP_HOOK_NO_FORWARD_MMA) && blockIdx.x == 0 && g == 0;
  const int tiles = (n + TM - 1) / TM;
  for (int tile = blockIdx.x * G + g; tile < tiles; tile += gridDim.x * G) {
    const int s = tile * TM + lt;
    // layer 1: A = the inputs of the tile, row lt (column 15 is the zero pad)
#pragma unroll
    for (int i = 0; i < K1; ++i)
      *reinterpret_cast<bf *>(Xs + cm_off(lt, i, K1)) =
          __float2bfloat16_rn((s < n && i < NI) ? X[(size_t)s * NI + i] : 0.0f);
    group_handoff(g);
    if (lt == 0 && !skip) {
      mma(tmem, dX, dW1, id12, 0u);
      commit(mbar);
    }
    pending = !skip;
    skip = false;
    ok = group_wait(S, g, lt, mbar, parity, spin);
    parity ^= 1u;
    if (!ok) break;
    tc_after_sync();
    epilogue(Gs.H, row, S.b1, lt);
    group_handoff(g);
    // layer 2: eight K = 16 slices (descriptor start + 256 B each)
    if (lt == 0) {
      for (uint32_t kk = 0; kk < NH / 16; ++kk) mma(tmem, dH + kk * 16u, dW2 + kk * 16u, id12, kk);
      commit(mbar);
    }
    pending = true;
    ok = group_wait(S, g, lt, mbar, parity, spin);
    parity ^= 1u;
    if (!ok) break;
    tc_after_sync();
    epilogue(Gs.H, row, S.b2, lt);
    group_handoff(g);
    // layer 3: N = 16 (outputs 0..2)
    if (lt == 0) {
      for (uint32_t kk = 0; kk < NH / 16; ++kk) mma(tmem, dH + kk * 16u, dW3 + kk * 16u, id3, kk);
      commit(mbar);
    }
    pending = true;
    ok = group_wait(S, g, lt, mbar, parity, spin);
    parity ^= 1u;
    if (!ok) break;
    tc_after_sync();
    float v[16];
    ld16(row, v);
    if (s < n) {
#pragma unroll
      for (int o = 0; o < NO; ++o) Y[(size_t)s * NO + o] = v[o] + S.b3[o];
    }
    tc_before_sync();
    group_bar(g);   // D, X and H are rewritten by the group's next tile
    tc_after_sync();
  }
  if (!ok && lt == 0) atomicExch(status, 1);
  // a wait that gave up on a committed MMA: wait once more (bounded) for it to finish writing
  // tensor memory before the memory is freed; the phase that ran out is the one before parity
  if (!ok && pending && lt == 32 * (g & 3)) wait_phase(mbar, parity ^ 1u, spin);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_slot), "r"(kCols) : "memory");
}

}  // namespace

// forward pass of the closure network on the tensor cores, enqueued on st; *status (device)
// becomes 1 if a wait gave up
int mlp_forward_tc(const float *P, const float *X, int n, float *Y, int *status, int spin, unsigned hook,
                   cudaStream_t st) {
  if (n <= 0) return PIC_EINVAL;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int tiles = (n + TM - 1) / TM;
  const int groups = (tiles + G - 1) / G;
  const int blocks = groups < sms ? groups : sms;   // one block (all of tensor memory) per SM
  const int smem = (int)sizeof(TcSmem);
  if (cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return PIC_ECUDA;
  k_mlp_fwd_tc<<<blocks, TM * G, smem, st>>>(P, X, n, Y, status, spin, hook);
  return cudaGetLastError() == cudaSuccess ? 0 : PIC_ECUDA;
}
