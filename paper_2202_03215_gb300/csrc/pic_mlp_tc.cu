// Closure-network inference on the 5th-generation tensor cores (tcgen05).
//
// One block of 128 threads takes 128 samples at a time (a persistent loop over
// tiles); thread t owns sample row t.  Each layer is one or eight
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
// Only thread 0 polls the mbarrier; a block barrier then hands completion to the
// other threads (which order their tensor-memory reads after it with
// tcgen05.fence::after_thread_sync), so the waiting threads issue nothing.
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
constexpr uint32_t kCols = 128;    // tensor-memory columns of a block
constexpr int kSpin = 1 << 20;     // polls of an mbarrier before giving up

using bf = __nv_bfloat16;

// byte offset of element (r, k) of an R x K BF16 matrix in the canonical K-major, no-swizzle layout
__host__ __device__ constexpr int cm_off(int r, int k, int K) {
  return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

struct __align__(1024) TcSmem {
  bf W1[NH * K1];   // N = 128 x K = 16
  bf W2[NH * NH];   // 128 x 128
  bf W3[N3 * NH];   // 16 x 128 (rows 3..15 zero)
  bf X[TM * K1];    // A of layer 1
  bf H[TM * NH];    // A of layers 2 and 3
  float b1[NH], b2[NH], b3[N3];
  unsigned long long mbar;
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

__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity) {
  for (int it = 0; it < kSpin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.b32 %0, 1, 0, P;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
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

// gelu(z) = z / (1 + exp(-2u)), u = sqrt(2/pi) (z + 0.044715 z^3): the tanh form
__device__ __forceinline__ float gelu(float z) {
  const float u = 0.7978845608028654f * (z + 0.044715f * z * z * z);
  return __fdividef(z, 1.0f + __expf(-2.0f * u));
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

// D row t (128 columns) + bias -> GELU -> BF16 -> row t of H (canonical layout)
__device__ __forceinline__ void epilogue(TcSmem &S, uint32_t taddr, const float *b, int t) {
  unsigned char *H = reinterpret_cast<unsigned char *>(S.H);
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

// all threads: operands written by this block become visible to the tensor core, and tensor
// memory reads before the barrier are ordered before MMAs after it
__device__ __forceinline__ void block_handoff() {
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
}

__global__ void __launch_bounds__(TM) k_mlp_fwd_tc(const float *__restrict__ P, const float *__restrict__ X, int n,
                                                   float *__restrict__ Y, int *status) {
  extern __shared__ __align__(1024) unsigned char raw[];
  TcSmem &S = *reinterpret_cast<TcSmem *>(raw + ((1024u - (smem_u32(raw) & 1023u)) & 1023u));
  const int t = threadIdx.x, w = t >> 5;
  unsigned char *W1 = reinterpret_cast<unsigned char *>(S.W1);
  unsigned char *W2 = reinterpret_cast<unsigned char *>(S.W2);
  unsigned char *W3 = reinterpret_cast<unsigned char *>(S.W3);
  unsigned char *Xs = reinterpret_cast<unsigned char *>(S.X);
  for (int q = t; q < NH * K1; q += TM) {
    const int h = q / K1, i = q % K1;
    *reinterpret_cast<bf *>(W1 + cm_off(h, i, K1)) = __float2bfloat16_rn(i < NI ? P[oW1 + h * NI + i] : 0.0f);
  }
  for (int q = t; q < NH * NH; q += TM) {
    const int h = q / NH, k = q % NH;
    *reinterpret_cast<bf *>(W2 + cm_off(h, k, NH)) = __float2bfloat16_rn(P[oW2 + q]);
  }
  for (int q = t; q < N3 * NH; q += TM) {
    const int o = q / NH, k = q % NH;
    *reinterpret_cast<bf *>(W3 + cm_off(o, k, NH)) = __float2bfloat16_rn(o < NO ? P[oW3 + o * NH + k] : 0.0f);
  }
  S.b1[t] = P[ob1 + t];
  S.b2[t] = P[ob2 + t];
  if (t < N3) S.b3[t] = t < NO ? P[ob3 + t] : 0.0f;
  const uint32_t mbar = smem_u32(&S.mbar);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  block_handoff();
  const uint32_t tmem = S.tmem_slot;
  const uint32_t row = tmem + ((uint32_t)(w * 32) << 16);   // this warp's 32 lanes
  const uint64_t dW1 = sdesc(S.W1, 128, K1 * 16), dW2 = sdesc(S.W2, 128, NH * 16), dW3 = sdesc(S.W3, 128, NH * 16);
  const uint64_t dX = sdesc(S.X, 128, K1 * 16), dH = sdesc(S.H, 128, NH * 16);
  constexpr uint32_t id12 = idesc(TM, NH), id3 = idesc(TM, N3);
  uint32_t parity = 0;
  int ok = 1;
  const int tiles = (n + TM - 1) / TM;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int s = tile * TM + t;
    // layer 1: A = the inputs of the tile, row t (column 15 is the zero pad)
#pragma unroll
    for (int i = 0; i < K1; ++i)
      *reinterpret_cast<bf *>(Xs + cm_off(t, i, K1)) =
          __float2bfloat16_rn((s < n && i < NI) ? X[(size_t)s * NI + i] : 0.0f);
    block_handoff();
    if (t == 0) {
      mma(tmem, dX, dW1, id12, 0u);
      commit(mbar);
    }
    ok = __syncthreads_and(ok && (t != 0 || wait_phase(mbar, parity)));   // thread 0 waits, the barrier tells the rest
    parity ^= 1u;
    if (!ok) break;
    tc_after_sync();
    epilogue(S, row, S.b1, t);
    block_handoff();
    // layer 2: eight K = 16 slices (descriptor start + 256 B each)
    if (t == 0) {
      for (uint32_t kk = 0; kk < NH / 16; ++kk) mma(tmem, dH + kk * 16u, dW2 + kk * 16u, id12, kk);
      commit(mbar);
    }
    ok = __syncthreads_and(ok && (t != 0 || wait_phase(mbar, parity)));   // thread 0 waits, the barrier tells the rest
    parity ^= 1u;
    if (!ok) break;
    tc_after_sync();
    epilogue(S, row, S.b2, t);
    block_handoff();
    // layer 3: N = 16 (outputs 0..2)
    if (t == 0) {
      for (uint32_t kk = 0; kk < NH / 16; ++kk) mma(tmem, dH + kk * 16u, dW3 + kk * 16u, id3, kk);
      commit(mbar);
    }
    ok = __syncthreads_and(ok && (t != 0 || wait_phase(mbar, parity)));   // thread 0 waits, the barrier tells the rest
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
    __syncthreads();   // D, X and H are rewritten by the next tile
    tc_after_sync();
  }
  if (!ok && t == 0) atomicExch(status, 1);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

}  // namespace

// forward pass of the closure network on the tensor cores, enqueued on st; *status (device)
// becomes 1 if a wait gave up
int mlp_forward_tc(const float *P, const float *X, int n, float *Y, int *status, cudaStream_t st) {
  if (n <= 0) return PIC_EINVAL;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int tiles = (n + TM - 1) / TM;
  const int blocks = tiles < 2 * sms ? tiles : 2 * sms;
  const int smem = (int)sizeof(TcSmem) + 1024;   // room to align the dynamic base to 1 KB
  if (cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return PIC_ECUDA;
  k_mlp_fwd_tc<<<blocks, TM, smem, st>>>(P, X, n, Y, status);
  return cudaGetLastError() == cudaSuccess ? 0 : PIC_ECUDA;
}
