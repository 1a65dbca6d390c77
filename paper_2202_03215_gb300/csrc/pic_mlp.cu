// Closure network of the quasi-neutral fluid screen: MLP 15 -> 128 -> 128 -> 3,
// GELU (tanh form) on the hidden layers, mean-squared-error loss, Adam.
// Training: BF16 operands on the tensor cores (mma.sync m16n8k16 fed by
// ldmatrix, FP32 accumulation), FP32 master weights and optimizer state.
// The forward pass of the fluid closure runs on tcgen05 (pic_mlp_tc.cu).
//
// One CTA of 16 warps trains on a tile of 64 samples: forward, backward and the
// weight gradients of its tile, written as a partial; a second kernel sums the
// partials in a fixed order (deterministic gradients) and applies Adam, which
// also refreshes the BF16 copy of the weights that the tile kernel stages with
// one bulk copy (TMA engine, completion on an mbarrier, bounded wait).
// Parameter layout (FP32, flat): W1[128][15], b1[128], W2[128][128], b2[128],
// W3[3][128], b3[3]  (row = output unit).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "pic.h"

namespace {

constexpr int NI = 15, NIP = 16, NH = 128, NO = 3, NOP = 16;
constexpr int LDI = NIP + 8, LDH = NH + 8, LDZ = NH + 8;   // padded rows: conflict-free ldmatrix
constexpr int S = 64;                 // samples per tile
constexpr int WR = S / 16;            // row groups of 16 samples
constexpr int WC = 4;                 // column quarters of the hidden layers
constexpr int WARPS = WR * WC;
constexpr int THREADS = WARPS * 32;
constexpr int oW1 = 0, ob1 = NH * NI, oW2 = ob1 + NH, ob2 = oW2 + NH * NH, oW3 = ob2 + NH, ob3 = oW3 + NO * NH;
constexpr int NPARAM = ob3 + NO;      // 18947
constexpr int GSTRIDE = (NPARAM + 3) & ~3;   // floats between the partials of two tiles (8-byte pairs stay aligned)
constexpr int kSpin = 200000;         // polls of an mbarrier (each suspends up to 10 us) before giving up

using bf = __nv_bfloat16;

// BF16 weights exactly as the tile kernel holds them in shared memory (padding zero)
struct WPack {
  bf W1[NH][LDI];
  bf W2[NH][LDH];
  bf W3[NOP][LDH];
};
static_assert(sizeof(WPack) % 16 == 0, "16-byte copies");
static_assert(oW2 % 2 == 0 && oW3 % 2 == 0 && GSTRIDE % 2 == 0, "8-byte pairs of partial gradients");

struct Smem {
  WPack w;
  bf X[S][LDI];
  bf A1[S][LDH];       // activations of layer 1
  bf A2[S][LDH];       // activations of layer 2
  bf D2[S][LDH];       // dL/dz2
  bf D1[S][LDH];       // dL/dz1
  bf dY[S][LDI];       // dL/dy (columns 3..15 zero)
  float G1[S][LDZ];    // gelu'(z1)
  float G2[S][LDZ];    // gelu'(z2)
  float b1[NH], b2[NH], b3[NOP];
  float cs1[WR][NH], cs2[WR][NH], cs3[WR][NOP];   // per-row-group column sums (bias gradients)
  float loss[WR];
  unsigned long long mbar;   // completion of the weight copy
  int ok;
};

// index of parameter p in WPack (in BF16 elements), -1 for biases
__host__ __device__ __forceinline__ int wpack_index(int p) {
  if (p < ob1) return (p / NI) * LDI + p % NI;
  if (p >= oW2 && p < ob2) return NH * LDI + ((p - oW2) / NH) * LDH + (p - oW2) % NH;
  if (p >= oW3 && p < ob3) return NH * LDI + NH * LDH + ((p - oW3) / NH) * LDH + (p - oW3) % NH;
  return -1;
}

__device__ __forceinline__ unsigned saddr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// four 8x8 BF16 matrices; lanes 8i..8i+7 give the row addresses of matrix i. Lane l receives
// row l/4, columns 2(l%4), 2(l%4)+1 of each (.trans: row 2(l%4), 2(l%4)+1 of column l/4)
__device__ __forceinline__ void ldsm4(unsigned r[4], const bf *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm4t(unsigned r[4], const bf *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(saddr(p)));
}

// one bulk copy global -> shared of `bytes` (multiple of 16, both addresses 16-byte aligned),
// completing on the mbarrier at mbar (initialised for one arrival by the calling thread)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *mbar) {
  const unsigned mb = saddr(mbar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(mb), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(mb)
               : "memory");
}
__device__ __forceinline__ bool wait_phase(unsigned long long *mbar, unsigned parity, int spin) {
  const unsigned mb = saddr(mbar);
  for (int it = 0; it < spin; ++it) {
    unsigned done;
    asm volatile(
        "{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, 10000;\nselp.b32 %0, 1, 0, P;\n}\n"
        : "=r"(done)
        : "r"(mb), "r"(parity)
        : "memory");
    if (done) return true;
    __nanosleep(64);
  }
  return false;
}

// programmatic dependent launch: let the next kernel of the stream start its launch now; wait
// for the previous kernel of the stream to complete (no-op without a programmatic dependency)
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void mma(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C[16 x 8 NT] (rows r0.., columns n0..) += A(16 x K) B(K x 8 NT), one warp, operands in shared memory.
// A(r, k) = A[r*lda + k], or A[k*lda + r] if AT; B(k, n) = B[n*ldb + k], or B[k*ldb + n] if BT.
// Fragment layout of m16n8k16 (g = lane/4, t = lane%4): A rows g, g+8 and columns 2t, 2t+1,
// 2t+8, 2t+9; B columns g and rows 2t, 2t+1, 2t+8, 2t+9; C rows g, g+8 and columns 2t, 2t+1.
template <int NT, bool AT, bool BT>
__device__ __forceinline__ void gemm(float c[NT][4], const bf *A, int lda, int r0, const bf *B, int ldb, int n0,
                                     int K) {
  static_assert(NT % 2 == 0, "two column tiles per B load");
  const int lane = threadIdx.x & 31, mi = lane >> 3, j = lane & 7;
  for (int k0 = 0; k0 < K; k0 += 16) {
    unsigned a[4];
    if (AT) ldsm4t(a, A + (k0 + j + (mi >> 1) * 8) * lda + r0 + (mi & 1) * 8);
    else    ldsm4(a, A + (r0 + j + (mi & 1) * 8) * lda + k0 + (mi >> 1) * 8);
#pragma unroll
    for (int np = 0; np < NT / 2; ++np) {
      const int n = n0 + 16 * np;
      unsigned b[4];   // b[0], b[1]: column tile 2np; b[2], b[3]: tile 2np + 1
      if (BT) ldsm4t(b, B + (k0 + j + (mi & 1) * 8) * ldb + n + (mi >> 1) * 8);
      else    ldsm4(b, B + (n + j + (mi >> 1) * 8) * ldb + k0 + (mi & 1) * 8);
      mma(c[2 * np], a, b[0], b[1]);
      mma(c[2 * np + 1], a, b[2], b[3]);
    }
  }
}

template <int NT>
__device__ __forceinline__ void zero(float c[NT][4]) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
}

__device__ __forceinline__ void st_bf2(bf *p, float x, float y) {
  *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(x, y);
}

// GELU (tanh form) and its derivative from th = tanh u, u = sqrt(2/pi)(z + 0.044715 z^3) (hardware
// tanh): gelu = z (1 + th)/2, gelu' = (1 + th)/2 + z (1 - th^2) du/dz / 2
__device__ __forceinline__ void gelu2(float z, float &y, float &dy) {
  const float c = 0.7978845608028654f, z2 = z * z;
  float th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(c * z * (1.0f + 0.044715f * z2)));
  const float h = 0.5f * (1.0f + th);
  y = z * h;
  dy = h + 0.5f * z * (1.0f - th * th) * c * (1.0f + 3.0f * 0.044715f * z2);
}

// sum of the two row values of a C fragment column over the 8 row groups (lanes t, t+4, ..)
__device__ __forceinline__ float colsum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

// hidden-layer epilogue of a row pass: z = c + b; gelu(z) -> H (BF16), gelu'(z) -> G (FP32)
template <int NT>
__device__ __forceinline__ void act_epilogue(const float c[NT][4], const float *b, float (*G)[LDZ], bf (*H)[LDH],
                                             int r0, int n0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int r = r0 + g + 8 * hr, col = n0 + 8 * nt + 2 * t;
      float y0, d0, y1, d1;
      gelu2(c[nt][2 * hr] + b[col], y0, d0);
      gelu2(c[nt][2 * hr + 1] + b[col + 1], y1, d1);
      *reinterpret_cast<float2 *>(&G[r][col]) = make_float2(d0, d1);
      st_bf2(&H[r][col], y0, y1);
    }
}

// backward epilogue of a row pass: dz = c * gelu'(z) -> D (BF16), column sums -> cs
template <int NT>
__device__ __forceinline__ void dz_epilogue(const float c[NT][4], const float (*G)[LDZ], bf (*D)[LDH], float *cs,
                                            int r0, int n0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    float bs[2] = {0.0f, 0.0f};
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int r = r0 + g + 8 * hr, col = n0 + 8 * nt + 2 * t;
      const float2 gd = *reinterpret_cast<const float2 *>(&G[r][col]);
      const float d0 = c[nt][2 * hr] * gd.x, d1 = c[nt][2 * hr + 1] * gd.y;
      bs[0] += d0;
      bs[1] += d1;
      st_bf2(&D[r][col], d0, d1);
    }
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      const float v = colsum(bs[o]);
      if (g == 0) cs[n0 + 8 * nt + 2 * t + o] = v;
    }
  }
}

// weight-gradient epilogue: 16 rows h0.. of a (rows x ncol) partial, columns n0.. (< ncol kept)
template <int NT>
__device__ __forceinline__ void wgrad_store(const float c[NT][4], float *gp, int h0, int n0, int ncol, int nrow) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int h = h0 + g + 8 * hr, col = n0 + 8 * nt + 2 * t;
      if (h >= nrow) continue;
      if (ncol % 2 == 0) {   // the pair is 8-byte aligned: partial and matrix offsets are even
        *reinterpret_cast<float2 *>(&gp[h * ncol + col]) = make_float2(c[nt][2 * hr], c[nt][2 * hr + 1]);
      } else {
        if (col < ncol) gp[h * ncol + col] = c[nt][2 * hr];
        if (col + 1 < ncol) gp[h * ncol + col + 1] = c[nt][2 * hr + 1];
      }
    }
}

// forward + backward of one tile of S samples; partial gradients (NPARAM floats at a stride of
// GSTRIDE) and loss per tile
__global__ void __launch_bounds__(THREADS) k_mlp_tile(const float *__restrict__ P, const WPack *__restrict__ Wb,
                                                      const float *__restrict__ X, const float *__restrict__ T, int n,
                                                      float inv_n3, float *__restrict__ gpart,
                                                      float *__restrict__ lpart, int *__restrict__ status, int spin,
                                                      unsigned hook) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, g = lane >> 2, t = lane & 3;
  const int rg = w % WR, ch = w / WR;          // row group, column half
  const int r0 = 16 * rg, c0 = (NH / WC) * ch;
  constexpr int NTH = NH / WC / 8;             // column tiles of a hidden-layer row pass
  const int tile = blockIdx.x, s0 = tile * S;
  // everything this kernel reads may come from the previous kernel of the stream (the inputs
  // from the caller's producer, the weights from the previous step's Adam update)
  pdl_launch_next();
  pdl_wait_prev();
  // the BF16 weights by one bulk copy, the FP32 biases and the tile's inputs
  if (tid == 0) {
    if (!(hook & PIC_MLP_HOOK_NO_WEIGHT_COPY)) {
      bulk_load(&sm.w, Wb, (unsigned)sizeof(WPack), &sm.mbar);
    } else {   // test hook: the barrier is armed but no copy will ever arrive on it
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&sm.mbar)) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  for (int q = tid; q < NH; q += THREADS) { sm.b1[q] = P[ob1 + q]; sm.b2[q] = P[ob2 + q]; }
  if (tid < NOP) sm.b3[tid] = tid < NO ? P[ob3 + tid] : 0.0f;
  {
    const int rows = min(S, n - s0);
    for (int q = tid; q < S * NI; q += THREADS) {
      const int r = q / NI, i = q % NI;
      sm.X[r][i] = __float2bfloat16_rn(r < rows ? X[(size_t)s0 * NI + q] : 0.0f);
    }
    for (int q = tid; q < S * (LDI - NI); q += THREADS) sm.X[q / (LDI - NI)][NI + q % (LDI - NI)] = __float2bfloat16_rn(0.0f);
  }
  if (tid == 0) {
    bool ok = wait_phase(&sm.mbar, 0, spin);
    if (!ok) {            // report, let the copy in flight land (bounded), skip the tile
      atomicExch(status, 1);
      wait_phase(&sm.mbar, 0, spin);
    }
    sm.ok = ok;
  }
  __syncthreads();
  if (!sm.ok) return;
  // layer 1, then layer 2: rows r0.., columns c0..
  {
    float c[NTH][4];
    zero<NTH>(c);
    gemm<NTH, false, false>(c, &sm.X[0][0], LDI, r0, &sm.w.W1[0][0], LDI, c0, NIP);
    act_epilogue<NTH>(c, sm.b1, sm.G1, sm.A1, r0, c0);
  }
  __syncthreads();
  {
    float c[NTH][4];
    zero<NTH>(c);
    gemm<NTH, false, false>(c, &sm.A1[0][0], LDH, r0, &sm.w.W2[0][0], LDH, c0, NH);
    act_epilogue<NTH>(c, sm.b2, sm.G2, sm.A2, r0, c0);
  }
  __syncthreads();
  // layer 3, outputs, dL/dy, loss (one warp per row group)
  if (ch == 0) {
    float c[2][4];
    zero<2>(c);
    gemm<2, false, false>(c, &sm.A2[0][0], LDH, r0, &sm.w.W3[0][0], LDH, 0, NH);
    float lsum = 0.0f, bsum[2] = {0.0f, 0.0f};
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int r = r0 + g + 8 * hr, s = s0 + r;
      float dy[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int o = 2 * t + e;
        dy[e] = 0.0f;
        if (o < NO && s < n) {
          const float d = c[0][2 * hr + e] + sm.b3[o] - T[(size_t)s * NO + o];
          lsum += d * d;
          dy[e] = 2.0f * d * inv_n3;
        }
        bsum[e] += dy[e];
      }
      st_bf2(&sm.dY[r][2 * t], dy[0], dy[1]);
      st_bf2(&sm.dY[r][8 + 2 * t], 0.0f, 0.0f);
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float v = colsum(bsum[e]);
      if (g == 0) sm.cs3[rg][2 * t + e] = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) sm.loss[rg] = lsum;
  }
  __syncthreads();
  float *gp = gpart + (size_t)tile * GSTRIDE;
  if (tid < NO) {
    float v = 0.0f;
    for (int q = 0; q < WR; ++q) v += sm.cs3[q][tid];
    gp[ob3 + tid] = v;
  }
  if (tid == 32) {
    float v = 0.0f;
    for (int q = 0; q < WR; ++q) v += sm.loss[q];
    lpart[tile] = v;
  }
  // dL/dW3 = dY^T A2 (outputs x hidden, summed over the tile): warp w < 8, hidden columns 16w..
  if (w < NH / 16) {
    float c[2][4];
    zero<2>(c);
    gemm<2, true, true>(c, &sm.dY[0][0], LDI, 0, &sm.A2[0][0], LDH, 16 * w, S);
    wgrad_store<2>(c, gp + oW3, 0, 16 * w, NH, NO);
  }
  // dL/dz2 = (dY W3) * gelu'(z2): rows r0.., columns c0..
  {
    float c[NTH][4];
    zero<NTH>(c);
    gemm<NTH, false, true>(c, &sm.dY[0][0], LDI, r0, &sm.w.W3[0][0], LDH, c0, NOP);
    dz_epilogue<NTH>(c, sm.G2, sm.D2, sm.cs2[rg], r0, c0);
  }
  __syncthreads();
  for (int q = tid; q < NH; q += THREADS) {
    float v = 0.0f;
    for (int k = 0; k < WR; ++k) v += sm.cs2[k][q];
    gp[ob2 + q] = v;
  }
  // dL/dW2 = dZ2^T A1: output rows 16 (w % 8).., columns 128 / (WARPS / 8) per warp
  {
    constexpr int NTW = NH / 8 / (WARPS / 8);
    const int h0 = 16 * (w % 8), n0 = NTW * 8 * (w / 8);
    float c[NTW][4];
    zero<NTW>(c);
    gemm<NTW, true, true>(c, &sm.D2[0][0], LDH, h0, &sm.A1[0][0], LDH, n0, S);
    wgrad_store<NTW>(c, gp + oW2, h0, n0, NH, NH);
  }
  // dL/dz1 = (dZ2 W2) * gelu'(z1): rows r0.., columns c0..
  {
    float c[NTH][4];
    zero<NTH>(c);
    gemm<NTH, false, true>(c, &sm.D2[0][0], LDH, r0, &sm.w.W2[0][0], LDH, c0, NH);
    dz_epilogue<NTH>(c, sm.G1, sm.D1, sm.cs1[rg], r0, c0);
  }
  __syncthreads();
  for (int q = tid; q < NH; q += THREADS) {
    float v = 0.0f;
    for (int k = 0; k < WR; ++k) v += sm.cs1[k][q];
    gp[ob1 + q] = v;
  }
  // dL/dW1 = dZ1^T X: warp w < 8, output rows 16w..
  if (w < NH / 16) {
    float c[2][4];
    zero<2>(c);
    gemm<2, true, true>(c, &sm.D1[0][0], LDH, 16 * w, &sm.X[0][0], LDI, 0, S);
    wgrad_store<2>(c, gp + oW1, 16 * w, 0, NI, NH);
  }
}

struct AdamArgs {
  int on;
  float lr, b1, b2, eps, c1, c2;
};

// g[p] = sum over tiles of the partials in a fixed order (tiles w, w+8, .. per warp, then the
// warps in order); optionally Adam (Kingma & Ba) on the FP32 master weights, refreshing the
// BF16 copy. Block 0 also sums the loss.
constexpr int RW = 16;  // warps of the reduction
__global__ void __launch_bounds__(RW * 32) k_mlp_reduce(const float *__restrict__ gpart, const float *__restrict__ lpart,
                                                        int ntiles, float *__restrict__ grad, double *__restrict__ loss,
                                                        float inv_n3, float *__restrict__ P, float *__restrict__ m,
                                                        float *__restrict__ v, bf *__restrict__ Wb, AdamArgs a,
                                                        const int *__restrict__ status) {
  __shared__ float part[RW][32];
  pdl_launch_next();
  pdl_wait_prev();
  // a tile whose wait gave up wrote no partial: leave gradient, loss, weights and moments as they are
  if (*status) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + lane;
  float s = 0.0f;
  if (p < NPARAM) {
#pragma unroll 8
    for (int q = w; q < ntiles; q += RW) s += gpart[(size_t)q * GSTRIDE + p];
  }
  part[w][lane] = s;
  __syncthreads();
  if (w == 0 && p < NPARAM) {
    float gr = 0.0f;
#pragma unroll
    for (int k = 0; k < RW; ++k) gr += part[k][lane];
    grad[p] = gr;
    if (a.on) {
      const float mm = a.b1 * m[p] + (1.0f - a.b1) * gr;
      const float vv = a.b2 * v[p] + (1.0f - a.b2) * gr * gr;
      m[p] = mm;
      v[p] = vv;
      const float x = P[p] - a.lr * (mm / a.c1) / (sqrtf(vv / a.c2) + a.eps);
      P[p] = x;
      const int q = wpack_index(p);
      if (q >= 0) Wb[q] = __float2bfloat16_rn(x);
    }
  }
  if (blockIdx.x == 0 && w == 1) {
    double l = 0.0;
    for (int q = lane; q < ntiles; q += 32) l += (double)lpart[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0) *loss = l * (double)inv_n3;
  }
}

// BF16 copy of the weights (the padding of the copy stays zero)
__global__ void k_mlp_pack(const float *__restrict__ P, bf *__restrict__ Wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const int q = wpack_index(p);
  if (q >= 0) Wb[q] = __float2bfloat16_rn(P[p]);
}

}  // namespace

int mlp_forward_tc(const float *P, const float *X, int n, float *Y, int *status, int spin, unsigned hook,
                   cudaStream_t st);

struct pic_mlp {
  float *P = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  float *gpart = nullptr, *lpart = nullptr;
  bf *Wb = nullptr;        // BF16 weights in the tile kernel's shared-memory layout
  double *loss = nullptr;
  int *status = nullptr;   // device: 1 once a bounded wait of the tensor-core forward gave up
  int cap_tiles = 0;
  int t = 0;   // Adam steps taken
  int spin = kSpin;        // polls of a bounded wait (pic_mlp_test_hook)
  unsigned hook = 0;       // PIC_MLP_HOOK_* (pic_mlp_test_hook)
  int latched = 0;         // PIC_ETIMEOUT once a wait gave up, until pic_mlp_set_params
};

namespace {

int ensure(pic_mlp *h, int n) {
  const int tiles = (n + S - 1) / S;
  if (tiles <= h->cap_tiles) return 0;
  cudaFree(h->gpart);
  cudaFree(h->lpart);
  h->gpart = nullptr;
  h->lpart = nullptr;
  if (cudaMalloc(&h->gpart, (size_t)tiles * GSTRIDE * 4) != cudaSuccess ||
      cudaMalloc(&h->lpart, (size_t)tiles * 4) != cudaSuccess)
    return PIC_ENOMEM;
  h->cap_tiles = tiles;
  return 0;
}

int run_forward(pic_mlp *h, const float *X, int n, float *Y, cudaStream_t st) {
  return mlp_forward_tc(h->P, X, n, Y, h->status, h->spin, h->hook, st);
}

int pack(pic_mlp *h) {
  k_mlp_pack<<<(NPARAM + 255) / 256, 256>>>(h->P, h->Wb);
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : PIC_ECUDA;
}

// partial gradients of n samples, reduced into h->grad (and h->loss); Adam if a.on
int run_tiles(pic_mlp *h, const float *X, const float *T, int n, const AdamArgs &a, cudaStream_t st) {
  if (n <= 0) return PIC_EINVAL;
  const int rc = ensure(h, n);
  if (rc) return rc;
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_mlp_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  });
  const int tiles = (n + S - 1) / S;
  const float inv_n3 = 1.0f / (3.0f * (float)n);
  // both kernels with programmatic stream serialization: each may be scheduled while the
  // previous kernel of the stream drains and waits for it (griddepcontrol.wait) before it
  // reads that kernel's results
  cudaLaunchAttribute pdl;
  pdl.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl.val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.stream = st;
  cfg.attrs = &pdl;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(tiles);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = sizeof(Smem);
  if (cudaLaunchKernelEx(&cfg, k_mlp_tile, (const float *)h->P, (const WPack *)h->Wb, X, T, n, inv_n3, h->gpart,
                         h->lpart, h->status, h->spin, h->hook) != cudaSuccess)
    return PIC_ECUDA;
  cfg.gridDim = dim3((NPARAM + 31) / 32);
  cfg.blockDim = dim3(RW * 32);
  cfg.dynamicSmemBytes = 0;
  if (cudaLaunchKernelEx(&cfg, k_mlp_reduce, (const float *)h->gpart, (const float *)h->lpart, tiles, h->grad, h->loss,
                         inv_n3, h->P, h->m, h->v, h->Wb, a, (const int *)h->status) != cudaSuccess)
    return PIC_ECUDA;
  return 0;
}

// splitmix64 (Steele, Lea, Flood 2014): seeds the initial weights
uint64_t splitmix(uint64_t &x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

// PIC_ETIMEOUT if a bounded wait of the handle's kernels gave up since the last call: the error
// latches on the handle (device flag cleared) until pic_mlp_set_params; synchronous (the
// handle's work must have completed)
int mlp_take_status(pic_mlp *h) {
  int st = 0;
  if (cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
  if (st) {
    cudaMemset(h->status, 0, sizeof(int));
    h->latched = PIC_ETIMEOUT;
  }
  return h->latched;
}

// forward pass enqueued on st without synchronising (used by the fluid closure)
int mlp_forward_async(pic_mlp *h, const float *X, int n, float *Y, cudaStream_t st) {
  if (!h || !X || !Y) return PIC_EINVAL;
  if (h->latched) return h->latched;
  return run_forward(h, X, n, Y, st);
}

extern "C" {

int pic_mlp_nparam(void) { return NPARAM; }

int pic_mlp_create(uint64_t seed, pic_mlp **out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  pic_mlp *h = new (std::nothrow) pic_mlp();
  if (!h) return PIC_ENOMEM;
  if (cudaMalloc(&h->P, NPARAM * 4) != cudaSuccess || cudaMalloc(&h->m, NPARAM * 4) != cudaSuccess ||
      cudaMalloc(&h->v, NPARAM * 4) != cudaSuccess || cudaMalloc(&h->grad, NPARAM * 4) != cudaSuccess ||
      cudaMalloc(&h->loss, 8) != cudaSuccess || cudaMalloc(&h->status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->Wb, sizeof(WPack)) != cudaSuccess) {
    pic_mlp_free(h);
    return PIC_ENOMEM;
  }
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for weights and biases
  std::vector<float> P(NPARAM);
  uint64_t st = seed;
  auto fill = [&](int off, int cnt, int fan_in) {
    const double b = 1.0 / std::sqrt((double)fan_in);
    for (int q = 0; q < cnt; ++q) P[off + q] = (float)((((double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0) * b);
  };
  fill(oW1, NH * NI, NI); fill(ob1, NH, NI); fill(oW2, NH * NH, NH); fill(ob2, NH, NH);
  fill(oW3, NO * NH, NH); fill(ob3, NO, NH);
  cudaMemcpy(h->P, P.data(), NPARAM * 4, cudaMemcpyHostToDevice);
  cudaMemset(h->m, 0, NPARAM * 4);
  cudaMemset(h->v, 0, NPARAM * 4);
  cudaMemset(h->status, 0, sizeof(int));
  cudaMemset(h->Wb, 0, sizeof(WPack));
  if (pack(h)) {
    pic_mlp_free(h);
    return PIC_ECUDA;
  }
  *out = h;
  return 0;
}

void pic_mlp_free(pic_mlp *h) {
  if (!h) return;
  cudaFree(h->P); cudaFree(h->m); cudaFree(h->v); cudaFree(h->grad); cudaFree(h->gpart); cudaFree(h->lpart);
  cudaFree(h->loss);
  cudaFree(h->status);
  cudaFree(h->Wb);
  delete h;
}

int pic_mlp_set_params(pic_mlp *h, const float *host, int n) {
  if (!h || !host || n != NPARAM) return PIC_EINVAL;
  if (cudaMemcpy(h->P, host, NPARAM * 4, cudaMemcpyHostToDevice) != cudaSuccess) return PIC_ECUDA;
  cudaMemset(h->m, 0, NPARAM * 4);
  cudaMemset(h->v, 0, NPARAM * 4);
  h->t = 0;
  h->latched = 0;
  return pack(h);
}

int pic_mlp_test_hook(pic_mlp *h, unsigned hook, int spin) {
  if (!h || spin < 0 || (hook & ~(unsigned)(PIC_MLP_HOOK_NO_WEIGHT_COPY | PIC_MLP_HOOK_NO_FORWARD_MMA))) return PIC_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return PIC_ECUDA;
  h->hook = hook;
  h->spin = spin > 0 ? spin : kSpin;
  return 0;
}

int pic_mlp_get_params(pic_mlp *h, float *host, int n) {
  if (!h || !host || n != NPARAM) return PIC_EINVAL;
  return cudaMemcpy(host, h->P, NPARAM * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : PIC_ECUDA;
}

int pic_mlp_forward(pic_mlp *h, const float *X, int n, float *Y, void *stream) {
  if (!h || !X || !Y) return PIC_EINVAL;
  if (h->latched) return h->latched;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int rc = run_forward(h, X, n, Y, st);
  if (rc) return rc;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PIC_ECUDA;
  return mlp_take_status(h);
}

int pic_mlp_grad(pic_mlp *h, const float *X, const float *T, int n, float *grad_host, double *loss, void *stream) {
  if (!h || !X || !T) return PIC_EINVAL;
  if (h->latched) return h->latched;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int rc = run_tiles(h, X, T, n, AdamArgs{0, 0, 0, 0, 0, 0, 0}, st);
  if (rc) return rc;
  if (grad_host && cudaMemcpyAsync(grad_host, h->grad, NPARAM * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PIC_ECUDA;
  if (loss && cudaMemcpyAsync(loss, h->loss, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return PIC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PIC_ECUDA;
  return mlp_take_status(h);
}

int pic_mlp_train(pic_mlp *h, const float *X, const float *T, int n, int batch, int steps, float lr,
                  double *last_loss, void *stream) {
  if (!h || !X || !T || n <= 0 || batch <= 0 || steps < 0) return PIC_EINVAL;
  if (h->latched) return h->latched;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int k = 0; k < steps; ++k) {
    const long long off = ((long long)k * batch) % n;
    const int nb = (int)((off + batch <= n) ? batch : n - off);
    h->t += 1;
    const float c1 = 1.0f - powf(b1, (float)h->t), c2 = 1.0f - powf(b2, (float)h->t);
    const int rc = run_tiles(h, X + off * NI, T + off * NO, nb, AdamArgs{1, lr, b1, b2, eps, c1, c2}, st);
    if (rc) return rc;
  }
  if (last_loss && cudaMemcpyAsync(last_loss, h->loss, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PIC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PIC_ECUDA;
  return mlp_take_status(h);
}

}  // extern "C"
