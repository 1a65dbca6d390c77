// Closure network of the quasi-neutral fluid screen: MLP 15 -> 128 -> 128 -> 3,
// GELU (tanh form) on the hidden layers, mean-squared-error loss, Adam.
// BF16 operands on the tensor cores (mma.sync m16n8k16, FP32 accumulation),
// FP32 master weights and optimizer state.
//
// One CTA trains on a tile of 64 samples: forward, backward and the weight
// gradients of its tile, written as a partial; a second kernel sums the
// partials in a fixed order (deterministic gradients), a third applies Adam.
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
constexpr int S = 64;                 // samples per tile
constexpr int WARPS = S / 16;         // one warp per 16 samples in the row passes
constexpr int THREADS = WARPS * 32;
constexpr int oW1 = 0, ob1 = NH * NI, oW2 = ob1 + NH, ob2 = oW2 + NH * NH, oW3 = ob2 + NH, ob3 = oW3 + NO * NH;
constexpr int NPARAM = ob3 + NO;      // 18947

using bf = __nv_bfloat16;

struct Smem {
  bf W1[NH][NIP];
  bf W2[NH][NH];
  bf W3[NOP][NH];
  bf X[S][NIP];
  bf A1[S][NH];        // activations of layer 1, later dL/dz1
  bf A2[S][NH];        // activations of layer 2, later dL/dz2
  bf dY[S][NOP];
  float Z1[S][NH];
  float Z2[S][NH];
  float b1[NH], b2[NH], b3[NOP];
  float cs[WARPS][NH]; // per-warp column sums (bias gradients)
  float loss[WARPS];
};

// a matrix in shared memory read element by element: (r, c) at p[r*ld + c], or p[c*ld + r] if tr
struct Mat {
  const bf *p;
  int ld;
  bool tr;
};
__device__ __forceinline__ unsigned short bits(bf x) { return *reinterpret_cast<unsigned short *>(&x); }
__device__ __forceinline__ unsigned at2(Mat m, int r, int c, int r2, int c2) {
  const bf lo = m.tr ? m.p[c * m.ld + r] : m.p[r * m.ld + c];
  const bf hi = m.tr ? m.p[c2 * m.ld + r2] : m.p[r2 * m.ld + c2];
  return (unsigned)bits(lo) | ((unsigned)bits(hi) << 16);
}

__device__ __forceinline__ void mma(float c[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[16 x 8 NT] (rows r0.., columns n0..) += A(16 x K) B(K x 8 NT), one warp.
// Fragment layout of m16n8k16 (g = lane/4, t = lane%4): A rows g, g+8 and columns 2t, 2t+1,
// 2t+8, 2t+9; B columns g and rows 2t, 2t+1, 2t+8, 2t+9; C rows g, g+8 and columns 2t, 2t+1.
template <int NT>
__device__ __forceinline__ void gemm(float c[NT][4], Mat A, int r0, Mat B, int n0, int K) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int k0 = 0; k0 < K; k0 += 16) {
    unsigned a[4];
    a[0] = at2(A, r0 + g, k0 + 2 * t, r0 + g, k0 + 2 * t + 1);
    a[1] = at2(A, r0 + g + 8, k0 + 2 * t, r0 + g + 8, k0 + 2 * t + 1);
    a[2] = at2(A, r0 + g, k0 + 2 * t + 8, r0 + g, k0 + 2 * t + 9);
    a[3] = at2(A, r0 + g + 8, k0 + 2 * t + 8, r0 + g + 8, k0 + 2 * t + 9);
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int n = n0 + 8 * nt + g;
      unsigned b[2];
      b[0] = at2(B, k0 + 2 * t, n, k0 + 2 * t + 1, n);
      b[1] = at2(B, k0 + 2 * t + 8, n, k0 + 2 * t + 9, n);
      mma(c[nt], a, b);
    }
  }
}

// GELU (tanh form) through s = (1 + tanh u)/2 = 1/(1 + exp(-2u)), u = sqrt(2/pi)(z + 0.044715 z^3):
// gelu = z s, gelu' = s + 2 z s (1 - s) du/dz
__device__ __forceinline__ float gelu(float z) {
  const float u = 0.7978845608028654f * (z + 0.044715f * z * z * z);
  return __fdividef(z, 1.0f + __expf(-2.0f * u));
}
__device__ __forceinline__ float gelu_d(float z) {
  const float c = 0.7978845608028654f;
  const float u = c * (z + 0.044715f * z * z * z);
  const float s = __fdividef(1.0f, 1.0f + __expf(-2.0f * u));
  return s + 2.0f * z * s * (1.0f - s) * c * (1.0f + 3.0f * 0.044715f * z * z);
}

// sum of the two row values of a C fragment column over the 8 row groups (lanes t, t+4, ..)
__device__ __forceinline__ float colsum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

// mode 0: forward + backward of the tile, partial gradients and loss; mode 1: forward only (Y)
__global__ void __launch_bounds__(THREADS) k_mlp_tile(const float *__restrict__ P, const float *__restrict__ X,
                                                      const float *__restrict__ T, int n, float inv_n3,
                                                      float *__restrict__ gpart, float *__restrict__ lpart,
                                                      float *__restrict__ Y, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, g = lane >> 2, t = lane & 3;
  const int tile = blockIdx.x, s0 = tile * S;
  // weights to BF16, biases FP32, the tile's inputs
  for (int q = tid; q < NH * NIP; q += THREADS) {
    const int h = q / NIP, i = q % NIP;
    sm.W1[h][i] = __float2bfloat16_rn(i < NI ? P[oW1 + h * NI + i] : 0.0f);
  }
  for (int q = tid; q < NH * NH; q += THREADS) sm.W2[q / NH][q % NH] = __float2bfloat16_rn(P[oW2 + q]);
  for (int q = tid; q < NOP * NH; q += THREADS) {
    const int o = q / NH, k = q % NH;
    sm.W3[o][k] = __float2bfloat16_rn(o < NO ? P[oW3 + o * NH + k] : 0.0f);
  }
  for (int q = tid; q < NH; q += THREADS) { sm.b1[q] = P[ob1 + q]; sm.b2[q] = P[ob2 + q]; }
  if (tid < NOP) sm.b3[tid] = tid < NO ? P[ob3 + tid] : 0.0f;
  for (int q = tid; q < S * NIP; q += THREADS) {
    const int r = q / NIP, i = q % NIP, s = s0 + r;
    sm.X[r][i] = __float2bfloat16_rn((s < n && i < NI) ? X[(size_t)s * NI + i] : 0.0f);
  }
  __syncthreads();
  const int r0 = 16 * w;
  // layer 1 and layer 2 (rows of this warp)
  {
    float c[16][4];
    for (int nt = 0; nt < 16; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
    gemm<16>(c, Mat{&sm.X[0][0], NIP, false}, r0, Mat{&sm.W1[0][0], NIP, true}, 0, NIP);
    for (int nt = 0; nt < 16; ++nt)
      for (int e = 0; e < 4; ++e) {
        const int r = r0 + g + (e >> 1) * 8, col = 8 * nt + 2 * t + (e & 1);
        const float z = c[nt][e] + sm.b1[col];
        sm.Z1[r][col] = z;
        sm.A1[r][col] = __float2bfloat16_rn(gelu(z));
      }
    __syncwarp();
    for (int nt = 0; nt < 16; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
    gemm<16>(c, Mat{&sm.A1[0][0], NH, false}, r0, Mat{&sm.W2[0][0], NH, true}, 0, NH);
    for (int nt = 0; nt < 16; ++nt)
      for (int e = 0; e < 4; ++e) {
        const int r = r0 + g + (e >> 1) * 8, col = 8 * nt + 2 * t + (e & 1);
        const float z = c[nt][e] + sm.b2[col];
        sm.Z2[r][col] = z;
        sm.A2[r][col] = __float2bfloat16_rn(gelu(z));
      }
    __syncwarp();
  }
  // layer 3, outputs, dL/dy
  {
    float c[1][4] = {{0.0f, 0.0f, 0.0f, 0.0f}};
    gemm<1>(c, Mat{&sm.A2[0][0], NH, false}, r0, Mat{&sm.W3[0][0], NH, true}, 0, NH);
    float lsum = 0.0f;
    float bsum[2] = {0.0f, 0.0f};
    for (int e = 0; e < 4; ++e) {
      const int r = r0 + g + (e >> 1) * 8, o = 2 * t + (e & 1), s = s0 + r;
      float dy = 0.0f;
      if (o < NO && s < n) {
        const float y = c[0][e] + sm.b3[o];
        if (mode == 1) {
          Y[(size_t)s * NO + o] = y;
        } else {
          const float d = y - T[(size_t)s * NO + o];
          lsum += d * d;
          dy = 2.0f * d * inv_n3;
        }
      }
      bsum[e & 1] += dy;
      sm.dY[r][o] = __float2bfloat16_rn(dy);
    }
    // dY columns 8..15 are zero padding
    for (int q = lane; q < 16 * 8; q += 32) sm.dY[r0 + q / 8][8 + q % 8] = __float2bfloat16_rn(0.0f);
    for (int o = 0; o < 2; ++o) {
      const float v = colsum(bsum[o]);
      if (g == 0 && 2 * t + o < NO) sm.cs[w][2 * t + o] = v;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) sm.loss[w] = lsum;
  }
  if (mode == 1) return;
  float *gp = gpart + (size_t)tile * NPARAM;
  __syncthreads();
  if (tid < NO) {
    float v = 0.0f;
    for (int q = 0; q < WARPS; ++q) v += sm.cs[q][tid];
    gp[ob3 + tid] = v;
  }
  if (tid == 0) {
    float v = 0.0f;
    for (int q = 0; q < WARPS; ++q) v += sm.loss[q];
    lpart[tile] = v;
  }
  // dL/dW3 = dY^T A2 (outputs x hidden, summed over the tile's samples); warp w: hidden columns 32w..32w+31
  {
    float c[4][4];
    for (int nt = 0; nt < 4; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
    gemm<4>(c, Mat{&sm.dY[0][0], NOP, true}, 0, Mat{&sm.A2[0][0], NH, false}, 32 * w, S);
    for (int nt = 0; nt < 4; ++nt)
      for (int e = 0; e < 2; ++e) {
        const int o = g, col = 32 * w + 8 * nt + 2 * t + e;
        if (o < NO) gp[oW3 + o * NH + col] = c[nt][e];
      }
  }
  __syncthreads();   // A2 is read above: from here on it holds dL/dz2
  // dL/dz2 = (dY W3) * gelu'(z2), rows of this warp
  {
    float c[16][4];
    for (int nt = 0; nt < 16; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
    gemm<16>(c, Mat{&sm.dY[0][0], NOP, false}, r0, Mat{&sm.W3[0][0], NH, false}, 0, NOP);
    for (int nt = 0; nt < 16; ++nt) {
      float bs[2] = {0.0f, 0.0f};
      for (int e = 0; e < 4; ++e) {
        const int r = r0 + g + (e >> 1) * 8, col = 8 * nt + 2 * t + (e & 1);
        const float dz = c[nt][e] * gelu_d(sm.Z2[r][col]);
        bs[e & 1] += dz;
        sm.A2[r][col] = __float2bfloat16_rn(dz);
      }
      for (int o = 0; o < 2; ++o) {
        const float v = colsum(bs[o]);
        if (g == 0) sm.cs[w][8 * nt + 2 * t + o] = v;
      }
    }
  }
  __syncthreads();
  for (int q = tid; q < NH; q += THREADS) {
    float v = 0.0f;
    for (int ww = 0; ww < WARPS; ++ww) v += sm.cs[ww][q];
    gp[ob2 + q] = v;
  }
  // dL/dW2 = dZ2^T A1; warp w: output rows 32w..32w+31 in two 16-row tiles
  for (int mt = 0; mt < 2; ++mt) {
    float c[16][4];
    for (int nt = 0; nt < 16; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
    const int h0 = 32 * w + 16 * mt;
    gemm<16>(c, Mat{&sm.A2[0][0], NH, true}, h0, Mat{&sm.A1[0][0], NH, false}, 0, S);
    for (int nt = 0; nt < 16; ++nt)
      for (int e = 0; e < 4; ++e) {
        const int h = h0 + g + (e >> 1) * 8, col = 8 * nt + 2 * t + (e & 1);
        gp[oW2 + h * NH + col] = c[nt][e];
      }
  }
  // dL/dz1 = (dZ2 W2) * gelu'(z1), rows of this warp, kept in registers until A1 is free
  float d1[16][4];
  for (int nt = 0; nt < 16; ++nt) d1[nt][0] = d1[nt][1] = d1[nt][2] = d1[nt][3] = 0.0f;
  gemm<16>(d1, Mat{&sm.A2[0][0], NH, false}, r0, Mat{&sm.W2[0][0], NH, false}, 0, NH);
  __syncthreads();   // A1 is read by dL/dW2 above: from here on it holds dL/dz1
  for (int nt = 0; nt < 16; ++nt) {
    float bs[2] = {0.0f, 0.0f};
    for (int e = 0; e < 4; ++e) {
      const int r = r0 + g + (e >> 1) * 8, col = 8 * nt + 2 * t + (e & 1);
      const float dz = d1[nt][e] * gelu_d(sm.Z1[r][col]);
      bs[e & 1] += dz;
      sm.A1[r][col] = __float2bfloat16_rn(dz);
    }
    for (int o = 0; o < 2; ++o) {
      const float v = colsum(bs[o]);
      if (g == 0) sm.cs[w][8 * nt + 2 * t + o] = v;
    }
  }
  __syncthreads();
  for (int q = tid; q < NH; q += THREADS) {
    float v = 0.0f;
    for (int ww = 0; ww < WARPS; ++ww) v += sm.cs[ww][q];
    gp[ob1 + q] = v;
  }
  // dL/dW1 = dZ1^T X; warp w: rows 32w..32w+31
  for (int mt = 0; mt < 2; ++mt) {
    float c[2][4];
    for (int nt = 0; nt < 2; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
    const int h0 = 32 * w + 16 * mt;
    gemm<2>(c, Mat{&sm.A1[0][0], NH, true}, h0, Mat{&sm.X[0][0], NIP, false}, 0, S);
    for (int nt = 0; nt < 2; ++nt)
      for (int e = 0; e < 4; ++e) {
        const int h = h0 + g + (e >> 1) * 8, i = 8 * nt + 2 * t + (e & 1);
        if (i < NI) gp[oW1 + h * NI + i] = c[nt][e];
      }
  }
}

// g[p] = sum over tiles of the partials, in tile order; loss likewise (block 0)
__global__ void k_mlp_reduce(const float *__restrict__ gpart, const float *__restrict__ lpart, int ntiles,
                             float *__restrict__ grad, double *__restrict__ loss, float inv_n3) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NPARAM) {
    float v = 0.0f;
    for (int q = 0; q < ntiles; ++q) v += gpart[(size_t)q * NPARAM + p];
    grad[p] = v;
  }
  if (p == 0) {
    double l = 0.0;
    for (int q = 0; q < ntiles; ++q) l += (double)lpart[q];
    *loss = l * (double)inv_n3;
  }
}

// Adam (Kingma & Ba) on the FP32 master weights
__global__ void k_mlp_adam(float *__restrict__ P, const float *__restrict__ grad, float *__restrict__ m,
                           float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const float gr = grad[p];
  const float mm = b1 * m[p] + (1.0f - b1) * gr;
  const float vv = b2 * v[p] + (1.0f - b2) * gr * gr;
  m[p] = mm;
  v[p] = vv;
  P[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

}  // namespace

int mlp_forward_tc(const float *P, const float *X, int n, float *Y, int *status, cudaStream_t st);

struct pic_mlp {
  float *P = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  float *gpart = nullptr, *lpart = nullptr;
  double *loss = nullptr;
  int *status = nullptr;   // device: 1 once a bounded wait of the tensor-core forward gave up
  int cap_tiles = 0;
  int t = 0;   // Adam steps taken
};

namespace {

int ensure(pic_mlp *h, int n) {
  const int tiles = (n + S - 1) / S;
  if (tiles <= h->cap_tiles) return 0;
  cudaFree(h->gpart);
  cudaFree(h->lpart);
  h->gpart = nullptr;
  h->lpart = nullptr;
  if (cudaMalloc(&h->gpart, (size_t)tiles * NPARAM * 4) != cudaSuccess ||
      cudaMalloc(&h->lpart, (size_t)tiles * 4) != cudaSuccess)
    return PIC_ENOMEM;
  h->cap_tiles = tiles;
  return 0;
}

int run_forward(pic_mlp *h, const float *X, int n, float *Y, cudaStream_t st) {
  return mlp_forward_tc(h->P, X, n, Y, h->status, st);
}

int run_tiles(pic_mlp *h, const float *X, const float *T, int n, float *Y, int mode, cudaStream_t st) {
  if (n <= 0) return PIC_EINVAL;
  if (mode == 0) {   // per-tile partial gradients only when training
    const int rc = ensure(h, n);
    if (rc) return rc;
  }
  const int tiles = (n + S - 1) / S;
  const float inv_n3 = 1.0f / (3.0f * (float)n);
  cudaFuncSetAttribute(k_mlp_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  k_mlp_tile<<<tiles, THREADS, sizeof(Smem), st>>>(h->P, X, T, n, inv_n3, h->gpart, h->lpart, Y, mode);
  if (mode == 0) k_mlp_reduce<<<(NPARAM + 255) / 256, 256, 0, st>>>(h->gpart, h->lpart, tiles, h->grad, h->loss, inv_n3);
  return cudaGetLastError() == cudaSuccess ? 0 : PIC_ECUDA;
}

// splitmix64 (Steele, Lea, Flood 2014): seeds the initial weights
uint64_t splitmix(uint64_t &x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

// PIC_ETIMEOUT (and the flag cleared) if a bounded wait of a forward pass gave up since the
// last call; synchronous (the handle's work must have completed)
int mlp_take_status(pic_mlp *h) {
  int st = 0;
  if (cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
  if (!st) return 0;
  cudaMemset(h->status, 0, sizeof(int));
  return PIC_ETIMEOUT;
}

// forward pass enqueued on st without synchronising (used by the fluid closure)
int mlp_forward_async(pic_mlp *h, const float *X, int n, float *Y, cudaStream_t st) {
  if (!h || !X || !Y) return PIC_EINVAL;
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
      cudaMalloc(&h->loss, 8) != cudaSuccess || cudaMalloc(&h->status, sizeof(int)) != cudaSuccess) {
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
  *out = h;
  return 0;
}

void pic_mlp_free(pic_mlp *h) {
  if (!h) return;
  cudaFree(h->P); cudaFree(h->m); cudaFree(h->v); cudaFree(h->grad); cudaFree(h->gpart); cudaFree(h->lpart);
  cudaFree(h->loss);
  cudaFree(h->status);
  delete h;
}

int pic_mlp_set_params(pic_mlp *h, const float *host, int n) {
  if (!h || !host || n != NPARAM) return PIC_EINVAL;
  if (cudaMemcpy(h->P, host, NPARAM * 4, cudaMemcpyHostToDevice) != cudaSuccess) return PIC_ECUDA;
  cudaMemset(h->m, 0, NPARAM * 4);
  cudaMemset(h->v, 0, NPARAM * 4);
  h->t = 0;
  return 0;
}

int pic_mlp_get_params(pic_mlp *h, float *host, int n) {
  if (!h || !host || n != NPARAM) return PIC_EINVAL;
  return cudaMemcpy(host, h->P, NPARAM * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : PIC_ECUDA;
}

int pic_mlp_forward(pic_mlp *h, const float *X, int n, float *Y, void *stream) {
  if (!h || !X || !Y) return PIC_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int rc = run_forward(h, X, n, Y, st);
  if (rc) return rc;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PIC_ECUDA;
  return mlp_take_status(h);
}

int pic_mlp_grad(pic_mlp *h, const float *X, const float *T, int n, float *grad_host, double *loss, void *stream) {
  if (!h || !X || !T) return PIC_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int rc = run_tiles(h, X, T, n, nullptr, 0, st);
  if (rc) return rc;
  if (grad_host && cudaMemcpyAsync(grad_host, h->grad, NPARAM * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PIC_ECUDA;
  if (loss && cudaMemcpyAsync(loss, h->loss, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return PIC_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? 0 : PIC_ECUDA;
}

int pic_mlp_train(pic_mlp *h, const float *X, const float *T, int n, int batch, int steps, float lr,
                  double *last_loss, void *stream) {
  if (!h || !X || !T || n <= 0 || batch <= 0 || steps < 0) return PIC_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int k = 0; k < steps; ++k) {
    const long long off = ((long long)k * batch) % n;
    const int nb = (int)((off + batch <= n) ? batch : n - off);
    int rc = run_tiles(h, X + off * NI, T + off * NO, nb, nullptr, 0, st);
    if (rc) return rc;
    h->t += 1;
    const float c1 = 1.0f - powf(b1, (float)h->t), c2 = 1.0f - powf(b2, (float)h->t);
    k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(h->P, h->grad, h->m, h->v, lr, b1, b2, eps, c1, c2);
  }
  if (last_loss && cudaMemcpyAsync(last_loss, h->loss, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PIC_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? 0 : PIC_ECUDA;
}

}  // extern "C"
