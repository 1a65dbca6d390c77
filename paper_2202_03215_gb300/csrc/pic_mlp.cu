// Closure network of the quasi-neutral fluid screen: MLP 15 -> 128 -> 128 -> 3,
// GELU (tanh form) on the hidden layers, mean-squared-error loss, Adam.
// BF16 operands on the 5th-generation tensor cores (tcgen05, FP32 accumulation in
// tensor memory), FP32 master weights and optimizer state.
//
// Training: persistent CTAs (at most one per SM) run forward, backward and the weight
// gradients of their tiles of 128 samples (pic_mlp_train_tc.cu) and write them as one
// partial per CTA; a second kernel here sums the partials in a fixed order (deterministic
// gradients for a given SM count)
// and applies Adam, which also refreshes the BF16 copy of the weights in the
// tensor cores' operand layout that the tile kernel stages with one bulk copy.
// The forward pass (inference) runs on tcgen05 too (pic_mlp_tc.cu).
// Parameter layout (FP32, flat): W1[128][15], b1[128], W2[128][128], b2[128],
// W3[3][128], b3[3]  (row = output unit).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "pic.h"
#include "pic_mlp_layout.cuh"

namespace {

using namespace mlpl;
constexpr int S = 128;                // samples per training tile
constexpr int kSpin = 200000;         // polls of an mbarrier (each suspends up to 10 us) before giving up

using bf = __nv_bfloat16;

// programmatic dependent launch: let the next kernel of the stream start its launch now; wait
// for the previous kernel of the stream to complete (no-op without a programmatic dependency)
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

struct AdamArgs {
  int on;
  float lr, b1, b2, eps, c1, c2;
};

// g[p] = sum of the CTAs' partials in a fixed order (partials w, w+16, .. per warp, then the
// warps in order); optionally Adam (Kingma & Ba) on the FP32 master weights, refreshing the
// BF16 copy. Block 0 also sums the loss.
constexpr int RW = 16;  // warps of the reduction
__global__ void __launch_bounds__(RW * 32) k_mlp_reduce(const float *__restrict__ gpart, const float *__restrict__ lpart,
                                                        int nparts, float *__restrict__ grad, double *__restrict__ loss,
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
    for (int q = w; q < nparts; q += RW) s += gpart[(size_t)q * GSTRIDE + p];
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
      const int q = windex(p);
      if (q >= 0) Wb[q] = __float2bfloat16_rn(x);
    }
  }
  if (blockIdx.x == 0 && w == 1) {
    double l = 0.0;
    for (int q = lane; q < nparts; q += 32) l += (double)lpart[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0) *loss = l * (double)inv_n3;
  }
}

// BF16 copy of the weights (the padding of the copy stays zero)
__global__ void k_mlp_pack(const float *__restrict__ P, bf *__restrict__ Wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const int q = windex(p);
  if (q >= 0) Wb[q] = __float2bfloat16_rn(P[p]);
}

}  // namespace

int mlp_forward_tc(const float *P, const float *X, int n, float *Y, int *status, int spin, unsigned hook,
                   cudaStream_t st);
int mlp_train_tiles_tc(const float *P, const void *Wb, const float *X, const float *T, int n, float inv_n3,
                       float *gpart, float *lpart, int ctas, int *status, int spin, unsigned hook, cudaStream_t st);

struct pic_mlp {
  float *P = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  float *gpart = nullptr, *lpart = nullptr;
  bf *Wb = nullptr;        // BF16 weights in the tensor cores' operand layout (TrainW)
  double *loss = nullptr;
  int *status = nullptr;   // device: 1 once a bounded wait of the tensor-core forward gave up
  int cap_parts = 0;       // partials gpart / lpart hold
  int nsm = 0;             // streaming multiprocessors: the training kernel's largest grid
  int t = 0;   // Adam steps taken
  int spin = kSpin;        // polls of a bounded wait (pic_mlp_test_hook)
  unsigned hook = 0;       // PIC_MLP_HOOK_* (pic_mlp_test_hook)
  int latched = 0;         // PIC_ETIMEOUT once a wait gave up, until pic_mlp_set_params
};

namespace {

// CTAs of the training kernel for n samples: one per tile, at most one per SM (each CTA then
// loops over tiles b, b + ctas, ..)
int train_ctas(const pic_mlp *h, int n) { return std::min((n + S - 1) / S, h->nsm); }

int ensure(pic_mlp *h, int n) {
  const int parts = train_ctas(h, n);
  if (parts <= h->cap_parts) return 0;
  cudaFree(h->gpart);
  cudaFree(h->lpart);
  h->gpart = nullptr;
  h->lpart = nullptr;
  if (cudaMalloc(&h->gpart, (size_t)parts * GSTRIDE * 4) != cudaSuccess ||
      cudaMalloc(&h->lpart, (size_t)parts * 4) != cudaSuccess)
    return PIC_ENOMEM;
  h->cap_parts = parts;
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
  const int parts = train_ctas(h, n);
  const float inv_n3 = 1.0f / (3.0f * (float)n);
  const int rc2 =
      mlp_train_tiles_tc(h->P, h->Wb, X, T, n, inv_n3, h->gpart, h->lpart, parts, h->status, h->spin, h->hook, st);
  if (rc2) return rc2;
  // the reduction with programmatic stream serialization: it may be scheduled while the tile
  // kernel drains and waits for it (griddepcontrol.wait) before it reads the partials
  cudaLaunchAttribute pdl;
  pdl.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl.val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.stream = st;
  cfg.attrs = &pdl;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((NPARAM + 31) / 32);
  cfg.blockDim = dim3(RW * 32);
  cfg.dynamicSmemBytes = 0;
  if (cudaLaunchKernelEx(&cfg, k_mlp_reduce, (const float *)h->gpart, (const float *)h->lpart, parts, h->grad, h->loss,
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
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || h->nsm <= 0) {
    delete h;
    return PIC_ECUDA;
  }
  if (cudaMalloc(&h->P, NPARAM * 4) != cudaSuccess || cudaMalloc(&h->m, NPARAM * 4) != cudaSuccess ||
      cudaMalloc(&h->v, NPARAM * 4) != cudaSuccess || cudaMalloc(&h->grad, NPARAM * 4) != cudaSuccess ||
      cudaMalloc(&h->loss, 8) != cudaSuccess || cudaMalloc(&h->status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->Wb, sizeof(TrainW)) != cudaSuccess) {
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
  cudaMemset(h->Wb, 0, sizeof(TrainW));
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
