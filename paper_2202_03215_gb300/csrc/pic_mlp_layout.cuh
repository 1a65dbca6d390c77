// Layouts shared by the closure network's kernels: the parameter vector, the partial
// gradients of the training tiles, and the BF16 weight image in the canonical K-major,
// no-swizzle operand layout of the tensor cores.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

namespace mlpl {

constexpr int NI = 15, NH = 128, NO = 3;
constexpr int K1 = 16;               // input width padded to one MMA K step
constexpr int N3 = 16;               // output width padded to the smallest N of an M = 128 MMA
constexpr int oW1 = 0, ob1 = NH * NI, oW2 = ob1 + NH, ob2 = oW2 + NH * NH, oW3 = ob2 + NH, ob3 = oW3 + NO * NH;
constexpr int NPARAM = ob3 + NO;     // 18947
constexpr int GSTRIDE = (NPARAM + 3) & ~3;   // floats between the partial gradients of two tiles (16-byte aligned)

// byte offset of element (r, k) of an R x K BF16 matrix in the canonical K-major, no-swizzle
// layout: 8-row x 16-byte core matrices, consecutive along K (128 B apart), 8-row groups K x 16 B apart
__host__ __device__ constexpr int cm_off(int r, int k, int K) {
  return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// BF16 weights as the training kernel reads them: W1 N = 128 x K = 16 (column 15 zero),
// W2 128 x 128, W3 16 x 128 (rows 3..15 zero); [out][in], K-major
struct TrainW {
  __nv_bfloat16 W1[NH * K1];
  __nv_bfloat16 W2[NH * NH];
  __nv_bfloat16 W3[N3 * NH];
};
static_assert(sizeof(TrainW) % 16 == 0, "16-byte bulk copy");

// index (in BF16 elements) of parameter p in TrainW, -1 for biases
__host__ __device__ __forceinline__ int windex(int p) {
  if (p < ob1) return cm_off(p / NI, p % NI, K1) / 2;
  if (p >= oW2 && p < ob2) return NH * K1 + cm_off((p - oW2) / NH, (p - oW2) % NH, NH) / 2;
  if (p >= oW3 && p < ob3) return NH * K1 + NH * NH + cm_off((p - oW3) / NH, (p - oW3) % NH, NH) / 2;
  return -1;
}

}  // namespace mlpl
