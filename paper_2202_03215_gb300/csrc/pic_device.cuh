// Device building blocks of the PIC-MCC step: Philox4x32-10, uniform
// conversions, the Gaussian table sampler, Marsaglia's isotropic direction,
// the leapfrog push with periodic wrap and the fixed-point charge weights.
// Every operation is IEEE +, -, *, /, sqrt or an exact conversion; the
// kernels are compiled with -fmad=false so that each expression rounds as
// written.
#pragma once
#include <cstdint>
#include <type_traits>

#include "pic_internal.cuh"

namespace pic {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit multiplies and a word permutation, key bumped by the Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;   // one 32x32->64 multiply each
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.y, (uint32_t)p0);
    if (r < 9) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
  }
  return c;
}

// the same function with its ten round keys given (rk[r] = key + r Weyl constants), so that
// a kernel whose key is a launch parameter reads them as constant operands
__device__ __forceinline__ uint4 philox10_rk(uint4 c, const uint32_t (&rk)[10][2]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[r][0], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk[r][1],
                   (uint32_t)p0);
  }
  return c;
}

__device__ __forceinline__ uint2 seed_key(uint64_t seed) {
  return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ float u24(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}
// decision uniform from one 32-bit word (collision test, process choice)
template <class R> __device__ __forceinline__ R u_dec(uint32_t w) {
  if constexpr (std::is_same<R, float>::value) return u24(w);
  else return (double)w * (1.0 / 4294967296.0);
}

// On-demand uniforms of one particle in one step, from blocks 1, 2, ...:
// four FP32 uniforms or two FP64 uniforms per Philox block.
template <class R> struct UStream {
  uint4 ctr;
  uint2 key;
  uint4 w;
  uint32_t c3, block;
  int pos;
  __device__ __forceinline__ UStream(uint2 k, uint64_t id, uint32_t step, uint32_t c3base)
      : key(k), c3(c3base), block(0), pos(4) {
    ctr = make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, 0u);
    w = make_uint4(0, 0, 0, 0);
  }
  __device__ __forceinline__ R next() {
    if (pos >= 4) {
      ++block;
      w = philox10(make_uint4(ctr.x, ctr.y, ctr.z, c3 | block), key);
      pos = 0;
    }
    if constexpr (std::is_same<R, float>::value) {
      const uint32_t x = pos == 0 ? w.x : pos == 1 ? w.y : pos == 2 ? w.z : w.w;
      ++pos;
      return u24(x);
    } else {
      const uint32_t a = pos == 0 ? w.x : w.z, b = pos == 0 ? w.y : w.w;
      pos += 2;
      return u53(a, b);
    }
  }
};

// linear interpolation of the Gaussian inverse-CDF table at u in [0,1)
template <class R> __device__ __forceinline__ R gauss(const float *__restrict__ T, R u) {
  const R x = u * (R)kGaussN;
  const int i = (int)x;
  const R fr = x - (R)i;
  const R a = (R)__ldg(T + i), b = (R)__ldg(T + i + 1);
  return a + fr * (b - a);
}

// Marsaglia (1972): a point uniform on the unit disc mapped to the sphere
template <class R> __device__ __forceinline__ void iso_dir(UStream<R> &us, R &nx, R &ny, R &nz) {
  R a = 0, b = 0, q = 0;
  bool ok = false;
  for (int t = 0; t < 64; ++t) {
    a = (R)2 * us.next() - (R)1;
    b = (R)2 * us.next() - (R)1;
    q = a * a + b * b;
    if (q < (R)1) { ok = true; break; }
  }
  if (!ok) { a = 0; b = 0; q = 0; }
  const R t2 = (R)2 * sqrt((R)1 - q);
  nx = a * t2; ny = b * t2; nz = (R)1 - (R)2 * q;
}

// leapfrog kick + drift in cell units with periodic re-injection; in a bounded column (Sec. V) a
// particle leaving [0, L) is taken by the electrode it crossed: returns -1 (cathode, x < 0, the
// record left at cell 0) or +1 (anode, x >= L, at cell N - 1), else 0
template <class R>
__device__ __forceinline__ int push(int N, bool bounded, R a, R d, R E, int32_t &cell, R &off, R &vx) {
  vx = vx + a * E;
  R f = off + vx * d;
  const R c = floor(f);
  f = f - c;
  int32_t cl = cell + (int32_t)c;
  if (f >= (R)1) { f = (R)0; cl += 1; }
  if (bounded) {
    if (cl < 0) { cell = 0; off = (R)0; return -1; }
    if (cl >= N) { cell = N - 1; off = (R)0; return 1; }
    cell = cl;
    off = f;
    return 0;
  }
  // cl mod N, without a division when the particle moved less than a column length
  if (cl >= N) cl = cl < 2 * N ? cl - N : cl % N;
  else if (cl < 0) {
    cl = cl >= -N ? cl + N : cl % N;
    if (cl < 0) cl += N;
  }
  cell = cl;
  off = f;
  return 0;
}

template <class R> __device__ __forceinline__ R gather(const R *E, int32_t cell, R off) {
  const R a = E[cell], b = E[cell + 1];
  return a + off * (b - a);
}

// cloud-in-cell weights as 2^32 fixed point: node cell gets 2^32 - k, node cell+1 gets k
template <class R> __device__ __forceinline__ unsigned long long wfix(R off) {
  return (unsigned long long)(off * (R)4294967296.0);
}

// the same weight as a 32-bit integer: off < 1, so off 2^32 < 2^32 (exact in both precisions)
template <class R> __device__ __forceinline__ uint32_t wfix32(R off) { return (uint32_t)(off * (R)4294967296.0); }

// collision-table position; above the table the last value is held
template <class R>
__device__ __forceinline__ int tab_pos(R eps, R inv_de, int ntab, R &fr, bool &ovf) {
  const R x = eps * inv_de;
  if (!(x < (R)(ntab - 1))) { fr = (R)1; ovf = true; return ntab - 2; }  // also NaN
  const int i = (int)x;
  fr = x - (R)i;
  ovf = false;
  return i;
}

template <class R> __device__ __forceinline__ R tab_at(const R *__restrict__ t, int i, R fr) {
  const R a = __ldg(t + i), b = __ldg(t + i + 1);
  return a + fr * (b - a);
}

}  // namespace pic
