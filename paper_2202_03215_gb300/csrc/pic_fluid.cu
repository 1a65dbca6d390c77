// Quasi-neutral three-moment fluid model (Sec. IV.A, eqs. 3-5, 8-12, 17)
// of many independent periodic columns: one thread block per column holds the
// whole column in shared memory (state, coefficient and face arrays, the two
// cyclic tridiagonal systems) and advances it through a chunk of steps with no
// global-memory round trip; the spectral record and the closure features are
// the only per-step outputs.  The step is written out in include/pic.h.
// The state is kept as FP32 pairs (hi + lo) advanced by exact two-sums, so that
// increments far below one FP32 ulp of n or Te still accumulate (slow growth at
// a small time step); every coefficient and flux is evaluated from hi in FP32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "pic.h"

int mlp_forward_async(pic_mlp *h, const float *X, int n, float *Y, cudaStream_t st);
int mlp_take_status(pic_mlp *h);

namespace {

constexpr int kThreads = 512;
constexpr int kMaxCells = 4096;
constexpr int kRows = kMaxCells / kThreads;   // rows per thread at the largest column
constexpr int kMaxModes = 64;
constexpr int kMaxT = 256;
constexpr int kNQ = 6;                          // muN, DN, mueN, DeN, nu_izN, lossN
constexpr int kArrays = 14;                     // shared-memory arrays of n_cells floats
constexpr int kChunk = 2000;                    // steps per launch without a closure
constexpr float kTd = 1e-21f;

struct ColK {
  int N, logN;
  long long off;       // first cell in the state arrays
  float dx, inv_dx, r, s, k;   // dx, 1/dx, dt/dx^2, dt/dx, 3/(2 dx)
  float GT, nu_w, mu_i, Ng, invNg;
  int pair;            // nu_w = <n nu>/<n> every step
};

struct FluidK {
  const ColK *cols;
  double *n, *T;                // state, all columns
  const float *tab;             // kNQ x nT (per gas density)
  int nT;
  float T0, inv_dT, Tmax, dt;
  int diag_every, n_modes;
  long long step0;
  int snap_base;                // buffer index of the first record of this launch
  float2 *modes;                // [snap][col][n_modes + 1]
  int n_cols;
  const float *corr;            // cells x 3 (scaled) or null
  const float *netY;            // cells x 3 (network outputs) or null
  float cs0, cs1, cs2;          // network output scales
  float nu_bound;               // |dnu| <= nu_bound nu_i (network corrections; <= 0: unbounded)
  float *feat;                  // cells x 15 or null: written after the last step
  float fs[15];                 // feature scales (divisors)
  int step;                     // stencil spacing of the features, cells
};

struct Sm {
  float *n, *nl, *T, *Tl, *u, *D, *A, *B, *G, *E, *pa, *pb, *pc, *pd;
};

__device__ __forceinline__ void tpos(const FluidK &K, float T, int &i, float &f) {
  float x = (T - K.T0) * K.inv_dT;
  x = fminf(fmaxf(x, 0.0f), (float)(K.nT - 1));
  i = min((int)x, K.nT - 2);
  f = x - (float)i;
}

// table value q at position (i, f); the table (a few KB) is read through the L1 cache
__device__ __forceinline__ float tq(const Sm &, const FluidK &K, int q, int i, float f) {
  const float a = __ldg(K.tab + q * K.nT + i), b = __ldg(K.tab + q * K.nT + i + 1);
  return a + f * (b - a);
}

// (hi, lo) += d with an exact two-sum (no contraction: -fmad=false)
__device__ __forceinline__ void add2(float &hi, float &lo, float d) {
  const float s = hi + d;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (d - bp);
  const float l = lo + e;
  hi = s + l;
  lo = l - (hi - s);
}

// periodic parallel cyclic reduction; N a power of two, N <= RP kThreads; row j:
// pa x_{j-1} + pb x_j + pc x_{j+1} = pd (fast divisions, a few ulp: the systems are
// diagonally dominant and well conditioned)
template <int RP>
__device__ void pcr(float *pa, float *pb, float *pc, float *pd, int N) {
  const int t = threadIdx.x;
  for (int s = 1; s < N; s <<= 1) {
    float na[RP], nb[RP], nc[RP], nd[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      const int j = t + r * kThreads;
      if (j < N) {
        const int jm = (j - s) & (N - 1), jp = (j + s) & (N - 1);
        const float al = -__fdividef(pa[j], pb[jm]), be = -__fdividef(pc[j], pb[jp]);
        na[r] = al * pa[jm];
        nc[r] = be * pc[jp];
        nb[r] = pb[j] + al * pc[jm] + be * pa[jp];
        nd[r] = pd[j] + al * pd[jm] + be * pd[jp];
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      const int j = t + r * kThreads;
      if (j < N) { pa[j] = na[r]; pb[j] = nb[r]; pc[j] = nc[r]; pd[j] = nd[r]; }
    }
    __syncthreads();
  }
}

// m (2, 4 or 8) consecutive floats at p (m-float aligned) into x[0..m), by vector loads
__device__ __forceinline__ void ld_rows(const float *p, int m, float (&x)[kRows]) {
  if (m == 8) {
    const float4 u = *reinterpret_cast<const float4 *>(p), v = *reinterpret_cast<const float4 *>(p + 4);
    x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w; x[4] = v.x; x[5] = v.y; x[6] = v.z; x[7] = v.w;
  } else if (m == 4) {
    const float4 u = *reinterpret_cast<const float4 *>(p);
    x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
  } else {
    const float2 u = *reinterpret_cast<const float2 *>(p);
    x[0] = u.x; x[1] = u.y;
  }
}
__device__ __forceinline__ void st_rows(float *p, int m, const float (&x)[kRows]) {
  if (m == 8) {
    *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
    *reinterpret_cast<float4 *>(p + 4) = make_float4(x[4], x[5], x[6], x[7]);
  } else if (m == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
  } else {
    *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
  }
}

// Periodic tridiagonal solve, N a power of two in [64, kMaxCells]; row j:
// pa x_{j-1} + pb x_j + pc x_{j+1} = pd; the solution is left in pd (pa, pb, pc are
// overwritten).  Partition method: thread p takes the m = max(2, N / kThreads) rows
// [p m, p m + m) into registers and eliminates them (a forward and a backward sweep)
// until every row couples only to the partition's own first and last unknowns; the
// first row then couples to the previous partition's last unknown and the last row to
// the next partition's first, so the first and last rows of all partitions form a
// periodic tridiagonal system of 2N/m rows, solved by parallel cyclic reduction; the
// interior unknowns follow by substitution.  The systems are diagonally dominant: no
// pivoting, fast reciprocals.
__device__ void solve(float *pa, float *pb, float *pc, float *pd, int N) {
  const int m = max(2, N / kThreads), P = N / m, t = threadIdx.x, j0 = t * m;
  float a[kRows], b[kRows], c[kRows], d[kRows];
  if (t < P) {
    ld_rows(pa + j0, m, a);
    ld_rows(pb + j0, m, b);
    ld_rows(pc + j0, m, c);
    ld_rows(pd + j0, m, d);
    // forward: rows 0 and 1 normalised; row i >= 2 loses x_{i-1} and gains x_0 (coefficient in a)
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float r = __fdividef(1.0f, b[i]);
      a[i] *= r; c[i] *= r; d[i] *= r;
    }
#pragma unroll
    for (int i = 2; i < kRows; ++i)
      if (i < m) {
        const float r = __fdividef(1.0f, b[i] - a[i] * c[i - 1]);
        d[i] = (d[i] - a[i] * d[i - 1]) * r;
        a[i] = -a[i] * a[i - 1] * r;
        c[i] *= r;
      }
    // backward: row i in [1, m - 3] loses x_{i+1} and gains x_{m-1} (coefficient in c)
#pragma unroll
    for (int i = kRows - 3; i >= 1; --i)
      if (i <= m - 3) {
        const float q = c[i];
        a[i] -= q * a[i + 1];
        d[i] -= q * d[i + 1];
        c[i] = -q * c[i + 1];
      }
    // row 0 loses x_1 (for m >= 3; for m == 2, x_1 is the last unknown already)
    if (m >= 3) {
      const float q = c[0], r = __fdividef(1.0f, 1.0f - q * a[1]);
      a[0] *= r;
      d[0] = (d[0] - q * d[1]) * r;
      c[0] = -q * c[1] * r;
    }
  }
  __syncthreads();   // every partition is in registers: the arrays take the reduced system
  if (t < P) {
    // the last row, m - 1 (selected explicitly: an index computed from m would put the rows in
    // local memory)
    const float aL = m == 8 ? a[7] : m == 4 ? a[3] : a[1];
    const float cL = m == 8 ? c[7] : m == 4 ? c[3] : c[1];
    const float dL = m == 8 ? d[7] : m == 4 ? d[3] : d[1];
    pa[2 * t] = a[0]; pb[2 * t] = 1.0f; pc[2 * t] = c[0]; pd[2 * t] = d[0];
    pa[2 * t + 1] = aL; pb[2 * t + 1] = 1.0f; pc[2 * t + 1] = cL; pd[2 * t + 1] = dL;
  }
  __syncthreads();
  pcr<2>(pa, pb, pc, pd, 2 * P);   // 2P = 2N/m <= 2 kThreads
  float x[kRows];
  if (t < P) {
    const float F = __fdividef(pd[2 * t], pa[2 * t] + pb[2 * t] + pc[2 * t]);
    const float L = __fdividef(pd[2 * t + 1], pa[2 * t + 1] + pb[2 * t + 1] + pc[2 * t + 1]);
#pragma unroll
    for (int i = 0; i < kRows; ++i) x[i] = (i == 0) ? F : (i == m - 1) ? L : d[i] - a[i] * F - c[i] * L;
  }
  __syncthreads();   // the reduced solution is read: pd takes the solution
  if (t < P) st_rows(pd + j0, m, x);
  __syncthreads();
}

// correction of cell j: scaled network outputs, or fixed corrections, or none
__device__ __forceinline__ void corr_at(const FluidK &K, long long g, float &cg, float &ch, float &cn) {
  if (K.netY) {
    cg = K.netY[g * 3 + 0] * K.cs0; ch = K.netY[g * 3 + 1] * K.cs1; cn = K.netY[g * 3 + 2] * K.cs2;
  } else if (K.corr) {
    cg = K.corr[g * 3 + 0]; ch = K.corr[g * 3 + 1]; cn = K.corr[g * 3 + 2];
  } else {
    cg = ch = cn = 0.0f;
  }
}

// coefficient arrays from T: D = D_e, A = a, B = mu_e (all cells)
__device__ void coeffs(const Sm &S, const FluidK &K, const ColK &c) {
  for (int j = threadIdx.x; j < c.N; j += kThreads) {
    int i; float f;
    tpos(K, S.T[j], i, f);
    const float mu_e = tq(S, K, 0, i, f) * c.invNg;
    S.D[j] = tq(S, K, 1, i, f) * c.invNg;
    S.A[j] = __fdividef(c.mu_i, mu_e + c.mu_i);
    S.B[j] = mu_e;
  }
}

// E at faces from the density in S.n into S.E; uses D, B (= mu_e):
// E = -d_x(n D_e) / (n mu_e) + Gamma_T / (n (mu_e + mu_i)), eq. 10 with the flux of eq. 12
__device__ void field(const Sm &S, const ColK &c) {
  const int N = c.N;
  for (int j = threadIdx.x; j < N; j += kThreads) {
    const int jp = (j + 1) & (N - 1);
    const float nD0 = S.n[j] * S.D[j], nD1 = S.n[jp] * S.D[jp];
    const float nf = 0.5f * (S.n[j] + S.n[jp]);
    const float muf = 0.5f * (S.B[j] + S.B[jp]);
    const float mf = 0.5f * ((S.B[j] + c.mu_i) + (S.B[jp] + c.mu_i));
    S.E[j] = -__fdividef(nD1 - nD0, c.dx * nf * muf) + __fdividef(c.GT, nf * mf);
  }
}

__device__ float block_sum(float v, float *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float s = 0.0f;
  for (int k = 0; k < kThreads / 32; ++k) s += red[k];
  return s;
}

// One step.  Both implicit systems are solved for the increment (n' = n + dn,
// T' = T + dT) with the residual of the starting state on the right-hand side,
// formed from flux differences: FP32 then rounds relative to the per-step
// change rather than to the state, which matters where the conduction term
// dt D_eps/dx^2 is in the thousands.
__device__ void step(const Sm &S, const FluidK &K, const ColK &c, float *red) {
  const int N = c.N, t = threadIdx.x;
  const bool has_corr = K.netY || K.corr;
  // 1. coefficients at the starting T; starting n kept in u; correction fluxes on faces (starting n);
  //    ionization frequency per cell in E (free until the field is formed)
  coeffs(S, K, c);
  float sn = 0.0f, snu = 0.0f;
  for (int j = t; j < N; j += kThreads) {
    S.u[j] = S.n[j];
    int i; float f;
    tpos(K, S.T[j], i, f);
    float nu = tq(S, K, 4, i, f) * c.Ng;
    if (has_corr) {
      const int jp = (j + 1) & (N - 1);
      float g0, h0, n0, g1, h1, n1;
      corr_at(K, c.off + j, g0, h0, n0);
      corr_at(K, c.off + jp, g1, h1, n1);
      const float gf = 0.5f * (g0 + g1);   // upwind correction flux at face j+1/2 (starting n)
      S.G[j] = fmaxf(gf, 0.0f) * S.n[j] + fminf(gf, 0.0f) * S.n[jp];
      if (K.netY && K.nu_bound > 0.0f) n0 = fminf(fmaxf(n0, -K.nu_bound * nu), K.nu_bound * nu);
      nu += n0;
    }
    S.E[j] = nu;
    sn += S.n[j];
    snu += S.n[j] * nu;
  }
  float nu_w = c.nu_w;
  if (c.pair) {
    const float a = block_sum(sn, red), b = block_sum(snu, red);
    nu_w = b / a;
  }
  __syncthreads();
  // 2. continuity: A dn = rhs - A n; the correction flux max(gf, 0) n'_j + min(gf, 0) n'_{j+1},
  //    gf = (g_j + g_{j+1}) / 2, is implicit (upwind advection by gf: in A, which stays an
  //    M-matrix), its value at the starting n in the residual
  for (int j = t; j < N; j += kThreads) {
    const int jm = (j - 1) & (N - 1), jp = (j + 1) & (N - 1);
    const float af = 0.5f * (S.A[j] + S.A[jp]), am = 0.5f * (S.A[jm] + S.A[j]);
    const float nu = S.E[j];
    float dGf = 0.0f, dGm = 0.0f, up = 0.0f, um = 0.0f, dp = 0.0f, dm = 0.0f;
    if (has_corr) {
      dGf = S.G[j];
      dGm = S.G[jm];
      float gm, g0, gp, h, q;
      corr_at(K, c.off + jm, gm, h, q);
      corr_at(K, c.off + j, g0, h, q);
      corr_at(K, c.off + jp, gp, h, q);
      const float gf = 0.5f * (g0 + gp), gb = 0.5f * (gm + g0);   // faces j+1/2, j-1/2
      up = fmaxf(gf, 0.0f); dp = fminf(gf, 0.0f);
      um = fmaxf(gb, 0.0f); dm = fminf(gb, 0.0f);
    }
    const float Dn = S.D[j] * S.n[j];
    S.pa[j] = -c.r * am * S.D[jm] - c.s * um;
    S.pb[j] = 1.0f + c.r * (af + am) * S.D[j] + K.dt * nu_w + c.s * (up - dm);   // losses implicit
    S.pc[j] = -c.r * af * S.D[jp] + c.s * dp;
    // b_{j+1/2} - b_{j-1/2} = -(a_{j+1/2} - a_{j-1/2}): taken from a, which is small, to keep its digits
    S.pd[j] = c.r * (af * (S.D[jp] * S.n[jp] - Dn) - am * (Dn - S.D[jm] * S.n[jm])) -
              c.s * (af - am) * c.GT + K.dt * S.n[j] * (nu - nu_w) - c.s * (dGf - dGm);
  }
  __syncthreads();
  solve(S.pa, S.pb, S.pc, S.pd, N);
  for (int j = t; j < N; j += kThreads) add2(S.n[j], S.nl[j], S.pd[j]);
  __syncthreads();
  // 3. flux and field at faces from n' (the correction flux too); energy coefficients into
  //    pa (mu_eps), pb (D_eps)
  field(S, c);
  for (int j = t; j < N; j += kThreads) {
    const int jp = (j + 1) & (N - 1);
    const float af = 0.5f * (S.A[j] + S.A[jp]);
    const float bf = 1.0f - af;
    float g = -af * (S.n[jp] * S.D[jp] - S.n[j] * S.D[j]) * c.inv_dx - bf * c.GT;
    if (has_corr) {
      float g0, h0, n0, g1, h1, n1;
      corr_at(K, c.off + j, g0, h0, n0);
      corr_at(K, c.off + jp, g1, h1, n1);
      const float gf = 0.5f * (g0 + g1);
      g += fmaxf(gf, 0.0f) * S.n[j] + fminf(gf, 0.0f) * S.n[jp];
    }
    S.G[j] = g;
    int i; float f;
    tpos(K, S.T[j], i, f);
    S.pa[j] = tq(S, K, 2, i, f) * c.invNg;
    S.pb[j] = tq(S, K, 3, i, f) * c.invNg;
  }
  __syncthreads();
  // energy flux of the starting T with n' (the correction's too: max(wf, 0) n'_j T_j +
  // min(wf, 0) n'_{j+1} T_{j+1}, wf = (h_j / T_j + h_{j+1} / T_{j+1}) / 2) on faces, into A (free
  // once the flux and field are formed)
  for (int j = t; j < N; j += kThreads) {
    const int jp = (j + 1) & (N - 1);
    const float mep = 0.5f * (S.pa[j] + S.pa[jp]);
    float h = -0.75f * mep * S.E[j] * (S.n[j] * S.T[j] + S.n[jp] * S.T[jp]) -
              c.k * (S.n[jp] * S.pb[jp] * S.T[jp] - S.n[j] * S.pb[j] * S.T[j]);
    if (has_corr) {
      float g0, h0, n0, g1, h1, n1;
      corr_at(K, c.off + j, g0, h0, n0);
      corr_at(K, c.off + jp, g1, h1, n1);
      const float wf = 0.5f * (__fdividef(h0, S.T[j]) + __fdividef(h1, S.T[jp]));
      h += fmaxf(wf, 0.0f) * S.n[j] * S.T[j] + fminf(wf, 0.0f) * S.n[jp] * S.T[jp];
    }
    S.A[j] = h;
  }
  __syncthreads();
  // 4. energy: A dT = rhs - A T, into D, B, pc, pd (rows read the neighbours' pa, pb; D and B
  //    are free once the field is formed); the correction flux is implicit in T' as upwind
  //    advection of n' T' by wf, w = h / T (T of the step's start)
  {
    for (int j = t; j < N; j += kThreads) {
      {
        const int jm = (j - 1) & (N - 1), jp = (j + 1) & (N - 1);
        const float P = -0.5f * (S.G[j] * S.E[j] + S.G[jm] * S.E[jm]);
        int i; float f;
        tpos(K, S.T[j], i, f);
        const float L = tq(S, K, 5, i, f) * c.Ng;
        const float dL = (__ldg(K.tab + 5 * K.nT + i + 1) - __ldg(K.tab + 5 * K.nT + i)) * K.inv_dT * c.Ng;
        const float mep = 0.5f * (S.pa[j] + S.pa[jp]), mem = 0.5f * (S.pa[jm] + S.pa[j]);
        const float Ep = S.E[j], Em = S.E[jm];
        const float n1 = S.n[j];
        float up = 0.0f, um = 0.0f, dp = 0.0f, dm = 0.0f;
        if (has_corr) {
          float g, q, hm, h0, hp;
          corr_at(K, c.off + jm, g, hm, q);
          corr_at(K, c.off + j, g, h0, q);
          corr_at(K, c.off + jp, g, hp, q);
          const float w0 = __fdividef(h0, S.T[j]);
          const float wf = 0.5f * (w0 + __fdividef(hp, S.T[jp])), wb = 0.5f * (__fdividef(hm, S.T[jm]) + w0);
          up = fmaxf(wf, 0.0f); dp = fminf(wf, 0.0f);
          um = fmaxf(wb, 0.0f); dm = fminf(wb, 0.0f);
        }
        S.B[j] = 1.5f * n1 + K.dt * n1 * dL + c.s * (-0.75f * mep * Ep + 0.75f * mem * Em) * n1 +
                 2.0f * c.s * c.k * n1 * S.pb[j] + c.s * (up - dm) * n1;
        S.pc[j] = c.s * (-0.75f * mep * Ep - c.k * S.pb[jp] + dp) * S.n[jp];
        S.D[j] = c.s * (0.75f * mem * Em - c.k * S.pb[jm] - um) * S.n[jm];
        S.pd[j] = 1.5f * (S.u[j] - n1) * S.T[j] + K.dt * P - K.dt * n1 * L - c.s * (S.A[j] - S.A[jm]);
      }
    }
    __syncthreads();
  }
  solve(S.D, S.B, S.pc, S.pd, N);
  for (int j = t; j < N; j += kThreads) {
    add2(S.T[j], S.Tl[j], S.pd[j]);
    if (S.T[j] < K.T0) { S.T[j] = K.T0; S.Tl[j] = 0.0f; }
    if (S.T[j] > K.Tmax) { S.T[j] = K.Tmax; S.Tl[j] = 0.0f; }
  }
  __syncthreads();
}

// spectral record of n: mean and c_m, m = 1..M (one warp per mode, modes strided over warps)
__device__ void record(const Sm &S, const FluidK &K, const ColK &c, int snap, float *red) {
  const int N = c.N, M = K.n_modes;
  float v = 0.0f;
  for (int j = threadIdx.x; j < N; j += kThreads) v += S.n[j] + S.nl[j];
  const float mean = block_sum(v, red) / (float)N;
  float2 *out = K.modes + ((size_t)snap * K.n_cols + blockIdx.x) * (M + 1);
  if (threadIdx.x == 0) out[0] = make_float2(mean, 0.0f);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int m = 1 + w; m <= M; m += kThreads / 32) {
    float re = 0.0f, im = 0.0f, rel = 0.0f, iml = 0.0f;   // hi and lo parts summed apart
    for (int j = l; j < N; j += 32) {
      const int ph = (m * j) & (N - 1);
      float sn, cs;
      sincospif(2.0f * (float)ph / (float)N, &sn, &cs);
      re += S.n[j] * cs;
      im -= S.n[j] * sn;
      rel += S.nl[j] * cs;
      iml -= S.nl[j] * sn;
    }
    re += rel;
    im += iml;
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (l == 0) out[m] = make_float2(re / (float)N, im / (float)N);
  }
  __syncthreads();
}

// closure features of the current state into K.feat
__device__ void features(const Sm &S, const FluidK &K, const ColK &c, float *red) {
  const int N = c.N;
  coeffs(S, K, c);
  __syncthreads();
  field(S, c);
  float v = 0.0f;
  for (int j = threadIdx.x; j < N; j += kThreads) v += S.n[j];
  const float mean = block_sum(v, red) / (float)N;   // (contains the barrier after field)
  for (int j = threadIdx.x; j < N; j += kThreads) {
    float *x = K.feat + (c.off + j) * 15;
#pragma unroll
    for (int d = -2; d <= 2; ++d) {
      const int q = (j + d * K.step) & (N - 1), qm = (q - 1) & (N - 1);
      x[d + 2] = S.n[q] / mean / K.fs[d + 2];
      x[d + 7] = 1.5f * S.T[q] / K.fs[d + 7];
      x[d + 12] = 0.5f * (S.E[q] + S.E[qm]) / (c.Ng * kTd) / K.fs[d + 12];
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1) k_fluid(FluidK K, int n_steps, int feat_only) {
  extern __shared__ float4 smem4[];
  float *base = reinterpret_cast<float *>(smem4);
  __shared__ float red[kThreads / 32];
  const ColK c = K.cols[blockIdx.x];
  const int N = c.N;
  Sm S;
  S.n = base;           S.nl = base + N;      S.T = base + 2 * N;   S.Tl = base + 3 * N;
  S.u = base + 4 * N;   S.D = base + 5 * N;   S.A = base + 6 * N;   S.B = base + 7 * N;
  S.G = base + 8 * N;   S.E = base + 9 * N;   S.pa = base + 10 * N; S.pb = base + 11 * N;
  S.pc = base + 12 * N; S.pd = base + 13 * N;
  for (int j = threadIdx.x; j < N; j += kThreads) {
    const double n = K.n[c.off + j], T = K.T[c.off + j];
    S.n[j] = (float)n;
    S.nl[j] = (float)(n - (double)S.n[j]);
    S.T[j] = (float)T;
    S.Tl[j] = (float)(T - (double)S.T[j]);
  }
  __syncthreads();
  if (!feat_only) {
    const long long first = K.diag_every > 0 ? K.step0 / K.diag_every : 0;
    for (int s = 0; s < n_steps; ++s) {
      step(S, K, c, red);
      const long long g = K.step0 + s;
      if (K.diag_every > 0 && K.n_modes >= 0 && (g + 1) % K.diag_every == 0)
        record(S, K, c, K.snap_base + (int)((g + 1) / K.diag_every - 1 - first), red);
    }
    for (int j = threadIdx.x; j < N; j += kThreads) {
      K.n[c.off + j] = (double)S.n[j] + (double)S.nl[j];
      K.T[c.off + j] = (double)S.T[j] + (double)S.Tl[j];
    }
  }
  if (K.feat) features(S, K, c, red);
}

size_t smem_bytes(int N) { return (size_t)kArrays * N * sizeof(float); }

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

}  // namespace

struct pic_fluid {
  int n_cols = 0, nT = 0, maxN = 0, diag_every = 0, n_modes = 0;
  long long cells = 0, step = 0;
  double dt = 0.0, T0 = 0.0, dT = 0.0;
  std::vector<ColK> hcols;
  ColK *cols = nullptr;
  double *n = nullptr, *T = nullptr;
  float *tab = nullptr;
  float2 *modes = nullptr;
  int snap_cap = 0, snap_count = 0;
  const float *corr = nullptr;
  pic_mlp *net = nullptr;
  int period = 0;
  float fs[15], cs[3];
  float nu_bound = 0.0f;
  int stencil = 1;
  float *X = nullptr, *Y = nullptr;
  bool y_valid = false;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  long long launches = 0;
  double last_ms = 0.0;
};

namespace {

FluidK make_k(pic_fluid *f) {
  FluidK K;
  std::memset(&K, 0, sizeof(K));
  K.cols = f->cols;
  K.n = f->n;
  K.T = f->T;
  K.tab = f->tab;
  K.nT = f->nT;
  K.T0 = (float)f->T0;
  K.inv_dT = (float)(1.0 / f->dT);
  K.Tmax = (float)(f->T0 + (f->nT - 1) * f->dT);
  K.dt = (float)f->dt;
  K.diag_every = f->diag_every;
  K.n_modes = f->n_modes;
  K.step0 = f->step;
  K.snap_base = f->snap_count;
  K.modes = f->modes;
  K.n_cols = f->n_cols;
  K.corr = f->corr;
  for (int k = 0; k < 15; ++k) K.fs[k] = f->fs[k];
  K.step = f->stencil;
  K.cs0 = f->cs[0]; K.cs1 = f->cs[1]; K.cs2 = f->cs[2];
  K.nu_bound = f->nu_bound;
  return K;
}

int launch(pic_fluid *f, FluidK K, int n_steps, int feat_only) {
  const size_t sm = smem_bytes(f->maxN);
  if (cudaFuncSetAttribute(k_fluid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return PIC_ECUDA;
  k_fluid<<<f->n_cols, kThreads, sm, f->st>>>(K, n_steps, feat_only);
  f->launches++;
  return cudaGetLastError() == cudaSuccess ? 0 : PIC_ECUDA;
}

// snapshot records produced by steps [step, step + n)
int n_records(const pic_fluid *f, long long n) {
  if (f->diag_every <= 0) return 0;
  return (int)((f->step + n) / f->diag_every - f->step / f->diag_every);
}

int ensure_snaps(pic_fluid *f, int need) {
  if (need <= f->snap_cap) return 0;
  int cap = std::max(need, 2 * f->snap_cap);
  float2 *m = nullptr;
  const size_t per = (size_t)f->n_cols * (f->n_modes + 1) * sizeof(float2);
  if (cudaMalloc(&m, per * cap) != cudaSuccess) return PIC_ENOMEM;
  if (f->snap_count && cudaMemcpyAsync(m, f->modes, per * f->snap_count, cudaMemcpyDeviceToDevice, f->st) != cudaSuccess)
    return PIC_ECUDA;
  cudaStreamSynchronize(f->st);
  cudaFree(f->modes);
  f->modes = m;
  f->snap_cap = cap;
  return 0;
}

int run(pic_fluid *f, long long n_steps) {
  long long done = 0;
  while (done < n_steps) {
    long long chunk = std::min<long long>(n_steps - done, f->net ? f->period : kChunk);
    int rc = ensure_snaps(f, f->snap_count + n_records(f, chunk));
    if (rc) return rc;
    FluidK K = make_k(f);
    if (f->net) {
      if (!f->y_valid) {   // features of the starting state -> network
        FluidK Kf = K;
        Kf.feat = f->X;
        if ((rc = launch(f, Kf, 0, 1))) return rc;
        if ((rc = mlp_forward_async(f->net, f->X, (int)f->cells, f->Y, f->st))) return rc;
        f->launches++;
      }
      K.netY = f->Y;
      K.corr = nullptr;
      K.feat = f->X;      // features of the state at the end of the chunk
    }
    if ((rc = launch(f, K, (int)chunk, 0))) return rc;
    if (f->net) {
      if ((rc = mlp_forward_async(f->net, f->X, (int)f->cells, f->Y, f->st))) return rc;
      f->launches++;
      f->y_valid = true;
    }
    f->snap_count += n_records(f, chunk);
    f->step += chunk;
    done += chunk;
  }
  return 0;
}

}  // namespace

extern "C" {

int pic_fluid_init(const pic_fluid_column *cols, int n_cols, const pic_transport *tr, int n_tr, int n_T,
                   double dt_s, int diag_every, int n_modes, pic_fluid **out) {
  if (!cols || n_cols <= 0 || !tr || n_tr < 2 || n_T < 2 || n_T > kMaxT || !(dt_s > 0.0) || diag_every < 0 ||
      n_modes < 0 || n_modes > kMaxModes || !out)
    return PIC_EINVAL;
  *out = nullptr;
  // resample the transport records onto a uniform Te grid
  std::vector<double> Te(n_tr);
  for (int k = 0; k < n_tr; ++k) {
    Te[k] = 2.0 / 3.0 * tr[k].mean_eps_eV;
    if (!std::isfinite(Te[k]) || (k && !(Te[k] > Te[k - 1]))) return PIC_EINVAL;
  }
  pic_fluid *f = new (std::nothrow) pic_fluid;
  if (!f) return PIC_ENOMEM;
  f->n_cols = n_cols;
  f->nT = n_T;
  f->dt = dt_s;
  f->diag_every = diag_every;
  f->n_modes = n_modes;
  f->T0 = Te[0];
  f->dT = (Te[n_tr - 1] - Te[0]) / (n_T - 1);
  std::vector<float> tab((size_t)kNQ * n_T);
  for (int q = 0; q < n_T; ++q) {
    const double x = (q == n_T - 1) ? Te[n_tr - 1] : Te[0] + q * f->dT;
    int k = 0;
    while (k + 2 < n_tr && Te[k + 1] <= x) ++k;
    const double w = std::min(1.0, std::max(0.0, (x - Te[k]) / (Te[k + 1] - Te[k])));
    const double *a = &tr[k].muN, *b = &tr[k + 1].muN;   // muN, DN, mueN, DeN, nu_izN, lossN are adjacent
    for (int p = 0; p < kNQ; ++p) tab[(size_t)p * n_T + q] = (float)(a[p] + w * (b[p] - a[p]));
  }
  f->hcols.resize(n_cols);
  long long off = 0;
  for (int c = 0; c < n_cols; ++c) {
    const pic_fluid_column &p = cols[c];
    if (!pow2(p.n_cells) || p.n_cells < 64 || p.n_cells > kMaxCells || !(p.L_m > 0.0) || !(p.N_gas_m3 > 0.0) ||
        !(p.mu_iN > 0.0) || !std::isfinite(p.Gamma_T) || !std::isfinite(p.nu_w) ||
        (p.loss != PIC_FLUID_LOSS_FIXED && p.loss != PIC_FLUID_LOSS_PAIR)) {
      delete f;
      return PIC_EINVAL;
    }
    ColK &k = f->hcols[c];
    k.N = p.n_cells;
    k.logN = 0;
    while ((1 << k.logN) < k.N) ++k.logN;
    k.off = off;
    const double dx = p.L_m / p.n_cells;
    k.dx = (float)dx;
    k.inv_dx = (float)(1.0 / dx);
    k.r = (float)(dt_s / (dx * dx));
    k.s = (float)(dt_s / dx);
    k.k = (float)(1.5 / dx);
    k.GT = (float)p.Gamma_T;
    k.nu_w = (float)p.nu_w;
    k.mu_i = (float)(p.mu_iN / p.N_gas_m3);
    k.Ng = (float)p.N_gas_m3;
    k.invNg = (float)(1.0 / p.N_gas_m3);
    k.pair = p.loss == PIC_FLUID_LOSS_PAIR;
    off += p.n_cells;
    f->maxN = std::max(f->maxN, p.n_cells);
  }
  f->cells = off;
  for (int k = 0; k < 15; ++k) f->fs[k] = 1.0f;
  for (int k = 0; k < 3; ++k) f->cs[k] = 1.0f;
  bool ok = cudaStreamCreateWithFlags(&f->st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&f->e0) == cudaSuccess && cudaEventCreate(&f->e1) == cudaSuccess &&
            cudaMalloc(&f->cols, sizeof(ColK) * n_cols) == cudaSuccess &&
            cudaMalloc(&f->n, sizeof(double) * off) == cudaSuccess &&
            cudaMalloc(&f->T, sizeof(double) * off) == cudaSuccess &&
            cudaMalloc(&f->tab, sizeof(float) * tab.size()) == cudaSuccess;
  if (ok)
    ok = cudaMemcpy(f->cols, f->hcols.data(), sizeof(ColK) * n_cols, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(f->tab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(f->n, 0, sizeof(double) * off) == cudaSuccess &&
         cudaMemset(f->T, 0, sizeof(double) * off) == cudaSuccess;
  if (!ok) {
    pic_fluid_free(f);
    return PIC_ENOMEM;
  }
  *out = f;
  return 0;
}

int pic_fluid_set_state(pic_fluid *f, int col, const double *n_m3, const double *Te_eV) {
  if (!f || col < 0 || col >= f->n_cols || !n_m3 || !Te_eV) return PIC_EINVAL;
  const ColK &c = f->hcols[col];
  for (int j = 0; j < c.N; ++j)
    if (!(n_m3[j] > 0.0) || !std::isfinite(n_m3[j]) || !std::isfinite(Te_eV[j])) return PIC_EINVAL;
  if (cudaMemcpyAsync(f->n + c.off, n_m3, 8 * c.N, cudaMemcpyHostToDevice, f->st) != cudaSuccess ||
      cudaMemcpyAsync(f->T + c.off, Te_eV, 8 * c.N, cudaMemcpyHostToDevice, f->st) != cudaSuccess ||
      cudaStreamSynchronize(f->st) != cudaSuccess)
    return PIC_ECUDA;
  f->y_valid = false;
  return 0;
}

int pic_fluid_get_state(pic_fluid *f, int col, double *n_m3, double *Te_eV) {
  if (!f || col < 0 || col >= f->n_cols || !n_m3 || !Te_eV) return PIC_EINVAL;
  const ColK &c = f->hcols[col];
  if (cudaMemcpyAsync(n_m3, f->n + c.off, 8 * c.N, cudaMemcpyDeviceToHost, f->st) != cudaSuccess ||
      cudaMemcpyAsync(Te_eV, f->T + c.off, 8 * c.N, cudaMemcpyDeviceToHost, f->st) != cudaSuccess ||
      cudaStreamSynchronize(f->st) != cudaSuccess)
    return PIC_ECUDA;
  return 0;
}

int pic_fluid_step(pic_fluid *f, int64_t n_steps) {
  if (!f || n_steps < 0) return PIC_EINVAL;
  f->launches = 0;
  if (cudaEventRecord(f->e0, f->st) != cudaSuccess) return PIC_ECUDA;
  const int rc = run(f, n_steps);
  if (rc) return rc;
  if (cudaEventRecord(f->e1, f->st) != cudaSuccess || cudaStreamSynchronize(f->st) != cudaSuccess) return PIC_ECUDA;
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, f->e0, f->e1);
  f->last_ms = ms;
  return f->net ? mlp_take_status(f->net) : 0;
}

int pic_fluid_modes(pic_fluid *f, float *out, int max_snaps, int *n_snaps) {
  if (!f || !n_snaps || max_snaps < 0 || (max_snaps > 0 && !out)) return PIC_EINVAL;
  const int n = std::min(max_snaps, f->snap_count);
  const size_t per = (size_t)f->n_cols * (f->n_modes + 1) * sizeof(float2);
  if (n && (cudaMemcpyAsync(out, f->modes, per * n, cudaMemcpyDeviceToHost, f->st) != cudaSuccess ||
            cudaStreamSynchronize(f->st) != cudaSuccess))
    return PIC_ECUDA;
  *n_snaps = n;
  const int lost = f->snap_count - n;
  f->snap_count = 0;
  return lost > 0 ? PIC_ECAPACITY : 0;
}

int pic_fluid_set_closure(pic_fluid *f, pic_mlp *net, int period, const float *feat_scale, const float *targ_scale,
                          float nu_bound, int stencil) {
  if (!f) return PIC_EINVAL;
  if (!net) {
    f->net = nullptr;
    f->y_valid = false;
    f->stencil = 1;
    return 0;
  }
  if (period <= 0 || !feat_scale || !targ_scale || stencil < 1) return PIC_EINVAL;
  for (const ColK &c : f->hcols)
    if (4 * stencil > c.N) return PIC_EINVAL;
  for (int k = 0; k < 15; ++k)
    if (!(feat_scale[k] != 0.0f)) return PIC_EINVAL;
  if (!f->X && (cudaMalloc(&f->X, sizeof(float) * 15 * f->cells) != cudaSuccess ||
                cudaMalloc(&f->Y, sizeof(float) * 3 * f->cells) != cudaSuccess))
    return PIC_ENOMEM;
  std::memcpy(f->fs, feat_scale, sizeof(f->fs));
  std::memcpy(f->cs, targ_scale, sizeof(f->cs));
  f->net = net;
  f->period = period;
  f->nu_bound = nu_bound;
  f->stencil = stencil;
  f->y_valid = false;
  return 0;
}

int pic_fluid_set_corrections(pic_fluid *f, const float *corr_dev) {
  if (!f) return PIC_EINVAL;
  f->corr = corr_dev;
  return 0;
}

int pic_fluid_features(pic_fluid *f, float *X_dev) {
  if (!f || !X_dev) return PIC_EINVAL;
  FluidK K = make_k(f);
  if (!f->net)
    for (int k = 0; k < 15; ++k) K.fs[k] = 1.0f;
  K.feat = X_dev;
  const int rc = launch(f, K, 0, 1);
  if (rc) return rc;
  return cudaStreamSynchronize(f->st) == cudaSuccess ? 0 : PIC_ECUDA;
}

int pic_fluid_elapsed(pic_fluid *f, double *ms, int64_t *launches) {
  if (!f) return PIC_EINVAL;
  if (ms) *ms = f->last_ms;
  if (launches) *launches = f->launches;
  return 0;
}

void *pic_fluid_stream(pic_fluid *f) { return f ? reinterpret_cast<void *>(f->st) : nullptr; }

void pic_fluid_free(pic_fluid *f) {
  if (!f) return;
  if (f->st) cudaStreamSynchronize(f->st);
  cudaFree(f->cols);
  cudaFree(f->n);
  cudaFree(f->T);
  cudaFree(f->tab);
  cudaFree(f->modes);
  cudaFree(f->X);
  cudaFree(f->Y);
  if (f->e0) cudaEventDestroy(f->e0);
  if (f->e1) cudaEventDestroy(f->e1);
  if (f->st) cudaStreamDestroy(f->st);
  delete f;
}

}  // extern "C"
