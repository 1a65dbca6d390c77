// Periodic counting sort of the particles by cell (stable), as an LSD radix
// sort on 7-bit digits of the cell index: two passes for up to 16384 cells.
// Each pass: per-tile digit histograms, a scan of the (digit, tile) counts,
// and a stable scatter in which every warp ranks its own contiguous run of
// particles.  Equal cells keep their slot order, so the result is the unique
// stable order that the CPU oracle's counting sort produces.
#include <cstdint>

#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr int kBits = 7;
constexpr int kBins = 1 << kBits;
constexpr int kWarps = 8;                         // warps per CTA
constexpr int kIters = 16;                        // 32-particle rows per warp and tile
constexpr int kTile = kWarps * kIters * 32;       // 4096 particles per tile
constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kInvalid = 0x7fffffff;

__device__ __forceinline__ int digit_of(int32_t cell, int shift) { return (cell >> shift) & (kBins - 1); }

// digit counts of every tile, stored digit-major: hist[d * ntiles + tile]
__global__ void __launch_bounds__(kWarps * 32)
k_sort_hist(const int32_t *__restrict__ cell, const long long *n_dev, int shift, unsigned *hist, int ntiles) {
  __shared__ unsigned h[kBins];
  const long long n = *n_dev;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    for (int d = threadIdx.x; d < kBins; d += blockDim.x) h[d] = 0u;
    __syncthreads();
    const long long start = (long long)tile * kTile + (long long)w * kIters * 32;
    for (int it = 0; it < kIters; ++it) {
      const long long p = start + it * 32 + lane;
      const int d = p < n ? digit_of(cell[p], shift) : kInvalid;
      const unsigned grp = __match_any_sync(kFullMask, d);
      if (d != kInvalid && lane == __ffs(grp) - 1) atomicAdd(&h[d], (unsigned)__popc(grp));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += blockDim.x) hist[(size_t)d * ntiles + tile] = h[d];
    __syncthreads();
  }
}

// one warp per digit: exclusive scan of its tile counts, digit totals
__global__ void k_sort_scan(unsigned *hist, int ntiles, unsigned *tot) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= kBins) return;
  unsigned *row = hist + (size_t)warp * ntiles;
  unsigned carry = 0;
  for (int base = 0; base < ntiles; base += 32) {
    const int t = base + lane;
    const unsigned v = t < ntiles ? row[t] : 0u;
    unsigned incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned x = __shfl_up_sync(kFullMask, incl, o);
      if (lane >= o) incl += x;
    }
    if (t < ntiles) row[t] = carry + incl - v;
    carry += __shfl_sync(kFullMask, incl, 31);
  }
  if (lane == 0) tot[warp] = carry;
}

template <class T>
__global__ void __launch_bounds__(kWarps * 32)
k_sort_scatter(const int32_t *__restrict__ cell, const T *__restrict__ rec, const uint64_t *__restrict__ id,
               int32_t *__restrict__ cell_o, T *__restrict__ rec_o, uint64_t *__restrict__ id_o,
               const long long *n_dev, int shift, const unsigned *__restrict__ hist, const unsigned *__restrict__ tot,
               int ntiles) {
  __shared__ unsigned dbase[kBins];
  const long long n = *n_dev;
  __shared__ unsigned woff[kWarps][kBins];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x < 32) {
    // exclusive scan of the 128 digit totals by one warp (4 per lane)
    unsigned v[4], s = 0;
    for (int k = 0; k < 4; ++k) { v[k] = tot[lane * 4 + k]; s += v[k]; }
    unsigned incl = s;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned x = __shfl_up_sync(kFullMask, incl, o);
      if (lane >= o) incl += x;
    }
    unsigned run = incl - s;
    for (int k = 0; k < 4; ++k) { dbase[lane * 4 + k] = run; run += v[k]; }
  }
  const unsigned lt = (1u << lane) - 1u;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    for (int d = lane; d < kBins; d += 32) woff[w][d] = 0u;
    __syncthreads();
    const long long start = (long long)tile * kTile + (long long)w * kIters * 32;
    for (int it = 0; it < kIters; ++it) {
      const long long p = start + it * 32 + lane;
      const int d = p < n ? digit_of(cell[p], shift) : kInvalid;
      const unsigned grp = __match_any_sync(kFullMask, d);
      if (d != kInvalid && lane == __ffs(grp) - 1) woff[w][d] += (unsigned)__popc(grp);
      __syncwarp();
    }
    __syncthreads();
    // running offsets: digit base + tile offset + counts of the earlier warps of this tile
    for (int d = threadIdx.x; d < kBins; d += blockDim.x) {
      unsigned run = dbase[d] + hist[(size_t)d * ntiles + tile];
      for (int ww = 0; ww < kWarps; ++ww) {
        const unsigned c = woff[ww][d];
        woff[ww][d] = run;
        run += c;
      }
    }
    __syncthreads();
    for (int it = 0; it < kIters; ++it) {
      const long long p = start + it * 32 + lane;
      const bool valid = p < n;
      const int32_t c = valid ? cell[p] : 0;
      const int d = valid ? digit_of(c, shift) : kInvalid;
      const unsigned grp = __match_any_sync(kFullMask, d);
      unsigned pos = 0;
      if (valid) pos = woff[w][d] + (unsigned)__popc(grp & lt);
      __syncwarp();
      if (valid && lane == __ffs(grp) - 1) woff[w][d] += (unsigned)__popc(grp);
      __syncwarp();
      if (valid) {
        cell_o[pos] = c;
        rec_o[pos] = rec[p];
        id_o[pos] = id[p];
      }
    }
    __syncthreads();
  }
}

template <class T>
__global__ void k_sort_copy(const int32_t *cell, const T *rec, const uint64_t *id, int32_t *cell_o, T *rec_o,
                            uint64_t *id_o, const long long *n_dev) {
  const long long n = *n_dev;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    cell_o[p] = cell[p];
    rec_o[p] = rec[p];
    id_o[p] = id[p];
  }
}

}  // namespace

int sort_passes(int n_cells) {
  int bits = 0;
  while ((1 << bits) < n_cells) ++bits;
  if (bits == 0) bits = 1;
  return (bits + kBits - 1) / kBits;
}

size_t sort_hist_words(int64_t cap) { return (size_t)kBins * (size_t)((cap + kTile - 1) / kTile) + kBins; }

// Sort the first *n_dev particles of s by cell; alt holds buffers of capacity cap.
template <class R>
void launch_sort(SpeciesDev s, SortBuf alt, const long long *n_dev, long long cap, int n_cells, int nsm,
                 cudaStream_t st) {
  using T = typename Rec<R>::T;
  const int ntiles = (int)((cap + kTile - 1) / kTile);
  const int grid = ntiles < nsm * 8 ? ntiles : nsm * 8;
  unsigned *hist = alt.hist, *tot = alt.hist + (size_t)kBins * ntiles;
  const int passes = sort_passes(n_cells);
  int32_t *ca = s.cell, *cb = alt.cell;
  T *ra = reinterpret_cast<T *>(s.rec), *rb = reinterpret_cast<T *>(alt.rec);
  uint64_t *ia = s.id, *ib = alt.id;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * kBits;
    k_sort_hist<<<grid, kWarps * 32, 0, st>>>(ca, n_dev, shift, hist, ntiles);
    k_sort_scan<<<(kBins * 32 + 255) / 256, 256, 0, st>>>(hist, ntiles, tot);
    k_sort_scatter<T><<<grid, kWarps * 32, 0, st>>>(ca, ra, ia, cb, rb, ib, n_dev, shift, hist, tot, ntiles);
    int32_t *tc = ca; ca = cb; cb = tc;
    T *tr = ra; ra = rb; rb = tr;
    uint64_t *ti = ia; ia = ib; ib = ti;
  }
  if (passes & 1) k_sort_copy<T><<<nsm * 8, 256, 0, st>>>(ca, ra, ia, s.cell, reinterpret_cast<T *>(s.rec), s.id, n_dev);
}

template void launch_sort<double>(SpeciesDev, SortBuf, const long long *, long long, int, int, cudaStream_t);
template void launch_sort<float>(SpeciesDev, SortBuf, const long long *, long long, int, int, cudaStream_t);

}  // namespace pic
