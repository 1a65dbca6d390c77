// Periodic counting sort of the particles by cell (stable), as an LSD radix
// sort on 7-bit digits of the cell index: two passes for up to 16384 cells.
// Each pass: per-tile digit histograms, a scan of the (digit, tile) counts,
// and a stable scatter.  The scatter reorders each tile in shared memory
// (every warp ranks its own contiguous run of particles) and then writes the
// tile's digit runs out in order, so that consecutive threads store to
// consecutive addresses.  Equal cells keep their slot order, so the result is
// the unique stable order that the CPU oracle's counting sort produces.
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
    int dg[kIters];   // every load of the warp's run issued before the first count
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
      const long long p = start + it * 32 + lane;
      dg[it] = p < n ? digit_of(cell[p], shift) : kInvalid;
    }
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
      const int d = dg[it];
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

// ---- the stable scatter of one tile through shared memory
constexpr int kSWarps = 16;                        // scatter: warps per CTA
constexpr int kSThreads = kSWarps * 32;
constexpr int kSRows = kTile / kSThreads;          // 32-particle rows ranked by each warp
constexpr int kSSlots = kTile / kSThreads;         // output slots per thread

struct ScatterSmem {
  uint4 buf[kTile];                  // one 16-byte word of every record, or the ids
  int32_t cell[kTile];               // the tile's cells in slot order
  uint16_t src[kTile];               // sorted position i -> tile-local index of its particle
  unsigned woff[kSWarps][kBins];     // per-warp digit counts, then running positions
  unsigned lstart[kBins];            // first sorted position of each digit within the tile
  unsigned gstart[kBins];            // global position of the tile's first particle of each digit
  unsigned dbase[kBins];             // first global position of each digit
};
constexpr size_t kScatterSmem = sizeof(ScatterSmem);

// exclusive scan of 128 counts by one warp (4 per lane); out may alias in
__device__ __forceinline__ void warp_scan_bins(const unsigned *in, unsigned *out, int lane) {
  unsigned v[4], s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) { v[k] = in[lane * 4 + k]; s += v[k]; }
  unsigned incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned x = __shfl_up_sync(kFullMask, incl, o);
    if (lane >= o) incl += x;
  }
  unsigned run = incl - s;
#pragma unroll
  for (int k = 0; k < 4; ++k) { out[lane * 4 + k] = run; run += v[k]; }
}

// Tile `tile` (particles [tile kTile, tile kTile + m)) of one column: rank each particle
// stably by its digit within the tile, then write the tile out digit run by digit run.
// tot: the column's digit totals; hist: its (digit, tile) exclusive offsets.
template <class T>
__device__ __forceinline__ void scatter_tile(ScatterSmem &s, const int32_t *__restrict__ cell,
                                             const T *__restrict__ rec, const uint64_t *__restrict__ id,
                                             int32_t *__restrict__ cell_o, T *__restrict__ rec_o,
                                             uint64_t *__restrict__ id_o, long long n, int tile, int shift,
                                             const unsigned *__restrict__ hist, const unsigned *__restrict__ tot,
                                             int ntiles) {
  constexpr int W = (int)(sizeof(T) / sizeof(uint4));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long t0 = (long long)tile * kTile;
  const int m = (int)min((long long)kTile, n - t0);
  if (m <= 0) return;                                  // uniform over the CTA
  // 1. the tile's cells (each warp a contiguous run) and the first record word, staged
  int32_t c[kSRows];
#pragma unroll
  for (int r = 0; r < kSRows; ++r) {
    const int i = (w * kSRows + r) * 32 + lane;
    c[r] = i < m ? cell[t0 + i] : 0;
  }
  const uint4 *rw = reinterpret_cast<const uint4 *>(rec + t0);
#pragma unroll
  for (int k = 0; k < kSSlots; ++k) {
    const int i = k * kSThreads + threadIdx.x;
    if (i < m) s.buf[i] = rw[(size_t)i * W];
  }
  for (int d = lane; d < kBins; d += 32) s.woff[w][d] = 0u;
  if (w == 0) warp_scan_bins(tot, s.dbase, lane);
  __syncwarp();
#pragma unroll
  for (int r = 0; r < kSRows; ++r) {
    const int i = (w * kSRows + r) * 32 + lane;
    const bool valid = i < m;
    if (valid) s.cell[i] = c[r];
    const int d = valid ? digit_of(c[r], shift) : kInvalid;
    const unsigned grp = __match_any_sync(kFullMask, d);
    if (valid && lane == __ffs(grp) - 1) s.woff[w][d] += (unsigned)__popc(grp);
    __syncwarp();
  }
  __syncthreads();
  // 2. the tile's digit counts, their exclusive scan, each warp's first position per digit
  if (threadIdx.x < kBins) {
    unsigned k = 0;
    for (int ww = 0; ww < kSWarps; ++ww) k += s.woff[ww][threadIdx.x];
    s.lstart[threadIdx.x] = k;
  }
  __syncthreads();
  if (w == 0) warp_scan_bins(s.lstart, s.lstart, lane);
  __syncthreads();
  if (threadIdx.x < kBins) {
    const int d = threadIdx.x;
    unsigned run = s.lstart[d];
    for (int ww = 0; ww < kSWarps; ++ww) {
      const unsigned k = s.woff[ww][d];
      s.woff[ww][d] = run;
      run += k;
    }
    s.gstart[d] = s.dbase[d] + hist[(size_t)d * ntiles + tile];
  }
  __syncthreads();
  // 3. stable ranks: equal digits keep their order within the warp's run, runs in warp order
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kSRows; ++r) {
    const int i = (w * kSRows + r) * 32 + lane;
    const bool valid = i < m;
    const int d = valid ? digit_of(c[r], shift) : kInvalid;
    const unsigned grp = __match_any_sync(kFullMask, d);
    if (valid) s.src[s.woff[w][d] + (unsigned)__popc(grp & lt)] = (uint16_t)i;
    __syncwarp();
    if (valid && lane == __ffs(grp) - 1) s.woff[w][d] += (unsigned)__popc(grp);
    __syncwarp();
  }
  __syncthreads();
  // 4. sorted position i of this thread: its particle and global destination; cells out
  int sidx[kSSlots];
  unsigned g[kSSlots];
#pragma unroll
  for (int k = 0; k < kSSlots; ++k) {
    const int i = k * kSThreads + threadIdx.x;
    sidx[k] = 0;
    g[k] = 0u;
    if (i < m) {
      const int src = s.src[i];
      const int32_t cv = s.cell[src];
      const int d = digit_of(cv, shift);
      sidx[k] = src;
      g[k] = s.gstart[d] + (unsigned)(i - (int)s.lstart[d]);
      cell_o[g[k]] = cv;
    }
  }
  // 5. records, one 16-byte word at a time (word 0 was staged in step 1)
  uint4 *ro = reinterpret_cast<uint4 *>(rec_o);
#pragma unroll
  for (int q = 0; q < W; ++q) {
    if (q > 0) {
#pragma unroll
      for (int k = 0; k < kSSlots; ++k) {
        const int i = k * kSThreads + threadIdx.x;
        if (i < m) s.buf[i] = rw[(size_t)i * W + q];
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kSSlots; ++k) {
      const int i = k * kSThreads + threadIdx.x;
      if (i < m) ro[(size_t)g[k] * W + q] = s.buf[sidx[k]];
    }
    __syncthreads();
  }
  // 6. ids
  uint64_t *sid = reinterpret_cast<uint64_t *>(s.buf);
#pragma unroll
  for (int k = 0; k < kSSlots; ++k) {
    const int i = k * kSThreads + threadIdx.x;
    if (i < m) sid[i] = id[t0 + i];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kSSlots; ++k) {
    const int i = k * kSThreads + threadIdx.x;
    if (i < m) id_o[g[k]] = sid[sidx[k]];
  }
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(kSThreads, 2)
k_sort_scatter(const int32_t *__restrict__ cell, const T *__restrict__ rec, const uint64_t *__restrict__ id,
               int32_t *__restrict__ cell_o, T *__restrict__ rec_o, uint64_t *__restrict__ id_o,
               const long long *n_dev, int shift, const unsigned *__restrict__ hist, const unsigned *__restrict__ tot,
               int ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem &s = *reinterpret_cast<ScatterSmem *>(smem_raw);
  const long long n = *n_dev;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    scatter_tile<T>(s, cell, rec, id, cell_o, rec_o, id_o, n, tile, shift, hist, tot, ntiles);
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

// ---- batches: one launch per phase for all columns of a batch (each global tile of
// kTile particles belongs to one column; a column's tiles are [tile0, tile0 + ntiles))

// the column of global tile t (columns in increasing tile0)
__device__ __forceinline__ int col_of(const SortCol *c, int ncols, int t) {
  int lo = 0, hi = ncols - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (c[mid].tile0 <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kWarps * 32)
k_sort_hist_b(const SortCol *__restrict__ cols, int ncols, int total, int shift, int src) {
  __shared__ unsigned h[kBins];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int gt = blockIdx.x; gt < total; gt += gridDim.x) {
    const SortCol &c = cols[col_of(cols, ncols, gt)];
    const int tile = gt - c.tile0;
    const long long n = *c.n;
    const int32_t *cell = c.cell[src];
    for (int d = threadIdx.x; d < kBins; d += blockDim.x) h[d] = 0u;
    __syncthreads();
    const long long start = (long long)tile * kTile + (long long)w * kIters * 32;
    int dg[kIters];
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
      const long long p = start + it * 32 + lane;
      dg[it] = p < n ? digit_of(cell[p], shift) : kInvalid;
    }
#pragma unroll
    for (int it = 0; it < kIters; ++it) {
      const int d = dg[it];
      const unsigned grp = __match_any_sync(kFullMask, d);
      if (d != kInvalid && lane == __ffs(grp) - 1) atomicAdd(&h[d], (unsigned)__popc(grp));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += blockDim.x) c.hist[(size_t)d * c.ntiles + tile] = h[d];
    __syncthreads();
  }
}

// one warp per (column, digit): exclusive scan of the column's tile counts, digit totals
__global__ void k_sort_scan_b(const SortCol *__restrict__ cols, int ncols) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= ncols * kBins) return;
  const SortCol &c = cols[warp / kBins];
  const int digit = warp % kBins;
  unsigned *row = c.hist + (size_t)digit * c.ntiles;
  unsigned carry = 0;
  for (int base = 0; base < c.ntiles; base += 32) {
    const int t = base + lane;
    const unsigned v = t < c.ntiles ? row[t] : 0u;
    unsigned incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned x = __shfl_up_sync(kFullMask, incl, o);
      if (lane >= o) incl += x;
    }
    if (t < c.ntiles) row[t] = carry + incl - v;
    carry += __shfl_sync(kFullMask, incl, 31);
  }
  if (lane == 0) c.hist[(size_t)kBins * c.ntiles + digit] = carry;
}

template <class T>
__global__ void __launch_bounds__(kSThreads, 2)
k_sort_scatter_b(const SortCol *__restrict__ cols, int ncols, int total, int shift, int src) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem &s = *reinterpret_cast<ScatterSmem *>(smem_raw);
  for (int gt = blockIdx.x; gt < total; gt += gridDim.x) {
    const SortCol &c = cols[col_of(cols, ncols, gt)];
    const int ntiles = c.ntiles;
    scatter_tile<T>(s, c.cell[src], reinterpret_cast<const T *>(c.rec[src]), c.id[src], c.cell[src ^ 1],
                    reinterpret_cast<T *>(c.rec[src ^ 1]), c.id[src ^ 1], *c.n, gt - c.tile0, shift, c.hist,
                    c.hist + (size_t)kBins * ntiles, ntiles);
  }
}

// after an odd number of passes: buffers 1 back into buffers 0, every column
template <class T>
__global__ void k_sort_copy_b(const SortCol *__restrict__ cols, int ncols, int total) {
  for (int gt = blockIdx.x; gt < total; gt += gridDim.x) {
    const SortCol &c = cols[col_of(cols, ncols, gt)];
    const long long n = *c.n, p0 = (long long)(gt - c.tile0) * kTile;
    const T *rec = reinterpret_cast<const T *>(c.rec[1]);
    T *rec_o = reinterpret_cast<T *>(c.rec[0]);
    for (long long p = p0 + threadIdx.x; p < n && p < p0 + kTile; p += blockDim.x) {
      c.cell[0][p] = c.cell[1][p];
      rec_o[p] = rec[p];
      c.id[0][p] = c.id[1][p];
    }
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
  const int sgrid = ntiles < nsm * 2 ? ntiles : nsm * 2;     // two scatter CTAs fit an SM's shared memory
  cudaFuncSetAttribute(k_sort_scatter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem);
  unsigned *hist = alt.hist, *tot = alt.hist + (size_t)kBins * ntiles;
  const int passes = sort_passes(n_cells);
  int32_t *ca = s.cell, *cb = alt.cell;
  T *ra = reinterpret_cast<T *>(s.rec), *rb = reinterpret_cast<T *>(alt.rec);
  uint64_t *ia = s.id, *ib = alt.id;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * kBits;
    k_sort_hist<<<grid, kWarps * 32, 0, st>>>(ca, n_dev, shift, hist, ntiles);
    k_sort_scan<<<(kBins * 32 + 255) / 256, 256, 0, st>>>(hist, ntiles, tot);
    k_sort_scatter<T><<<sgrid, kSThreads, kScatterSmem, st>>>(ca, ra, ia, cb, rb, ib, n_dev, shift, hist, tot,
                                                               ntiles);
    int32_t *tc = ca; ca = cb; cb = tc;
    T *tr = ra; ra = rb; rb = tr;
    uint64_t *ti = ia; ia = ib; ib = ti;
  }
  if (passes & 1) k_sort_copy<T><<<nsm * 8, 256, 0, st>>>(ca, ra, ia, s.cell, reinterpret_cast<T *>(s.rec), s.id, n_dev);
}

int sort_tiles(int64_t cap) { return (int)((cap + kTile - 1) / kTile); }

// Sort every column of a batch (one species) by cell: one launch per phase for all columns.
// cols: device array of ncols columns in increasing tile0, tile0 = sum of the earlier columns'
// ntiles (= sort_tiles(cap)); passes = sort_passes of the largest column (a pass on bits above a
// column's cells keeps its order).  Same result, particle for particle, as launch_sort per column.
template <class R>
void launch_sort_batch(const SortCol *cols, int ncols, int total_tiles, int passes, int nsm, cudaStream_t st) {
  using T = typename Rec<R>::T;
  const int grid = total_tiles < nsm * 8 ? total_tiles : nsm * 8;
  const int sgrid = total_tiles < nsm * 2 ? total_tiles : nsm * 2;
  cudaFuncSetAttribute(k_sort_scatter_b<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem);
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * kBits, src = pass & 1;
    k_sort_hist_b<<<grid, kWarps * 32, 0, st>>>(cols, ncols, total_tiles, shift, src);
    k_sort_scan_b<<<(ncols * kBins * 32 + 255) / 256, 256, 0, st>>>(cols, ncols);
    k_sort_scatter_b<T><<<sgrid, kSThreads, kScatterSmem, st>>>(cols, ncols, total_tiles, shift, src);
  }
  if (passes & 1) k_sort_copy_b<T><<<grid, 256, 0, st>>>(cols, ncols, total_tiles);
}

template void launch_sort<double>(SpeciesDev, SortBuf, const long long *, long long, int, int, cudaStream_t);
template void launch_sort<float>(SpeciesDev, SortBuf, const long long *, long long, int, int, cudaStream_t);
template void launch_sort_batch<double>(const SortCol *, int, int, int, int, cudaStream_t);
template void launch_sort_batch<float>(const SortCol *, int, int, int, int, cudaStream_t);

}  // namespace pic
