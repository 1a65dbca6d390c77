// pic_field_periodic_noalloc: the periodic Poisson solve of pic_field_periodic
// for callers that must not allocate device memory during a call.
//
// Why: pic_field_periodic obtains its scratch with cudaMalloc and releases it
// with cudaFree.  cudaFree waits for the whole device to go idle, which stalls
// every other stream of an application that runs its own work beside the
// solve, and callers that manage device memory through their own pool (a
// framework's caching allocator, a fixed-budget embedded deployment) may not
// be allowed to allocate behind the pool's back at all.  This entry point
// takes the same inputs and outputs from the caller and keeps its scratch in a
// fixed array compiled into the library instead.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (525 KiB) until the process exits.  Host code cannot
// use the array's name as a device address, so every call looks the address
// up with cudaGetSymbolAddress on the current device (a lookup, no
// allocation); the first call on a device also loads the library's device
// code there, so make it before any stream capture.  Every call shares the
// one array and overwrites it, so calls that overlap on the GPU (two streams,
// or two host threads on one device) race and must be ordered by the caller.
#include "pic_internal.cuh"

namespace {

constexpr int kNoAllocMaxCells = 65536;
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffCtl = 0;
constexpr size_t kOffScan = align256(sizeof(pic::Ctl));
constexpr size_t kOffEf = kOffScan + align256(sizeof(pic::FieldScan));
constexpr size_t kScratchBytes = kOffEf + align256(((size_t)kNoAllocMaxCells + 1) * 8);

// scratch of the no-allocation field solve: control block, block partials of
// the exact prefix sums, field copy; see the file comment for its rules
static __device__ __align__(256) unsigned char g_field_scratch[kScratchBytes];

// device address of the scratch on the current device, looked up on every call
// (a cached address would outlive a cudaDeviceReset, which reloads the module)
cudaError_t scratch_address(unsigned char **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_field_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char *>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" {

int pic_field_periodic_noalloc(const int64_t *Q_i, const int64_t *Q_e, int n_cells, double C, double E0, double *E,
                               double *E_half, void *stream) {
  if (!Q_i || !Q_e || !E || !E_half || n_cells < 3) return PIC_EINVAL;
  if (n_cells > kNoAllocMaxCells) return PIC_EINVAL;  // beyond the fixed scratch
  unsigned char *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return PIC_ECUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  pic::Ctl *ctl = reinterpret_cast<pic::Ctl *>(base + kOffCtl);
  pic::FieldScan *fs = reinterpret_cast<pic::FieldScan *>(base + kOffScan);
  double *Ef = reinterpret_cast<double *>(base + kOffEf);
  // the control block keeps the previous call's status: start it from zero
  pic::Ctl c{};
  c.E0 = E0;
  e = cudaMemcpyAsync(ctl, &c, sizeof c, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return PIC_ECUDA;
  // the reduction's completion ticket must start at zero
  e = cudaMemsetAsync(&fs->ticket, 0, sizeof fs->ticket, st);
  if (e != cudaSuccess) return PIC_ECUDA;
  pic::FieldK f{};
  f.N = n_cells;
  f.field_mode = PIC_FIELD_POISSON;
  f.smem = 0;  // the net-charge array lives in the scratch array
  f.seg = (n_cells + pic::kFieldThreads - 1) / pic::kFieldThreads;
  f.Cf = C / ((double)n_cells * (double)n_cells);
  pic::launch_field<double>(f, reinterpret_cast<const unsigned long long *>(Q_e),
                            reinterpret_cast<const unsigned long long *>(Q_i), ctl, E, E_half, Ef, pic::Moments{}, fs,
                            false, false, st);
  e = cudaGetLastError();
  unsigned int status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &ctl->status, sizeof status, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return PIC_ECUDA;
  if (status & pic::kStNonFinite) return PIC_ENONFINITE;
  return 0;
}

}  // extern "C"
