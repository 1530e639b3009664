// cell_list_static.cu -- the cell-list build for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a cell
// list: a host application that has already handed the device memory to its
// own pool allocator (PyTorch's caching allocator, for one, may hold nearly
// all of it, so a fresh cudaMalloc fails), or a time loop that must not take
// the implicit device-wide synchronisation that cudaMalloc/cudaFree can cause.
// bl_cell_list_build_static builds the same list as bl_cell_list_get but
// keeps its scratch -- the bin of every cell and two counters per bin -- in
// one fixed-size array that this library reserves in device memory on every
// GPU that loads it, held until the process exits.  The caller still passes
// the positions and the output arrays, all in device memory.
//
// Set-up: the first call on a device looks up the device address of that
// array (cudaGetSymbolAddress) with the device current and caches it; make
// this first call before any stream capture.  The cache is kept per device
// ordinal for the life of the process: it assumes the device's primary
// context (the one the CUDA runtime and PyTorch use) and no cudaDeviceReset
// between calls, after which the cached address would be stale.  Every later call on the device
// reuses the same array, so calls that overlap on the GPU (on different
// streams, or from several threads) race on it and must be serialised by the
// caller.  The counters are cleared at the start of each call.
#include <mutex>

#include "../../include/bloodlb.h"
#include "bl_internal.cuh"

namespace {

constexpr int kMaxCells = 1 << 16;  // cells per call
constexpr int kMaxBins = 1 << 18;   // nb0 * nb1 * nb2 per call
constexpr int kMaxDevices = 64;

// bin of each cell, then the per-bin counts, then the per-bin cursors
// (2.25 MiB of device memory per GPU)
static __device__ __align__(256) int g_cell_list_scratch[kMaxCells + 2 * kMaxBins];

std::mutex g_mu;
int *g_scratch_dev[kMaxDevices] = {};

int scratch_of_current_device(int **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return BL_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return BL_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_cell_list_scratch) != cudaSuccess || !p) return BL_ECUDA;
    g_scratch_dev[dev] = static_cast<int *>(p);
  }
  *out = g_scratch_dev[dev];
  return BL_OK;
}

}  // namespace

extern "C" int bl_cell_list_build_static(const double *X, int n, const int32_t dims[3], double r_cut, int32_t nb[3],
                                         int32_t *start, int32_t *ids, void *cuda_stream) {
  if (!dims || !nb || n < 0 || !(r_cut > 0.0)) return BL_EINVAL;
  if (n > kMaxCells) return BL_EINVAL;  // more cells than the reserved scratch holds
  if (n > 0 && (!X || !ids)) return BL_EINVAL;
  if (!start) return BL_EINVAL;
  // bin counts in double, checked against the reserved scratch before any
  // conversion to int (a tiny r_cut gives quotients far beyond INT_MAX);
  // nb is written only once the request is accepted
  int nbk[3];
  double nbins_d = 1.0;
  for (int k = 0; k < 3; ++k) {
    if (dims[k] < 1) return BL_EINVAL;
    const double b = fmax(1.0, floor((double)dims[k] / r_cut));
    if (!(b <= (double)kMaxBins)) return BL_EINVAL;
    nbk[k] = (int)b;
    nbins_d *= b;
  }
  if (!(nbins_d <= (double)kMaxBins)) return BL_EINVAL;  // more bins than the reserved scratch holds
  const long long nbins = (long long)nbins_d;
  int *scratch = nullptr;
  int rc = scratch_of_current_device(&scratch);
  if (rc != BL_OK) return rc;
  for (int k = 0; k < 3; ++k) nb[k] = nbk[k];
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  bl::CellListView cl{};
  for (int k = 0; k < 3; ++k) cl.nb[k] = nb[k];
  cl.nbins = (int)nbins;
  cl.bin_of = scratch;
  cl.count = scratch + kMaxCells;
  cl.cursor = scratch + kMaxCells + kMaxBins;
  cl.start = start;
  cl.ids = ids;
  if (cudaMemsetAsync(cl.count, 0, sizeof(int) * (size_t)nbins, st) != cudaSuccess ||
      cudaMemsetAsync(cl.cursor, 0, sizeof(int) * (size_t)nbins, st) != cudaSuccess)
    return BL_ECUDA;
  if (n == 0) {
    if (cudaMemsetAsync(start, 0, sizeof(int32_t) * (size_t)(nbins + 1), st) != cudaSuccess) return BL_ECUDA;
    return BL_OK;
  }
  bl::LatticeView lv{};
  lv.nx = dims[0];
  lv.ny = dims[1];
  lv.nz = dims[2];
  bl::PartView pv{};
  pv.n = n;
  pv.X = const_cast<double *>(X);
  int64_t launched = 0;
  bl::launch_cell_list(lv, pv, cl, st, &launched);
  return cudaGetLastError() == cudaSuccess ? BL_OK : BL_ECUDA;
}
