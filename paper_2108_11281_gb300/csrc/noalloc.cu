// Allocation-free column dots.
//
// mlmc_column_dots allocates its scratch (per-chunk partial sums) with
// cudaMalloc and frees it with cudaFree on every call.  Some callers cannot
// do that: code that runs while a CUDA graph is being captured on the stream
// (cudaMalloc and cudaFree are not stream operations and break the capture),
// applications whose memory manager owns every device allocation or whose
// memory budget forbids a library from allocating, and latency-critical
// loops that must avoid the device-wide synchronisation cudaFree implies.
// mlmc_column_dots_noalloc gives them the same computation with its scratch
// in a fixed array of this file.
#include <mutex>

#include "mlmc.h"
#include "mlmc_internal.cuh"

namespace {

// Largest scratch the entry point may need: 608 row chunks x 256 columns x
// one complex double.  2,490,368 bytes, held by every GPU that loads the
// library until the process exits.
constexpr size_t kMaxParts = 608;
constexpr size_t kMaxColumns = 256;
constexpr size_t kScratchBytes = kMaxParts * kMaxColumns * 16;

static __device__ __align__(256) unsigned char g_dots_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

thread_local std::string g_err;

// Device address of the scratch array on the current device.  In host code
// g_dots_scratch only names a host-side stand-in, so the address is looked
// up once per device, with that device current, and cached.
int scratch_address(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return MLMC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    g_err = "device ordinal out of range";
    return MLMC_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dots_scratch);
    if (e != cudaSuccess) {
      g_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return MLMC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return MLMC_OK;
}

}  // namespace

extern "C" int mlmc_column_dots_noalloc(int complex_data, const void *x, const void *y, int n, int k, void *out,
                                        void *stream) {
  if (!x || !y || !out || n < 1 || k < 1) {
    g_err = "bad column-dot arguments";
    return MLMC_ERR_INVALID_ARG;
  }
  if ((size_t)k > kMaxColumns) {
    g_err = "k exceeds the 256 columns the fixed scratch holds";
    return MLMC_ERR_INVALID_ARG;
  }
  void *scratch = nullptr;
  int st = scratch_address(&scratch);
  if (st != MLMC_OK) return st;
  const int parts = mlmc::multidot_parts((size_t)n, k);   // at most 608
  if ((size_t)parts * k * 16 > kScratchBytes) {
    g_err = "scratch too small";
    return MLMC_ERR_INVALID_ARG;
  }
  // The partial sums are written in full by the first kernel before the second
  // reads them, so nothing in the array needs clearing between calls.
  try {
    mlmc::DType t = complex_data ? mlmc::C64 : mlmc::F64;
    mlmc::launch_multidot(t, x, (size_t)n * k, 1, y, (size_t)n, k, scratch, parts, out, t, (cudaStream_t)stream);
    mlmc::check_cuda(cudaStreamSynchronize((cudaStream_t)stream), "sync");
  } catch (const mlmc::cuda_error &e) {
    g_err = std::string(e.where) + ": " + cudaGetErrorString(e.code);
    return MLMC_ERR_CUDA;
  }
  return MLMC_OK;
}

extern "C" const char *mlmc_noalloc_last_error(void) { return g_err.c_str(); }
