// Allocation-free column dots.
//
// mlmc_column_dots allocates its scratch (per-chunk partial sums) on every
// call and frees it again.  Some callers cannot let a library do that:
// applications whose own memory manager owns every byte of device memory (a
// pool sized up front, a fixed budget per process), and latency-critical
// loops that must not pay an allocator's synchronisation or its failure
// modes in the middle of a run.  mlmc_column_dots_noalloc gives them the same
// computation with its scratch in a fixed array of this file.  Like
// mlmc_column_dots it returns once `out` has been written.
#include <cstdint>
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
// Per device ordinal: the array's device address and the id of the context it
// was looked up in (0 = not yet).  A context created after a device reset
// loads the module again, possibly at another address, and gets a new id.
void *g_scratch_ptr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};

thread_local std::string g_err;

// Driver calls reached through the runtime's entry-point table (the library
// links only the runtime): the current context and its process-unique id.
typedef int (*ctx_get_current_fn)(void **ctx);
typedef int (*ctx_get_id_fn)(void *ctx, unsigned long long *id);

// Id of the current context, 0 if none is current yet or the driver cannot say.
unsigned long long current_context_id() {
  static ctx_get_current_fn get_current = nullptr;
  static ctx_get_id_fn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void *f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (ctx_get_current_fn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (ctx_get_id_fn)f;
  });
  if (!get_current || !get_id) return 0;
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on the current device.  In host code
// g_dots_scratch only names a host-side stand-in, so the address is looked
// up with the device current, the first time the device is used (and again
// if its context has been replaced since, e.g. after cudaDeviceReset), and
// cached.
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
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dots_scratch);   // also makes the device's primary context current
    if (e != cudaSuccess) {
      g_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return MLMC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = current_context_id();
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
