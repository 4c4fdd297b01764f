// tp_slice_norms_noalloc: slice norms with no memory allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs while a framework owns
// the whole device memory pool, real-time or embedded callers that forbid
// allocation after start-up, and callers that must not trigger the device
// synchronisation a cudaMalloc/cudaFree may imply.  For them this entry point
// runs the same norm kernels as tp_slice_norms, with their partial sums kept
// in a fixed array in device global memory that belongs to the library.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its kNoAllocScratch doubles (8 MiB) until the process exits.
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in object), so its device address is looked up with
// cudaGetSymbolAddress on the first call made with a device current, and
// cached for that device and its CUDA context.  A call under a different
// context (after cudaDeviceReset, or with another context made current
// through the driver API) sees the context change and looks the address up
// again, since the module may then live at a new address.
#include <cuda.h>

#include <mutex>

#include "tp_internal.cuh"

namespace tp {
namespace {

constexpr size_t kNoAllocScratch = size_t(1) << 20;   // doubles (8 MiB)

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

constexpr int kMaxDevices = 64;
struct ScratchSlot {
  CUcontext ctx = nullptr;
  double* addr = nullptr;
};
ScratchSlot g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

typedef CUresult (*PFN_ctx_get_current)(CUcontext*);

// The current CUDA context (driver API, reached through the runtime so that
// the library needs no link against libcuda); null if it cannot be read.
CUcontext current_context() {
  static PFN_ctx_get_current fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_ctx_get_current>(p);
    cudaGetLastError();
  });
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Device address of the scratch array on the current device and context.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_error("tp_slice_norms_noalloc: no usable current CUDA device");
    return TP_ECUDA;
  }
  // null before the runtime has made a context current: the lookup below
  // then runs (and creates the primary context), and the next call caches
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  ScratchSlot& slot = g_scratch[dev];
  if (!slot.addr || !ctx || slot.ctx != ctx) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("tp_slice_norms_noalloc: cudaGetSymbolAddress failed: %s",
                cudaGetErrorString(e));
      return TP_ECUDA;
    }
    slot.addr = static_cast<double*>(p);
    slot.ctx = ctx;
  }
  *out = slot.addr;
  return TP_OK;
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" {

size_t tp_slice_norms_noalloc_capacity(void) { return kNoAllocScratch; }

int tp_slice_norms_noalloc(const float* X, int64_t n1, int64_t n2, int64_t n3, int which,
                           double* out, void* stream) {
  if (!X || !out) { set_error("tp_slice_norms_noalloc: NULL pointer"); return TP_ENULL; }
  if (n1 < 1 || n2 < 1 || n3 < 1 || n1 > (int64_t(1) << 31) || n2 > (int64_t(1) << 31) ||
      n3 > (int64_t(1) << 31) || (n2 * n3) / n3 != n2) {
    set_error("tp_slice_norms_noalloc: invalid sizes");
    return TP_EINVAL;
  }
  if (which != 0 && which != 1) {
    set_error("tp_slice_norms_noalloc: which must be 0 or 1");
    return TP_EINVAL;
  }
  const size_t need = norms_partial_count(n1, n2, n3, which);
  if (need > kNoAllocScratch) {
    set_error("tp_slice_norms_noalloc: needs %zu scratch doubles, the fixed array holds %zu "
              "(lateral norms need n2*n3 <= %zu); use tp_slice_norms instead",
              need, kNoAllocScratch, kNoAllocScratch);
    return TP_EINVAL;
  }
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  // Every partial slot the kernels read is written first in the same call,
  // so nothing in the array has to start at zero.
  // the default launch shape: no autotuning (it would time and synchronise)
  return launch_slice_norms(X, n1, n2, n3, which, out, scratch, as_stream(stream), false);
}

}  // extern "C"
