// Host runtime of libtprod.so: error reporting, launch accounting and the
// library-managed workspace (one growing buffer per device).
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "tp_internal.cuh"

namespace tp {

namespace {
thread_local char g_err[512] = "";
std::atomic<uint64_t> g_launches{0};

struct DevBuf {
  void* ptr = nullptr;
  size_t size = 0;
};
constexpr int kMaxDev = 64;
DevBuf g_ws[kMaxDev];
std::mutex g_ws_mu;
}  // namespace

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int launch_status(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return TP_ECUDA;
  }
  return TP_OK;
}

void note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int set_smem_attr(const void* func, size_t bytes, const char* name) {
  const cudaError_t e =
      cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("%s: cannot allow %zu bytes of dynamic shared memory: %s", name, bytes,
              cudaGetErrorString(e));
    return TP_ECUDA;
  }
  return TP_OK;
}

int sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return 152;
  }
  int sms = cache[dev].load(std::memory_order_relaxed);
  if (sms > 0) return sms;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    sms = 152;
  }
  cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

namespace {
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
};
struct ProfTotal {
  std::string name;
  double ms = 0.0;
  int64_t launches = 0;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<ProfRec> g_prof_recs;
std::vector<ProfTotal> g_prof_tot;
constexpr size_t kMaxProfRecs = 1 << 16;
}  // namespace

KernelScope::KernelScope(const char* n, cudaStream_t s, bool c)
    : name(n), st(s), slot(-1), count(c) {
  if (!g_prof_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;   // launches inside a graph capture are not timed one by one
  }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on || g_prof_recs.size() >= kMaxProfRecs) return;
  ProfRec r{n, nullptr, nullptr};
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaEventRecord(r.a, st);
  slot = int(g_prof_recs.size());
  g_prof_recs.push_back(r);
}

KernelScope::~KernelScope() {
  if (count) note_launches(1);
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot < int(g_prof_recs.size())) cudaEventRecord(g_prof_recs[slot].b, st);
}

int acquire_workspace(const tp_opts* opts, size_t need, Arena* out) {
  if (opts && opts->workspace) {
    if ((reinterpret_cast<uintptr_t>(opts->workspace) & 255) != 0) {
      set_error("workspace must be 256-byte aligned");
      return TP_EALIGN;
    }
    if (opts->workspace_bytes < need) {
      set_error("workspace of %zu bytes is smaller than the %zu this call needs",
                opts->workspace_bytes, need);
      return TP_EWORKSPACE;
    }
    out->base = static_cast<char*>(opts->workspace);
    out->size = opts->workspace_bytes;
    out->off = 0;
    return TP_OK;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    set_error("no current CUDA device");
    return TP_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_ws_mu);
  DevBuf& b = g_ws[dev];
  if (b.size < need) {
    // growing: earlier calls may still use the old buffer on any stream
    if (cudaDeviceSynchronize() != cudaSuccess) {
      set_error("cudaDeviceSynchronize before workspace growth failed");
      return TP_ECUDA;
    }
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.size = 0;
    size_t sz = need < (size_t(1) << 20) ? (size_t(1) << 20) : need;
    if (cudaMalloc(&b.ptr, sz) != cudaSuccess) {
      cudaGetLastError();
      set_error("cannot allocate a %zu-byte workspace", sz);
      return TP_ENOMEM;
    }
    b.size = sz;
  }
  out->base = static_cast<char*>(b.ptr);
  out->size = b.size;
  out->off = 0;
  return TP_OK;
}

}  // namespace tp

extern "C" {

const char* tp_status_string(int s) {
  switch (s) {
    case TP_OK: return "TP_OK";
    case TP_EINVAL: return "TP_EINVAL: invalid size or mode";
    case TP_ENULL: return "TP_ENULL: required pointer is NULL";
    case TP_EALIGN: return "TP_EALIGN: misaligned pointer";
    case TP_ENOMEM: return "TP_ENOMEM: workspace allocation failed";
    case TP_ECUDA: return "TP_ECUDA: CUDA error";
    case TP_EWORKSPACE: return "TP_EWORKSPACE: workspace too small";
    case TP_EUNSUPPORTED: return "TP_EUNSUPPORTED: not supported by this library";
    default: return "unknown tp_status";
  }
}

const char* tp_last_error(void) { return tp::g_err; }

int tp_sync_status(void* stream, const int32_t* status_dev, int32_t* status_host) {
  if (status_dev && !status_host) { tp::set_error("tp_sync_status: NULL status_host"); return TP_ENULL; }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    tp::set_error("asynchronous CUDA error: %s", cudaGetErrorString(e));
    return TP_ECUDA;
  }
  if (status_dev) {
    if (cudaMemcpy(status_host, status_dev, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      tp::set_error("tp_sync_status: reading the status word failed");
      return TP_ECUDA;
    }
  }
  return TP_OK;
}

int tp_release(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= tp::kMaxDev) return TP_ECUDA;
  std::lock_guard<std::mutex> lk(tp::g_ws_mu);
  tp::DevBuf& b = tp::g_ws[dev];
  if (b.ptr) {
    cudaDeviceSynchronize();
    cudaFree(b.ptr);
  }
  b.ptr = nullptr;
  b.size = 0;
  return TP_OK;
}

uint64_t tp_launch_count(void) { return tp::g_launches.load(); }

int tp_version(void) { return 1; }

int tp_profile_start(void) {
  std::lock_guard<std::mutex> lk(tp::g_prof_mu);
  tp::g_prof_on = true;
  return TP_OK;
}

int tp_profile_stop(void) {
  std::lock_guard<std::mutex> lk(tp::g_prof_mu);
  tp::g_prof_on = false;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    tp::set_error("tp_profile_stop: device synchronisation failed");
    return TP_ECUDA;
  }
  for (auto& r : tp::g_prof_recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      ms = 0.f;
    }
    tp::ProfTotal* t = nullptr;
    for (auto& x : tp::g_prof_tot)
      if (x.name == r.name) t = &x;
    if (!t) {
      tp::g_prof_tot.push_back(tp::ProfTotal{r.name, 0.0, 0});
      t = &tp::g_prof_tot.back();
    }
    t->ms += ms;
    t->launches += 1;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  tp::g_prof_recs.clear();
  return TP_OK;
}

int tp_profile_entry(int i, char* name, int name_len, double* total_ms, int64_t* launches) {
  std::lock_guard<std::mutex> lk(tp::g_prof_mu);
  if (i < 0 || i >= int(tp::g_prof_tot.size())) return TP_EINVAL;
  const auto& t = tp::g_prof_tot[i];
  if (name && name_len > 0) {
    snprintf(name, size_t(name_len), "%s", t.name.c_str());
  }
  if (total_ms) *total_ms = t.ms;
  if (launches) *launches = t.launches;
  return TP_OK;
}

int tp_profile_reset(void) {
  std::lock_guard<std::mutex> lk(tp::g_prof_mu);
  tp::g_prof_tot.clear();
  return TP_OK;
}

}  // extern "C"
