// Launch-shape autotuner.  A tunable launch offers a few candidate shapes
// (tile widths, blocks per SM) that all compute bit-identical results; the
// first call with a given problem key (sizes taken by their size class, the
// bit length, so that problems within a factor of two share a choice) times
// each candidate on the caller's stream with CUDA events (one warm-up and
// three timed launches each), keeps the fastest, and every later call with
// that key launches it directly.  A stream being captured into a CUDA graph
// is never timed: the call takes the cached choice or the default.  The
// table can be listed, saved to and loaded from a text file (one "key
// choice" line per entry), and tuning can be switched off (the default
// candidate everywhere; environment variable TP_AUTOTUNE=0 at load) or
// forced to one candidate (for tests).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tp_internal.cuh"

namespace tp {
namespace {

struct TuneEntry {
  int choice = 0;
  int ncand = 0;
  int dflt = 0;
  std::vector<double> ms;   // per candidate, empty when loaded from a file
};

std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune;
int g_tune_mode = -1;   // -1: not read from the environment yet
int g_tune_force = -1;

int tune_mode_locked() {
  if (g_tune_mode < 0) {
    const char* e = std::getenv("TP_AUTOTUNE");
    g_tune_mode = (e && e[0] == '0') ? TP_TUNE_OFF : TP_TUNE_ON;
  }
  return g_tune_mode;
}

std::string make_key(const char* op, const int64_t* key, int nkey) {
  std::string s(op);
  for (int i = 0; i < nkey; ++i) s += (i ? "," : ":") + std::to_string(key[i]);
  return s;
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;   // unknown: do not time
  }
  return cs != cudaStreamCaptureStatusNone;
}

}  // namespace

int autotune_pick(const char* op, const int64_t* key, int nkey, int ncand, int dflt,
                  const std::function<int(int)>& launch, cudaStream_t st, int* choice) {
  *choice = dflt;
  const std::string k = make_key(op, key, nkey);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune_force >= 0) {
      *choice = g_tune_force < ncand ? g_tune_force : ncand - 1;
      return TP_OK;
    }
    if (tune_mode_locked() == TP_TUNE_OFF) return TP_OK;
    auto it = g_tune.find(k);
    if (it != g_tune.end()) {
      if (it->second.choice >= 0 && it->second.choice < ncand) *choice = it->second.choice;
      return TP_OK;
    }
  }
  if (ncand < 2 || capturing(st)) return TP_OK;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    return TP_OK;   // untimed: the default
  }
  TuneEntry e;
  e.ncand = ncand;
  e.dflt = dflt;
  e.ms.assign(size_t(ncand), -1.0);
  int rc = TP_OK;
  double best = 0.0;
  int best_c = dflt;
  for (int c = 0; c < ncand && rc == TP_OK; ++c) {
    if ((rc = launch(c))) break;   // warm-up
    cudaEventRecord(a, st);
    for (int r = 0; r < 3 && rc == TP_OK; ++r) rc = launch(c);
    cudaEventRecord(b, st);
    if (rc) break;
    float ms = 0.f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
      cudaGetLastError();
      set_error("autotune %s: timing failed", k.c_str());
      rc = TP_ECUDA;
      break;
    }
    e.ms[size_t(c)] = ms / 3.0;
    if (c == 0 || e.ms[size_t(c)] < best) {
      best = e.ms[size_t(c)];
      best_c = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  e.choice = best_c;
  *choice = best_c;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[k] = e;
  return TP_OK;
}

}  // namespace tp

using namespace tp;

extern "C" {

int tp_autotune_mode(int mode) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const int prev = tune_mode_locked();
  if (mode == TP_TUNE_OFF || mode == TP_TUNE_ON) g_tune_mode = mode;
  return prev;
}

int tp_autotune_force(int candidate) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const int prev = g_tune_force;
  g_tune_force = candidate < 0 ? -1 : candidate;
  return prev;
}

int tp_autotune_count(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return int(g_tune.size());
}

int tp_autotune_entry(int i, char* key, int key_len, int* choice, int* ncand, double* best_ms,
                      double* default_ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (i < 0 || i >= int(g_tune.size())) return TP_EINVAL;
  auto it = g_tune.begin();
  std::advance(it, i);
  if (key && key_len > 0) {
    std::strncpy(key, it->first.c_str(), size_t(key_len) - 1);
    key[key_len - 1] = '\0';
  }
  const TuneEntry& e = it->second;
  if (choice) *choice = e.choice;
  if (ncand) *ncand = e.ncand;
  const bool timed = !e.ms.empty();
  if (best_ms) *best_ms = timed ? e.ms[size_t(e.choice)] : -1.0;
  if (default_ms) *default_ms = timed ? e.ms[size_t(e.dflt)] : -1.0;
  return TP_OK;
}

int tp_autotune_reset(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  return TP_OK;
}

int tp_autotune_save(const char* path) {
  if (!path) { set_error("tp_autotune_save: NULL path"); return TP_ENULL; }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE* f = std::fopen(path, "w");
  if (!f) { set_error("tp_autotune_save: cannot open %s", path); return TP_EINVAL; }
  for (const auto& kv : g_tune) std::fprintf(f, "%s %d\n", kv.first.c_str(), kv.second.choice);
  std::fclose(f);
  return TP_OK;
}

int tp_autotune_load(const char* path) {
  if (!path) { set_error("tp_autotune_load: NULL path"); return TP_ENULL; }
  FILE* f = std::fopen(path, "r");
  if (!f) { set_error("tp_autotune_load: cannot open %s", path); return TP_EINVAL; }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  char key[512];
  int choice = 0;
  int rc = TP_OK;
  while (true) {
    const int got = std::fscanf(f, "%511s %d", key, &choice);
    if (got == EOF) break;
    if (got != 2 || choice < 0) {
      set_error("tp_autotune_load: malformed line in %s", path);
      rc = TP_EINVAL;
      break;
    }
    TuneEntry e;
    e.choice = choice;
    g_tune[key] = e;
  }
  std::fclose(f);
  return rc;
}

}  // extern "C"
