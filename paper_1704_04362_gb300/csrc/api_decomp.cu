// C entry points of the decomposition paths (filled in by later kernels).
#include "tp_internal.cuh"

namespace tp {
size_t workspace_for(int op, const int64_t* d, int nd) {
  (void)op; (void)d; (void)nd;
  return 0;
}
}  // namespace tp

using namespace tp;

extern "C" {
int tsvd(const float*, int64_t, int64_t, int64_t, float*, float*, float*, const tp_opts*, void*) {
  set_error("tsvd: not built yet");
  return TP_EUNSUPPORTED;
}
int tsvd_randomized(const float*, int64_t, int64_t, int64_t, int, int, int, uint64_t, float*,
                    float*, float*, const tp_opts*, void*) {
  set_error("tsvd_randomized: not built yet");
  return TP_EUNSUPPORTED;
}
int tcomplete_svt(const float*, const uint8_t*, int64_t, int64_t, int64_t, int, double, double,
                  float*, float*, float*, double*, const tp_opts*, void*) {
  set_error("tcomplete_svt: not built yet");
  return TP_EUNSUPPORTED;
}
}
