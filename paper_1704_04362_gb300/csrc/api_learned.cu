// C entry points of the per-frequency truncation ranks: sketch spectra, the
// plain rank rule and the learned predictor (argument checks, workspace,
// kernel sequencing on the caller's stream).
#include "tp_internal.cuh"

namespace tp {
int rsvd_run(const float* X, int64_t n1, int64_t n2, int64_t n3, int k, int p, int q,
             uint64_t seed, float* U, float* S, float* V, const tp_opts* opts, cudaStream_t st,
             float* sig_out, const int32_t* rank_per_freq, int sketch_mode,
             const int32_t* sketch_per_freq = nullptr);
size_t rsvd_ws(int64_t n1, int64_t n2, int64_t n3, int64_t k, int64_t p, int prec = TP_FP32);
bool fft_supported(int64_t n3);
size_t mlp_partial_count(int64_t B);
int launch_rank_rule(const float* sig, int64_t h, int l, int cap, double tol, int32_t* out,
                     cudaStream_t st);
int launch_rank_features(const float* sig, int64_t h, int l, void* feat, cudaStream_t st);
int launch_mlp_forward(const void* w16, const void* x16, int64_t B, float* y, cudaStream_t st);
int launch_mlp_round(const float* theta, void* w16, cudaStream_t st);
int launch_mlp_grad(const void* w16, const void* x16, const float* tgt, int64_t B, float* part,
                    float* grad, cudaStream_t st);
int launch_mlp_adam(float* theta, float* m, float* v, const float* grad, void* w16, int step,
                    float lr, cudaStream_t st);
constexpr int kMlpParams = 16 * 128 + 128 + 128 * 128 + 128 + 2 * 128 + 2;

size_t mlp_ws(int64_t B) { return ws_bytes(mlp_partial_count(B), 4); }
}  // namespace tp

using namespace tp;

extern "C" {

int tp_sketch_spectrum(const float* X, int64_t n1, int64_t n2, int64_t n3, int l, int q,
                       uint64_t seed, float* sig_out, const tp_opts* opts, void* stream) {
  if (!X || !sig_out) { set_error("tp_sketch_spectrum: NULL pointer"); return TP_ENULL; }
  if (n1 < 1 || n2 < 1 || n3 < 1 || n1 > (int64_t(1) << 31) || n2 > (int64_t(1) << 31)) {
    set_error("tp_sketch_spectrum: invalid sizes");
    return TP_EINVAL;
  }
  const int64_t m = n1 < n2 ? n1 : n2;
  if (l < 1 || q < 0 || l > m || l > 96) {
    set_error("tp_sketch_spectrum: need 1 <= l <= min(n1, n2, 96) and q >= 0");
    return TP_EINVAL;
  }
  if (n3 > 512 && !fft_supported(n3)) {
    set_error("tp_sketch_spectrum: n3 > 512 must factor into radices 2..13");
    return TP_EUNSUPPORTED;
  }
  return rsvd_run(X, n1, n2, n3, l, 0, q, seed, nullptr, nullptr, nullptr, opts,
                  as_stream(stream), sig_out, nullptr, TP_SKETCH_SIGNS);
}

int tp_rank_rule(const float* sig, int64_t h, int l, int cap, double tol, int32_t* rank_out,
                 void* stream) {
  if (!sig || !rank_out) { set_error("tp_rank_rule: NULL pointer"); return TP_ENULL; }
  if (h < 0 || l < 1 || cap < 1 || !(tol >= 0.0)) {
    set_error("tp_rank_rule: need h >= 0, l >= 1, cap >= 1, tol >= 0");
    return TP_EINVAL;
  }
  if (h == 0) return TP_OK;
  return launch_rank_rule(sig, h, l, cap, tol, rank_out, as_stream(stream));
}

int tp_rank_features(const float* sig, int64_t h, int l, void* feat_out, void* stream) {
  if (!sig || !feat_out) { set_error("tp_rank_features: NULL pointer"); return TP_ENULL; }
  if (h < 0 || l < 17) { set_error("tp_rank_features: need l >= 17 singular values"); return TP_EINVAL; }
  if (h == 0) return TP_OK;
  return launch_rank_features(sig, h, l, feat_out, as_stream(stream));
}

int tp_mlp_param_count(void) { return kMlpParams; }

int tp_mlp_round(const float* theta, void* w16, void* stream) {
  if (!theta || !w16) { set_error("tp_mlp_round: NULL pointer"); return TP_ENULL; }
  return launch_mlp_round(theta, w16, as_stream(stream));
}

int tp_mlp_forward(const void* w16, const void* x16, int64_t batch, float* y, void* stream) {
  if (!w16 || !x16 || !y) { set_error("tp_mlp_forward: NULL pointer"); return TP_ENULL; }
  if (batch < 0 || batch > (int64_t(1) << 31)) { set_error("tp_mlp_forward: invalid batch"); return TP_EINVAL; }
  return launch_mlp_forward(w16, x16, batch, y, as_stream(stream));
}

int tp_mlp_train_step(float* theta, void* w16, float* adam_m, float* adam_v, int step, float lr,
                      const void* x16, const float* target, int64_t batch, float* grad_out,
                      const tp_opts* opts, void* stream) {
  if (!theta || !w16 || !x16 || !target || !grad_out || (lr != 0.f && (!adam_m || !adam_v))) {
    set_error("tp_mlp_train_step: NULL pointer");
    return TP_ENULL;
  }
  if (batch < 1 || batch > (int64_t(1) << 31) || step < 1 || !(lr >= 0.f)) {
    set_error("tp_mlp_train_step: need batch >= 1, step >= 1, lr >= 0");
    return TP_EINVAL;
  }
  Arena ws;
  int rc = acquire_workspace(opts, mlp_ws(batch), &ws);
  if (rc) return rc;
  float* part = ws.take<float>(mlp_partial_count(batch));
  cudaStream_t st = as_stream(stream);
  if ((rc = launch_mlp_grad(w16, x16, target, batch, part, grad_out, st))) return rc;
  if (lr == 0.f) return TP_OK;
  return launch_mlp_adam(theta, adam_m, adam_v, grad_out, w16, step, lr, st);
}

}  // extern "C"
