// C entry points of the decomposition paths (filled in by later kernels).
#include <cmath>

#include "tp_internal.cuh"

namespace tp {
size_t tsvd_ws(int64_t n1, int64_t n2, int64_t n3);
bool fft_supported(int64_t n3);
size_t rsvd_ws(int64_t n1, int64_t n2, int64_t n3, int64_t k, int64_t p, int prec = TP_FP32);
size_t svt_ws(int64_t n1, int64_t n2, int64_t n3, int prec = TP_FP32);
size_t svt_batched_ws_dims(const int64_t* dims, int nd, int prec);
size_t mlp_ws(int64_t B);
int svt_batched_run(int ntens, const tp_tensor_desc* d, int iters, double rho, double mu_max,
                    const tp_opts* opts, cudaStream_t st, const double* lams = nullptr);
int svt_run(const float* X, const uint8_t* mask, int64_t n1, int64_t n2, int64_t n3, int iters,
            double rho, double mu_max, float* L, float* E, float* Y, double* mu,
            const tp_opts* opts, cudaStream_t st, double lam);
size_t tcx_ws(int64_t n1, int64_t n2, int64_t n3);
int tcx_run(const float* A, int64_t n1, int64_t n2, int64_t n3, int64_t c, uint64_t seed,
            int prob_mode, const double* p_given, float* Z, int32_t* idx_out, int64_t* count_out,
            const tp_opts* opts, cudaStream_t st);
size_t tcur_ws(int64_t n1, int64_t n2, int64_t n3);
int tcur_run(const float* A, int64_t n1, int64_t n2, int64_t n3, int64_t c, int64_t l, int rank,
             uint64_t seed, int prob_mode, const double* p_cols, const double* p_rows, float* Z,
             int32_t* col_idx, int64_t* col_count, int32_t* row_idx, int64_t* row_count,
             double* row_prob, const tp_opts* opts, cudaStream_t st);
size_t cur_tnn_ws(int64_t n1, int64_t n2, int64_t n3);
int cur_tnn_run(const float* X, const uint8_t* mask, int64_t n1, int64_t n2, int64_t n3,
                int64_t c, int64_t l, int rank, uint64_t seed, int prob_mode, const double* p_cols,
                const double* p_rows, int iters, double lambda, double mu0, double rho,
                double mu_max, double rtol, float* Lout, float* Ct_out, float* Rt_out,
                int32_t* col_idx, int64_t* col_count, int32_t* row_idx, int64_t* row_count,
                double* row_prob, const tp_opts* opts, cudaStream_t st);
int rsvd_run(const float* X, int64_t n1, int64_t n2, int64_t n3, int k, int p, int q,
             uint64_t seed, float* U, float* S, float* V, const tp_opts* opts, cudaStream_t st,
             float* sig_out, const int32_t* rank_per_freq, int sketch_mode,
             const int32_t* sketch_per_freq = nullptr);
int tsvd_run(const float* X, int64_t n1, int64_t n2, int64_t n3, float* U, float* S, float* V,
             const tp_opts* opts, cudaStream_t st);

size_t workspace_for(int op, const int64_t* d, int nd, const tp_opts* opts) {
  switch (op) {
    case TP_OP_TSVD: return nd >= 3 ? tsvd_ws(d[0], d[1], d[2]) : 0;
    case TP_OP_TSVD_RANDOMIZED:
      return nd >= 5 ? rsvd_ws(d[0], d[1], d[2], d[3], d[4], opts ? opts->precision : TP_FP32) : 0;
    case TP_OP_TCOMPLETE_SVT:
    case TP_OP_TRPCA:
      return nd >= 3 ? svt_ws(d[0], d[1], d[2], opts ? opts->precision : TP_FP32) : 0;
    case TP_OP_TCOMPLETE_SVT_BATCHED:
      return nd >= 3 ? svt_batched_ws_dims(d, nd, opts ? opts->precision : TP_FP32) : 0;
    case TP_OP_SKETCH_SPECTRUM: return nd >= 4 ? rsvd_ws(d[0], d[1], d[2], d[3], 0) : 0;
    case TP_OP_MLP_TRAIN: return nd >= 1 ? mlp_ws(d[0]) : 0;
    case TP_OP_TCX: return nd >= 3 ? tcx_ws(d[0], d[1], d[2]) : 0;
    case TP_OP_TCUR: return nd >= 3 ? tcur_ws(d[0], d[1], d[2]) : 0;
    case TP_OP_CUR_TNN: return nd >= 3 ? cur_tnn_ws(d[0], d[1], d[2]) : 0;
    default: return 0;
  }
}

namespace {
bool dims3_ok(int64_t n1, int64_t n2, int64_t n3) {
  return n1 >= 1 && n2 >= 1 && n3 >= 1 && n1 <= (int64_t(1) << 31) && n2 <= (int64_t(1) << 31) &&
         n3 <= (int64_t(1) << 31) && n1 * n2 <= (int64_t(1) << 40) / n3;
}
}  // namespace
}  // namespace tp

using namespace tp;

extern "C" {
int tsvd(const float* X, int64_t n1, int64_t n2, int64_t n3, float* U, float* S, float* V,
         const tp_opts* opts, void* stream) {
  if (!X || !U || !S || !V) { set_error("tsvd: NULL pointer"); return TP_ENULL; }
  if (!dims3_ok(n1, n2, n3)) { set_error("tsvd: invalid sizes"); return TP_EINVAL; }
  const int64_t m = n1 < n2 ? n1 : n2;
  if (m > 512) { set_error("tsvd: min(n1, n2) = %lld > 512 not supported", (long long)m); return TP_EUNSUPPORTED; }
  if (n3 > 512 && !fft_supported(n3)) {
    set_error("tsvd: n3 = %lld > 512 must factor into radices 2..13", (long long)n3);
    return TP_EUNSUPPORTED;
  }
  return tsvd_run(X, n1, n2, n3, U, S, V, opts, as_stream(stream));
}
int tsvd_randomized(const float* X, int64_t n1, int64_t n2, int64_t n3, int k, int p, int q,
                    uint64_t seed, int sketch_mode, const int32_t* rank_per_freq,
                    const int32_t* sketch_per_freq, float* U, float* S, float* V,
                    const tp_opts* opts, void* stream) {
  if (!X || !U || !S || !V) { set_error("tsvd_randomized: NULL pointer"); return TP_ENULL; }
  if (!dims3_ok(n1, n2, n3)) { set_error("tsvd_randomized: invalid sizes"); return TP_EINVAL; }
  const int64_t m = n1 < n2 ? n1 : n2;
  if (k < 1 || p < 0 || q < 0 || int64_t(k) + p > m || k + p > 96) {
    set_error("tsvd_randomized: need 1 <= k, 0 <= p, q and k + p <= min(n1, n2, 96)");
    return TP_EINVAL;
  }
  if (n3 > 512 && !fft_supported(n3)) {
    set_error("tsvd_randomized: n3 = %lld > 512 must factor into radices 2..13", (long long)n3);
    return TP_EUNSUPPORTED;
  }
  if (sketch_mode != TP_SKETCH_SIGNS && sketch_mode != TP_SKETCH_SLICES) {
    set_error("tsvd_randomized: unknown sketch_mode %d", sketch_mode);
    return TP_EINVAL;
  }
  return rsvd_run(X, n1, n2, n3, k, p, q, seed, U, S, V, opts, as_stream(stream), nullptr,
                  rank_per_freq, sketch_mode, sketch_per_freq);
}
int tcomplete_svt(const float* X, const uint8_t* mask, int64_t n1, int64_t n2, int64_t n3,
                  int iters, double rho, double mu_max, float* L, float* E, float* Y, double* mu,
                  const tp_opts* opts, void* stream) {
  if (!X || !mask || !L || !E || !Y || !mu) { set_error("tcomplete_svt: NULL pointer"); return TP_ENULL; }
  if (!dims3_ok(n1, n2, n3) || iters < 0 || !(rho > 0.0) || !(mu_max > 0.0)) {
    set_error("tcomplete_svt: invalid sizes or constants");
    return TP_EINVAL;
  }
  const int64_t m = n1 < n2 ? n1 : n2;
  if (m > 512) { set_error("tcomplete_svt: min(n1, n2) > 512 not supported"); return TP_EUNSUPPORTED; }
  if (n3 > 512 && !fft_supported(n3)) {
    set_error("tcomplete_svt: n3 > 512 must factor into radices 2..13");
    return TP_EUNSUPPORTED;
  }
  return svt_run(X, mask, n1, n2, n3, iters, rho, mu_max, L, E, Y, mu, opts, as_stream(stream),
                 0.0);
}

int trpca_admm(const float* X, int64_t n1, int64_t n2, int64_t n3, int iters, double lambda,
               double rho, double mu_max, float* L, float* E, float* Y, double* mu,
               const tp_opts* opts, void* stream) {
  if (!X || !L || !E || !Y || !mu) { set_error("trpca_admm: NULL pointer"); return TP_ENULL; }
  if (!dims3_ok(n1, n2, n3) || iters < 0 || !(rho > 0.0) || !(mu_max > 0.0) || lambda < 0.0) {
    set_error("trpca_admm: invalid sizes or constants");
    return TP_EINVAL;
  }
  if ((n1 < n2 ? n1 : n2) > 512) { set_error("trpca_admm: min(n1, n2) > 512 not supported"); return TP_EUNSUPPORTED; }
  if (n3 > 512 && !fft_supported(n3)) {
    set_error("trpca_admm: n3 > 512 must factor into radices 2..13");
    return TP_EUNSUPPORTED;
  }
  const double lam = lambda > 0.0 ? lambda : 1.0 / sqrt(double(n1 > n2 ? n1 : n2) * double(n3));
  return svt_run(X, nullptr, n1, n2, n3, iters, rho, mu_max, L, E, Y, mu, opts, as_stream(stream),
                 lam);
}

int tcomplete_svt_batched(int ntens, const tp_tensor_desc* descs, int iters, double rho,
                          double mu_max, const tp_opts* opts, void* stream) {
  if (!descs) { set_error("tcomplete_svt_batched: NULL descs"); return TP_ENULL; }
  if (ntens < 1 || iters < 0 || !(rho > 0.0) || !(mu_max > 0.0)) {
    set_error("tcomplete_svt_batched: invalid count or constants");
    return TP_EINVAL;
  }
  for (int i = 0; i < ntens; ++i) {
    const tp_tensor_desc& t = descs[i];
    if (!t.X || !t.mask || !t.L || !t.E || !t.Y || !t.mu) {
      set_error("tcomplete_svt_batched: tensor %d has a NULL pointer", i);
      return TP_ENULL;
    }
    if (!dims3_ok(t.n1, t.n2, t.n3)) {
      set_error("tcomplete_svt_batched: tensor %d has invalid sizes", i);
      return TP_EINVAL;
    }
    if ((t.n1 < t.n2 ? t.n1 : t.n2) > 512) {
      set_error("tcomplete_svt_batched: tensor %d has min(n1, n2) > 512", i);
      return TP_EUNSUPPORTED;
    }
    if (t.n3 > 512 && !fft_supported(t.n3)) {
      set_error("tcomplete_svt_batched: tensor %d: n3 > 512 must factor into radices 2..13", i);
      return TP_EUNSUPPORTED;
    }
  }
  return svt_batched_run(ntens, descs, iters, rho, mu_max, opts, as_stream(stream));
}

int tcx(const float* A, int64_t n1, int64_t n2, int64_t n3, int64_t c, uint64_t seed,
        int prob_mode, const double* p_given, float* Z, int32_t* idx_out, int64_t* count_out,
        const tp_opts* opts, void* stream) {
  if (!A || !Z) { set_error("tcx: NULL tensor"); return TP_ENULL; }
  if (!dims3_ok(n1, n2, n3) || c < 1) { set_error("tcx: invalid sizes"); return TP_EINVAL; }
  if (prob_mode != TP_PROB_A2 && prob_mode != TP_PROB_GIVEN) {
    set_error("tcx: prob_mode must be TP_PROB_A2 or TP_PROB_GIVEN");
    return TP_EINVAL;
  }
  if (prob_mode == TP_PROB_GIVEN && !p_given) { set_error("tcx: TP_PROB_GIVEN needs p_given"); return TP_ENULL; }
  if ((n1 < n2 ? n1 : n2) > 512 || n2 > 4096) {
    set_error("tcx: needs min(n1, n2) <= 512 and n2 <= 4096");
    return TP_EUNSUPPORTED;
  }
  if (n3 > 512) { set_error("tcx: n3 > 512 not supported (the gathered transform is direct)"); return TP_EUNSUPPORTED; }
  return tcx_run(A, n1, n2, n3, c, seed, prob_mode, p_given, Z, idx_out, count_out, opts,
                 as_stream(stream));
}

int tcur(const float* A, int64_t n1, int64_t n2, int64_t n3, int64_t c, int64_t l, int rank,
         uint64_t seed, int prob_mode, const double* p_cols, const double* p_rows, float* Z, int32_t* col_idx,
         int64_t* col_count, int32_t* row_idx, int64_t* row_count, double* row_prob,
         const tp_opts* opts, void* stream) {
  if (!A || !Z) { set_error("tcur: NULL tensor"); return TP_ENULL; }
  if (!dims3_ok(n1, n2, n3) || c < 1 || l < 1 || rank < 0) { set_error("tcur: invalid sizes"); return TP_EINVAL; }
  if (prob_mode != TP_PROB_A2 && prob_mode != TP_PROB_GIVEN) {
    set_error("tcur: prob_mode must be TP_PROB_A2 or TP_PROB_GIVEN");
    return TP_EINVAL;
  }
  if (prob_mode == TP_PROB_GIVEN && !p_cols) { set_error("tcur: TP_PROB_GIVEN needs p_cols"); return TP_ENULL; }
  if ((n1 < n2 ? n1 : n2) > 512 || (n1 > n2 ? n1 : n2) > 4096) {
    set_error("tcur: needs min(n1, n2) <= 512 and max(n1, n2) <= 4096");
    return TP_EUNSUPPORTED;
  }
  if (n3 > 512) { set_error("tcur: n3 > 512 not supported (the gathered transform is direct)"); return TP_EUNSUPPORTED; }
  return tcur_run(A, n1, n2, n3, c, l, rank, seed, prob_mode, p_cols, p_rows, Z, col_idx, col_count,
                  row_idx, row_count, row_prob, opts, as_stream(stream));
}

int cur_tnn(const float* X, const uint8_t* mask, int64_t n1, int64_t n2, int64_t n3, int64_t c,
            int64_t l, int rank, uint64_t seed, int prob_mode, const double* p_cols,
            const double* p_rows, int iters, double lambda, double mu0, double rho, double mu_max,
            double pinv_rtol, float* L, float* Ct, float* Rt, int32_t* col_idx,
            int64_t* col_count, int32_t* row_idx, int64_t* row_count, double* row_prob,
            const tp_opts* opts, void* stream) {
  if (!X || !L) { set_error("cur_tnn: NULL tensor"); return TP_ENULL; }
  if (!dims3_ok(n1, n2, n3) || c < 1 || l < 1 || rank < 0 || iters < 0 || !(mu0 > 0.0) ||
      !(rho > 0.0) || !(mu_max > 0.0) || lambda < 0.0 || pinv_rtol < 0.0) {
    set_error("cur_tnn: invalid sizes or constants");
    return TP_EINVAL;
  }
  if (prob_mode != TP_PROB_A2 && prob_mode != TP_PROB_GIVEN) {
    set_error("cur_tnn: prob_mode must be TP_PROB_A2 or TP_PROB_GIVEN");
    return TP_EINVAL;
  }
  if (prob_mode == TP_PROB_GIVEN && !p_cols) { set_error("cur_tnn: TP_PROB_GIVEN needs p_cols"); return TP_ENULL; }
  if ((n1 < n2 ? n1 : n2) > 512 || (n1 > n2 ? n1 : n2) > 4096) {
    set_error("cur_tnn: needs min(n1, n2) <= 512 and max(n1, n2) <= 4096");
    return TP_EUNSUPPORTED;
  }
  if (n3 > 512 && !fft_supported(n3)) {
    set_error("cur_tnn: n3 > 512 must factor into radices 2..13");
    return TP_EUNSUPPORTED;
  }
  return cur_tnn_run(X, mask, n1, n2, n3, c, l, rank, seed, prob_mode, p_cols, p_rows, iters,
                     lambda, mu0, rho, mu_max, pinv_rtol, L, Ct, Rt, col_idx, col_count, row_idx,
                     row_count, row_prob, opts, as_stream(stream));
}
}
