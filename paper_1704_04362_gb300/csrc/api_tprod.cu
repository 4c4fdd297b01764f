// C entry points of the t-product path: tprod (Algorithm 1), tprod_sampled
// (Algorithm 2) and their stages.  Host code only: argument checks,
// workspace carving and kernel sequencing on the caller's stream.
#include "tp_internal.cuh"

namespace tp {

int launch_cgemm_simt(const CGemm& g, cudaStream_t st);
int launch_cgemm_tc(const CGemm& g, cudaStream_t st);

int launch_cgemm(const CGemm& g, cudaStream_t st) {
  if (g.precision == TP_FP32) return launch_cgemm_simt(g, st);
  if (g.b_conj_trans) {
    set_error("cgemm: a conjugate-transposed B is supported by the FP32 path only");
    return TP_EINVAL;
  }
  if (g.precision == TP_TF32X3 || g.precision == TP_BF16X3) return launch_cgemm_tc(g, st);
  set_error("unknown precision %d", g.precision);
  return TP_EINVAL;
}

namespace {

constexpr int64_t kMaxElems = int64_t(1) << 40;

bool dims_ok(std::initializer_list<int64_t> d) {
  int64_t prod = 1;
  for (int64_t v : d) {
    if (v < 1 || v > (int64_t(1) << 31)) return false;
    if (prod > kMaxElems / v) return false;
    prod *= v;
  }
  return true;
}

int opt_precision(const tp_opts* o) { return o ? o->precision : TP_FP32; }

inline int64_t pad4(int64_t v) { return (v + 3) / 4 * 4; }
bool is_tc(int prec) { return prec == TP_TF32X3 || prec == TP_BF16X3; }
// K leading dimension: 16-byte rows for the tensor maps (4 floats or 8 bf16)
inline int64_t pad_k(int64_t v, int prec) {
  return prec == TP_BF16X3 ? (v + 7) / 8 * 8 : prec == TP_TF32X3 ? pad4(v) : v;
}

// Fourier-domain operand storage of one call: plain planar FP32 for the SIMT
// GEMM, or the 3xTF32 split (hi/lo planes) with leading dimensions padded to
// 4 floats for the tensor-core GEMM's TMA tiles.
struct Planes {
  float *re, *im, *re_lo, *im_lo;
};
size_t planes_bytes(size_t elems, bool tc) { return (tc ? 4 : 2) * ws_bytes(elems, 4); }
Planes take_planes(Arena& ws, size_t elems, bool tc) {
  Planes p{};
  p.re = ws.take<float>(elems);
  p.im = ws.take<float>(elems);
  if (tc) {
    p.re_lo = ws.take<float>(elems);
    p.im_lo = ws.take<float>(elems);
  }
  return p;
}

// Operand layouts.  SIMT: A_hat_k is n1 x K column-major (leading dimension
// n1).  Tensor cores: A_hat_k is stored K-major, element (i, kk) at
// kk + lk*i with lk = K padded to 16 bytes (4 floats for 3xTF32, 8 bf16 for
// BF16x3).  B_hat_k is K-major in both (leading dimension K, padded likewise
// for the tensor cores).  The planes are sized as floats in both splits.
size_t tprod_ws(int64_t n1, int64_t n2, int64_t n4, int64_t n3, int prec) {
  const size_t h = size_t(half_len(n3));
  const bool tc = is_tc(prec);
  const int64_t lk = pad_k(n2, prec);
  return planes_bytes(size_t(tc ? lk : n2) * n1 * h, tc) + planes_bytes(size_t(lk) * n4 * h, tc) +
         2 * ws_bytes(size_t(n1) * n4 * h, 4);
}

size_t sampled_ws(int64_t n1, int64_t n2, int64_t n4, int64_t n3, int prec) {
  const size_t h = size_t(half_len(n3));
  const bool tc = is_tc(prec);
  const int64_t lk = pad_k(n2, prec);
  size_t part = norms_partial_count(n1, n2, n3, 0);
  const size_t p2 = norms_partial_count(n2, n4, n3, 1);
  if (p2 > part) part = p2;
  return 2 * ws_bytes(size_t(n2), 8) + ws_bytes(part, 8) + ws_bytes(size_t(n2), 4) +
         ws_bytes(size_t(n2), 4) + ws_bytes(1, 8) + planes_bytes(size_t(lk) * n1 * h, tc) +
         planes_bytes(size_t(lk) * n4 * h, tc) + 2 * ws_bytes(size_t(n1) * n4 * h, 4) +
         draw_scratch_bytes(n2);
}

}  // namespace

size_t workspace_for(int op, const int64_t* d, int nd, const tp_opts* opts);

}  // namespace tp

using namespace tp;

extern "C" {

int tprod(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t n4,
          int64_t n3, const tp_opts* opts, void* stream) {
  if (!A || !B || !C) { set_error("tprod: NULL tensor"); return TP_ENULL; }
  if (!dims_ok({n1, n2, n3}) || !dims_ok({n2, n4, n3}) || !dims_ok({n1, n4, n3})) {
    set_error("tprod: invalid sizes n1=%lld n2=%lld n4=%lld n3=%lld", (long long)n1,
              (long long)n2, (long long)n4, (long long)n3);
    return TP_EINVAL;
  }
  if (n3 > 512) { set_error("tprod: n3 = %lld > 512 not supported", (long long)n3); return TP_EUNSUPPORTED; }
  const int prec = opt_precision(opts);
  if (prec < TP_FP32 || prec > TP_BF16X3) { set_error("tprod: unknown precision %d", prec); return TP_EINVAL; }
  const bool tc = is_tc(prec);
  cudaStream_t st = as_stream(stream);
  Arena ws;
  int rc = acquire_workspace(opts, tprod_ws(n1, n2, n4, n3, prec), &ws);
  if (rc) return rc;
  const int64_t h = half_len(n3);
  const int64_t lk = pad_k(n2, prec);              // K leading dimension
  const int64_t la = tc ? lk : n1;                 // A leading dimension
  Planes Ah = take_planes(ws, size_t(lk) * n1 * h, tc);
  Planes Bh = take_planes(ws, size_t(lk) * n4 * h, tc);
  float* Cr = ws.take<float>(size_t(n1) * n4 * h);
  float* Ci = ws.take<float>(size_t(n1) * n4 * h);

  DftGather ga{A, n1, n2, 1, n1, n1 * n2, nullptr, nullptr, nullptr, 0, n3,
               Ah.re, Ah.im, la, la * (tc ? n1 : n2), Ah.re_lo, Ah.im_lo, tc ? 1 : 0,
               prec == TP_BF16X3 ? 1 : 0};
  if ((rc = launch_rdft(ga, st))) return rc;
  DftGather gb{B, n2, n4, 1, n2, n2 * n4, nullptr, nullptr, nullptr, 0, n3,
               Bh.re, Bh.im, lk, lk * n4, Bh.re_lo, Bh.im_lo, 0, prec == TP_BF16X3 ? 1 : 0};
  if ((rc = launch_rdft(gb, st))) return rc;
  CGemm g{Ah.re, Ah.im, Bh.re, Bh.im, Cr, Ci, n1, n4, n2, nullptr,
          la, lk, n1, la * (tc ? n1 : n2), lk * n4, n1 * n4, h, n3, prec,
          Ah.re_lo, Ah.im_lo, Bh.re_lo, Bh.im_lo, n2, opts ? opts->status : nullptr,
          opts ? opts->pipeline_wait_limit : 0};
  if ((rc = launch_cgemm(g, st))) return rc;
  return launch_irdft(Cr, Ci, n1 * n4, n1 * n4, n3, C, st);
}

int tprod_sampled(const float* A, const float* B, float* Z, int64_t n1, int64_t n2, int64_t n4,
                  int64_t n3, int64_t c, uint64_t seed, int prob_mode, int sample_mode,
                  const double* p_given, int32_t* idx_out, int64_t* count_out,
                  const tp_opts* opts, void* stream) {
  if (!A || !B || !Z) { set_error("tprod_sampled: NULL tensor"); return TP_ENULL; }
  if (!dims_ok({n1, n2, n3}) || !dims_ok({n2, n4, n3}) || !dims_ok({n1, n4, n3})) {
    set_error("tprod_sampled: invalid sizes");
    return TP_EINVAL;
  }
  if (c < 1) { set_error("tprod_sampled: c must be >= 1"); return TP_EINVAL; }
  if (prob_mode < TP_PROB_AB || prob_mode > TP_PROB_GIVEN) {
    set_error("tprod_sampled: unknown prob_mode %d", prob_mode);
    return TP_EINVAL;
  }
  if (sample_mode != TP_SAMPLE_BERNOULLI && sample_mode != TP_SAMPLE_IID) {
    set_error("tprod_sampled: unknown sample_mode %d", sample_mode);
    return TP_EINVAL;
  }
  if (sample_mode == TP_SAMPLE_IID && c > n2) {
    set_error("tprod_sampled: TP_SAMPLE_IID needs c <= n2");
    return TP_EINVAL;
  }
  if (prob_mode == TP_PROB_GIVEN && !p_given) {
    set_error("tprod_sampled: TP_PROB_GIVEN needs p_given");
    return TP_ENULL;
  }
  if (n3 > 512) { set_error("tprod_sampled: n3 > 512 not supported"); return TP_EUNSUPPORTED; }
  const int prec = opt_precision(opts);
  if (prec < TP_FP32 || prec > TP_BF16X3) { set_error("tprod_sampled: unknown precision %d", prec); return TP_EINVAL; }
  const bool tc = is_tc(prec);
  cudaStream_t st = as_stream(stream);
  Arena ws;
  int rc = acquire_workspace(opts, sampled_ws(n1, n2, n4, n3, prec), &ws);
  if (rc) return rc;
  const int64_t h = half_len(n3);
  const int64_t lk = pad_k(n2, prec);              // K (picked-slice) leading dimension capacity
  const int64_t la = tc ? lk : n1;
  size_t part_n = norms_partial_count(n1, n2, n3, 0);
  const size_t p2 = norms_partial_count(n2, n4, n3, 1);
  if (p2 > part_n) part_n = p2;
  double* a2 = ws.take<double>(n2);
  double* b2 = ws.take<double>(n2);
  double* part = ws.take<double>(part_n);
  int32_t* idx_ws = ws.take<int32_t>(n2);
  float* scale = ws.take<float>(n2);
  int64_t* cnt_ws = ws.take<int64_t>(1);
  Planes Ch = take_planes(ws, size_t(lk) * n1 * h, tc);
  Planes Rh = take_planes(ws, size_t(lk) * n4 * h, tc);
  float* Zr = ws.take<float>(size_t(n1) * n4 * h);
  float* Zi = ws.take<float>(size_t(n1) * n4 * h);
  char* dscr = ws.take<char>(draw_scratch_bytes(n2));
  int32_t* idx = idx_out ? idx_out : idx_ws;
  int64_t* cnt = count_out ? count_out : cnt_ws;

  // S2-S4: slice norms, probabilities and the picking loop
  if (prob_mode != TP_PROB_GIVEN) {
    if ((rc = launch_slice_norms(A, n1, n2, n3, 0, a2, part, st))) return rc;
    if (prob_mode == TP_PROB_AB)
      if ((rc = launch_slice_norms(B, n2, n4, n3, 1, b2, part, st))) return rc;
  }
  const double* w = prob_mode == TP_PROB_GIVEN ? p_given : a2;
  if ((rc = launch_draw(w, b2, n2, c, seed, prob_mode, 0u, idx, scale, cnt, nullptr, dscr, st,
                        sample_mode)))
    return rc;
  // S5 + S1: rescaled gathers fused into the forward transforms.
  // C_hat_k is n1 x c' (capacity n2 columns): column-major for the SIMT GEMM,
  // K-major (picked index contiguous) for the tensor cores.
  DftGather gc{A, n1, n2, 1, n1, n1 * n2, idx, scale, cnt, 2, n3,
               Ch.re, Ch.im, la, la * (tc ? n1 : n2), Ch.re_lo, Ch.im_lo, tc ? 1 : 0,
               prec == TP_BF16X3 ? 1 : 0};
  if ((rc = launch_rdft(gc, st))) return rc;
  // R_hat_k is c' x n4 (leading dimension lk, capacity n2 rows).
  DftGather gr{B, n2, n4, 1, n2, n2 * n4, idx, scale, cnt, 1, n3,
               Rh.re, Rh.im, lk, lk * n4, Rh.re_lo, Rh.im_lo, 0, prec == TP_BF16X3 ? 1 : 0};
  if ((rc = launch_rdft(gr, st))) return rc;
  // S6: facewise products with inner dimension c' read on the device
  CGemm g{Ch.re, Ch.im, Rh.re, Rh.im, Zr, Zi, n1, n4, 0, cnt,
          la, lk, n1, la * (tc ? n1 : n2), lk * n4, n1 * n4, h, n3, prec,
          Ch.re_lo, Ch.im_lo, Rh.re_lo, Rh.im_lo, n2, opts ? opts->status : nullptr,
          opts ? opts->pipeline_wait_limit : 0};
  if ((rc = launch_cgemm(g, st))) return rc;
  // S7: inverse transform
  return launch_irdft(Zr, Zi, n1 * n4, n1 * n4, n3, Z, st);
}

int tp_rdft3(const float* X, int64_t rows, int64_t n3, float* Xr, float* Xi, void* stream) {
  if (!X || !Xr || !Xi) { set_error("tp_rdft3: NULL pointer"); return TP_ENULL; }
  if (!dims_ok({rows, n3})) { set_error("tp_rdft3: invalid sizes"); return TP_EINVAL; }
  DftGather g{X, rows, 1, 1, 0, rows, nullptr, nullptr, nullptr, 0, n3, Xr, Xi, rows, rows,
              nullptr, nullptr, 0};
  return launch_rdft(g, as_stream(stream));
}

int tp_irdft3(const float* Xr, const float* Xi, int64_t rows, int64_t n3, float* Out,
              void* stream) {
  if (!Xr || !Xi || !Out) { set_error("tp_irdft3: NULL pointer"); return TP_ENULL; }
  if (!dims_ok({rows, n3})) { set_error("tp_irdft3: invalid sizes"); return TP_EINVAL; }
  return launch_irdft(Xr, Xi, rows, rows, n3, Out, as_stream(stream));
}

int tp_slice_norms(const float* X, int64_t n1, int64_t n2, int64_t n3, int which, double* out,
                   const tp_opts* opts, void* stream) {
  if (!X || !out) { set_error("tp_slice_norms: NULL pointer"); return TP_ENULL; }
  if (!dims_ok({n1, n2, n3})) { set_error("tp_slice_norms: invalid sizes"); return TP_EINVAL; }
  if (which != 0 && which != 1) { set_error("tp_slice_norms: which must be 0 or 1"); return TP_EINVAL; }
  Arena ws;
  int rc = acquire_workspace(opts, ws_bytes(norms_partial_count(n1, n2, n3, which), 8), &ws);
  if (rc) return rc;
  double* part = ws.take<double>(norms_partial_count(n1, n2, n3, which));
  return launch_slice_norms(X, n1, n2, n3, which, out, part, as_stream(stream));
}

int tp_sample_draw(const double* w, const double* w2, int64_t n, int64_t c, uint64_t seed,
                   int prob_mode, int sample_mode, uint32_t stream_id, int32_t* idx, float* scale,
                   int64_t* count, double* q_out, void* stream) {
  if (!w || !idx || !count) { set_error("tp_sample_draw: NULL pointer"); return TP_ENULL; }
  if (prob_mode == TP_PROB_AB && !w2) { set_error("tp_sample_draw: TP_PROB_AB needs w2"); return TP_ENULL; }
  if (prob_mode < TP_PROB_AB || prob_mode > TP_PROB_GIVEN) { set_error("tp_sample_draw: bad mode"); return TP_EINVAL; }
  if (n < 1 || n > (int64_t(1) << 31) - 1 || c < 1) { set_error("tp_sample_draw: invalid sizes"); return TP_EINVAL; }
  if (sample_mode != TP_SAMPLE_BERNOULLI && sample_mode != TP_SAMPLE_IID) { set_error("tp_sample_draw: bad sample_mode"); return TP_EINVAL; }
  if (sample_mode == TP_SAMPLE_IID && c > n) { set_error("tp_sample_draw: TP_SAMPLE_IID needs c <= n"); return TP_EINVAL; }
  Arena ws;
  int rc = acquire_workspace(nullptr, draw_scratch_bytes(n), &ws);
  if (rc) return rc;
  return launch_draw(w, w2, n, c, seed, prob_mode, stream_id, idx, scale, count, q_out, ws.base,
                     as_stream(stream), sample_mode);
}

int tp_philox4x32_10(const uint32_t* counters, uint32_t k0, uint32_t k1, int64_t n,
                     uint32_t* out, void* stream) {
  if (n < 0 || n > (int64_t(1) << 40)) { set_error("tp_philox4x32_10: invalid n"); return TP_EINVAL; }
  if (n > 0 && (!counters || !out)) { set_error("tp_philox4x32_10: NULL pointer"); return TP_ENULL; }
  return launch_philox_words(counters, k0, k1, n, out, as_stream(stream));
}

size_t tp_workspace_query(int op, const int64_t* d, int nd, const tp_opts* opts) {
  if (!d) return 0;
  switch (op) {
    case TP_OP_TPROD: return nd >= 4 ? tprod_ws(d[0], d[1], d[2], d[3], opt_precision(opts)) : 0;
    case TP_OP_TPROD_SAMPLED:
      return nd >= 4 ? sampled_ws(d[0], d[1], d[2], d[3], opt_precision(opts)) : 0;
    case TP_OP_SLICE_NORMS:
      if (nd < 3) return 0;
      {
        size_t a = norms_partial_count(d[0], d[1], d[2], 0), b = norms_partial_count(d[0], d[1], d[2], 1);
        return ws_bytes(a > b ? a : b, 8);
      }
    default: return tp::workspace_for(op, d, nd, opts);
  }
}

}  // extern "C"
