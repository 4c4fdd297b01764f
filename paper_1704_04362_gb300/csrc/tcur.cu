// t-CUR (Algorithm 5).  Lateral slices are picked as in t-CX (probability
// min{1, c p_j}, Philox stream 0) and rescaled by 1/sqrt(q_j): C.  Horizontal
// slices are picked with probability min{1, l p_i} (Philox stream 1), p_i the
// row leverage of C (eq. colprob_rows_exact with beta = 1: the squared row
// norms of the left singular vectors of every Fourier slice C_hat_k that pass
// MATLAB's pinv cut-off, summed over all n3 frequencies, normalised) or given
// by the caller, and rescaled by D = diag(1/sqrt(q_i)).  Per half-spectrum
// slice k
//     R_hat_k = D S^T A_hat_k,  W_k = D S^T C_hat_k,  U_hat_k = W_k^dagger,
//     Z_hat_k = C_hat_k U_hat_k R_hat_k,
// with W_k^dagger = V_k Sigma_k^{-1} U_k^H over the singular values of W_k
// above MATLAB's cut-off max(l', c') eps(s_max).  Only the picked columns and
// rows of A are transformed (gathering DFTs); the two SVDs are the
// float32-sweeps + float64-refinement ones of svd.cu and the three products
// (C_hat V Sigma^{-1}) (U^H R_hat) run on the facewise complex GEMM in FP32.
// The pick counts c' and l' are read back to the host (the SVDs are sized by
// them).
#include <cmath>

#include "tp_internal.cuh"

namespace tp {

int launch_cgemm(const CGemm& g, cudaStream_t st);
int hybrid_svd(const float* xr, const float* xi, int64_t sX, int64_t ldx, bool conj, int p, int q,
               int batch, float* fr, float* fi, float* qr, float* qi, float* qsig, double* tr,
               double* ti, double* gr, double* gi, double* wr, double* wi, double* sig,
               const int* real_flags, int max_sweeps, int32_t* status, cudaStream_t st);

namespace {

unsigned grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return unsigned(b);
}

// op(X_k) of every rows x cols slice X_k (leading dimension ld, slice stride
// `slice`) into the dense SVD work matrix: X_k itself or its conjugate
// transpose.
__global__ void work_kernel(const float* __restrict__ xr, const float* __restrict__ xi,
                            int64_t rows, int64_t cols, int64_t ld, int64_t slice, int64_t h,
                            bool transpose, float* __restrict__ gr, float* __restrict__ gi) {
  const int64_t per = rows * cols, total = per * h;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = e / per, r = e - k * per;
    const int64_t i = r % rows, j = r / rows;
    const float vr = xr[k * slice + i + ld * j], vi = xi[k * slice + i + ld * j];
    if (!transpose) {
      gr[e] = vr;
      gi[e] = vi;
    } else {
      gr[k * per + j + cols * i] = vr;
      gi[k * per + j + cols * i] = -vi;
    }
  }
}

__global__ void flags_kernel(int* flags, int64_t h, int64_t n3) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < h) flags[k] = (k == 0 || (n3 % 2 == 0 && k == h - 1)) ? 1 : 0;
}

// MATLAB's pinv cut-off of slice k: dim * eps(max_j sig_kj), eps(s) = 2^(e-53)
// for s = f 2^e, f in [0.5, 1).
__global__ void cut_kernel(const double* __restrict__ sig, int m, int64_t h, int64_t dim,
                           double* __restrict__ cut) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= h) return;
  double smax = 0.0;
  for (int j = 0; j < m; ++j) smax = fmax(smax, sig[k * m + j]);
  int ex = 0;
  frexp(smax, &ex);
  cut[k] = smax > 0.0 ? double(dim) * ldexp(1.0, ex - 53) : 0.0;
}

// lev[i] = sum over all n3 frequencies of the squared modulus of row i of the
// kept left singular vectors; the half spectrum stands for its conjugate
// partner, so slices other than 0 and n3/2 count twice.  One thread per row,
// frequencies and columns in a fixed order (deterministic).
__global__ void leverage_kernel(const double* __restrict__ ur, const double* __restrict__ ui,
                                int64_t sU, int64_t ldU, const double* __restrict__ sig,
                                const double* __restrict__ cut, int m, int64_t n1, int64_t h,
                                int64_t n3, double* __restrict__ lev) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n1) return;
  double acc = 0.0;
  for (int64_t k = 0; k < h; ++k) {
    const double w = (k == 0 || (n3 % 2 == 0 && k == h - 1)) ? 1.0 : 2.0;
    double s = 0.0;
    for (int j = 0; j < m; ++j) {
      const double sj = sig[k * m + j];
      if (sj > cut[k] && sj > 0.0) {
        const double a = ur[k * sU + i + ldU * j], b = ui[k * sU + i + ldU * j];
        s += a * a + b * b;
      }
    }
    acc += w * s;
  }
  lev[i] = acc;
}

// p_i = lev_i / sum lev (zeros when the sum is zero).  One block; the sum is
// a fixed-order tree.
__global__ void normalize_kernel(const double* __restrict__ lev, int64_t n,
                                 double* __restrict__ p) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += lev[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double tot = red[0];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) p[i] = tot > 0.0 ? lev[i] / tot : 0.0;
}

// W_k = D S^T C_hat_k: row r of W_k is row idx[r] of C_hat_k times scale[r].
__global__ void row_gather_kernel(const float* __restrict__ cr, const float* __restrict__ ci,
                                  int64_t n1, int64_t cp, const int32_t* __restrict__ idx,
                                  const float* __restrict__ scale, int64_t lp, int64_t h,
                                  float* __restrict__ wr, float* __restrict__ wi) {
  const int64_t per = lp * cp, total = per * h;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = e / per, rem = e - k * per;
    const int64_t r = rem % lp, j = rem / lp;
    const int64_t src = k * n1 * cp + idx[r] + n1 * j;
    const float s = scale[r];
    wr[e] = s * cr[src];
    wi[e] = s * ci[src];
  }
}

// The pseudo-inverse's two factors from the SVD W_k = U Sigma V^H (lp x cp,
// m = min(lp, cp) singular triplets): Vs = V Sigma^{-1} (cp x m) and
// Uh = U^H (m x lp), float32; triplets at or below the cut-off are zero.
__global__ void pinv_factors_kernel(const double* __restrict__ ur, const double* __restrict__ ui,
                                    int64_t sU, const double* __restrict__ vr,
                                    const double* __restrict__ vi, int64_t sV,
                                    const double* __restrict__ sig,
                                    const double* __restrict__ cut, int m, int64_t lp, int64_t cp,
                                    int64_t h, float* __restrict__ vsr, float* __restrict__ vsi,
                                    float* __restrict__ uhr, float* __restrict__ uhi) {
  const int64_t per_v = cp * m, per_u = lp * m;
  const int64_t total = (per_v + per_u) * h;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    if (e < per_v * h) {
      const int64_t k = e / per_v, rem = e - k * per_v;
      const int64_t i = rem % cp, j = rem / cp;
      const double sj = sig[k * m + j];
      const bool keep = sj > cut[k] && sj > 0.0;
      vsr[e] = keep ? float(vr[k * sV + i + cp * j] / sj) : 0.f;
      vsi[e] = keep ? float(vi[k * sV + i + cp * j] / sj) : 0.f;
    } else {
      const int64_t f = e - per_v * h;
      const int64_t k = f / per_u, rem = f - k * per_u;
      const int64_t i = rem % lp, j = rem / lp;       // U(i, j) -> Uh(j, i)
      const double sj = sig[k * m + j];
      const bool keep = sj > cut[k] && sj > 0.0;
      uhr[k * per_u + j + int64_t(m) * i] = keep ? float(ur[k * sU + i + lp * j]) : 0.f;
      uhi[k * per_u + j + int64_t(m) * i] = keep ? float(-ui[k * sU + i + lp * j]) : 0.f;
    }
  }
}

__global__ void zero_kernel(double* p, int64_t n, int64_t* count) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0;
  if (i == 0 && count) *count = 0;
}

int read_count(const int64_t* dev, int64_t* host, const char* what, cudaStream_t st) {
  if (cudaMemcpyAsync(host, dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    set_error(what);
    return TP_ECUDA;
  }
  return TP_OK;
}

}  // namespace

size_t tcur_ws(int64_t n1, int64_t n2, int64_t n3) {
  const size_t h = size_t(half_len(n3));
  const size_t m = size_t(n1 < n2 ? n1 : n2);
  const size_t P = size_t(n1 > n2 ? n1 : n2);
  const size_t N1 = size_t(n1), N2 = size_t(n2);
  const size_t part = norms_partial_count(n1, n2, n3, 0);
  return ws_bytes(N2, 8) + ws_bytes(part, 8)               // lateral norms
         + ws_bytes(N2, 4) + ws_bytes(N2, 4) + ws_bytes(1, 8)  // column picks
         + ws_bytes(N1, 4) + ws_bytes(N1, 4) + ws_bytes(1, 8)  // row picks
         + 2 * ws_bytes(N1, 8)                             // leverage, row probabilities
         + ws_bytes(h, 8) + ws_bytes(h, 4)                 // cut-offs, real-slice flags
         + 2 * ws_bytes(N1 * N2 * h, 4)                    // C_hat (c' <= n2)
         + 2 * ws_bytes(N1 * N2 * h, 4)                    // R_hat (l' <= n1)
         + 2 * ws_bytes(N1 * N2 * h, 4)                    // W = D S^T C_hat
         + 2 * ws_bytes(P * m * h, 4)                      // SVD: float32 work matrix
         + 2 * ws_bytes(m * m * h, 4) + ws_bytes(m * h, 4) // SVD: float32 rotations, norms
         + 2 * ws_bytes(m * m * h, 8)                      // SVD: Newton-Schulz factor
         + 2 * ws_bytes(P * m * h, 8)                      // SVD: G
         + 2 * ws_bytes(m * m * h, 8)                      // SVD: V of the Jacobi
         + ws_bytes(m * h, 8)                              // singular values
         + 2 * ws_bytes(N2 * m * h, 4)                     // V Sigma^{-1}
         + 2 * ws_bytes(m * N1 * h, 4)                     // U^H
         + 2 * ws_bytes(N1 * m * h, 4)                     // C_hat V Sigma^{-1}
         + 2 * ws_bytes(m * N2 * h, 4)                     // U^H R_hat
         + 2 * ws_bytes(N1 * N2 * h, 4);                   // Z_hat
}

int tcur_run(const float* A, int64_t n1, int64_t n2, int64_t n3, int64_t c, int64_t l,
             uint64_t seed, int prob_mode, const double* p_cols, const double* p_rows, float* Z,
             int32_t* col_idx, int64_t* col_count, int32_t* row_idx, int64_t* row_count,
             double* row_prob, const tp_opts* opts, cudaStream_t st) {
  const int64_t h = half_len(n3);
  Arena ws;
  int rc = acquire_workspace(opts, tcur_ws(n1, n2, n3), &ws);
  if (rc) return rc;
  int32_t* status = opts ? opts->status : nullptr;
  const int64_t m_cap = n1 < n2 ? n1 : n2;
  const int64_t P_cap = n1 > n2 ? n1 : n2;
  double* a2 = ws.take<double>(n2);
  double* part = ws.take<double>(norms_partial_count(n1, n2, n3, 0));
  int32_t* cidx_ws = ws.take<int32_t>(n2);
  float* cscale = ws.take<float>(n2);
  int64_t* ccnt_ws = ws.take<int64_t>(1);
  int32_t* ridx_ws = ws.take<int32_t>(n1);
  float* rscale = ws.take<float>(n1);
  int64_t* rcnt_ws = ws.take<int64_t>(1);
  double* lev = ws.take<double>(n1);
  double* prow_ws = ws.take<double>(n1);
  double* cut = ws.take<double>(h);
  int* flags = ws.take<int>(h);
  float* Cr = ws.take<float>(size_t(n1) * n2 * h);
  float* Ci = ws.take<float>(size_t(n1) * n2 * h);
  float* Rr = ws.take<float>(size_t(n1) * n2 * h);
  float* Ri = ws.take<float>(size_t(n1) * n2 * h);
  float* Wr = ws.take<float>(size_t(n1) * n2 * h);
  float* Wi = ws.take<float>(size_t(n1) * n2 * h);
  float* Fr = ws.take<float>(size_t(P_cap) * m_cap * h);
  float* Fi = ws.take<float>(size_t(P_cap) * m_cap * h);
  float* Qr = ws.take<float>(size_t(m_cap) * m_cap * h);
  float* Qi = ws.take<float>(size_t(m_cap) * m_cap * h);
  float* qsig = ws.take<float>(size_t(m_cap) * h);
  double* NSr = ws.take<double>(size_t(m_cap) * m_cap * h);
  double* NSi = ws.take<double>(size_t(m_cap) * m_cap * h);
  double* Gr = ws.take<double>(size_t(P_cap) * m_cap * h);
  double* Gi = ws.take<double>(size_t(P_cap) * m_cap * h);
  double* Vr = ws.take<double>(size_t(m_cap) * m_cap * h);
  double* Vi = ws.take<double>(size_t(m_cap) * m_cap * h);
  double* sig = ws.take<double>(size_t(m_cap) * h);
  float* VSr = ws.take<float>(size_t(n2) * m_cap * h);
  float* VSi = ws.take<float>(size_t(n2) * m_cap * h);
  float* UHr = ws.take<float>(size_t(m_cap) * n1 * h);
  float* UHi = ws.take<float>(size_t(m_cap) * n1 * h);
  float* Xr = ws.take<float>(size_t(n1) * m_cap * h);
  float* Xi = ws.take<float>(size_t(n1) * m_cap * h);
  float* Yr = ws.take<float>(size_t(m_cap) * n2 * h);
  float* Yi = ws.take<float>(size_t(m_cap) * n2 * h);
  float* Zr = ws.take<float>(size_t(n1) * n2 * h);
  float* Zi = ws.take<float>(size_t(n1) * n2 * h);
  int32_t* cidx = col_idx ? col_idx : cidx_ws;
  int64_t* ccnt = col_count ? col_count : ccnt_ws;
  int32_t* ridx = row_idx ? row_idx : ridx_ws;
  int64_t* rcnt = row_count ? row_count : rcnt_ws;
  double* prow = row_prob ? row_prob : prow_ws;
  const int sweeps = (opts && opts->max_sweeps > 0) ? opts->max_sweeps : 30;
  const size_t zbytes = sizeof(float) * size_t(n1) * n2 * n3;

  // 1. lateral picks (Algorithm 4's draw, stream 0)
  if (prob_mode == TP_PROB_A2)
    if ((rc = launch_slice_norms(A, n1, n2, n3, 0, a2, part, st))) return rc;
  const double* w = prob_mode == TP_PROB_GIVEN ? p_cols : a2;
  if ((rc = launch_draw(w, nullptr, n2, c, seed, prob_mode, 0u, cidx, cscale, ccnt, nullptr, st)))
    return rc;
  int64_t cp = 0;
  if ((rc = read_count(ccnt, &cp, "tcur: reading the number of picked lateral slices failed", st)))
    return rc;
  if (cp == 0) {
    {
      KernelScope ks("tcur_zero", st);
      zero_kernel<<<grid_n(n1), 256, 0, st>>>(prow, n1, rcnt);
    }
    if (cudaMemsetAsync(Z, 0, zbytes, st) != cudaSuccess) {
      set_error("tcur: cudaMemsetAsync failed");
      return TP_ECUDA;
    }
    return launch_status("tcur_zero");
  }
  // 2. C_hat: gathering DFT of the picked lateral slices, rescaled
  DftGather gc{A, n1, cp, 1, n1, n1 * n2, cidx, cscale, ccnt, 2, n3, Cr, Ci, n1, n1 * cp,
               nullptr, nullptr, 0, 0};
  if ((rc = launch_rdft(gc, st))) return rc;
  {
    KernelScope ks("tcur_flags", st);
    flags_kernel<<<unsigned((h + 255) / 256), 256, 0, st>>>(flags, h, n3);
  }

  // 3. row probabilities: leverage of C (or given)
  if (!p_rows) {
    const bool tr = n1 < cp;
    const int64_t p = tr ? cp : n1, q = tr ? n1 : cp;
    {
      KernelScope ks("tcur_work", st);
      work_kernel<<<grid_n(n1 * cp * h), 256, 0, st>>>(Cr, Ci, n1, cp, n1, n1 * cp, h, tr, Fr, Fi);
    }
    if ((rc = hybrid_svd(Cr, Ci, n1 * cp, n1, tr, int(p), int(q), int(h), Fr, Fi, Qr, Qi, qsig,
                         NSr, NSi, Gr, Gi, Vr, Vi, sig, flags, sweeps, status, st)))
      return rc;
    {
      KernelScope ks("tcur_leverage", st);
      cut_kernel<<<unsigned((h + 255) / 256), 256, 0, st>>>(sig, int(q), h, p, cut);
      // left singular vectors of C_hat_k: G (n1 x q) or, transposed, V (n1 x n1)
      if (!tr)
        leverage_kernel<<<grid_n(n1), 256, 0, st>>>(Gr, Gi, p * q, n1, sig, cut, int(q), n1, h,
                                                    n3, lev);
      else
        leverage_kernel<<<grid_n(n1), 256, 0, st>>>(Vr, Vi, q * q, n1, sig, cut, int(q), n1, h,
                                                    n3, lev);
      normalize_kernel<<<1, 256, 0, st>>>(lev, n1, prow);
    }
    note_launches(2);
    if ((rc = launch_status("tcur_leverage"))) return rc;
  } else if (prow != p_rows) {
    if (cudaMemcpyAsync(prow, p_rows, sizeof(double) * n1, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess) {
      set_error("tcur: copying the given row probabilities failed");
      return TP_ECUDA;
    }
  }

  // 4. horizontal picks (stream 1)
  if ((rc = launch_draw(prow, nullptr, n1, l, seed, TP_PROB_GIVEN, 1u, ridx, rscale, rcnt, nullptr,
                        st)))
    return rc;
  int64_t lp = 0;
  if ((rc = read_count(rcnt, &lp, "tcur: reading the number of picked horizontal slices failed",
                       st)))
    return rc;
  if (lp == 0) {
    if (cudaMemsetAsync(Z, 0, zbytes, st) != cudaSuccess) {
      set_error("tcur: cudaMemsetAsync failed");
      return TP_ECUDA;
    }
    return TP_OK;
  }

  // 5. R_hat = D S^T A_hat (gathering DFT of the picked rows), W = D S^T C_hat
  DftGather gr{A, lp, n2, 1, n1, n1 * n2, ridx, rscale, rcnt, 1, n3, Rr, Ri, lp, lp * n2,
               nullptr, nullptr, 0, 0};
  if ((rc = launch_rdft(gr, st))) return rc;
  const bool tw = lp < cp;
  const int64_t pw = tw ? cp : lp, qw = tw ? lp : cp;   // m = qw triplets
  {
    KernelScope ks("tcur_wgather", st);
    row_gather_kernel<<<grid_n(lp * cp * h), 256, 0, st>>>(Cr, Ci, n1, cp, ridx, rscale, lp, h,
                                                           Wr, Wi);
    work_kernel<<<grid_n(lp * cp * h), 256, 0, st>>>(Wr, Wi, lp, cp, lp, lp * cp, h, tw, Fr, Fi);
  }
  note_launches(1);
  // 6. W = U Sigma V^H
  if ((rc = hybrid_svd(Wr, Wi, lp * cp, lp, tw, int(pw), int(qw), int(h), Fr, Fi, Qr, Qi, qsig,
                       NSr, NSi, Gr, Gi, Vr, Vi, sig, flags, sweeps, status, st)))
    return rc;
  {
    KernelScope ks("tcur_pinv", st);
    cut_kernel<<<unsigned((h + 255) / 256), 256, 0, st>>>(sig, int(qw), h, pw, cut);
    // not transposed: U = G (lp x m), V = Jacobi V (cp x cp); transposed
    // (SVD of W^H): V = G (cp x m), U = Jacobi V (lp x lp)
    const int64_t per = (cp + lp) * qw * h;
    if (!tw)
      pinv_factors_kernel<<<grid_n(per), 256, 0, st>>>(Gr, Gi, pw * qw, Vr, Vi, qw * qw, sig, cut,
                                                       int(qw), lp, cp, h, VSr, VSi, UHr, UHi);
    else
      pinv_factors_kernel<<<grid_n(per), 256, 0, st>>>(Vr, Vi, qw * qw, Gr, Gi, pw * qw, sig, cut,
                                                       int(qw), lp, cp, h, VSr, VSi, UHr, UHi);
  }
  note_launches(1);
  if ((rc = launch_status("tcur_pinv"))) return rc;
  const int64_t m = qw;
  // 7. X = C_hat (V Sigma^{-1}) (n1 x m), Y = U^H R_hat (m x n2), Z_hat = X Y
  CGemm g1{Cr, Ci, VSr, VSi, Xr, Xi, n1, m, cp, nullptr, n1, cp, n1, n1 * cp, cp * m, n1 * m, h,
           n3, TP_FP32, nullptr, nullptr, nullptr, nullptr, cp, status};
  if ((rc = launch_cgemm(g1, st))) return rc;
  CGemm g2{UHr, UHi, Rr, Ri, Yr, Yi, m, n2, lp, nullptr, m, lp, m, m * lp, lp * n2, m * n2, h, n3,
           TP_FP32, nullptr, nullptr, nullptr, nullptr, lp, status};
  if ((rc = launch_cgemm(g2, st))) return rc;
  CGemm g3{Xr, Xi, Yr, Yi, Zr, Zi, n1, n2, m, nullptr, n1, m, n1, n1 * m, m * n2, n1 * n2, h, n3,
           TP_FP32, nullptr, nullptr, nullptr, nullptr, m, status};
  if ((rc = launch_cgemm(g3, st))) return rc;
  return launch_irdft(Zr, Zi, n1 * n2, n1 * n2, n3, Z, st);
}

}  // namespace tp
