// t-CUR (Algorithm 5) and CUR t-NN (Algorithm 6).
//
// t-CUR.  Lateral slices are picked as in t-CX (probability
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
// them).  With a rank parameter r > 0 (Algorithm 5's input) the leverage uses
// only the top r left singular vectors of each slice.
//
// CUR t-NN.  The lateral picks C and horizontal picks R of X (not rescaled;
// rows by the top-r leverage of C) are each denoised by the ADMM of
// Algorithm 7: the robust form of problem tlow7, or with a mask the
// completion form of problem tlow6.  The two ADMM runs are independent and
// run concurrently (the batched runner of svt.cu, graph-replayed
// iterations).  Then W~ = the picked rows of C~, U~ = W~^dagger over the
// singular values above rtol * s_max, and L~ = C~ * U~ * R~.
#include <cmath>

#include "tp_internal.cuh"

namespace tp {

int launch_cgemm(const CGemm& g, cudaStream_t st);
size_t svt_ws(int64_t n1, int64_t n2, int64_t n3, int prec = TP_FP32);
int svt_batched_run(int ntens, const tp_tensor_desc* d, int iters, double rho, double mu_max,
                    const tp_opts* opts, cudaStream_t st, const double* lams);
int hybrid_svd(const float* xr, const float* xi, int64_t sX, int64_t ldx, bool conj, int p, int q,
               int batch, float* fr, float* fi, float* qr, float* qi, float* qsig, double* tr,
               double* ti, double* gr, double* gi, double* wr, double* wi, double* sig,
               const int* real_flags, int max_sweeps, int32_t* status, cudaStream_t st,
               bool polish = true);

namespace {

unsigned grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > int64_t(sm_count()) * 16) b = int64_t(sm_count()) * 16;
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

// Which singular triplets of slice k are kept: sig_kj above the cut-off and,
// with rank > 0, among the `rank` largest of the slice (ties broken by the
// index).  The cut-off is rtol * s_max for rtol > 0, else MATLAB's pinv
// default dim * eps(s_max), eps(s) = 2^(e-53) for s = f 2^e, f in [0.5, 1).
// One thread per (k, j).
__global__ void keep_kernel(const double* __restrict__ sig, int m, int64_t h, int64_t dim,
                            double rtol, int rank, uint8_t* __restrict__ keep) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= h * m) return;
  const int64_t k = e / m;
  const int j = int(e - k * m);
  const double* s = sig + k * m;
  double smax = 0.0;
  int above = 0;
  for (int i = 0; i < m; ++i) {
    smax = fmax(smax, s[i]);
    above += (s[i] > s[j] || (s[i] == s[j] && i < j)) ? 1 : 0;
  }
  int ex = 0;
  frexp(smax, &ex);
  const double cut = rtol > 0.0 ? rtol * smax : (smax > 0.0 ? double(dim) * ldexp(1.0, ex - 53) : 0.0);
  keep[e] = (s[j] > cut && s[j] > 0.0 && (rank <= 0 || above < rank)) ? 1 : 0;
}

// lev[i] = sum over all n3 frequencies of the squared modulus of row i of the
// kept left singular vectors; the half spectrum stands for its conjugate
// partner, so slices other than 0 and n3/2 count twice.  One thread per row,
// frequencies and columns in a fixed order (deterministic).
__global__ void leverage_kernel(const double* __restrict__ ur, const double* __restrict__ ui,
                                int64_t sU, int64_t ldU, const uint8_t* __restrict__ keep, int m,
                                int64_t n1, int64_t h, int64_t n3, double* __restrict__ lev) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n1) return;
  double acc = 0.0;
  for (int64_t k = 0; k < h; ++k) {
    const double w = (k == 0 || (n3 % 2 == 0 && k == h - 1)) ? 1.0 : 2.0;
    double s = 0.0;
    for (int j = 0; j < m; ++j) {
      if (keep[k * m + j]) {
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

// W_k = D S^T C_hat_k: row r of W_k is row idx[r] of C_hat_k times scale[r]
// (1 without a scale).
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
    const float s = scale ? scale[r] : 1.0f;
    wr[e] = s * cr[src];
    wi[e] = s * ci[src];
  }
}

// The pseudo-inverse's two factors from the SVD W_k = U Sigma V^H (lp x cp,
// m = min(lp, cp) singular triplets): Vs = V Sigma^{-1} (cp x m) and
// Uh = U^H (m x lp), float32; triplets not kept are zero.
__global__ void pinv_factors_kernel(const double* __restrict__ ur, const double* __restrict__ ui,
                                    int64_t sU, const double* __restrict__ vr,
                                    const double* __restrict__ vi, int64_t sV,
                                    const double* __restrict__ sig,
                                    const uint8_t* __restrict__ keep, int m, int64_t lp, int64_t cp,
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
      const bool kept = keep[k * m + j] != 0;
      vsr[e] = kept ? float(vr[k * sV + i + cp * j] / sj) : 0.f;
      vsi[e] = kept ? float(vi[k * sV + i + cp * j] / sj) : 0.f;
    } else {
      const int64_t f = e - per_v * h;
      const int64_t k = f / per_u, rem = f - k * per_u;
      const int64_t i = rem % lp, j = rem / lp;       // U(i, j) -> Uh(j, i)
      const bool kept = keep[k * m + j] != 0;
      uhr[k * per_u + j + int64_t(m) * i] = kept ? float(ur[k * sU + i + lp * j]) : 0.f;
      uhi[k * per_u + j + int64_t(m) * i] = kept ? float(-ui[k * sU + i + lp * j]) : 0.f;
    }
  }
}

__global__ void zero_kernel(double* p, int64_t n, int64_t* count) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    p[i] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && count) *count = 0;
}

// P_Omega(X): the entries the mask marks observed, zero elsewhere.
__global__ void observed_kernel(const float* __restrict__ x, const uint8_t* __restrict__ mask,
                                int64_t n, float* __restrict__ out) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x)
    out[e] = mask[e] ? x[e] : 0.f;
}

// The picked lateral slices X(:, idx, :) as a compact n1 x cp x n3 tensor
// (and the same slices of the mask).
__global__ void lateral_gather_kernel(const float* __restrict__ x, const uint8_t* __restrict__ mask,
                                      int64_t n1, int64_t n2, int64_t cp, int64_t n3,
                                      const int32_t* __restrict__ idx, float* __restrict__ out,
                                      uint8_t* __restrict__ mout) {
  const int64_t total = n1 * cp * n3;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e % n1, r = e / n1;
    const int64_t j = r % cp, t = r / cp;
    const int64_t src = i + n1 * (int64_t(idx[j]) + n2 * t);
    out[e] = x[src];
    if (mask) mout[e] = mask[src];
  }
}

// The picked horizontal slices X(idx, :, :) as a compact lp x n2 x n3 tensor.
__global__ void horizontal_gather_kernel(const float* __restrict__ x,
                                         const uint8_t* __restrict__ mask, int64_t n1, int64_t n2,
                                         int64_t lp, int64_t n3, const int32_t* __restrict__ idx,
                                         float* __restrict__ out, uint8_t* __restrict__ mout) {
  const int64_t total = lp * n2 * n3;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e % lp, c = e / lp;             // c = j + n2 t
    const int64_t src = int64_t(idx[r]) + n1 * c;
    out[e] = x[src];
    if (mask) mout[e] = mask[src];
  }
}

__global__ void set_kernel(double* p, int n, double v) {
  if (int(threadIdx.x) < n) p[threadIdx.x] = v;
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

// Scratch of the leverage and pseudo-inverse stages, sized for the largest
// pick counts (c' <= n2, l' <= n1).
struct CurBufs {
  int* flags;
  uint8_t* keep;
  double* lev;
  float *Wr, *Wi, *Fr, *Fi, *Qr, *Qi, *qsig;
  double *NSr, *NSi, *Gr, *Gi, *Vr, *Vi, *sig;
  float *VSr, *VSi, *UHr, *UHi, *Xr, *Xi, *Yr, *Yi, *Zr, *Zi;
};

size_t cur_bufs_ws(int64_t n1, int64_t n2, int64_t n3) {
  const size_t h = size_t(half_len(n3));
  const size_t m = size_t(n1 < n2 ? n1 : n2);
  const size_t P = size_t(n1 > n2 ? n1 : n2);
  const size_t N1 = size_t(n1), N2 = size_t(n2);
  return ws_bytes(h, 4) + ws_bytes(m * h, 1) + ws_bytes(N1, 8)
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

CurBufs cur_carve(Arena& ws, int64_t n1, int64_t n2, int64_t n3) {
  const size_t h = size_t(half_len(n3));
  const size_t m = size_t(n1 < n2 ? n1 : n2);
  const size_t P = size_t(n1 > n2 ? n1 : n2);
  const size_t N1 = size_t(n1), N2 = size_t(n2);
  CurBufs b{};
  b.flags = ws.take<int>(h);
  b.keep = ws.take<uint8_t>(m * h);
  b.lev = ws.take<double>(N1);
  b.Wr = ws.take<float>(N1 * N2 * h);
  b.Wi = ws.take<float>(N1 * N2 * h);
  b.Fr = ws.take<float>(P * m * h);
  b.Fi = ws.take<float>(P * m * h);
  b.Qr = ws.take<float>(m * m * h);
  b.Qi = ws.take<float>(m * m * h);
  b.qsig = ws.take<float>(m * h);
  b.NSr = ws.take<double>(m * m * h);
  b.NSi = ws.take<double>(m * m * h);
  b.Gr = ws.take<double>(P * m * h);
  b.Gi = ws.take<double>(P * m * h);
  b.Vr = ws.take<double>(m * m * h);
  b.Vi = ws.take<double>(m * m * h);
  b.sig = ws.take<double>(m * h);
  b.VSr = ws.take<float>(N2 * m * h);
  b.VSi = ws.take<float>(N2 * m * h);
  b.UHr = ws.take<float>(m * N1 * h);
  b.UHi = ws.take<float>(m * N1 * h);
  b.Xr = ws.take<float>(N1 * m * h);
  b.Xi = ws.take<float>(N1 * m * h);
  b.Yr = ws.take<float>(m * N2 * h);
  b.Yi = ws.take<float>(m * N2 * h);
  b.Zr = ws.take<float>(N1 * N2 * h);
  b.Zi = ws.take<float>(N1 * N2 * h);
  return b;
}

// Row probabilities from the half spectrum of C (n1 x cp per slice, leading
// dimension n1, slice stride n1 cp): the (top-rank) leverage, normalised.
int row_leverage(const float* Cr, const float* Ci, int64_t n1, int64_t cp, int64_t n3, int rank,
                 const CurBufs& b, double* prow, int sweeps, int32_t* status, cudaStream_t st) {
  const int64_t h = half_len(n3);
  const bool tr = n1 < cp;
  const int64_t p = tr ? cp : n1, q = tr ? n1 : cp;
  {
    KernelScope ks("cur_work", st);
    work_kernel<<<grid_n(n1 * cp * h), 256, 0, st>>>(Cr, Ci, n1, cp, n1, n1 * cp, h, tr, b.Fr, b.Fi);
    flags_kernel<<<unsigned((h + 255) / 256), 256, 0, st>>>(b.flags, h, n3);
  }
  note_launches(1);
  int rc = hybrid_svd(Cr, Ci, n1 * cp, n1, tr, int(p), int(q), int(h), b.Fr, b.Fi, b.Qr, b.Qi,
                      b.qsig, b.NSr, b.NSi, b.Gr, b.Gi, b.Vr, b.Vi, b.sig, b.flags, sweeps, status,
                      st);
  if (rc) return rc;
  {
    KernelScope ks("cur_leverage", st);
    keep_kernel<<<grid_n(h * q), 256, 0, st>>>(b.sig, int(q), h, p, 0.0, rank, b.keep);
    // left singular vectors of C_hat_k: G (n1 x q) or, transposed, V (n1 x n1)
    if (!tr)
      leverage_kernel<<<grid_n(n1), 256, 0, st>>>(b.Gr, b.Gi, p * q, n1, b.keep, int(q), n1, h, n3,
                                                  b.lev);
    else
      leverage_kernel<<<grid_n(n1), 256, 0, st>>>(b.Vr, b.Vi, q * q, n1, b.keep, int(q), n1, h, n3,
                                                  b.lev);
    normalize_kernel<<<1, 256, 0, st>>>(b.lev, n1, prow);
  }
  note_launches(2);
  return launch_status("cur_leverage");
}

// Z = ifft(C_hat_k (D S^T C_hat_k)^dagger R_hat_k): C_hat n1 x cp (leading
// dimension n1, slice stride n1 cp), R_hat lp x n2 (lp, lp n2), rows idx and
// optional scale of the horizontal picks; pseudo-inverse over the singular
// values above rtol * s_max (MATLAB's default cut-off for rtol <= 0).
int cur_combine(const float* Cr, const float* Ci, const float* Rr, const float* Ri,
                const int32_t* ridx, const float* rscale, int64_t n1, int64_t n2, int64_t n3,
                int64_t cp, int64_t lp, double rtol, const CurBufs& b, float* Z, int sweeps,
                int32_t* status, cudaStream_t st) {
  const int64_t h = half_len(n3);
  const bool tw = lp < cp;
  const int64_t pw = tw ? cp : lp, qw = tw ? lp : cp;   // m = qw triplets
  {
    KernelScope ks("cur_wgather", st);
    row_gather_kernel<<<grid_n(lp * cp * h), 256, 0, st>>>(Cr, Ci, n1, cp, ridx, rscale, lp, h,
                                                           b.Wr, b.Wi);
    work_kernel<<<grid_n(lp * cp * h), 256, 0, st>>>(b.Wr, b.Wi, lp, cp, lp, lp * cp, h, tw, b.Fr,
                                                     b.Fi);
    flags_kernel<<<unsigned((h + 255) / 256), 256, 0, st>>>(b.flags, h, n3);
  }
  note_launches(2);
  // W = U Sigma V^H
  int rc = hybrid_svd(b.Wr, b.Wi, lp * cp, lp, tw, int(pw), int(qw), int(h), b.Fr, b.Fi, b.Qr,
                      b.Qi, b.qsig, b.NSr, b.NSi, b.Gr, b.Gi, b.Vr, b.Vi, b.sig, b.flags, sweeps,
                      status, st);
  if (rc) return rc;
  {
    KernelScope ks("cur_pinv", st);
    keep_kernel<<<grid_n(h * qw), 256, 0, st>>>(b.sig, int(qw), h, pw, rtol, 0, b.keep);
    // not transposed: U = G (lp x m), V = Jacobi V (cp x cp); transposed
    // (SVD of W^H): V = G (cp x m), U = Jacobi V (lp x lp)
    const int64_t per = (cp + lp) * qw * h;
    if (!tw)
      pinv_factors_kernel<<<grid_n(per), 256, 0, st>>>(b.Gr, b.Gi, pw * qw, b.Vr, b.Vi, qw * qw,
                                                       b.sig, b.keep, int(qw), lp, cp, h, b.VSr,
                                                       b.VSi, b.UHr, b.UHi);
    else
      pinv_factors_kernel<<<grid_n(per), 256, 0, st>>>(b.Vr, b.Vi, qw * qw, b.Gr, b.Gi, pw * qw,
                                                       b.sig, b.keep, int(qw), lp, cp, h, b.VSr,
                                                       b.VSi, b.UHr, b.UHi);
  }
  note_launches(1);
  if ((rc = launch_status("cur_pinv"))) return rc;
  const int64_t m = qw;
  // X = C_hat (V Sigma^{-1}) (n1 x m), Y = U^H R_hat (m x n2), Z_hat = X Y
  CGemm g1{Cr, Ci, b.VSr, b.VSi, b.Xr, b.Xi, n1, m, cp, nullptr, n1, cp, n1, n1 * cp, cp * m,
           n1 * m, h, n3, TP_FP32, nullptr, nullptr, nullptr, nullptr, cp, status};
  if ((rc = launch_cgemm(g1, st))) return rc;
  CGemm g2{b.UHr, b.UHi, Rr, Ri, b.Yr, b.Yi, m, n2, lp, nullptr, m, lp, m, m * lp, lp * n2, m * n2,
           h, n3, TP_FP32, nullptr, nullptr, nullptr, nullptr, lp, status};
  if ((rc = launch_cgemm(g2, st))) return rc;
  CGemm g3{b.Xr, b.Xi, b.Yr, b.Yi, b.Zr, b.Zi, n1, n2, m, nullptr, n1, m, n1, n1 * m, m * n2,
           n1 * n2, h, n3, TP_FP32, nullptr, nullptr, nullptr, nullptr, m, status};
  if ((rc = launch_cgemm(g3, st))) return rc;
  return launch_irdft(b.Zr, b.Zi, n1 * n2, n1 * n2, n3, Z, st);
}

int zero_output(float* Z, size_t bytes, cudaStream_t st) {
  if (cudaMemsetAsync(Z, 0, bytes, st) != cudaSuccess) {
    set_error("cudaMemsetAsync of the output failed");
    return TP_ECUDA;
  }
  return TP_OK;
}

}  // namespace

size_t tcur_ws(int64_t n1, int64_t n2, int64_t n3) {
  const size_t h = size_t(half_len(n3));
  const size_t N1 = size_t(n1), N2 = size_t(n2);
  const size_t part = norms_partial_count(n1, n2, n3, 0);
  return ws_bytes(N2, 8) + ws_bytes(part, 8)                   // lateral norms
         + ws_bytes(N2, 4) + ws_bytes(N2, 4) + ws_bytes(1, 8)  // column picks
         + ws_bytes(N1, 4) + ws_bytes(N1, 4) + ws_bytes(1, 8)  // row picks
         + ws_bytes(N1, 8)                                     // row probabilities
         + 2 * ws_bytes(N1 * N2 * h, 4)                        // C_hat (c' <= n2)
         + 2 * ws_bytes(N1 * N2 * h, 4)                        // R_hat (l' <= n1)
         + draw_scratch_bytes(n1 > n2 ? n1 : n2)
         + cur_bufs_ws(n1, n2, n3);
}

int tcur_run(const float* A, int64_t n1, int64_t n2, int64_t n3, int64_t c, int64_t l, int rank,
             uint64_t seed, int prob_mode, const double* p_cols, const double* p_rows, float* Z,
             int32_t* col_idx, int64_t* col_count, int32_t* row_idx, int64_t* row_count,
             double* row_prob, const tp_opts* opts, cudaStream_t st) {
  const int64_t h = half_len(n3);
  Arena ws;
  int rc = acquire_workspace(opts, tcur_ws(n1, n2, n3), &ws);
  if (rc) return rc;
  int32_t* status = opts ? opts->status : nullptr;
  double* a2 = ws.take<double>(n2);
  double* part = ws.take<double>(norms_partial_count(n1, n2, n3, 0));
  int32_t* cidx_ws = ws.take<int32_t>(n2);
  float* cscale = ws.take<float>(n2);
  int64_t* ccnt_ws = ws.take<int64_t>(1);
  int32_t* ridx_ws = ws.take<int32_t>(n1);
  float* rscale = ws.take<float>(n1);
  int64_t* rcnt_ws = ws.take<int64_t>(1);
  double* prow_ws = ws.take<double>(n1);
  float* Cr = ws.take<float>(size_t(n1) * n2 * h);
  float* Ci = ws.take<float>(size_t(n1) * n2 * h);
  float* Rr = ws.take<float>(size_t(n1) * n2 * h);
  float* Ri = ws.take<float>(size_t(n1) * n2 * h);
  char* dscr = ws.take<char>(draw_scratch_bytes(n1 > n2 ? n1 : n2));
  const CurBufs b = cur_carve(ws, n1, n2, n3);
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
  if ((rc = launch_draw(w, nullptr, n2, c, seed, prob_mode, 0u, cidx, cscale, ccnt, nullptr, dscr,
                        st)))
    return rc;
  int64_t cp = 0;
  if ((rc = read_count(ccnt, &cp, "tcur: reading the number of picked lateral slices failed", st)))
    return rc;
  if (cp == 0) {
    {
      KernelScope ks("cur_zero", st);
      zero_kernel<<<grid_n(n1), 256, 0, st>>>(prow, n1, rcnt);
    }
    if ((rc = zero_output(Z, zbytes, st))) return rc;
    return launch_status("cur_zero");
  }
  // 2. C_hat: gathering DFT of the picked lateral slices, rescaled
  DftGather gc{A, n1, cp, 1, n1, n1 * n2, cidx, cscale, ccnt, 2, n3, Cr, Ci, n1, n1 * cp,
               nullptr, nullptr, 0, 0};
  if ((rc = launch_rdft(gc, st))) return rc;
  // 3. row probabilities: leverage of C (or given)
  if (!p_rows) {
    if ((rc = row_leverage(Cr, Ci, n1, cp, n3, rank, b, prow, sweeps, status, st))) return rc;
  } else if (prow != p_rows) {
    if (cudaMemcpyAsync(prow, p_rows, sizeof(double) * n1, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess) {
      set_error("tcur: copying the given row probabilities failed");
      return TP_ECUDA;
    }
  }
  // 4. horizontal picks (stream 1)
  if ((rc = launch_draw(prow, nullptr, n1, l, seed, TP_PROB_GIVEN, 1u, ridx, rscale, rcnt, nullptr,
                        dscr, st)))
    return rc;
  int64_t lp = 0;
  if ((rc = read_count(rcnt, &lp, "tcur: reading the number of picked horizontal slices failed",
                       st)))
    return rc;
  if (lp == 0) return zero_output(Z, zbytes, st);
  // 5. R_hat = D S^T A_hat (gathering DFT of the picked rows)
  DftGather gr{A, lp, n2, 1, n1, n1 * n2, ridx, rscale, rcnt, 1, n3, Rr, Ri, lp, lp * n2,
               nullptr, nullptr, 0, 0};
  if ((rc = launch_rdft(gr, st))) return rc;
  // 6-7. Z_hat = C_hat (D S^T C_hat)^dagger R_hat with MATLAB's cut-off
  return cur_combine(Cr, Ci, Rr, Ri, ridx, rscale, n1, n2, n3, cp, lp, 0.0, b, Z, sweeps, status,
                     st);
}

size_t cur_tnn_ws(int64_t n1, int64_t n2, int64_t n3) {
  const size_t h = size_t(half_len(n3));
  const size_t N1 = size_t(n1), N2 = size_t(n2), N = N1 * N2 * size_t(n3);
  const size_t part = norms_partial_count(n1, n2, n3, 0);
  return ws_bytes(N2, 8) + ws_bytes(part, 8)                   // lateral norms
         + ws_bytes(N2, 4) + ws_bytes(N2, 4) + ws_bytes(1, 8)  // column picks
         + ws_bytes(N1, 4) + ws_bytes(N1, 4) + ws_bytes(1, 8)  // row picks
         + ws_bytes(N1, 8) + ws_bytes(2, 8)                    // row probabilities, mu
         + ws_bytes(N, 4)                                      // P_Omega(X)
         + 2 * ws_bytes(N, 4) + 2 * ws_bytes(N, 1)             // C, R and their masks
         + 6 * ws_bytes(N, 4)                                  // ADMM states L, E, Y of C and R
         + 2 * svt_ws(n1, n2, n3)                        // the two ADMM workspaces
         + 2 * ws_bytes(N1 * N2 * h, 4)                        // C~_hat
         + 2 * ws_bytes(N1 * N2 * h, 4)                        // R~_hat
         + draw_scratch_bytes(n1 > n2 ? n1 : n2)
         + cur_bufs_ws(n1, n2, n3);
}

int cur_tnn_run(const float* X, const uint8_t* mask, int64_t n1, int64_t n2, int64_t n3,
                int64_t c, int64_t l, int rank, uint64_t seed, int prob_mode, const double* p_cols,
                const double* p_rows, int iters, double lambda, double mu0, double rho,
                double mu_max, double rtol, float* Lout, float* Ct_out, float* Rt_out,
                int32_t* col_idx, int64_t* col_count, int32_t* row_idx, int64_t* row_count,
                double* row_prob, const tp_opts* opts, cudaStream_t st) {
  const int64_t h = half_len(n3);
  const size_t N = size_t(n1) * n2 * n3;
  Arena ws;
  int rc = acquire_workspace(opts, cur_tnn_ws(n1, n2, n3), &ws);
  if (rc) return rc;
  int32_t* status = opts ? opts->status : nullptr;
  double* a2 = ws.take<double>(n2);
  double* part = ws.take<double>(norms_partial_count(n1, n2, n3, 0));
  int32_t* cidx_ws = ws.take<int32_t>(n2);
  float* cscale = ws.take<float>(n2);
  int64_t* ccnt_ws = ws.take<int64_t>(1);
  int32_t* ridx_ws = ws.take<int32_t>(n1);
  float* rscale = ws.take<float>(n1);
  int64_t* rcnt_ws = ws.take<int64_t>(1);
  double* prow_ws = ws.take<double>(n1);
  double* mu = ws.take<double>(2);
  float* Xo = ws.take<float>(N);
  float* C = ws.take<float>(N);
  float* R = ws.take<float>(N);
  uint8_t* Cm = ws.take<uint8_t>(N);
  uint8_t* Rm = ws.take<uint8_t>(N);
  float* st_ws[6];
  for (int i = 0; i < 6; ++i) st_ws[i] = ws.take<float>(N);
  char* admm_ws = ws.take<char>(2 * svt_ws(n1, n2, n3));
  float* Chr = ws.take<float>(size_t(n1) * n2 * h);
  float* Chi = ws.take<float>(size_t(n1) * n2 * h);
  float* Rhr = ws.take<float>(size_t(n1) * n2 * h);
  float* Rhi = ws.take<float>(size_t(n1) * n2 * h);
  char* dscr = ws.take<char>(draw_scratch_bytes(n1 > n2 ? n1 : n2));
  const CurBufs b = cur_carve(ws, n1, n2, n3);
  int32_t* cidx = col_idx ? col_idx : cidx_ws;
  int64_t* ccnt = col_count ? col_count : ccnt_ws;
  int32_t* ridx = row_idx ? row_idx : ridx_ws;
  int64_t* rcnt = row_count ? row_count : rcnt_ws;
  double* prow = row_prob ? row_prob : prow_ws;
  float* Ct = Ct_out ? Ct_out : st_ws[0];
  float* Rt = Rt_out ? Rt_out : st_ws[3];
  const int sweeps = (opts && opts->max_sweeps > 0) ? opts->max_sweeps : 30;
  const size_t zbytes = sizeof(float) * N;

  // 1. the observed data P_Omega(X) and the lateral picks (stream 0)
  const float* Xd = X;
  if (mask) {
    {
      KernelScope ks("cur_observed", st);
      observed_kernel<<<grid_n(int64_t(N)), 256, 0, st>>>(X, mask, int64_t(N), Xo);
    }
    if ((rc = launch_status("cur_observed"))) return rc;
    Xd = Xo;
  }
  if (prob_mode == TP_PROB_A2)
    if ((rc = launch_slice_norms(Xd, n1, n2, n3, 0, a2, part, st))) return rc;
  const double* w = prob_mode == TP_PROB_GIVEN ? p_cols : a2;
  if ((rc = launch_draw(w, nullptr, n2, c, seed, prob_mode, 0u, cidx, cscale, ccnt, nullptr, dscr,
                        st)))
    return rc;
  int64_t cp = 0;
  if ((rc = read_count(ccnt, &cp, "cur_tnn: reading the number of picked lateral slices failed",
                       st)))
    return rc;
  if (cp == 0) {
    {
      KernelScope ks("cur_zero", st);
      zero_kernel<<<grid_n(n1), 256, 0, st>>>(prow, n1, rcnt);
    }
    if ((rc = zero_output(Lout, zbytes, st))) return rc;
    return launch_status("cur_zero");
  }
  // 2. C = the picked lateral slices (not rescaled), its half spectrum
  {
    KernelScope ks("cur_lateral_gather", st);
    lateral_gather_kernel<<<grid_n(n1 * cp * n3), 256, 0, st>>>(Xd, mask, n1, n2, cp, n3, cidx, C,
                                                                 Cm);
  }
  if ((rc = launch_status("cur_lateral_gather"))) return rc;
  // 3. row probabilities: top-rank leverage of C (or given)
  if (!p_rows) {
    DftGather gc{C, n1 * cp, 1, 1, 0, n1 * cp, nullptr, nullptr, nullptr, 0, n3, Chr, Chi,
                 n1 * cp, n1 * cp, nullptr, nullptr, 0, 0};
    if ((rc = launch_rdft(gc, st))) return rc;
    if ((rc = row_leverage(Chr, Chi, n1, cp, n3, rank, b, prow, sweeps, status, st))) return rc;
  } else if (prow != p_rows) {
    if (cudaMemcpyAsync(prow, p_rows, sizeof(double) * n1, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess) {
      set_error("cur_tnn: copying the given row probabilities failed");
      return TP_ECUDA;
    }
  }
  // 4. horizontal picks (stream 1), R = the picked rows (not rescaled)
  if ((rc = launch_draw(prow, nullptr, n1, l, seed, TP_PROB_GIVEN, 1u, ridx, rscale, rcnt, nullptr,
                        dscr, st)))
    return rc;
  int64_t lp = 0;
  if ((rc = read_count(rcnt, &lp,
                       "cur_tnn: reading the number of picked horizontal slices failed", st)))
    return rc;
  if (lp == 0) return zero_output(Lout, zbytes, st);
  {
    KernelScope ks("cur_horizontal_gather", st);
    horizontal_gather_kernel<<<grid_n(lp * n2 * n3), 256, 0, st>>>(Xd, mask, n1, n2, lp, n3, ridx,
                                                                     R, Rm);
  }
  if ((rc = launch_status("cur_horizontal_gather"))) return rc;
  // 5. C~ = ADMM(C), R~ = ADMM(R), concurrently
  if (cudaMemsetAsync(Ct, 0, sizeof(float) * n1 * cp * n3, st) != cudaSuccess ||
      cudaMemsetAsync(Rt, 0, sizeof(float) * lp * n2 * n3, st) != cudaSuccess) {
    set_error("cur_tnn: clearing the ADMM state failed");
    return TP_ECUDA;
  }
  for (int i : {1, 2, 4, 5})
    if (cudaMemsetAsync(st_ws[i], 0, zbytes, st) != cudaSuccess) {
      set_error("cur_tnn: clearing the ADMM state failed");
      return TP_ECUDA;
    }
  {
    KernelScope ks("cur_mu", st);
    set_kernel<<<1, 32, 0, st>>>(mu, 2, mu0);
  }
  tp_tensor_desc d[2] = {
      {C, mask ? Cm : nullptr, Ct, st_ws[1], st_ws[2], mu, n1, cp, n3},
      {R, mask ? Rm : nullptr, Rt, st_ws[4], st_ws[5], mu + 1, lp, n2, n3}};
  double lams[2] = {0.0, 0.0};
  if (!mask) {
    lams[0] = lambda > 0.0 ? lambda : 1.0 / sqrt(double(n1 > cp ? n1 : cp) * double(n3));
    lams[1] = lambda > 0.0 ? lambda : 1.0 / sqrt(double(lp > n2 ? lp : n2) * double(n3));
  }
  tp_opts sub{};
  if (opts) sub = *opts;
  sub.workspace = admm_ws;
  sub.workspace_bytes = 2 * svt_ws(n1, n2, n3);
  if ((rc = svt_batched_run(2, d, iters, rho, mu_max, &sub, st, lams))) return rc;
  // 6-7. W~ = rows ridx of C~, L~ = C~ W~^dagger R~ per Fourier slice
  DftGather gc2{Ct, n1 * cp, 1, 1, 0, n1 * cp, nullptr, nullptr, nullptr, 0, n3, Chr, Chi,
                n1 * cp, n1 * cp, nullptr, nullptr, 0, 0};
  if ((rc = launch_rdft(gc2, st))) return rc;
  DftGather gr2{Rt, lp * n2, 1, 1, 0, lp * n2, nullptr, nullptr, nullptr, 0, n3, Rhr, Rhi,
                lp * n2, lp * n2, nullptr, nullptr, 0, 0};
  if ((rc = launch_rdft(gr2, st))) return rc;
  return cur_combine(Chr, Chi, Rhr, Rhi, ridx, nullptr, n1, n2, n3, cp, lp, rtol, b, Lout, sweeps,
                     status, st);
}

}  // namespace tp
