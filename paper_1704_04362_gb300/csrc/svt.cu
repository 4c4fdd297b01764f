// Tensor completion by ADMM with tensor singular-value thresholding
// (Algorithm 7 in the completion form of problem (tlow6)).  Per iteration,
// with tau = 1/mu (mu held on the device):
//   M = X_obs - E - Y/mu                         (admm_pre_kernel)
//   L = ifft(SVT_tau(fft(M)))                     (half spectrum, per slice)
//   E = (X_obs - L - Y/mu) off the mask, 0 on it
//   Y = Y + mu (L + E - X_obs)                    (admm_post_kernel)
//   mu = min(rho mu, mu_max)                      (admm_mu_kernel)
// X_obs is X where the mask is set and 0 elsewhere.  The slice SVT takes the
// right singular vectors V from the float32 one-sided Jacobi of svd.cu on a
// copy of M_hat_k (or its conjugate transpose when n1 < n2), warm-started
// from the previous iteration's V (the ADMM iterate moves little between
// iterations, so a sweep or two re-converges), then forms
// H = M_hat_k V in float64 and the singular values as Rayleigh quotients
// s_j = ||h_j|| / ||v_j||: their error is second order in the error of v_j,
// which matters because max(s_j - tau, 0) amplifies the error of any s_j
// close to tau.  The shrunk slice is
// sum_j max(s_j - tau, 0) u_j v_j^H = sum_j c_j h_j v_j^H,
// c_j = max(s_j - tau, 0) / (s_j ||v_j||^2).
#include "tp_internal.cuh"

namespace tp {

int jacobi_float_launch(float* gr, float* gi, int64_t sG, float* vr, float* vi, int64_t sV,
                        float* sig, int p, int q, int batch, int max_sweeps,
                        const int* real_flags, int32_t* status, bool init_v, cudaStream_t st);
int launch_cgemm(const CGemm& g, cudaStream_t st);
int zgemm64_from_float(const float* ar, const float* ai, int64_t sA, int64_t lda, bool conj_a,
                       const float* br, const float* bi, int64_t sB, int64_t ldb, double* cr,
                       double* ci, int64_t sC, int64_t ldc, int M, int N, int K, int batch,
                       cudaStream_t st);

namespace {

__global__ void admm_pre_kernel(const float* __restrict__ X, const uint8_t* __restrict__ mask,
                                const float* __restrict__ E, const float* __restrict__ Y,
                                const double* __restrict__ mu, int64_t n, float* __restrict__ M) {
  const float inv_mu = float(1.0 / *mu);
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x) {
    const float x = mask[e] ? X[e] : 0.f;
    M[e] = x - E[e] - Y[e] * inv_mu;
  }
}

__global__ void admm_post_kernel(const float* __restrict__ X, const uint8_t* __restrict__ mask,
                                 const float* __restrict__ L, float* __restrict__ E,
                                 float* __restrict__ Y, const double* __restrict__ mu, int64_t n) {
  const float m = float(*mu);
  const float inv_mu = float(1.0 / *mu);
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x) {
    const bool obs = mask[e] != 0;
    const float x = obs ? X[e] : 0.f;
    const float y = Y[e];
    const float l = L[e];
    const float enew = obs ? 0.f : (x - l - y * inv_mu);
    E[e] = enew;
    Y[e] = y + m * (l + enew - x);
  }
}

__global__ void admm_mu_kernel(double* mu, double rho, double mu_max) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *mu = fmin(rho * *mu, mu_max);
}

// Work matrix of every slice: G = M_hat_k (n1 x n2) or, when transposed,
// G = M_hat_k^H (n2 x n1).
__global__ void to_work_kernel(const float* __restrict__ xr, const float* __restrict__ xi,
                               int64_t n1, int64_t n2, int64_t h, bool transpose,
                               float* __restrict__ gr, float* __restrict__ gi) {
  const int64_t per = n1 * n2, total = per * h;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = e / per, r = e - k * per;
    const int64_t i = r % n1, j = r / n1;
    if (!transpose) {
      gr[e] = xr[e];
      gi[e] = xi[e];
    } else {
      gr[k * per + j + n2 * i] = xr[e];
      gi[k * per + j + n2 * i] = -xi[e];
    }
  }
}

// Shrinks and rebuilds every slice from V (q x q, float32) and H = W V
// (p x q, float64; W the work matrix): the p x q work-shaped result
// R = sum_j c_j h_j v_j^H, written as the n1 x n2 slice itself, or as its
// conjugate transpose when the work matrix was M_hat^H.
__global__ void svt_rebuild_kernel(const double* __restrict__ hr, const double* __restrict__ hi,
                                   int64_t sH, const float* __restrict__ wr,
                                   const float* __restrict__ wi, int64_t sW, int p, int q,
                                   const double* __restrict__ mu, bool transpose, int64_t n1,
                                   float* __restrict__ outr, float* __restrict__ outi) {
  extern __shared__ float coef[];   // q factors c_j
  const int64_t f = blockIdx.x;
  const double tau = 1.0 / *mu;
  const double* Hr = hr + f * sH;
  const double* Hi = hi + f * sH;
  const float* Wr = wr + f * sW;
  const float* Wi = wi + f * sW;
  for (int j = threadIdx.x; j < q; j += blockDim.x) {
    double nv = 0.0, nh = 0.0;
    for (int b = 0; b < q; ++b) {
      const double x = Wr[b + int64_t(q) * j], y = Wi[b + int64_t(q) * j];
      nv += x * x + y * y;
    }
    for (int a = 0; a < p; ++a) {
      const double x = Hr[a + int64_t(p) * j], y = Hi[a + int64_t(p) * j];
      nh += x * x + y * y;
    }
    const double s = nv > 0.0 ? sqrt(nh / nv) : 0.0;
    coef[j] = s > tau ? float((s - tau) / (s * nv)) : 0.f;
  }
  __syncthreads();
  const int64_t per = int64_t(p) * q;
  for (int64_t e = threadIdx.x; e < per; e += blockDim.x) {
    const int64_t a = e % p, b = e / p;
    float sr = 0.f, si = 0.f;
    for (int j = 0; j < q; ++j) {
      const float c = coef[j];
      if (c == 0.f) continue;
      const float ur = float(Hr[a + int64_t(p) * j]), ui = float(Hi[a + int64_t(p) * j]);
      const float vr = Wr[b + int64_t(q) * j], vi = -Wi[b + int64_t(q) * j];   // conj(V(b, j))
      sr = fmaf(c, ur * vr - ui * vi, sr);
      si = fmaf(c, ur * vi + ui * vr, si);
    }
    if (!transpose) {            // R is the n1 x n2 slice itself
      outr[f * per + a + int64_t(p) * b] = sr;
      outi[f * per + a + int64_t(p) * b] = si;
    } else {                     // R = slice^H: slice(b, a) = conj(R(a, b)), slice is n1 x n2, n1 = q
      outr[f * per + b + n1 * a] = sr;
      outi[f * per + b + n1 * a] = -si;
    }
  }
}

__global__ void flags_kernel(int* flags, int64_t h, int64_t n3) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < h) flags[k] = (k == 0 || (n3 % 2 == 0 && k == h - 1)) ? 1 : 0;
}

unsigned grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return unsigned(b);
}

}  // namespace

size_t svt_ws(int64_t n1, int64_t n2, int64_t n3) {
  const size_t h = size_t(half_len(n3));
  const size_t p = size_t(n1 > n2 ? n1 : n2), q = size_t(n1 < n2 ? n1 : n2);
  const size_t n = size_t(n1) * n2;
  return ws_bytes(n * n3, 4)                  // M (and L, reused)
         + 2 * ws_bytes(n * h, 4)             // M_hat / L_hat
         + 2 * ws_bytes(p * q * h, 4)         // G
         + 2 * ws_bytes(q * q * h, 4)         // V
         + 2 * ws_bytes(p * q * h, 4)         // work matrix (warm start: G = work V)
         + 2 * ws_bytes(p * q * h, 8)         // H = W V (float64)
         + ws_bytes(q * h, 4) + ws_bytes(h, 4);
}

int svt_run(const float* X, const uint8_t* mask, int64_t n1, int64_t n2, int64_t n3, int iters,
            double rho, double mu_max, float* L, float* E, float* Y, double* mu,
            const tp_opts* opts, cudaStream_t st) {
  const int64_t h = half_len(n3);
  const bool transpose = n1 < n2;
  const int64_t p = transpose ? n2 : n1, q = transpose ? n1 : n2;
  const int64_t n = n1 * n2 * n3;
  Arena ws;
  int rc = acquire_workspace(opts, svt_ws(n1, n2, n3), &ws);
  if (rc) return rc;
  int32_t* status = opts ? opts->status : nullptr;
  float* M = ws.take<float>(size_t(n));
  float* Mr = ws.take<float>(size_t(n1) * n2 * h);
  float* Mi = ws.take<float>(size_t(n1) * n2 * h);
  float* Gr = ws.take<float>(size_t(p) * q * h);
  float* Gi = ws.take<float>(size_t(p) * q * h);
  float* Wr = ws.take<float>(size_t(q) * q * h);
  float* Wi = ws.take<float>(size_t(q) * q * h);
  float* Kr = ws.take<float>(size_t(p) * q * h);
  float* Ki = ws.take<float>(size_t(p) * q * h);
  double* Hr = ws.take<double>(size_t(p) * q * h);
  double* Hi = ws.take<double>(size_t(p) * q * h);
  float* sig = ws.take<float>(size_t(q) * h);
  int* flags = ws.take<int>(size_t(h));
  {
    KernelScope ks("svt_flags", st);
    flags_kernel<<<unsigned((h + 255) / 256), 256, 0, st>>>(flags, h, n3);
  }
  const int sweeps = (opts && opts->max_sweeps > 0) ? opts->max_sweeps : 30;
  for (int it = 0; it < iters; ++it) {
    {
      KernelScope ks("admm_pre", st);
      admm_pre_kernel<<<grid_n(n), 256, 0, st>>>(X, mask, E, Y, mu, n, M);
    }
    DftGather gm{M, n1 * n2, 1, 1, 0, n1 * n2, nullptr, nullptr, nullptr, 0, n3, Mr, Mi,
                 n1 * n2, n1 * n2, nullptr, nullptr, 0};
    if ((rc = launch_rdft(gm, st))) return rc;
    const bool warm = it > 0;
    {
      KernelScope ks("svt_work", st);
      to_work_kernel<<<grid_n(n1 * n2 * h), 256, 0, st>>>(Mr, Mi, n1, n2, h, transpose,
                                                         warm ? Kr : Gr, warm ? Ki : Gi);
    }
    if (warm) {   // G = work V_prev
      CGemm gw{Kr, Ki, Wr, Wi, Gr, Gi, p, q, q, nullptr, p, q, p, p * q, q * q, p * q, h, n3,
               TP_FP32, nullptr, nullptr, nullptr, nullptr, q, status};
      if ((rc = launch_cgemm(gw, st))) return rc;
    }
    if ((rc = jacobi_float_launch(Gr, Gi, p * q, Wr, Wi, q * q, sig, int(p), int(q), int(h),
                                  sweeps, flags, status, !warm, st)))
      return rc;
    // H = W V in float64 from the untouched half spectrum (W = M_hat or M_hat^H)
    if ((rc = zgemm64_from_float(Mr, Mi, n1 * n2, n1, transpose, Wr, Wi, q * q, q, Hr, Hi, p * q,
                                 p, int(p), int(q), int(q), int(h), st)))
      return rc;
    {
      KernelScope ks("svt_rebuild", st);
      svt_rebuild_kernel<<<unsigned(h), 256, size_t(q) * sizeof(float), st>>>(
          Hr, Hi, p * q, Wr, Wi, q * q, int(p), int(q), mu, transpose, n1, Mr, Mi);
    }
    if ((rc = launch_irdft(Mr, Mi, n1 * n2, n1 * n2, n3, L, st))) return rc;
    {
      KernelScope ks("admm_post", st);
      admm_post_kernel<<<grid_n(n), 256, 0, st>>>(X, mask, L, E, Y, mu, n);
    }
    {
      KernelScope ks("admm_mu", st);
      admm_mu_kernel<<<1, 32, 0, st>>>(mu, rho, mu_max);
    }
    if ((rc = launch_status("admm iteration"))) return rc;
  }
  return TP_OK;
}

}  // namespace tp
