// t-CX (Algorithm 4): pick lateral slices of A with probability min{1, c p_j}
// (Algorithm 2's picking loop, p_j = ||A(:,j,:)||_F^2 / ||A||_F^2 or given),
// C = the picked slices rescaled by 1/sqrt(q_j), and return the t-project
// Z = C * C^dagger * A (Algorithm 3): per half-spectrum slice
// Z_hat_k = P_k A_hat_k with P_k = C_hat_k C_hat_k^dagger the orthogonal
// projector onto range(C_hat_k).  P_k = U_r U_r^H where U_r are the left
// singular vectors of C_hat_k (float64 one-sided Jacobi) whose singular values
// exceed MATLAB's pinv cut-off max(n1, c') eps(s_max).  The SVD is the
// float32-sweeps + float64-refinement one of svd.cu (float64 accuracy).  The
// number of picks is read back to the host once (the SVD is sized by it).
#include <cmath>

#include "tp_internal.cuh"

namespace tp {

int launch_cgemm(const CGemm& g, cudaStream_t st);
int hybrid_svd(const float* xr, const float* xi, int64_t sX, int64_t ldx, bool conj, int p, int q,
               int batch, float* fr, float* fi, float* qr, float* qi, float* qsig, double* tr,
               double* ti, double* gr, double* gi, double* wr, double* wi, double* sig,
               const int* real_flags, int max_sweeps, int32_t* status, cudaStream_t st,
               bool polish = true);

namespace {

__global__ void work_kernel(const float* __restrict__ xr, const float* __restrict__ xi,
                            int64_t n1, int64_t c, int64_t ld, int64_t slice, int64_t h,
                            bool transpose, float* __restrict__ gr, float* __restrict__ gi) {
  const int64_t per = n1 * c, total = per * h;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = e / per, r = e - k * per;
    const int64_t i = r % n1, j = r / n1;
    const float vr = xr[k * slice + i + ld * j], vi = xi[k * slice + i + ld * j];
    if (!transpose) {
      gr[e] = vr;
      gi[e] = vi;
    } else {
      gr[k * per + j + c * i] = vr;
      gi[k * per + j + c * i] = -vi;
    }
  }
}

// U_r (n1 x m) and U_r^H (m x n1) of every slice, float32 planar; columns
// whose singular value is at or below the cut-off are zero.  `uvec` is the
// matrix holding the left singular vectors (G when not transposed, else W),
// with leading dimension n1.
__global__ void range_basis_kernel(const double* __restrict__ ur, const double* __restrict__ ui,
                                   int64_t sU, const double* __restrict__ sig, int m, int64_t n1,
                                   int64_t cprime, float* __restrict__ br, float* __restrict__ bi,
                                   float* __restrict__ hr, float* __restrict__ hi) {
  __shared__ double cut;
  const int64_t f = blockIdx.x;
  if (threadIdx.x == 0) {
    double smax = 0.0;
    for (int j = 0; j < m; ++j) smax = fmax(smax, sig[f * m + j]);
    int ex = 0;
    frexp(smax, &ex);   // smax = fr * 2^ex, fr in [0.5, 1): eps(smax) = 2^(ex - 53)
    const double eps_s = smax > 0.0 ? ldexp(1.0, ex - 53) : 0.0;
    cut = double(n1 > cprime ? n1 : cprime) * eps_s;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < n1 * m; e += blockDim.x) {
    const int64_t i = e % n1, j = e / n1;
    const bool keep = sig[f * m + j] > cut && sig[f * m + j] > 0.0;
    const float vr = keep ? float(ur[f * sU + i + n1 * j]) : 0.f;
    const float vi = keep ? float(ui[f * sU + i + n1 * j]) : 0.f;
    br[f * n1 * m + e] = vr;
    bi[f * n1 * m + e] = vi;
    hr[f * n1 * m + j + int64_t(m) * i] = vr;
    hi[f * n1 * m + j + int64_t(m) * i] = -vi;
  }
}

__global__ void flags_kernel(int* flags, int64_t h, int64_t n3) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < h) flags[k] = (k == 0 || (n3 % 2 == 0 && k == h - 1)) ? 1 : 0;
}

unsigned grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > int64_t(sm_count()) * 16) b = int64_t(sm_count()) * 16;
  if (b < 1) b = 1;
  return unsigned(b);
}

}  // namespace

size_t tcx_ws(int64_t n1, int64_t n2, int64_t n3) {
  const size_t h = size_t(half_len(n3));
  const size_t m = size_t(n1 < n2 ? n1 : n2);
  const size_t P = size_t(n1 > n2 ? n1 : n2);
  const size_t part = norms_partial_count(n1, n2, n3, 0);
  return ws_bytes(size_t(n2), 8) + ws_bytes(part, 8) + ws_bytes(size_t(n2), 4) +
         ws_bytes(size_t(n2), 4) + ws_bytes(1, 8) +
         2 * ws_bytes(size_t(n1) * n2 * h, 4)      // C_hat (capacity n2 columns)
         + 2 * ws_bytes(size_t(n1) * n2 * h, 4)    // A_hat
         + 2 * ws_bytes(P * m * h, 8)              // SVD: G
         + 2 * ws_bytes(size_t(n2) * n2 * h, 8)    // SVD: W (q <= n2)
         + 2 * ws_bytes(P * m * h, 4)              // SVD: float32 work matrix
         + 2 * ws_bytes(m * m * h, 4)              // SVD: float32 rotations
         + ws_bytes(m * h, 4)                      // SVD: float32 norms
         + 2 * ws_bytes(m * m * h, 8)              // SVD: Newton-Schulz factor
         + ws_bytes(size_t(n2) * h, 8) + ws_bytes(h, 4)
         + 4 * ws_bytes(size_t(n1) * m * h, 4)     // U_r and U_r^H
         + 2 * ws_bytes(m * n2 * h, 4)             // U_r^H A_hat
         + 2 * ws_bytes(size_t(n1) * n2 * h, 4)    // Z_hat
         + draw_scratch_bytes(n2);
}

int tcx_run(const float* A, int64_t n1, int64_t n2, int64_t n3, int64_t c, uint64_t seed,
            int prob_mode, const double* p_given, float* Z, int32_t* idx_out, int64_t* count_out,
            const tp_opts* opts, cudaStream_t st) {
  const int64_t h = half_len(n3);
  Arena ws;
  int rc = acquire_workspace(opts, tcx_ws(n1, n2, n3), &ws);
  if (rc) return rc;
  int32_t* status = opts ? opts->status : nullptr;
  const int64_t m_cap = n1 < n2 ? n1 : n2;
  const int64_t P_cap = n1 > n2 ? n1 : n2;
  double* a2 = ws.take<double>(n2);
  double* part = ws.take<double>(norms_partial_count(n1, n2, n3, 0));
  int32_t* idx_ws = ws.take<int32_t>(n2);
  float* scale = ws.take<float>(n2);
  int64_t* cnt_ws = ws.take<int64_t>(1);
  float* Cr = ws.take<float>(size_t(n1) * n2 * h);
  float* Ci = ws.take<float>(size_t(n1) * n2 * h);
  float* Ar = ws.take<float>(size_t(n1) * n2 * h);
  float* Ai = ws.take<float>(size_t(n1) * n2 * h);
  double* Gr = ws.take<double>(size_t(P_cap) * m_cap * h);
  double* Gi = ws.take<double>(size_t(P_cap) * m_cap * h);
  double* Wr = ws.take<double>(size_t(n2) * n2 * h);
  double* Wi = ws.take<double>(size_t(n2) * n2 * h);
  float* Fr = ws.take<float>(size_t(P_cap) * m_cap * h);
  float* Fi = ws.take<float>(size_t(P_cap) * m_cap * h);
  float* Qr = ws.take<float>(size_t(m_cap) * m_cap * h);
  float* Qi = ws.take<float>(size_t(m_cap) * m_cap * h);
  float* qsig = ws.take<float>(size_t(m_cap) * h);
  double* NSr = ws.take<double>(size_t(m_cap) * m_cap * h);
  double* NSi = ws.take<double>(size_t(m_cap) * m_cap * h);
  double* sig = ws.take<double>(size_t(n2) * h);
  int* flags = ws.take<int>(size_t(h));
  float* Br = ws.take<float>(size_t(n1) * m_cap * h);
  float* Bi = ws.take<float>(size_t(n1) * m_cap * h);
  float* Hr = ws.take<float>(size_t(n1) * m_cap * h);
  float* Hi = ws.take<float>(size_t(n1) * m_cap * h);
  float* Tr = ws.take<float>(size_t(m_cap) * n2 * h);
  float* Ti = ws.take<float>(size_t(m_cap) * n2 * h);
  float* Zr = ws.take<float>(size_t(n1) * n2 * h);
  float* Zi = ws.take<float>(size_t(n1) * n2 * h);
  char* dscr = ws.take<char>(draw_scratch_bytes(n2));
  int32_t* idx = idx_out ? idx_out : idx_ws;
  int64_t* cnt = count_out ? count_out : cnt_ws;

  if (prob_mode == TP_PROB_A2)
    if ((rc = launch_slice_norms(A, n1, n2, n3, 0, a2, part, st))) return rc;
  const double* w = prob_mode == TP_PROB_GIVEN ? p_given : a2;
  if ((rc = launch_draw(w, nullptr, n2, c, seed, prob_mode, 0u, idx, scale, cnt, nullptr, dscr,
                        st)))
    return rc;
  int64_t cprime = 0;
  if (cudaMemcpyAsync(&cprime, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    set_error("tcx: reading the number of picked slices failed");
    return TP_ECUDA;
  }
  if (cprime == 0) {
    if (cudaMemsetAsync(Z, 0, sizeof(float) * size_t(n1) * n2 * n3, st) != cudaSuccess) {
      set_error("tcx: cudaMemsetAsync failed");
      return TP_ECUDA;
    }
    return TP_OK;
  }
  DftGather gc{A, n1, n2, 1, n1, n1 * n2, idx, scale, cnt, 2, n3, Cr, Ci, n1, n1 * n2,
               nullptr, nullptr, 0};
  if ((rc = launch_rdft(gc, st))) return rc;
  DftGather ga{A, n1 * n2, 1, 1, 0, n1 * n2, nullptr, nullptr, nullptr, 0, n3, Ar, Ai,
               n1 * n2, n1 * n2, nullptr, nullptr, 0};
  if ((rc = launch_rdft(ga, st))) return rc;

  const bool transpose = n1 < cprime;
  const int64_t p = transpose ? cprime : n1, q = transpose ? n1 : cprime;
  const int64_t m = q;   // number of left singular vectors (= min(n1, c'))
  {
    KernelScope ks("tcx_work", st);
    work_kernel<<<grid_n(n1 * cprime * h), 256, 0, st>>>(Cr, Ci, n1, cprime, n1, n1 * n2, h,
                                                         transpose, Fr, Fi);
    flags_kernel<<<unsigned((h + 255) / 256), 256, 0, st>>>(flags, h, n3);
  }
  note_launches(1);
  const int sweeps = (opts && opts->max_sweeps > 0) ? opts->max_sweeps : 30;
  if ((rc = hybrid_svd(Cr, Ci, n1 * n2, n1, transpose, int(p), int(q), int(h), Fr, Fi, Qr, Qi, qsig,
                       NSr, NSi, Gr, Gi, Wr, Wi, sig, flags, sweeps, status, st)))
    return rc;
  {
    KernelScope ks("tcx_basis", st);
    // left singular vectors of C_hat: G (n1 x m) when not transposed, W (n1 x n1) otherwise
    if (!transpose)
      range_basis_kernel<<<unsigned(h), 256, 0, st>>>(Gr, Gi, p * q, sig, int(m), n1, cprime, Br,
                                                      Bi, Hr, Hi);
    else
      range_basis_kernel<<<unsigned(h), 256, 0, st>>>(Wr, Wi, q * q, sig, int(m), n1, cprime, Br,
                                                      Bi, Hr, Hi);
  }
  if ((rc = launch_status("tcx_basis"))) return rc;
  // T = U_r^H A_hat (m x n2), Z_hat = U_r T (n1 x n2)
  CGemm g1{Hr, Hi, Ar, Ai, Tr, Ti, m, n2, n1, nullptr, m, n1, m, m * n1, n1 * n2, m * n2, h, n3,
           TP_FP32, nullptr, nullptr, nullptr, nullptr, n1, status};
  if ((rc = launch_cgemm(g1, st))) return rc;
  CGemm g2{Br, Bi, Tr, Ti, Zr, Zi, n1, n2, m, nullptr, n1, m, n1, n1 * m, m * n2, n1 * n2, h, n3,
           TP_FP32, nullptr, nullptr, nullptr, nullptr, m, status};
  if ((rc = launch_cgemm(g2, st))) return rc;
  return launch_irdft(Zr, Zi, n1 * n2, n1 * n2, n3, Z, st);
}

}  // namespace tp
