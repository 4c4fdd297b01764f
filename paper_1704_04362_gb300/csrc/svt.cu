// ADMM with tensor singular-value thresholding: Algorithm 7 as printed
// (robust TNN, problem tlow7: E-step = entrywise soft threshold of
// X - L - Y/mu at lambda/mu, every entry observed) and its completion form
// (problem tlow6, below).  Per iteration of the completion form,
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
// iterations, so a sweep or two re-converges), then forms H = W V from the
// unrotated work matrix W and the singular values as Rayleigh quotients
// s_j = ||h_j|| / ||v_j||: their error is second order in the error of v_j
// (the Jacobi's own column norms carry the rounding of every rotation), which
// matters because max(s_j - tau, 0) amplifies the error of any s_j close to
// tau.  The shrunk slice is
// sum_j max(s_j - tau, 0) u_j v_j^H = sum_j c_j h_j v_j^H,
// c_j = max(s_j - tau, 0) / (s_j ||v_j||^2).
//
// Split forms (opts->precision TP_TF32X3 / TP_BF16X3): the iteration's three
// GEMMs (G = W V_prev, H = W V, the rebuild) run on the tcgen05 tensor cores
// with hi + lo operand planes.  Their operands are stored K-major: W and H
// row-major (element (a, k) at k + lq a), V and the small rebuild operand
// column-major; H is formed as its transpose H^T = V^T W^T, which comes out
// of the GEMM already row-major, so no operand needs a transpose pass but W's.
#include <vector>

#include "dft_common.cuh"
#include "tp_internal.cuh"

namespace tp {

int jacobi_float_launch(float* gr, float* gi, int64_t sG, float* vr, float* vi, int64_t sV,
                        float* sig, int p, int q, int batch, int max_sweeps,
                        const int* real_flags, int32_t* status, bool init_v, cudaStream_t st);
bool jacobi_blocked_applies(int p, int q);
bool jacobi_cluster_applies(int q, int batch);
int jacobi_float_cluster_launch(float* gr, float* gi, int64_t sG, float* vr, float* vi,
                                int64_t sV, float* sig, int p, int q, int batch, int max_sweeps,
                                const int* real_flags, int32_t* status, bool init_v,
                                cudaStream_t st);
int jacobi_float_blocked_launch(float* gr, float* gi, int64_t sG, float* vr, float* vi,
                                int64_t sV, float* sig, int p, int q, int batch, int max_sweeps,
                                const int* real_flags, int32_t* status, bool init_v,
                                cudaStream_t st);
// Slices too large for the shared-memory Jacobi take the blocked one
// (jacobi_blocked.cu); -DTP_SVT_BLOCKED=0 keeps them on the global-memory form.
#ifndef TP_SVT_BLOCKED
#define TP_SVT_BLOCKED 1
#endif
int launch_cgemm(const CGemm& g, cudaStream_t st);

namespace {

__global__ void admm_pre_kernel(const float* __restrict__ X, const uint8_t* __restrict__ mask,
                                const float* __restrict__ E, const float* __restrict__ Y,
                                const double* __restrict__ mu, int64_t n, float* __restrict__ M) {
  const float inv_mu = float(1.0 / *mu);
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x) {
    const float x = (mask == nullptr || mask[e]) ? X[e] : 0.f;   // robust form: no mask
    M[e] = x - E[e] - Y[e] * inv_mu;
  }
}

// E and Y updates.  lam > 0: robust form, E = soft(X - L - Y/mu, lam/mu) on
// every entry; else completion form, E = X_obs - L - Y/mu off the mask, 0 on it.
__global__ void admm_post_kernel(const float* __restrict__ X, const uint8_t* __restrict__ mask,
                                 const float* __restrict__ L, float* __restrict__ E,
                                 float* __restrict__ Y, const double* __restrict__ mu, int64_t n,
                                 double lam) {
  const float m = float(*mu);
  const float inv_mu = float(1.0 / *mu);
  const float thr = float(lam / *mu);
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x) {
    const float y = Y[e];
    const float l = L[e];
    float x, enew;
    if (lam > 0.0) {
      x = X[e];
      const float v = x - l - y * inv_mu;
      enew = copysignf(fmaxf(fabsf(v) - thr, 0.f), v);
    } else {
      const bool obs = mask[e] != 0;
      x = obs ? X[e] : 0.f;
      enew = obs ? 0.f : (x - l - y * inv_mu);
    }
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
                               float* __restrict__ gr, float* __restrict__ gi,
                               float* __restrict__ g2r, float* __restrict__ g2i) {
  const int64_t per = n1 * n2, total = per * h;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = e / per, r = e - k * per;
    const int64_t i = r % n1, j = r / n1;
    const int64_t o = transpose ? k * per + j + n2 * i : e;
    const float vr = xr[e], vi = transpose ? -xi[e] : xi[e];
    gr[o] = vr;
    gi[o] = vi;
    if (g2r) {   // second copy (the Jacobi rotates the first in place)
      g2r[o] = vr;
      g2i[o] = vi;
    }
  }
}

// Shrink factors of every slice from V (q x q) and H = W V (p x q; W the
// work matrix): with n_j = ||v_j|| and s_j = ||h_j|| / n_j (norms accumulated
// in float64), c_j = max(s_j - tau, 0) / (s_j n_j^2), so that the shrunk
// work-shaped slice is R = sum_j c_j h_j v_j^H = H diag(c) V^H.  Writes the
// small operand of the rebuilding product: D V^H (q x q, entry (j, b) =
// c_j conj(V(b, j))) when the slice is R itself, or V D (entry (b, j) =
// V(b, j) c_j) when the slice is R^H = V D H^H.
__global__ void svt_coef_kernel(const float* __restrict__ hr, const float* __restrict__ hi,
                                int64_t sH, int64_t h_row, int64_t h_col,
                                const float* __restrict__ vr,
                                const float* __restrict__ vi, int64_t sV, int p, int q,
                                const double* __restrict__ mu, bool transpose,
                                float* __restrict__ outr, float* __restrict__ outi) {
  extern __shared__ float coef[];   // q factors c_j
  const int64_t f = blockIdx.x;
  const double tau = 1.0 / *mu;
  const float* Hr = hr + f * sH;
  const float* Hi = hi + f * sH;
  const float* Vr = vr + f * sV;
  const float* Vi = vi + f * sV;
  for (int j = threadIdx.x; j < q; j += blockDim.x) {
    double nv = 0.0, nh = 0.0;
    for (int b = 0; b < q; ++b) {
      const double x = Vr[b + int64_t(q) * j], y = Vi[b + int64_t(q) * j];
      nv += x * x + y * y;
    }
    for (int a = 0; a < p; ++a) {   // H(a, j) at a h_row + j h_col
      const double x = Hr[a * h_row + j * h_col], y = Hi[a * h_row + j * h_col];
      nh += x * x + y * y;
    }
    const double s = nv > 0.0 ? sqrt(nh / nv) : 0.0;
    coef[j] = s > tau ? float((s - tau) / (s * nv)) : 0.f;
  }
  __syncthreads();
  float* Or = outr + f * sV;
  float* Oi = outi + f * sV;
  const int64_t qq = int64_t(q) * q;
  for (int64_t e = threadIdx.x; e < qq; e += blockDim.x) {
    const int64_t r = e % q, c = e / q;
    if (!transpose) {   // (j = r, b = c): c_j conj(V(b, j))
      const float cj = coef[r];
      Or[e] = cj * Vr[c + int64_t(q) * r];
      Oi[e] = -cj * Vi[c + int64_t(q) * r];
    } else {            // (b = r, j = c): V(b, j) c_j
      const float cj = coef[c];
      Or[e] = cj * Vr[e];
      Oi[e] = cj * Vi[e];
    }
  }
}

// Split planes of a batch of matrices (rows x cols, column-major, leading
// dimension ld_src, batch stride s_src) at f*s_dst + r + ld_dst*c; rows
// [rows, ld_dst) are zero; the imaginary part negated when conj.
__global__ void svt_split_kernel(const float* __restrict__ sr, const float* __restrict__ si,
                                 int64_t rows, int64_t cols, int64_t ld_src, int64_t s_src,
                                 int64_t h, int64_t ld_dst, int64_t s_dst, int conj, int bf16,
                                 float* __restrict__ p0, float* __restrict__ p1,
                                 float* __restrict__ p2, float* __restrict__ p3) {
  const int64_t per = ld_dst * cols, total = per * h;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t f = e / per, rem = e - f * per;
    const int64_t c = rem / ld_dst, r = rem - c * ld_dst;
    float vr = 0.f, vi = 0.f;
    if (r < rows) {
      vr = sr[f * s_src + r + ld_src * c];
      vi = si[f * s_src + r + ld_src * c];
      if (conj) vi = -vi;
    }
    dftc::put_split(p0, p1, bf16 != 0, e, vr);
    dftc::put_split(p2, p3, bf16 != 0, e, vi);
  }
}

// The same split of the transposes: element (r, c) of matrix f (rows x cols,
// column-major, ld rows) goes to f*s_dst + c + ld_dst*r (the K-major, i.e.
// row-major, operand); 32 x 32 tiles through shared memory.
__global__ void svt_split_t_kernel(const float* __restrict__ sr, const float* __restrict__ si,
                                   int64_t rows, int64_t cols, int64_t ld_dst, int64_t s_dst,
                                   int bf16, float* __restrict__ p0, float* __restrict__ p1,
                                   float* __restrict__ p2, float* __restrict__ p3) {
  __shared__ float tr[32][33], ti[32][33];
  const int64_t f = blockIdx.z;
  const int64_t r0 = int64_t(blockIdx.x) * 32, c0 = int64_t(blockIdx.y) * 32;
  const float* xr = sr + f * rows * cols;
  const float* xi = si + f * rows * cols;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int64_t r = r0 + threadIdx.x, c = c0 + dy;
    tr[dy][threadIdx.x] = (r < rows && c < cols) ? xr[r + rows * c] : 0.f;
    ti[dy][threadIdx.x] = (r < rows && c < cols) ? xi[r + rows * c] : 0.f;
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int64_t c = c0 + threadIdx.x, r = r0 + dy;
    if (r < rows && c < ld_dst) {   // c in [cols, ld_dst): the zero K padding
      const int64_t o = f * s_dst + c + ld_dst * r;
      dftc::put_split(p0, p1, bf16 != 0, o, tr[threadIdx.x][dy]);
      dftc::put_split(p2, p3, bf16 != 0, o, ti[threadIdx.x][dy]);
    }
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

// K leading dimension of the split operand planes (16-byte rows for TMA).
int64_t svt_ld(int64_t k, int prec) {
  return prec == TP_BF16X3 ? (k + 7) / 8 * 8 : (k + 3) / 4 * 4;
}
bool svt_tc(int prec) { return prec == TP_TF32X3 || prec == TP_BF16X3; }

size_t svt_ws(int64_t n1, int64_t n2, int64_t n3, int prec) {
  const size_t h = size_t(half_len(n3));
  const size_t p = size_t(n1 > n2 ? n1 : n2), q = size_t(n1 < n2 ? n1 : n2);
  const size_t n = size_t(n1) * n2;
  const size_t lq = size_t(svt_ld(int64_t(q), prec)), esz = prec == TP_BF16X3 ? 2 : 4;
  const size_t split = svt_tc(prec) ? 4 * (2 * ws_bytes(lq * p * h, esz)      // W, H planes
                                           + 2 * ws_bytes(lq * q * h, esz))   // V, rebuild planes
                                    : 0;
  return split + ws_bytes(n * n3, 4)          // M (and L, reused)
         + 2 * ws_bytes(n * h, 4)             // M_hat / L_hat
         + 2 * ws_bytes(p * q * h, 4)         // G (rotated by the Jacobi)
         + 2 * ws_bytes(q * q * h, 4)         // V
         + 2 * ws_bytes(p * q * h, 4)         // work matrix W
         + 2 * ws_bytes(p * q * h, 4)         // H = W V
         + ws_bytes(q * h, 4) + ws_bytes(h, 4);
}

// One tensor of a completion run: its ADMM state (caller's buffers) and its
// workspace.
struct SvtTensor {
  const float* X;
  const uint8_t* mask;
  float *L, *E, *Y;
  double* mu;
  double lam;   // > 0: robust form (no mask), else completion form
  int64_t n1, n2, n3, h, p, q;
  bool transpose;
  float *M, *Mr, *Mi, *Gr, *Gi, *Vr, *Vi, *Kr, *Ki, *Hr, *Hi, *sig;
  int* flags;
  // split forms: precision, K leading dimension lq, operand planes (re hi,
  // re lo, im hi, im lo): W and H row-major, V and the rebuild operand
  // column-major (or row-major for V D)
  int prec;
  int64_t lq;
  float *WP[4], *HP[4], *VP[4], *BP[4];
  // a lone tensor (not one of a batch sharing the GPU): its Jacobi may spread
  // each slice over a thread-block cluster when the slices are fewer than SMs
  bool alone = false;
};

SvtTensor svt_carve(const float* X, const uint8_t* mask, int64_t n1, int64_t n2, int64_t n3,
                    float* L, float* E, float* Y, double* mu, Arena& ws, int prec) {
  SvtTensor t{};
  t.prec = prec;
  t.X = X;
  t.mask = mask;
  t.L = L;
  t.E = E;
  t.Y = Y;
  t.mu = mu;
  t.n1 = n1;
  t.n2 = n2;
  t.n3 = n3;
  t.h = half_len(n3);
  t.transpose = n1 < n2;
  t.p = t.transpose ? n2 : n1;
  t.q = t.transpose ? n1 : n2;
  const size_t h = size_t(t.h), pq = size_t(t.p) * t.q, qq = size_t(t.q) * t.q;
  t.M = ws.take<float>(size_t(n1) * n2 * n3);
  t.Mr = ws.take<float>(size_t(n1) * n2 * h);
  t.Mi = ws.take<float>(size_t(n1) * n2 * h);
  t.Gr = ws.take<float>(pq * h);
  t.Gi = ws.take<float>(pq * h);
  t.Vr = ws.take<float>(qq * h);
  t.Vi = ws.take<float>(qq * h);
  t.Kr = ws.take<float>(pq * h);
  t.Ki = ws.take<float>(pq * h);
  t.Hr = ws.take<float>(pq * h);
  t.Hi = ws.take<float>(pq * h);
  t.sig = ws.take<float>(size_t(t.q) * h);
  t.flags = ws.take<int>(h);
  t.lq = svt_ld(t.q, prec);
  if (svt_tc(prec)) {
    const size_t lq = size_t(t.lq);
    auto planes = [&](float** P, size_t elems) {
      for (int i = 0; i < 4; ++i)
        P[i] = prec == TP_BF16X3 ? reinterpret_cast<float*>(ws.take<uint16_t>(elems))
                                 : ws.take<float>(elems);
    };
    planes(t.WP, lq * size_t(t.p) * h);
    planes(t.HP, lq * size_t(t.p) * h);
    planes(t.VP, lq * size_t(t.q) * h);
    planes(t.BP, lq * size_t(t.q) * h);
  }
  return t;
}

int svt_init(const SvtTensor& t, cudaStream_t st) {
  {
    KernelScope ks("svt_flags", st);
    flags_kernel<<<unsigned((t.h + 255) / 256), 256, 0, st>>>(t.flags, t.h, t.n3);
  }
  return launch_status("svt_flags");
}

// One ADMM iteration of one tensor on stream st.  warm: start the Jacobi from
// the V left by the previous iteration of this tensor.
int svt_iteration(const SvtTensor& t, bool warm, double rho, double mu_max, int sweeps,
                  int32_t* status, cudaStream_t st) {
  int rc;
  const int64_t n = t.n1 * t.n2 * t.n3, n12 = t.n1 * t.n2;
  const int64_t p = t.p, q = t.q, h = t.h;
  {
    KernelScope ks("admm_pre", st);
    admm_pre_kernel<<<grid_n(n), 256, 0, st>>>(t.X, t.mask, t.E, t.Y, t.mu, n, t.M);
  }
  DftGather gm{t.M, n12, 1, 1, 0, n12, nullptr, nullptr, nullptr, 0, t.n3, t.Mr, t.Mi,
               n12, n12, nullptr, nullptr, 0};
  if ((rc = launch_rdft(gm, st))) return rc;
  {   // work matrix W (kept in K), and G = W for a cold start
    KernelScope ks("svt_work", st);
    to_work_kernel<<<grid_n(n12 * h), 256, 0, st>>>(t.Mr, t.Mi, t.n1, t.n2, h, t.transpose, t.Kr,
                                                    t.Ki, warm ? nullptr : t.Gr,
                                                    warm ? nullptr : t.Gi);
  }
  const bool tc = svt_tc(t.prec);
  const int bf = t.prec == TP_BF16X3 ? 1 : 0;
  const int64_t lq = t.lq;
  // tensor-core GEMM C = A B over the h slices, A (M x K) and B (K x N) split
  // planes stored K-major with leading dimension lq, C column-major (ldc)
  auto gemm_tc = [&](float* const* A, float* const* B, float* cr, float* ci, int64_t M,
                     int64_t N, int64_t ldc) {
    CGemm g{A[0], A[2], B[0], B[2], cr, ci, M, N, q, nullptr, lq, lq, ldc, lq * M, lq * N,
            M * N, h, t.n3, t.prec, A[1], A[3], B[1], B[3], lq, status};
    return launch_cgemm(g, st);
  };
  auto split = [&](const float* sr, const float* si, int64_t rows, int64_t cols, int conj,
                   float* const* P) {
    {
      KernelScope ks("svt_split", st);
      svt_split_kernel<<<grid_n(lq * cols * h), 256, 0, st>>>(
          sr, si, rows, cols, rows, rows * cols, h, lq, lq * cols, conj, bf, P[0], P[1], P[2],
          P[3]);
    }
    return launch_status("svt_split_kernel");
  };
  // row-major split of the column-major rows x cols matrices (K = cols)
  auto split_t = [&](const float* sr, const float* si, int64_t rows, int64_t cols,
                     float* const* P) {
    {
      KernelScope ks("svt_split_t", st);
      svt_split_t_kernel<<<dim3(unsigned((rows + 31) / 32), unsigned((lq + 31) / 32),
                                unsigned(h)),
                           dim3(32, 8), 0, st>>>(sr, si, rows, cols, lq, lq * rows, bf, P[0],
                                                 P[1], P[2], P[3]);
    }
    return launch_status("svt_split_t_kernel");
  };
  if (tc && (rc = split_t(t.Kr, t.Ki, p, q, t.WP))) return rc;   // W, row-major
  if (warm) {   // G = W V_prev
    if (tc) {
      if ((rc = gemm_tc(t.WP, t.VP, t.Gr, t.Gi, p, q, p))) return rc;
    } else {
      CGemm gw{t.Kr, t.Ki, t.Vr, t.Vi, t.Gr, t.Gi, p, q, q, nullptr, p, q, p, p * q, q * q, p * q,
               h, t.n3, TP_FP32, nullptr, nullptr, nullptr, nullptr, q, status};
      if ((rc = launch_cgemm(gw, st))) return rc;
    }
  }
  if (t.alone && jacobi_cluster_applies(int(q), int(h)))
    rc = jacobi_float_cluster_launch(t.Gr, t.Gi, p * q, t.Vr, t.Vi, q * q, t.sig, int(p), int(q),
                                     int(h), sweeps, t.flags, status, !warm, st);
  else if (TP_SVT_BLOCKED && jacobi_blocked_applies(int(p), int(q)))
    rc = jacobi_float_blocked_launch(t.Gr, t.Gi, p * q, t.Vr, t.Vi, q * q, t.sig, int(p), int(q),
                                     int(h), sweeps, t.flags, status, !warm, st);
  else
    rc = jacobi_float_launch(t.Gr, t.Gi, p * q, t.Vr, t.Vi, q * q, t.sig, int(p), int(q),
                             int(h), sweeps, t.flags, status, !warm, st);
  if (rc) return rc;
  if (tc) {
    // V's planes (also V_prev of the next iteration's G = W V_prev), then
    // H^T = V^T W^T (q x p, column-major: H row-major) from the unrotated W
    if ((rc = split(t.Vr, t.Vi, q, q, 0, t.VP))) return rc;
    if ((rc = gemm_tc(t.VP, t.WP, t.Hr, t.Hi, q, p, q))) return rc;
  } else {   // H = W V from the unrotated work matrix
    CGemm gh{t.Kr, t.Ki, t.Vr, t.Vi, t.Hr, t.Hi, p, q, q, nullptr, p, q, p, p * q, q * q, p * q,
             h, t.n3, TP_FP32, nullptr, nullptr, nullptr, nullptr, q, status};
    if ((rc = launch_cgemm(gh, st))) return rc;
  }
  {   // shrink factors into the small operand (in G, free after the Jacobi)
    KernelScope ks("svt_coef", st);
    svt_coef_kernel<<<unsigned(h), 256, size_t(q) * sizeof(float), st>>>(
        t.Hr, t.Hi, p * q, tc ? q : 1, tc ? 1 : p, t.Vr, t.Vi, q * q, int(p), int(q), t.mu,
        t.transpose, t.Gr, t.Gi);
  }
  if (tc) {
    if (!t.transpose) {   // slice (p x q) = H (D V^H)
      if ((rc = split(t.Hr, t.Hi, q, p, 0, t.HP))) return rc;     // H row-major
      if ((rc = split(t.Gr, t.Gi, q, q, 0, t.BP))) return rc;     // D V^H column-major
      if ((rc = gemm_tc(t.HP, t.BP, t.Mr, t.Mi, p, q, p))) return rc;
    } else {              // slice (q x p) = (V D) H^H
      if ((rc = split(t.Hr, t.Hi, q, p, 1, t.HP))) return rc;     // conj(H) row-major
      if ((rc = split_t(t.Gr, t.Gi, q, q, t.BP))) return rc;      // V D row-major
      if ((rc = gemm_tc(t.BP, t.HP, t.Mr, t.Mi, q, p, q))) return rc;
    }
  } else if (!t.transpose) {   // slice = H (D V^H): n1 x n2 = p x q
    CGemm gr{t.Hr, t.Hi, t.Gr, t.Gi, t.Mr, t.Mi, p, q, q, nullptr, p, q, p, p * q, q * q, p * q,
             h, t.n3, TP_FP32, nullptr, nullptr, nullptr, nullptr, q, status};
    if ((rc = launch_cgemm(gr, st))) return rc;
  } else {              // slice = (V D) H^H: n1 x n2 = q x p
    CGemm gr{t.Gr, t.Gi, t.Hr, t.Hi, t.Mr, t.Mi, q, p, q, nullptr, q, p, q, q * q, p * q, q * p,
             h, t.n3, TP_FP32, nullptr, nullptr, nullptr, nullptr, q, status};
    gr.b_conj_trans = 1;
    if ((rc = launch_cgemm(gr, st))) return rc;
  }
  if ((rc = launch_irdft(t.Mr, t.Mi, n12, n12, t.n3, t.L, st))) return rc;
  {
    KernelScope ks("admm_post", st);
    admm_post_kernel<<<grid_n(n), 256, 0, st>>>(t.X, t.mask, t.L, t.E, t.Y, t.mu, n, t.lam);
  }
  {
    KernelScope ks("admm_mu", st);
    admm_mu_kernel<<<1, 32, 0, st>>>(t.mu, rho, mu_max);
  }
  return launch_status("admm iteration");
}

// mask null and lam > 0: the robust form; else the completion form.
int svt_run(const float* X, const uint8_t* mask, int64_t n1, int64_t n2, int64_t n3, int iters,
            double rho, double mu_max, float* L, float* E, float* Y, double* mu,
            const tp_opts* opts, cudaStream_t st, double lam) {
  const int prec = opts ? opts->precision : TP_FP32;
  if (prec != TP_FP32 && !svt_tc(prec)) {
    set_error("admm: unknown precision %d", prec);
    return TP_EINVAL;
  }
  Arena ws;
  int rc = acquire_workspace(opts, svt_ws(n1, n2, n3, prec), &ws);
  if (rc) return rc;
  int32_t* status = opts ? opts->status : nullptr;
  const int sweeps = (opts && opts->max_sweeps > 0) ? opts->max_sweeps : 30;
  SvtTensor t = svt_carve(X, mask, n1, n2, n3, L, E, Y, mu, ws, prec);
  t.lam = lam;
  t.alone = true;
  if ((rc = svt_init(t, st))) return rc;
  for (int it = 0; it < iters; ++it)
    if ((rc = svt_iteration(t, it > 0, rho, mu_max, sweeps, status, st))) return rc;
  return TP_OK;
}

size_t svt_batched_ws(int ntens, const tp_tensor_desc* d, int prec) {
  size_t total = 0;
  for (int i = 0; i < ntens; ++i) total += svt_ws(d[i].n1, d[i].n2, d[i].n3, prec);
  return total;
}

size_t svt_batched_ws_dims(const int64_t* dims, int nd, int prec) {
  size_t total = 0;
  for (int i = 0; i + 2 < nd; i += 3) total += svt_ws(dims[i], dims[i + 1], dims[i + 2], prec);
  return total;
}

namespace {
constexpr int kSideStreams = 8;

// Forks the tensors of one iteration over the side streams and joins them
// back into st (event record / wait pairs: valid eagerly and under capture).
// The captured iteration is recorded on a private non-blocking stream (the
// legacy default stream cannot be captured) and its graph launched on the
// caller's stream.
int svt_fork_join(std::vector<SvtTensor>& T, bool warm, bool init, double rho, double mu_max,
                  int sweeps, int32_t* status, cudaStream_t st, cudaStream_t* side,
                  cudaEvent_t fork, cudaEvent_t* join, int ns) {
  int rc = TP_OK;
  if (cudaEventRecord(fork, st) != cudaSuccess) return TP_ECUDA;
  for (int s = 0; s < ns; ++s)
    if (cudaStreamWaitEvent(side[s], fork, 0) != cudaSuccess) return TP_ECUDA;
  for (size_t i = 0; i < T.size() && rc == TP_OK; ++i) {
    cudaStream_t ss = side[i % size_t(ns)];
    if (init) rc = svt_init(T[i], ss);
    if (rc == TP_OK) rc = svt_iteration(T[i], warm, rho, mu_max, sweeps, status, ss);
  }
  for (int s = 0; s < ns; ++s) {
    if (cudaEventRecord(join[s], side[s]) != cudaSuccess ||
        cudaStreamWaitEvent(st, join[s], 0) != cudaSuccess)
      return TP_ECUDA;
  }
  return rc;
}
}  // namespace

int svt_batched_run(int ntens, const tp_tensor_desc* d, int iters, double rho, double mu_max,
                    const tp_opts* opts, cudaStream_t st, const double* lams) {
  const int prec = opts ? opts->precision : TP_FP32;
  if (prec != TP_FP32 && !svt_tc(prec)) {
    set_error("tcomplete_svt_batched: unknown precision %d", prec);
    return TP_EINVAL;
  }
  Arena ws;
  int rc = acquire_workspace(opts, svt_batched_ws(ntens, d, prec), &ws);
  if (rc) return rc;
  if (iters <= 0) return TP_OK;
  int32_t* status = opts ? opts->status : nullptr;
  const int sweeps = (opts && opts->max_sweeps > 0) ? opts->max_sweeps : 30;
  std::vector<SvtTensor> T;
  T.reserve(size_t(ntens));
  for (int i = 0; i < ntens; ++i) {
    T.push_back(svt_carve(d[i].X, d[i].mask, d[i].n1, d[i].n2, d[i].n3, d[i].L, d[i].E, d[i].Y,
                          d[i].mu, ws, prec));
    if (lams) T.back().lam = lams[i];   // > 0: robust form of problem tlow7
  }
  const int ns = ntens < kSideStreams ? ntens : kSideStreams;
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t join[kSideStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;   // capture stream (the caller's may be the legacy stream)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess;
  for (int s = 0; s < ns && ok; ++s)
    ok = cudaStreamCreateWithFlags(&side[s], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&join[s], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    set_error("tcomplete_svt_batched: creating streams or events failed");
    rc = TP_ECUDA;
  }
  // iteration 1: cold Jacobi start, launched directly
  if (rc == TP_OK)
    rc = svt_fork_join(T, false, true, rho, mu_max, sweeps, status, st, side, fork, join, ns);
  // iterations 2..iters: one captured iteration, replayed
  if (rc == TP_OK && iters > 1) {
    const uint64_t before = tp_launch_count();
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      set_error("tcomplete_svt_batched: stream capture could not begin");
      rc = TP_ECUDA;
    } else {
      rc = svt_fork_join(T, true, false, rho, mu_max, sweeps, status, cap, side, fork, join, ns);
      const cudaError_t e = cudaStreamEndCapture(cap, &graph);
      if (rc == TP_OK && e != cudaSuccess) {
        set_error("tcomplete_svt_batched: stream capture failed (%s)", cudaGetErrorString(e));
        rc = TP_ECUDA;
      }
    }
    const uint64_t per_iter = tp_launch_count() - before;   // counted once at capture
    if (rc == TP_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      set_error("tcomplete_svt_batched: graph instantiation failed");
      rc = TP_ECUDA;
    }
    {
      // the replays as one profiled region (tp_profile_*): their time over
      // iters - 1 is the warm iteration time
      KernelScope region("svt_graph_replays", st, false);
      for (int it = 1; it < iters && rc == TP_OK; ++it)
        if (cudaGraphLaunch(exec, st) != cudaSuccess) {
          set_error("tcomplete_svt_batched: graph launch failed");
          rc = TP_ECUDA;
        }
    }
    if (rc == TP_OK && iters > 2) note_launches(per_iter * uint64_t(iters - 2));
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == TP_OK) {
    set_error("tcomplete_svt_batched: %s", cudaGetErrorString(cudaGetLastError()));
    rc = TP_ECUDA;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  for (int s = 0; s < ns; ++s) {
    if (join[s]) cudaEventDestroy(join[s]);
    if (side[s]) cudaStreamDestroy(side[s]);
  }
  if (fork) cudaEventDestroy(fork);
  if (cap) cudaStreamDestroy(cap);
  cudaGetLastError();
  return rc;
}

}  // namespace tp
