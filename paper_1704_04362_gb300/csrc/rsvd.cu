// Randomized low-tubal-rank t-SVD: per half-spectrum slice X_hat_f the range
// finder with power iterations of Halko, Martinsson and Tropp (2011):
//   Y = X_hat Omega;  Q = orth(Y)
//   q times: Z = orth(X_hat^H Q), Q = orth(X_hat Z)
//   B^H = X_hat^H Q  (n2 x l);  B^H = V_B diag(s) W^H (one-sided Jacobi, float64)
//   U_f = Q W[:, :k],  V_f = V_B[:, :k],  S_f = diag(s[:k])
// followed by the inverse DFT of U, S, V (Theorem 2.6's form, tubal rank k).
// The test matrix has random-sign entries from Philox stream 2 (see
// tsvd_randomized in tprod.h).  orth() is a float32 Householder QR in shared
// memory for slices of at most 256 rows; taller slices take CholeskyQR2
// (Fukaya et al. 2014): G = Y^H Y and its Cholesky factor R in float64,
// Y <- Y R^{-1}, twice; if a Cholesky fails, the Gram matrix is shifted
// (shifted CholeskyQR, Fukaya et al. 2020) and one more pass is made; a
// failure after that sets TP_DEV_BREAKDOWN.  Every product with X_hat is a plain column-major batched
// complex GEMM because X_hat^H is formed once.
#include <cfloat>
#include <cmath>

#include "dft_common.cuh"
#include "philox.cuh"

namespace tp {

int launch_cgemm(const CGemm& g, cudaStream_t st);
int jacobi_double_launch(double* gr, double* gi, int64_t sG, double* vr, double* vi, int64_t sV,
                         double* sig, int p, int q, int batch, int max_sweeps,
                         const int* real_flags, int32_t* status, cudaStream_t st);

namespace {

constexpr int QR_THREADS = 256;

// X^H of every slice: out(j, i) = conj(in(i, j)), in n1 x n2, out n2 x n1.
__global__ void conj_transpose_kernel(const float* __restrict__ ir, const float* __restrict__ ii,
                                      int64_t n1, int64_t n2, float* __restrict__ orr,
                                      float* __restrict__ oi) {
  __shared__ float tr[32][33], ti[32][33];
  const int64_t f = blockIdx.z;
  const int64_t i0 = int64_t(blockIdx.x) * 32, j0 = int64_t(blockIdx.y) * 32;
  const float* sr = ir + f * n1 * n2;
  const float* si = ii + f * n1 * n2;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int64_t i = i0 + threadIdx.x, j = j0 + dy;
    if (i < n1 && j < n2) {
      tr[dy][threadIdx.x] = sr[i + n1 * j];
      ti[dy][threadIdx.x] = si[i + n1 * j];
    }
  }
  __syncthreads();
  float* dr = orr + f * n1 * n2;
  float* di = oi + f * n1 * n2;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int64_t j = j0 + threadIdx.x, i = i0 + dy;
    if (i < n1 && j < n2) {
      dr[j + n2 * i] = tr[threadIdx.x][dy];
      di[j + n2 * i] = -ti[threadIdx.x][dy];
    }
  }
}

// Split operand planes (tensor-core products) of a batch of column-major
// complex matrices: element (r, c) of matrix f (rows x cols, at
// f*s_src + r + ld_src*c) goes to f*s_dst + r + ld_dst*c of the hi/lo
// planes (3xTF32 float or BF16x3 bf16 pairs), the imaginary part negated
// when conj; rows [rows, ld_dst) are zero (the K padding of the tiles).
// The split planes of X_hat transposed without conjugation, for the
// tensor-core products X_hat B: element (i, j) of X_hat (n1 x n2,
// column-major) goes to j + ldk i of each plane (K-major, rows j from n2 to
// ldk zero), through a 32 x 32 shared-memory tile as conj_transpose_kernel
// moves it.
__global__ void transpose_split_kernel(const float* __restrict__ ir, const float* __restrict__ ii,
                                       int64_t n1, int64_t n2, int64_t ldk, int bf16,
                                       float* __restrict__ re_hi, float* __restrict__ re_lo,
                                       float* __restrict__ im_hi, float* __restrict__ im_lo) {
  __shared__ float tr[32][33], ti[32][33];
  const int64_t f = blockIdx.z;
  const int64_t i0 = int64_t(blockIdx.x) * 32, j0 = int64_t(blockIdx.y) * 32;
  const float* sr = ir + f * n1 * n2;
  const float* si = ii + f * n1 * n2;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int64_t i = i0 + threadIdx.x, j = j0 + dy;
    const bool in = i < n1 && j < n2;
    tr[dy][threadIdx.x] = in ? sr[i + n1 * j] : 0.f;
    ti[dy][threadIdx.x] = in ? si[i + n1 * j] : 0.f;
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int64_t j = j0 + threadIdx.x, i = i0 + dy;
    if (i < n1 && j < ldk) {
      const int64_t o = f * ldk * n1 + j + ldk * i;
      dftc::put_split(re_hi, re_lo, bf16 != 0, o, tr[threadIdx.x][dy]);
      dftc::put_split(im_hi, im_lo, bf16 != 0, o, ti[threadIdx.x][dy]);
    }
  }
}

__global__ void split_planes_kernel(const float* __restrict__ sr, const float* __restrict__ si,
                                    int64_t rows, int64_t cols, int64_t ld_src, int64_t s_src,
                                    int64_t h, int64_t ld_dst, int64_t s_dst, int conj, int bf16,
                                    float* __restrict__ re_hi, float* __restrict__ re_lo,
                                    float* __restrict__ im_hi, float* __restrict__ im_lo) {
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
    const int64_t o = f * s_dst + r + ld_dst * c;
    dftc::put_split(re_hi, re_lo, bf16 != 0, o, vr);
    dftc::put_split(im_hi, im_lo, bf16 != 0, o, vi);
  }
}

// Omega(r, c, f) at e = r + n2*(c + l*f): (s0 + i s1)/sqrt(2) from the top bits
// of Philox(e, stream 2); the real slices take s0.
__global__ void sketch_kernel(float* __restrict__ om_r, float* __restrict__ om_i, int64_t n2,
                              int64_t l, int64_t h, int64_t n3, uint64_t seed) {
  const int64_t total = n2 * l * h;
  const float inv_sqrt2 = 0.70710678118654752f;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    uint32_t c[4] = {uint32_t(e), uint32_t(uint64_t(e) >> 32), 2u, 0u};
    philox4x32_10(c, uint32_t(seed), uint32_t(seed >> 32));
    const float s0 = (c[0] >> 31) ? -1.f : 1.f;
    const float s1 = (c[1] >> 31) ? -1.f : 1.f;
    const int64_t f = e / (n2 * l);
    const bool real = f == 0 || (n3 % 2 == 0 && f == h - 1);
    om_r[e] = real ? s0 : s0 * inv_sqrt2;
    om_i[e] = real ? 0.f : s1 * inv_sqrt2;
  }
}

// Gram of the columns of Y (p x l, float32 planar, column-major) into
// G (l x l, float64, interleaved re/im, full Hermitian).
__device__ void gram(const float* __restrict__ yr, const float* __restrict__ yi, int p, int l,
                     double* G) {
  const int npairs = l * (l + 1) / 2;
  for (int e = threadIdx.x; e < npairs; e += blockDim.x) {
    // e -> (a, b), a <= b, row-major upper triangle
    int a = 0, rem = e;
    while (rem >= l - a) { rem -= l - a; ++a; }
    const int b = a + rem;
    const float* xa_r = yr + int64_t(a) * p;
    const float* xa_i = yi + int64_t(a) * p;
    const float* xb_r = yr + int64_t(b) * p;
    const float* xb_i = yi + int64_t(b) * p;
    double sr = 0.0, si = 0.0;
    for (int r = 0; r < p; ++r) {
      const double ar = xa_r[r], ai = xa_i[r], br = xb_r[r], bi = xb_i[r];
      sr += ar * br + ai * bi;
      si += ar * bi - ai * br;
    }
    G[2 * (a * l + b)] = sr;
    G[2 * (a * l + b) + 1] = si;
    G[2 * (b * l + a)] = sr;
    G[2 * (b * l + a) + 1] = -si;
  }
}

// In-place upper Cholesky G = R^H R (R in the upper triangle of G).
// Returns false on a non-positive pivot.
__device__ bool cholesky(double* G, int l, int* fail) {
  for (int j = 0; j < l; ++j) {
    __syncthreads();
    if (threadIdx.x == 0) {
      double d = G[2 * (j * l + j)];
      for (int i = 0; i < j; ++i) {
        const double rr = G[2 * (i * l + j)], ri = G[2 * (i * l + j) + 1];
        d -= rr * rr + ri * ri;
      }
      if (!(d > 0.0) || !isfinite(d)) *fail = 1;
      G[2 * (j * l + j)] = (d > 0.0 && isfinite(d)) ? sqrt(d) : 1.0;
      G[2 * (j * l + j) + 1] = 0.0;
    }
    __syncthreads();
    const double djj = G[2 * (j * l + j)];
    for (int k = j + 1 + threadIdx.x; k < l; k += blockDim.x) {
      double sr = G[2 * (j * l + k)], si = G[2 * (j * l + k) + 1];
      for (int i = 0; i < j; ++i) {
        // subtract conj(R_ij) R_ik
        const double ar = G[2 * (i * l + j)], ai = G[2 * (i * l + j) + 1];
        const double br = G[2 * (i * l + k)], bi = G[2 * (i * l + k) + 1];
        sr -= ar * br + ai * bi;
        si -= ar * bi - ai * br;
      }
      G[2 * (j * l + k)] = sr / djj;
      G[2 * (j * l + k) + 1] = si / djj;
    }
  }
  __syncthreads();
  return *fail == 0;
}

// Y <- Y R^{-1}, row by row (x R = y by forward substitution), in place.
__device__ void right_solve(float* yr, float* yi, int p, int l, const double* R) {
  for (int r = threadIdx.x; r < p; r += blockDim.x) {
    for (int j = 0; j < l; ++j) {
      double sr = yr[r + int64_t(p) * j], si = yi[r + int64_t(p) * j];
      for (int i = 0; i < j; ++i) {
        const double xr = yr[r + int64_t(p) * i], xi = yi[r + int64_t(p) * i];
        const double ar = R[2 * (i * l + j)], ai = R[2 * (i * l + j) + 1];
        sr -= xr * ar - xi * ai;
        si -= xr * ai + xi * ar;
      }
      const double d = R[2 * (j * l + j)];
      yr[r + int64_t(p) * j] = float(sr / d);
      yi[r + int64_t(p) * j] = float(si / d);
    }
  }
}

// CholeskyQR2 (with a shifted retry) of every slice's p x l block.
__global__ void __launch_bounds__(QR_THREADS) cholqr2_kernel(float* y_re, float* y_im, int64_t sY,
                                                             int p, int lfull,
                                                             const int32_t* lcols,
                                                             int32_t* status) {
  extern __shared__ double G[];   // 2 * l * l
  __shared__ int fail;
  // per-slice column count (the per-frequency sketch size): the columns from
  // l on are set to zero
  const int l = lcols ? min(max(int(lcols[blockIdx.x]), 1), lfull) : lfull;
  float* yr = y_re + int64_t(blockIdx.x) * sY;
  float* yi = y_im + int64_t(blockIdx.x) * sY;
  for (int64_t e = int64_t(p) * l + threadIdx.x; e < int64_t(p) * lfull; e += blockDim.x) {
    yr[e] = 0.f;
    yi[e] = 0.f;
  }
  int passes_left = 2;
  bool shifted = false;
  for (int it = 0; it < 4 && passes_left > 0; ++it) {
    if (threadIdx.x == 0) fail = 0;
    gram(yr, yi, p, l, G);
    __syncthreads();
    if (shifted) {
      // shift s = 11 (p l + l (l + 1)) u ||Y||_F^2 on the diagonal
      if (threadIdx.x == 0) {
        double tr = 0.0;
        for (int j = 0; j < l; ++j) tr += G[2 * (j * l + j)];
        const double s = 11.0 * (double(p) * l + double(l) * (l + 1)) * 1.1102230246251565e-16 * tr;
        for (int j = 0; j < l; ++j) G[2 * (j * l + j)] += s;
      }
      __syncthreads();
    }
    const bool ok = cholesky(G, l, &fail);
    if (!ok) {
      if (shifted) {
        if (threadIdx.x == 0 && status) atomicOr(status, TP_DEV_BREAKDOWN);
        return;
      }
      shifted = true;   // retry this pass with a shift, then two plain passes
      passes_left = 3;
      continue;
    }
    __syncthreads();
    right_solve(yr, yi, p, l, G);
    __syncthreads();
    shifted = false;
    --passes_left;
  }
}

// ---------------------------------------------------------------- Householder QR in shared memory
// orth() of one slice's Y (p x l, p >= l, float32) held in shared memory:
// the Householder QR Y = Q R with reflectors H_j = I - tau_j v_j v_j^H
// (v_j(j) = 1, zero above) chosen as LAPACK's zlarfg chooses them, so that
// H_j^H maps rows j.. of column j onto beta_j e_j with beta_j real; then
// Q = H_0 H_1 ... H_{l-1} [I_l; 0] formed in place by backward accumulation.
// Householder QR is backward stable whatever the conditioning of Y: Q is
// orthonormal to float32 rounding in one pass and cannot break down, and it
// spans the columns of Y (completed by the reflectors where Y is rank
// deficient), which is all the range finder uses.  A step's reflector sits
// in registers (lane r % 32 holds rows r); each warp applies it to its
// columns k = j + 1 + warp (mod warps), and the owner of column j + 1 forms
// the next reflector at once (look-ahead), so a step costs one barrier.
constexpr int HQR_THREADS = 256;
constexpr int HQR_WARPS = HQR_THREADS / 32;
constexpr int HQR_MAX_L = 96;

__device__ __forceinline__ float hqr_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Two (four) warp sums at once by exchanging halves of the values at the
// first (two) levels instead of reducing each value separately: 5 + 2
// broadcasts (6 + 4) shuffles instead of 10 (20); every lane gets every sum.
__device__ __forceinline__ void hqr_sum2(float& a, float& b, int lane) {
  const bool up = lane & 16;
  float k = up ? b : a;
  k += __shfl_xor_sync(0xffffffffu, up ? a : b, 16);   // a in the low half, b in the high
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  a = __shfl_sync(0xffffffffu, k, 0);
  b = __shfl_sync(0xffffffffu, k, 16);
}
__device__ __forceinline__ void hqr_sum4(float (&d)[4], int lane) {
  const bool up = lane & 16, mid = lane & 8;
  float k0 = up ? d[2] : d[0], k1 = up ? d[3] : d[1];
  k0 += __shfl_xor_sync(0xffffffffu, up ? d[0] : d[2], 16);
  k1 += __shfl_xor_sync(0xffffffffu, up ? d[1] : d[3], 16);
  float k = mid ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, mid ? k0 : k1, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  // lanes 0-7 hold sum 0, 8-15 sum 1, 16-23 sum 2, 24-31 sum 3
#pragma unroll
  for (int u = 0; u < 4; ++u) d[u] = __shfl_sync(0xffffffffu, k, 8 * u);
}

// Reflector of column a (rows j .. p-1), one warp: rows j+1.. become v,
// row j becomes beta; returns tau (0 when the column is already beta e_j with
// beta real).
__device__ float2 hqr_reflector(float2* a, int j, int p, int lane) {
  const float2 al = a[j];
  float s = 0.f;
  for (int r = j + 1 + lane; r < p; r += 32) {
    const float2 x = a[r];
    s = fmaf(x.x, x.x, fmaf(x.y, x.y, s));
  }
  s = hqr_sum(s);
  if (s == 0.f && al.y == 0.f) return make_float2(0.f, 0.f);
  const float nrm = sqrtf(fmaf(al.x, al.x, fmaf(al.y, al.y, s)));
  const float beta = al.x >= 0.f ? -nrm : nrm;
  // v = x / (alpha - beta); |alpha - beta| >= nrm > 0 by the sign of beta
  const float dr = al.x - beta, di = al.y;
  const float den = fmaf(dr, dr, di * di);
  const float sr = dr / den, si = -di / den;
  for (int r = j + 1 + lane; r < p; r += 32) {
    const float2 x = a[r];
    a[r] = make_float2(x.x * sr - x.y * si, x.x * si + x.y * sr);
  }
  __syncwarp();
  if (lane == 0) a[j] = make_float2(beta, 0.f);
  return make_float2((beta - al.x) / beta, -al.y / beta);
}

// v_j of column a into registers: row r = lane + 32 t, 1 at row j, 0 above.
// FULL: p == 32 RPL, so that every lane's rows exist; rows above j then
// need no predicate (v is zero there, so they are read and rewritten
// unchanged).
template <int RPL, bool FULL>
__device__ __forceinline__ void hqr_load_v(const float2* a, int j, int p, int lane,
                                           float2 (&v)[RPL]) {
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int r = lane + 32 * t;
    if (FULL) {
      const float2 x = a[r];
      v[t] = r > j ? x : make_float2(r == j ? 1.f : 0.f, 0.f);
    } else {
      v[t] = (r <= j || r >= p) ? make_float2(r == j ? 1.f : 0.f, 0.f) : a[r];
    }
  }
}

// c <- c - f v (v^H c) on rows j .. p-1 (f = conj(tau) applies H^H, f = tau H)
template <int RPL, bool FULL>
__device__ __forceinline__ void hqr_apply(const float2 (&v)[RPL], float2* c, int j, int p,
                                          float2 f, int lane) {
  float2 x[RPL];
  float dr = 0.f, di = 0.f;
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int r = lane + 32 * t;
    x[t] = (FULL || (r >= j && r < p)) ? c[r] : make_float2(0.f, 0.f);
    dr = fmaf(v[t].x, x[t].x, fmaf(v[t].y, x[t].y, dr));    // Re(conj(v) x)
    di = fmaf(v[t].x, x[t].y, fmaf(-v[t].y, x[t].x, di));   // Im(conj(v) x)
  }
  hqr_sum2(dr, di, lane);
  const float gr = f.x * dr - f.y * di, gi = f.x * di + f.y * dr;
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int r = lane + 32 * t;
    if (FULL || (r >= j && r < p))
      c[r] = make_float2(x[t].x - (v[t].x * gr - v[t].y * gi),
                         x[t].y - (v[t].x * gi + v[t].y * gr));
  }
}

// hqr_apply on two columns at once (their sums interleave in the shuffles)
template <int RPL, bool FULL>
__device__ __forceinline__ void hqr_apply2(const float2 (&v)[RPL], float2* c0, float2* c1, int j,
                                           int p, float2 f, int lane) {
  float2 x0[RPL], x1[RPL];
  float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int r = lane + 32 * t;
    const bool in = FULL || (r >= j && r < p);
    x0[t] = in ? c0[r] : make_float2(0.f, 0.f);
    x1[t] = in ? c1[r] : make_float2(0.f, 0.f);
    d[0] = fmaf(v[t].x, x0[t].x, fmaf(v[t].y, x0[t].y, d[0]));
    d[1] = fmaf(v[t].x, x0[t].y, fmaf(-v[t].y, x0[t].x, d[1]));
    d[2] = fmaf(v[t].x, x1[t].x, fmaf(v[t].y, x1[t].y, d[2]));
    d[3] = fmaf(v[t].x, x1[t].y, fmaf(-v[t].y, x1[t].x, d[3]));
  }
  hqr_sum4(d, lane);
  const float g0r = f.x * d[0] - f.y * d[1], g0i = f.x * d[1] + f.y * d[0];
  const float g1r = f.x * d[2] - f.y * d[3], g1i = f.x * d[3] + f.y * d[2];
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int r = lane + 32 * t;
    if (FULL || (r >= j && r < p)) {
      c0[r] = make_float2(x0[t].x - (v[t].x * g0r - v[t].y * g0i),
                          x0[t].y - (v[t].x * g0i + v[t].y * g0r));
      c1[r] = make_float2(x1[t].x - (v[t].x * g1r - v[t].y * g1i),
                          x1[t].y - (v[t].x * g1i + v[t].y * g1r));
    }
  }
}

// Column k of Q from its reflector (stored in place): H_k e_k restricted to
// rows k.. -- 1 - tau at row k, -tau v below -- and zeros above.
__device__ __forceinline__ void hqr_materialize(float2* a, int k, int p, float2 tau, int lane) {
  for (int r = lane; r < p; r += 32) {
    float2 y;
    if (r < k) {
      y = make_float2(0.f, 0.f);
    } else if (r == k) {
      y = make_float2(1.f - tau.x, -tau.y);
    } else {
      const float2 v = a[r];
      y = make_float2(-(tau.x * v.x - tau.y * v.y), -(tau.x * v.y + tau.y * v.x));
    }
    a[r] = y;
  }
}

// One CTA per slice; RPL rows per lane (p <= 32 RPL).
// keep_phase: column j of Q is multiplied by sign(R(j, j)) (R's diagonal is
// real), so that for Y with nearly orthonormal columns Q(:, j) stays close
// to Y(:, j) instead of possibly flipping its sign.
// Split planes (sp non-null): Q also leaves as the hi/lo planes (bf16 or
// tf32, dftc::put_split) of the next tensor-core product's B operand,
// K-major with leading dimension ldk >= p (rows p .. ldk-1 and the columns
// from l on zero), slice stride ldk * lfull -- the operand split fused.
struct HqrSplit {
  float* p0;
  float* p1;
  float* p2;
  float* p3;
  int64_t ldk;
  int bf16;
};

template <int RPL, bool FULL>
__global__ void __launch_bounds__(HQR_THREADS) householder_qr_kernel(float* y_re, float* y_im,
                                                                     int64_t sY, int p, int lfull,
                                                                     const int32_t* lcols,
                                                                     int keep_phase, HqrSplit sp) {
  extern __shared__ float2 hqr_a[];   // Y, then Q: p x l column-major
  __shared__ float2 tau_s[HQR_MAX_L];
  __shared__ float sgn_s[HQR_MAX_L];   // sign of R(j, j)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // per-slice column count (the per-frequency sketch size): the columns from
  // l on are left zero
  const int l = lcols ? min(max(int(lcols[blockIdx.x]), 1), lfull) : lfull;
  float* yr = y_re + int64_t(blockIdx.x) * sY;
  float* yi = y_im + int64_t(blockIdx.x) * sY;
  float2* A = hqr_a;
  for (int e = threadIdx.x; e < p * l; e += HQR_THREADS) A[e] = make_float2(yr[e], yi[e]);
  __syncthreads();
  if (warp == 0) {
    const float2 t = hqr_reflector(A, 0, p, lane);
    if (lane == 0) {
      tau_s[0] = t;
      sgn_s[0] = A[0].x < 0.f ? -1.f : 1.f;
    }
  }
  __syncthreads();
  // factorisation: step j applies H_j^H to columns j+1 .. l-1
  for (int j = 0; j + 1 < l; ++j) {
    const float2 tau = tau_s[j];
    float2 v[RPL];
    hqr_load_v<RPL, FULL>(A + int64_t(j) * p, j, p, lane, v);
    const bool live = tau.x != 0.f || tau.y != 0.f;
    const float2 f = make_float2(tau.x, -tau.y);
    int k = j + 1 + warp;
    if (warp == 0) {   // look-ahead: column j + 1 first, then its reflector
      float2* c = A + int64_t(k) * p;
      if (live) hqr_apply<RPL, FULL>(v, c, j, p, f, lane);
      __syncwarp();
      const float2 t = hqr_reflector(c, k, p, lane);
      if (lane == 0) {
        tau_s[k] = t;
        sgn_s[k] = c[k].x < 0.f ? -1.f : 1.f;
      }
      k += HQR_WARPS;
    }
    if (live) {
      for (; k + HQR_WARPS < l; k += 2 * HQR_WARPS)
        hqr_apply2<RPL, FULL>(v, A + int64_t(k) * p, A + int64_t(k + HQR_WARPS) * p, j, p, f, lane);
      if (k < l) hqr_apply<RPL, FULL>(v, A + int64_t(k) * p, j, p, f, lane);
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{l-1} [I; 0]: step i applies H_i to columns i+1 .. l-1,
  // whose first (column i + 1) its owner first turns from reflector storage
  // into H_{i+1} e_{i+1}
  for (int i = l - 2; i >= 0; --i) {
    const float2 tau = tau_s[i];
    float2 v[RPL];
    hqr_load_v<RPL, FULL>(A + int64_t(i) * p, i, p, lane, v);
    int k = i + 1 + warp;
    if (warp == 0) {
      hqr_materialize(A + int64_t(k) * p, k, p, tau_s[k], lane);
      __syncwarp();
    }
    if (tau.x != 0.f || tau.y != 0.f) {
      for (; k + HQR_WARPS < l; k += 2 * HQR_WARPS)
        hqr_apply2<RPL, FULL>(v, A + int64_t(k) * p, A + int64_t(k + HQR_WARPS) * p, i, p, tau, lane);
      if (k < l) hqr_apply<RPL, FULL>(v, A + int64_t(k) * p, i, p, tau, lane);
    }
    __syncthreads();
  }
  if (warp == 0) hqr_materialize(A, 0, p, tau_s[0], lane);
  __syncthreads();
  for (int e = threadIdx.x; e < p * l; e += HQR_THREADS) {
    const float2 q = A[e];
    const float sg = keep_phase ? sgn_s[e / p] : 1.f;
    yr[e] = sg * q.x;
    yi[e] = sg * q.y;
  }
  for (int e = p * l + threadIdx.x; e < p * lfull; e += HQR_THREADS) {
    yr[e] = 0.f;
    yi[e] = 0.f;
  }
  if (sp.p0) {
    const int64_t base = int64_t(blockIdx.x) * sp.ldk * lfull;
    for (int64_t e = threadIdx.x; e < sp.ldk * lfull; e += HQR_THREADS) {
      const int c = int(e / sp.ldk), r = int(e - int64_t(c) * sp.ldk);
      float2 q = make_float2(0.f, 0.f);
      if (r < p && c < l) {
        q = A[c * p + r];
        if (keep_phase) {
          q.x *= sgn_s[c];
          q.y *= sgn_s[c];
        }
      }
      dftc::put_split(sp.p0, sp.p1, sp.bf16 != 0, base + e, q.x);
      dftc::put_split(sp.p2, sp.p3, sp.bf16 != 0, base + e, q.y);
    }
  }
}

// ---------------------------------------------------------------- core eigensolver
__device__ __forceinline__ float eig_warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Householder reduction of the Hermitian l x l matrix G (row stride ls, both
// triangles held) to a real symmetric tridiagonal T = Q^H G Q with
// Q = H_0 H_1 ... H_{l-2}.  Step j takes the reflector H_j = I - tau_j v v^H
// of column j below the diagonal (chosen as LAPACK's zlarfg chooses it, so
// that the new off-diagonal beta_j is real; the last step, on a single
// entry, only makes the last off-diagonal real) and applies H_j^H . H_j to
// the trailing block as the rank-2 change A - v w^H - w v^H with y = tau A v
// and w = y - (1/2) tau (y^H v) v.  On exit d and e hold T's diagonal and
// off-diagonal; v_j (after its leading 1) sits in row j of G right of
// column j + 1, tau_j in tau.
__device__ void hermitian_tridiag(float2* G, int l, int ls, float* d, float* e, float2* tau,
                                  float2* vbuf, float2* ybuf) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j + 1 < l; ++j) {
    const int m = l - 1 - j;
    float2* row = G + j * ls + j + 1;   // conj of column j below the diagonal
    if (warp == 0) {
      float s = 0.f;
      for (int t = 1 + lane; t < m; t += 32) {
        const float2 x = row[t];
        s = fmaf(x.x, x.x, fmaf(x.y, x.y, s));
      }
      s = eig_warp_sum(s);
      const float2 al = make_float2(row[0].x, -row[0].y);
      float2 tj = make_float2(0.f, 0.f);
      float beta = al.x;
      float sr = 0.f, si = 0.f;   // 1 / (alpha - beta), 0 when H_j = I
      if (!(s == 0.f && al.y == 0.f)) {
        const float nrm = sqrtf(fmaf(al.x, al.x, fmaf(al.y, al.y, s)));
        beta = al.x >= 0.f ? -nrm : nrm;
        tj = make_float2((beta - al.x) / beta, -al.y / beta);
        const float dr = al.x - beta, di = al.y, den = fmaf(dr, dr, di * di);
        sr = dr / den;
        si = -di / den;
      }
      for (int t = 1 + lane; t < m; t += 32) {
        const float2 x = make_float2(row[t].x, -row[t].y);
        const float2 v = make_float2(x.x * sr - x.y * si, x.x * si + x.y * sr);
        row[t] = v;
        vbuf[t] = v;
      }
      if (lane == 0) {
        vbuf[0] = make_float2(1.f, 0.f);
        tau[j] = tj;
        e[j] = beta;
      }
    }
    __syncthreads();
    const float2 tj = tau[j];
    if (tj.x != 0.f || tj.y != 0.f) {   // block-uniform
      // y = tau A v over the trailing block A = G(j+1:, j+1:), four threads a row
      for (int base = 0; base < m; base += int(blockDim.x) >> 2) {
        const int i = base + (tid >> 2), part = tid & 3;
        float ar = 0.f, ai = 0.f;
        if (i < m) {
          const float2* Ai = G + (j + 1 + i) * ls + (j + 1);
          for (int t = part; t < m; t += 4) {
            const float2 a = Ai[t], v = vbuf[t];
            ar = fmaf(a.x, v.x, fmaf(-a.y, v.y, ar));
            ai = fmaf(a.x, v.y, fmaf(a.y, v.x, ai));
          }
        }
        ar += __shfl_xor_sync(0xffffffffu, ar, 1);
        ai += __shfl_xor_sync(0xffffffffu, ai, 1);
        ar += __shfl_xor_sync(0xffffffffu, ar, 2);
        ai += __shfl_xor_sync(0xffffffffu, ai, 2);
        if (i < m && part == 0)
          ybuf[i] = make_float2(tj.x * ar - tj.y * ai, tj.x * ai + tj.y * ar);
      }
      __syncthreads();
      // tau (y^H v) is real (|tau|^2 v^H A v): alpha' = -Re(tau y^H v) / 2
      float hr = 0.f, hi = 0.f;
      for (int t = lane; t < m; t += 32) {
        const float2 y = ybuf[t], v = vbuf[t];
        hr = fmaf(y.x, v.x, fmaf(y.y, v.y, hr));
        hi = fmaf(y.x, v.y, fmaf(-y.y, v.x, hi));
      }
      hr = eig_warp_sum(hr);
      hi = eig_warp_sum(hi);
      const float ap = -0.5f * (tj.x * hr - tj.y * hi);
      for (int i = warp; i < m; i += nw) {
        const float2 vi = vbuf[i], yi = ybuf[i];
        const float2 wi = make_float2(fmaf(ap, vi.x, yi.x), fmaf(ap, vi.y, yi.y));
        float2* Ai = G + (j + 1 + i) * ls + (j + 1);
        for (int t = lane; t < m; t += 32) {
          const float2 vt = vbuf[t], yt = ybuf[t];
          const float2 wt = make_float2(fmaf(ap, vt.x, yt.x), fmaf(ap, vt.y, yt.y));
          // v_i conj(w_t) + w_i conj(v_t)
          const float re = vi.x * wt.x + vi.y * wt.y + wi.x * vt.x + wi.y * vt.y;
          const float im = vi.y * wt.x - vi.x * wt.y + wi.y * vt.x - wi.x * vt.y;
          float2 a = Ai[t];
          a.x -= re;
          a.y -= im;
          Ai[t] = a;
        }
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < l; i += blockDim.x) {
    d[i] = G[i * ls + i].x;
    if (i == l - 1) e[i] = 0.f;
  }
  __syncthreads();
}

// Q = H_0 H_1 ... H_{l-2} into W (column-major, column stride ls) by
// backward accumulation from W = I: step j applies H_j to rows j+1.. of
// columns j+1.. (a warp per column).
__device__ void tridiag_form_q(const float2* G, float2* W, int l, int ls, const float2* tau) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int c = e / l, r = e - c * l;
    W[c * ls + r] = make_float2(r == c ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  for (int j = l - 2; j >= 0; --j) {
    const float2 tj = tau[j];
    if (tj.x != 0.f || tj.y != 0.f) {
      const int m = l - 1 - j;
      const float2* vr = G + j * ls + j + 1;
      for (int c = j + 1 + warp; c < l; c += nw) {
        float2* z = W + c * ls + j + 1;
        float dr = 0.f, di = 0.f;
        for (int t = lane; t < m; t += 32) {
          const float2 v = t == 0 ? make_float2(1.f, 0.f) : vr[t];
          const float2 x = z[t];
          dr = fmaf(v.x, x.x, fmaf(v.y, x.y, dr));    // conj(v) x
          di = fmaf(v.x, x.y, fmaf(-v.y, x.x, di));
        }
        dr = eig_warp_sum(dr);
        di = eig_warp_sum(di);
        const float gr = tj.x * dr - tj.y * di, gi = tj.x * di + tj.y * dr;
        for (int t = lane; t < m; t += 32) {
          const float2 v = t == 0 ? make_float2(1.f, 0.f) : vr[t];
          float2 x = z[t];
          x.x -= v.x * gr - v.y * gi;
          x.y -= v.x * gi + v.y * gr;
          z[t] = x;
        }
      }
    }
    __syncthreads();
  }
}

// Eigenvalues of the real symmetric tridiagonal (d, e) -- d[i * stride],
// e[i * stride], e[l-1] = 0 -- by the implicit QL algorithm with
// Wilkinson's shift from the leading 2 x 2 (Bowdler, Martin, Reinsch and
// Wilkinson, 1968), run by one thread: each chase goes from the bottom of
// the unreduced block to its top, deflating off-diagonals below
// FLT_EPSILON (|d_m| + |d_m+1|), and its plane rotations are appended to
// log (at most cap; rotation i mixes columns i and i + 1, code i, or
// -(i + 1) for a chase's first rotation).  T is first scaled by a power of
// two to a largest entry near 1 (exact; only the eigenvectors are used), so
// that the squares stay in range and one refined reciprocal square root
// forms each rotation.  Returns false if an eigenvalue took more
// than max_iter chases (its off-diagonal is then dropped) or the log was
// full (the chase stops there); *count gets the log's length.
struct QlRot {
  int code;
  float c, s;
};

__device__ bool ql_chase(float* __restrict__ d, float* __restrict__ e, int stride, int l,
                         QlRot* __restrict__ log, int cap, int max_iter, int* count) {
#define D(i) d[(i) * stride]
#define E(i) e[(i) * stride]
  float mx = 0.f;
  for (int i = 0; i < l; ++i) mx = fmaxf(mx, fmaxf(fabsf(D(i)), fabsf(E(i))));
  if (mx > 0.f && isfinite(mx)) {
    int ex;
    frexpf(mx, &ex);
    for (int i = 0; i < l; ++i) {
      D(i) = ldexpf(D(i), -ex);
      E(i) = ldexpf(E(i), -ex);
    }
  }
  bool ok = true;
  int cnt = 0, l0 = 0, it = 0;
  while (l0 < l) {
    int m = l0;
    for (; m + 1 < l; ++m) {
      const float dd = fabsf(D(m)) + fabsf(D(m + 1));
      if (fabsf(E(m)) <= FLT_EPSILON * dd) break;
    }
    if (m == l0) {
      ++l0;
      it = 0;
      continue;
    }
    if (cnt + (m - l0) > cap || ++it > max_iter) {
      ok = false;
      E(l0) = 0.f;
      continue;
    }
    float g = (D(l0 + 1) - D(l0)) / (2.f * E(l0));
    const float r0 = hypotf(g, 1.f);
    g = D(m) - D(l0) + E(l0) / (g + copysignf(r0, g));
    float s = 1.f, c = 1.f, pp = 0.f;
    float dn = D(m);   // d[i + 1] of the step below, carried
    bool early = false;
    // e[i] and d[i] of the next step are loaded a step ahead (a step writes
    // only index i + 1), off the chain of dependent arithmetic
    float ei_n = E(m - 1), di_n = D(m - 1);
    for (int i = m - 1; i >= l0; --i) {
      const float ei = ei_n, di = di_n;
      if (i > l0) {
        ei_n = E(i - 1);
        di_n = D(i - 1);
      }
      const float f = s * ei, b = c * ei;
      // r = sqrt(f^2 + g^2) and 1/r from the hardware reciprocal square root
      // refined by one Newton-Raphson step y (3 - x y^2) / 2 (subnormal x:
      // the rounded square root and reciprocal)
      const float x = fmaf(f, f, g * g);
      float r, inv;
      if (x >= FLT_MIN) {
        float y = rsqrtf(x);
        y *= fmaf(-0.5f * x, y * y, 1.5f);
        inv = y;
        r = x * y;
      } else {
        r = sqrtf(x);
        inv = r > 0.f ? __frcp_rn(r) : 0.f;
      }
      E(i + 1) = r;
      if (r == 0.f) {   // the chase splits: restart from the new block
        D(i + 1) = dn - pp;
        E(m) = 0.f;
        early = true;
        break;
      }
      s = f * inv;
      c = g * inv;
      g = dn - pp;
      r = fmaf(di - g, s, 2.f * c * b);
      pp = s * r;
      D(i + 1) = g + pp;
      g = fmaf(c, r, -b);
      dn = di;
      log[cnt++] = QlRot{i == m - 1 ? -(i + 1) : i, c, s};
    }
    if (!early) {
      D(l0) = D(l0) - pp;
      E(l0) = g;
      E(m) = 0.f;
    }
  }
#undef D
#undef E
  *count = cnt;
  return ok;
}

// W <- W S for the logged rotations (W column-major, column stride ls), a
// thread per row and component (threads 0 .. 2l-1), one chunk of the log
// (in shared memory) at a time: the column the next rotation of a chase
// reuses is carried in a register (prev, carry) from chunk to chunk, and
// ql_replay_end stores the last one.
__device__ __forceinline__ void ql_replay(float2* W, int l, int ls,
                                          const QlRot* __restrict__ log, int cnt, int& prev,
                                          float& carry) {
  if (int(threadIdx.x) >= 2 * l) return;
  // W(r, i), component t & 1 of row r = t >> 1, at float index 2 ls i + t
  float* __restrict__ z = reinterpret_cast<float*>(W) + threadIdx.x;
  const int cs = 2 * ls;
#pragma unroll 4
  for (int q = 0; q < cnt; ++q) {
    const QlRot R = log[q];
    const int i = R.code < 0 ? -R.code - 1 : R.code;
    if (R.code < 0) {   // a new chase: the previous one's last column first
      if (prev >= 0) z[cs * prev] = carry;
      carry = z[cs * (i + 1)];
    }
    const float zi = z[cs * i];
    z[cs * (i + 1)] = fmaf(R.s, zi, R.c * carry);
    carry = fmaf(R.c, zi, -R.s * carry);
    prev = i;
  }
}
__device__ __forceinline__ void ql_replay_end(float2* W, int l, int ls, int prev, float carry) {
  if (int(threadIdx.x) < 2 * l && prev >= 0)
    reinterpret_cast<float*>(W)[threadIdx.x + 2 * ls * prev] = carry;
}

// Core SVD through the l x l Gram of B^H (n2 x l, read from global memory,
// which the previous product left in L2): G = B B^H = W diag(s^2) W^H by the
// Householder tridiagonalization and implicit QL above (float32).  The
// singular values are then the Rayleigh quotients s_j = ||B^H w_j|| (float32
// products, float64 sums of squares), whose error is second order in the
// error of w_j -- the square roots of G's float32 eigenvalues would carry an
// error u ||G|| / (2 s_j) that grows as 1/s_j.  B^H itself is a float32
// product of float32 data, so its singular values are only defined to about
// u32 s_1 (absolute), which is also the eigensolver's accuracy; a
// relatively accurate (Jacobi) solve would not change the result beyond
// that.  The top k give W_k (left singular vectors of B), S = diag(s) and
// V_k = B^H W_k S^{-1}.
constexpr int EIG_THREADS = 256;
constexpr int EIG_CHUNK = 32;   // rows of B^H staged per step of the Gram

__global__ void __launch_bounds__(EIG_THREADS) core_tridiag_kernel(
    const float* __restrict__ bh_re, const float* __restrict__ bh_im, int p, int l,
    float* __restrict__ d_out, float* __restrict__ e_out, float2* __restrict__ z_out) {
  extern __shared__ double dyn[];
  const int ls = l | 1;                                     // odd stride
  const int L2 = l * ls;
  float2* Gf = reinterpret_cast<float2*>(dyn);              // l x l Gram (row stride ls)
  float2* Wf = Gf + L2;                                     // l x l Q (column stride ls)
  float2* tau = Wf + L2;                                    // l: reflectors of the reduction
  float2* vbuf = tau + l;                                   // l
  float2* ybuf = vbuf + l;                                  // l
  float* dv = reinterpret_cast<float*>(ybuf + l);           // l: tridiagonal
  float* ev = dv + l;                                       // l
  const int64_t f = blockIdx.x;
  const float* br = bh_re + f * int64_t(p) * l;
  const float* bi = bh_im + f * int64_t(p) * l;
  // G(a, b) = sum_r conj(B^H(r, a)) B^H(r, b), a <= b, Hermitian fill: rows of
  // B^H staged EIG_CHUNK at a time (in W's space, before W is set)
  float2* chunk = Wf;                                       // EIG_CHUNK x l, row stride l
  const int npairs = l * (l + 1) / 2;
  constexpr int PPT = 6;                                    // pairs per thread and pass
  for (int base = 0; base < npairs; base += PPT * EIG_THREADS) {
    int pa[PPT], pb[PPT];
    float gr[PPT], gi[PPT];
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      const int e = base + u * EIG_THREADS + threadIdx.x;
      int a = 0, rem = e;
      while (a < l && rem >= l - a) { rem -= l - a; ++a; }
      pa[u] = e < npairs ? a : -1;
      pb[u] = a + rem;
      gr[u] = 0.f;
      gi[u] = 0.f;
    }
    const int ch = min(EIG_CHUNK, ls);   // the chunk (ch x l) fits in W's l x ls
    for (int r0 = 0; r0 < p; r0 += ch) {
      const int nr = min(ch, p - r0);
      __syncthreads();
      for (int e = threadIdx.x; e < nr * l; e += EIG_THREADS) {
        const int c = e / nr, r = e - c * nr;
        chunk[r * l + c] = make_float2(__ldg(br + r0 + r + int64_t(p) * c),
                                       __ldg(bi + r0 + r + int64_t(p) * c));
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < PPT; ++u) {
        if (pa[u] < 0) continue;
        for (int r = 0; r < nr; ++r) {
          const float2 x = chunk[r * l + pa[u]], y = chunk[r * l + pb[u]];
          gr[u] = fmaf(x.x, y.x, fmaf(x.y, y.y, gr[u]));
          gi[u] = fmaf(x.x, y.y, fmaf(-x.y, y.x, gi[u]));
        }
      }
    }
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      if (pa[u] < 0) continue;
      Gf[pa[u] * ls + pb[u]] = make_float2(gr[u], gi[u]);
      Gf[pb[u] * ls + pa[u]] = make_float2(gr[u], -gi[u]);
    }
  }
  __syncthreads();
  hermitian_tridiag(Gf, l, ls, dv, ev, tau, vbuf, ybuf);
  tridiag_form_q(Gf, Wf, l, ls, tau);
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    d_out[f * l + i] = dv[i];
    e_out[f * l + i] = ev[i];
  }
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int c = e / l, r = e - c * l;
    z_out[f * l * l + e] = Wf[c * ls + r];
  }
}

// The QL chase of every slice in a block of its own (lane 0 chases, d and e
// in shared memory), away from the blocks that form and use the
// eigenvectors: the chases of different slices run concurrently on every
// SM, and no lane waits on another slice's chase.
constexpr int QL_THREADS = 32;
constexpr int QL_LOG_PER_L = 100;   // log capacity per slice: 100 l rotations

__global__ void __launch_bounds__(QL_THREADS) core_ql_kernel(
    const float* __restrict__ d_in, const float* __restrict__ e_in, int l,
    QlRot* __restrict__ log, int32_t* __restrict__ log_count, int max_iter, int32_t* status) {
  extern __shared__ float qsm[];   // d (l), e (l)
  const int64_t f = blockIdx.x;
  if (threadIdx.x != 0) return;
  float* d = qsm;
  float* e = qsm + l;
  for (int i = 0; i < l; ++i) {
    d[i] = d_in[f * l + i];
    e[i] = i + 1 < l ? e_in[f * l + i] : 0.f;
  }
  const int cap = QL_LOG_PER_L * l;
  int cnt = 0;
  const bool ok = ql_chase(d, e, 1, l, log + f * cap, cap, max_iter, &cnt);
  log_count[f] = cnt;
  if (!ok && status) atomicOr(status, TP_DEV_NOCONV);
}

constexpr int FIN_RB = 64;   // rows of B^H staged per step of P = B^H W

__global__ void __launch_bounds__(EIG_THREADS) core_finish_kernel(
    const float* __restrict__ bh_re, const float* __restrict__ bh_im, int p, int l, int k,
    const float2* __restrict__ z_in, const QlRot* __restrict__ log,
    const int32_t* __restrict__ log_count, float* __restrict__ wkr, float* __restrict__ wki,
    float* __restrict__ vkr, float* __restrict__ vki, float* __restrict__ sr_out,
    float* __restrict__ si_out, float2* __restrict__ pscratch, const int32_t* __restrict__ rank,
    const float* __restrict__ q_re, const float* __restrict__ q_im, int n1,
    float* __restrict__ ur, float* __restrict__ ui) {
  extern __shared__ double dyn[];
  const int ls = l | 1;
  double* sig2 = dyn;                                       // l: ||B^H w_j||^2
  float2* Wf = reinterpret_cast<float2*>(dyn + ((l + 1) & ~1));   // l x l (column stride ls)
  float2* stage = Wf + size_t(l) * ls;                      // FIN_RB x l: log chunks, rows of B^H
  __shared__ int order[128];
  const int64_t f = blockIdx.x;
  const float* br = bh_re + f * int64_t(p) * l;
  const float* bi = bh_im + f * int64_t(p) * l;
  float2* P = pscratch + f * int64_t(p) * l;                // B^H W (p x l), column-major
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int c = e / l, r = e - c * l;
    Wf[c * ls + r] = z_in[f * l * l + e];
  }
  for (int j = threadIdx.x; j < l; j += blockDim.x) sig2[j] = 0.0;
  // replay the QL log on W, a chunk of it in shared memory at a time
  {
    QlRot* chunk = reinterpret_cast<QlRot*>(stage);
    const int ccap = int(size_t(FIN_RB) * l * sizeof(float2) / sizeof(QlRot));
    const QlRot* lg = log + f * int64_t(QL_LOG_PER_L) * l;
    const int cnt = log_count[f];
    int prev = -1;
    float carry = 0.f;
    for (int q0 = 0; q0 < cnt; q0 += ccap) {
      const int nq = min(ccap, cnt - q0);
      __syncthreads();
      for (int e = threadIdx.x; e < nq; e += blockDim.x) chunk[e] = lg[q0 + e];
      __syncthreads();
      ql_replay(Wf, l, ls, chunk, nq, prev, carry);
    }
    ql_replay_end(Wf, l, ls, prev, carry);
  }
  // P = B^H W and s_j^2 = ||P(:, j)||^2, FIN_RB rows of B^H at a time in
  // shared memory: a warp per column, lanes over rows
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int r0 = 0; r0 < p; r0 += FIN_RB) {
    const int nr = min(FIN_RB, p - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * l; e += blockDim.x) {
      const int m = e / nr, rr = e - m * nr;
      stage[m * FIN_RB + rr] = make_float2(__ldg(br + r0 + rr + int64_t(p) * m),
                                           __ldg(bi + r0 + rr + int64_t(p) * m));
    }
    __syncthreads();
    for (int j = warp; j < l; j += nwarp) {
      const float2* wj = Wf + j * ls;
      double acc = 0.0;
      for (int rr = lane; rr < nr; rr += 32) {
        float pr = 0.f, pim = 0.f;
        for (int m = 0; m < l; ++m) {
          const float2 b = stage[m * FIN_RB + rr];
          const float2 w = wj[m];
          pr = fmaf(b.x, w.x, fmaf(-b.y, w.y, pr));
          pim = fmaf(b.x, w.y, fmaf(b.y, w.x, pim));
        }
        P[r0 + rr + int64_t(p) * j] = make_float2(pr, pim);
        acc += double(pr) * pr + double(pim) * pim;
      }
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) sig2[j] += acc;   // column j belongs to this warp in every chunk
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < l; j += blockDim.x) {
    const double lj = sig2[j];
    int rank = 0;
    for (int m = 0; m < l; ++m) {
      const double lm = sig2[m];
      rank += (lm > lj) || (lm == lj && m < j);
    }
    order[rank] = j;
  }
  __syncthreads();
  // the slice keeps its top kr triplets (per-frequency rank), zeros after
  const int kr = rank ? min(max(int(rank[f]), 0), k) : k;
  for (int e = threadIdx.x; e < l * k; e += blockDim.x) {
    const int i = e % l, c = e / l;
    const float2 w = c < kr ? Wf[order[c] * ls + i] : make_float2(0.f, 0.f);
    wkr[f * l * k + e] = w.x;
    wki[f * l * k + e] = w.y;
  }
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e % k, c = e / k;
    sr_out[f * k * k + e] = (i == c && c < kr) ? float(sqrt(sig2[order[c]])) : 0.f;
    si_out[f * k * k + e] = 0.f;
  }
  // V_k = B^H W_k S^{-1}: the columns of P in order, scaled
  for (int c = warp; c < k; c += nwarp) {
    const int j = order[c];
    const double sg = sqrt(sig2[j]);
    const float inv = (sg > 0.0 && c < kr) ? float(1.0 / sg) : 0.f;
    for (int r = lane; r < p; r += 32) {
      const float2 v = P[r + int64_t(p) * j];
      vkr[f * int64_t(p) * k + r + int64_t(p) * c] = v.x * inv;
      vki[f * int64_t(p) * k + r + int64_t(p) * c] = v.y * inv;
    }
  }
  // U_hat = Q W_k (ur non-null): FIN_RB rows of Q (n1 x l) at a time in
  // shared memory, a warp per column
  if (ur) {
    const float* qrf = q_re + f * int64_t(n1) * l;
    const float* qif = q_im + f * int64_t(n1) * l;
    for (int r0 = 0; r0 < n1; r0 += FIN_RB) {
      const int nr = min(FIN_RB, n1 - r0);
      __syncthreads();
      for (int e = threadIdx.x; e < nr * l; e += blockDim.x) {
        const int m = e / nr, rr = e - m * nr;
        stage[m * FIN_RB + rr] = make_float2(__ldg(qrf + r0 + rr + int64_t(n1) * m),
                                             __ldg(qif + r0 + rr + int64_t(n1) * m));
      }
      __syncthreads();
      for (int c = warp; c < k; c += nwarp) {
        const float2* wj = Wf + order[c] * ls;
        for (int rr = lane; rr < nr; rr += 32) {
          float pr = 0.f, pim = 0.f;
          if (c < kr)
            for (int m = 0; m < l; ++m) {
              const float2 q = stage[m * FIN_RB + rr];
              const float2 w = wj[m];
              pr = fmaf(q.x, w.x, fmaf(-q.y, w.y, pr));
              pim = fmaf(q.x, w.y, fmaf(q.y, w.x, pim));
            }
          ur[f * int64_t(n1) * k + r0 + rr + int64_t(n1) * c] = pr;
          ui[f * int64_t(n1) * k + r0 + rr + int64_t(n1) * c] = pim;
        }
      }
    }
  }
}

size_t core_tridiag_smem(int l) {
  const size_t L2 = size_t(l) * (l | 1);
  return 2 * L2 * 8 + size_t(l) * (3 * 8 + 2 * 4);
}
size_t core_finish_smem(int l) {
  const size_t L2 = size_t(l) * (l | 1);
  return size_t((l + 1) & ~1) * 8 + L2 * 8 + size_t(FIN_RB) * l * 8;
}

// Sorts the l Jacobi singular triplets of every slice, keeps the top k and
// writes: Wk (l x k, float32 planar; right factor of the small problem, the
// columns of W), Vk (n2 x k, float32; left singular vectors of B^H = right
// ones of X_hat), S (k x k diagonal).
__global__ void pick_topk_kernel(const double* __restrict__ gr, const double* __restrict__ gi,
                                 int64_t sG, const double* __restrict__ wr,
                                 const double* __restrict__ wi, int64_t sW,
                                 const double* __restrict__ sig, int p, int l, int k,
                                 float* __restrict__ wkr, float* __restrict__ wki,
                                 float* __restrict__ vkr, float* __restrict__ vki,
                                 float* __restrict__ sr, float* __restrict__ si) {
  extern __shared__ int order[];
  const int64_t f = blockIdx.x;
  const double* s = sig + f * l;
  for (int j = threadIdx.x; j < l; j += blockDim.x) {
    const double sj = s[j];
    int rank = 0;
    for (int m = 0; m < l; ++m) rank += (s[m] > sj) || (s[m] == sj && m < j);
    order[rank] = j;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < l * k; e += blockDim.x) {
    const int i = e % l, c = e / l;
    const int j = order[c];
    wkr[f * l * k + e] = float(wr[f * sW + i + int64_t(l) * j]);
    wki[f * l * k + e] = float(wi[f * sW + i + int64_t(l) * j]);
  }
  for (int64_t e = threadIdx.x; e < int64_t(p) * k; e += blockDim.x) {
    const int64_t i = e % p, c = e / p;
    const int j = order[c];
    vkr[f * p * k + e] = float(gr[f * sG + i + int64_t(p) * j]);
    vki[f * p * k + e] = float(gi[f * sG + i + int64_t(p) * j]);
  }
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e % k, c = e / k;
    sr[f * k * k + e] = (i == c) ? float(s[order[c]]) : 0.f;
    si[f * k * k + e] = 0.f;
  }
}

// Per-frequency truncation: columns c >= r_f of W_k (l x k), V (p x k) and the
// diagonal of S (k x k) of frequency f are zeroed.  One block per frequency.
// Zero the columns c >= l_f of slice f (rows x l, column-major, slice
// stride rows * l): the per-frequency sketch size.
__global__ void sketch_cols_kernel(float* __restrict__ re, float* __restrict__ im, int64_t rows,
                                   int64_t l, const int32_t* __restrict__ sizes) {
  const int64_t f = blockIdx.x;
  const int64_t lf = min(max(int64_t(sizes[f]), int64_t(1)), l);
  for (int64_t e = lf * rows + threadIdx.x; e < l * rows; e += blockDim.x) {
    re[f * rows * l + e] = 0.f;
    im[f * rows * l + e] = 0.f;
  }
}

__global__ void rank_mask_kernel(const int32_t* __restrict__ rank, int l, int p, int k,
                                 float* __restrict__ wkr, float* __restrict__ wki,
                                 float* __restrict__ vkr, float* __restrict__ vki,
                                 float* __restrict__ sr, float* __restrict__ si) {
  const int64_t f = blockIdx.x;
  const int r = min(max(rank[f], 0), k);
  if (r == k) return;
  for (int e = threadIdx.x + l * r; e < l * k; e += blockDim.x) {
    wkr[f * l * k + e] = 0.f;
    wki[f * l * k + e] = 0.f;
  }
  for (int64_t e = threadIdx.x + int64_t(p) * r; e < int64_t(p) * k; e += blockDim.x) {
    vkr[f * p * k + e] = 0.f;
    vki[f * p * k + e] = 0.f;
  }
  for (int c = threadIdx.x + r; c < k; c += blockDim.x) {
    sr[f * k * k + c + int64_t(k) * c] = 0.f;
    si[f * k * k + c + int64_t(k) * c] = 0.f;
  }
}

__global__ void to_double_kernel(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x)
    b[e] = a[e];
}

__global__ void real_flags2_kernel(int* flags, int64_t h, int64_t n3) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < h) flags[k] = (k == 0 || (n3 % 2 == 0 && k == h - 1)) ? 1 : 0;
}

unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > int64_t(sm_count()) * 16) b = int64_t(sm_count()) * 16;
  if (b < 1) b = 1;
  return unsigned(b);
}

// Launch of householder_qr_kernel with RPL = 2, 4 or 8 rows per lane (p
// up to 64, 128, 256) and the predicate-free form when p fills the lanes.
int launch_hqr(float* yr, float* yi, int64_t sY, int p, int l, const int32_t* lcols,
               bool keep_phase, int64_t batch, cudaStream_t st, HqrSplit sp = HqrSplit{}) {
  const size_t smem = size_t(p) * l * sizeof(float2);
  const int kp = keep_phase ? 1 : 0;
  const unsigned grid = unsigned(batch);
  KernelScope ks("householder_qr", st);
#define TP_HQR(R, F)                                                                      \
  do {                                                                                    \
    TP_SET_SMEM((householder_qr_kernel<R, F>), smem);                                     \
    householder_qr_kernel<R, F><<<grid, HQR_THREADS, smem, st>>>(yr, yi, sY, p, l, lcols, kp, \
                                                                 sp);                            \
  } while (0)
  if (p == 64) TP_HQR(2, true);
  else if (p < 64) TP_HQR(2, false);
  else if (p == 128) TP_HQR(4, true);
  else if (p < 128) TP_HQR(4, false);
  else if (p == 256) TP_HQR(8, true);
  else TP_HQR(8, false);
#undef TP_HQR
  return launch_status("householder_qr_kernel");
}

}  // namespace

// K leading dimension of the split operand planes (16-byte rows for TMA).
int64_t split_ld(int64_t k, int prec) {
  return prec == TP_BF16X3 ? (k + 7) / 8 * 8 : (k + 3) / 4 * 4;
}

// Householder orthonormalisation of `batch` slices Y (p x l, column-major,
// slice stride sY) in place, float32 in shared memory: p <= 256 and
// l <= 96 (else TP_EUNSUPPORTED).  keep_phase multiplies column j by
// sign(R(j, j)), so that nearly orthonormal columns stay close to their
// input.
int householder_orth_launch(float* yr, float* yi, int64_t sY, int p, int l, int64_t batch,
                            bool keep_phase, cudaStream_t st) {
  if (p > 256 || l > HQR_MAX_L || l > p) {
    set_error("householder_orth: needs l <= p <= 256 and l <= %d", HQR_MAX_L);
    return TP_EUNSUPPORTED;
  }
  if (batch <= 0 || l <= 0) return TP_OK;
  return launch_hqr(yr, yi, sY, p, l, nullptr, keep_phase, batch, st);
}

size_t rsvd_ws(int64_t n1, int64_t n2, int64_t n3, int64_t k, int64_t p, int prec) {
  const size_t h = size_t(half_len(n3));
  const size_t l = size_t(k + p);
  const bool tc = prec == TP_TF32X3 || prec == TP_BF16X3;
  const size_t ln = size_t(split_ld(n1, prec)), lm = size_t(split_ld(n2, prec));
  const size_t lb = ln > lm ? ln : lm;
  const size_t split = tc ? 4 * ws_bytes(lm * n1 * h, 4)      // X_hat, K-major (for X_hat .)
                                + 4 * ws_bytes(ln * n2 * h, 4)  // X_hat^H, K-major
                                + 4 * ws_bytes(lb * l * h, 4)   // B operand (Omega, Q or Z)
                          : 0;
  return split + 2 * ws_bytes(size_t(n1) * n2 * h, 4)   // X_hat
         + 2 * ws_bytes(size_t(n1) * n2 * h, 4) // X_hat^H
         + 2 * ws_bytes(size_t(n2) * l * h, 4)  // Omega
         + 2 * ws_bytes(size_t(n1) * l * h, 4)  // Y / Q
         + 2 * ws_bytes(size_t(n2) * l * h, 4)  // Z / B^H
         + 2 * ws_bytes(size_t(n2) * l * h, 8)  // Jacobi G (float64)
         + 2 * ws_bytes(l * l * h, 8)           // Jacobi W (float64)
         + ws_bytes(l * h, 8) + ws_bytes(h, 4)  // singular values, real flags
         + ws_bytes(size_t(QL_LOG_PER_L) * l * h, sizeof(QlRot)) + ws_bytes(h, 4)   // QL logs
         + 2 * ws_bytes(l * size_t(k) * h, 4)   // W_k
         + 2 * ws_bytes(size_t(n1) * k * h, 4)  // U_hat
         + 2 * ws_bytes(size_t(k) * k * h, 4)   // S_hat
         + 2 * ws_bytes(size_t(n2) * k * h, 4)  // V_hat
         // slice sketch: lateral norms, picks, draw scratch
         + ws_bytes(size_t(n2), 8) + ws_bytes(norms_partial_count(n1, n2, n3, 0), 8) +
         ws_bytes(l, 4) + ws_bytes(l, 4) + ws_bytes(1, 8) + draw_scratch_bytes(n2);
}

namespace {
// Test matrix of the slice (t-CX) sketch: Omega_f(j_c, c) = scale_c for the
// c-th of the `count` with-replacement picks at every frequency f, zero
// elsewhere (X_hat_f Omega_f is the rescaled picked columns).
__global__ void slice_sketch_kernel(float* __restrict__ om_r, float* __restrict__ om_i, int64_t n2,
                                    int64_t l, int64_t h, const int32_t* __restrict__ idx,
                                    const float* __restrict__ scale,
                                    const int64_t* __restrict__ count) {
  const int64_t cnt = *count;
  const int64_t total = n2 * l * h;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e % n2, c = (e / n2) % l;
    om_r[e] = (c < cnt && idx[c] == r) ? scale[c] : 0.f;
    om_i[e] = 0.f;
  }
}

// Diagonal of every k x k half-spectrum slice of S: sig[f * k + j] = S_f(j, j).
__global__ void diag_kernel(const float* __restrict__ sr, int k, int64_t h, float* __restrict__ sig) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= h * k) return;
  const int64_t f = e / k;
  const int j = int(e - f * k);
  sig[e] = sr[f * k * k + j * (k + 1)];
}
}  // namespace

// sig_out non-null: only the core singular values of every frequency are
// wanted (descending, h x k, float32); U, S, V are not formed.  rank_per_freq
// non-null (device int32[h]): frequency f keeps its top min(max(r_f, 0), k)
// triplets, the others are zero.  sketch_per_freq non-null (device
// int32[h]): frequency f sketches with the first l_f = min(max(s_f, 1), l)
// columns; its other columns of Omega, Y and Z are held at zero, so that the
// products (run over l columns for every slice) leave them zero, the
// orthonormalisations factor only the first l_f columns, and the core Gram
// has an exact zero block beyond l_f (zero singular values, zero factors).
int rsvd_run(const float* X, int64_t n1, int64_t n2, int64_t n3, int k, int p, int q,
             uint64_t seed, float* U, float* S, float* V, const tp_opts* opts, cudaStream_t st,
             float* sig_out, const int32_t* rank_per_freq, int sketch_mode,
             const int32_t* sketch_per_freq) {
  const int64_t h = half_len(n3);
  const int64_t l = k + p;
  const int prec = opts ? opts->precision : TP_FP32;
  if (prec != TP_FP32 && prec != TP_TF32X3 && prec != TP_BF16X3) {
    set_error("tsvd_randomized: unknown precision %d", prec);
    return TP_EINVAL;
  }
  const bool tc = prec != TP_FP32;
  Arena ws;
  int rc = acquire_workspace(opts, rsvd_ws(n1, n2, n3, k, p, prec), &ws);
  if (rc) return rc;
  int32_t* status = opts ? opts->status : nullptr;
  // tensor-core form: split planes of X_hat (K-major for X_hat Omega and
  // X_hat Z), of X_hat^H (K-major for X_hat^H Q) and of the B operand
  const int64_t ln = split_ld(n1, prec), lm = split_ld(n2, prec), lb = ln > lm ? ln : lm;
  float* XA[4] = {};
  float* XH[4] = {};
  float* BP[4] = {};
  if (tc) {
    for (int i = 0; i < 4; ++i) XA[i] = ws.take<float>(size_t(lm) * n1 * h);
    for (int i = 0; i < 4; ++i) XH[i] = ws.take<float>(size_t(ln) * n2 * h);
    for (int i = 0; i < 4; ++i) BP[i] = ws.take<float>(size_t(lb) * l * h);
  }
  float* Xr = ws.take<float>(size_t(n1) * n2 * h);
  float* Xi = ws.take<float>(size_t(n1) * n2 * h);
  float* Hr = ws.take<float>(size_t(n1) * n2 * h);
  float* Hi = ws.take<float>(size_t(n1) * n2 * h);
  float* Or = ws.take<float>(size_t(n2) * l * h);
  float* Oi = ws.take<float>(size_t(n2) * l * h);
  float* Yr = ws.take<float>(size_t(n1) * l * h);
  float* Yi = ws.take<float>(size_t(n1) * l * h);
  float* Zr = ws.take<float>(size_t(n2) * l * h);
  float* Zi = ws.take<float>(size_t(n2) * l * h);
  double* Gr = ws.take<double>(size_t(n2) * l * h);
  double* Gi = ws.take<double>(size_t(n2) * l * h);
  double* Wr = ws.take<double>(size_t(l) * l * h);
  double* Wi = ws.take<double>(size_t(l) * l * h);
  double* sig = ws.take<double>(size_t(l) * h);
  int* flags = ws.take<int>(size_t(h));
  QlRot* qlog = ws.take<QlRot>(size_t(QL_LOG_PER_L) * l * h);
  int32_t* qcnt = ws.take<int32_t>(size_t(h));
  float* Wkr = ws.take<float>(size_t(l) * k * h);
  float* Wki = ws.take<float>(size_t(l) * k * h);
  float* Ur = ws.take<float>(size_t(n1) * k * h);
  float* Ui = ws.take<float>(size_t(n1) * k * h);
  float* Sr = ws.take<float>(size_t(k) * k * h);
  float* Si = ws.take<float>(size_t(k) * k * h);
  float* Vr = ws.take<float>(size_t(n2) * k * h);
  float* Vi = ws.take<float>(size_t(n2) * k * h);
  double* a2 = ws.take<double>(size_t(n2));
  double* part = ws.take<double>(norms_partial_count(n1, n2, n3, 0));
  int32_t* pidx = ws.take<int32_t>(size_t(l));
  float* pscale = ws.take<float>(size_t(l));
  int64_t* pcnt = ws.take<int64_t>(1);
  char* dscr = ws.take<char>(draw_scratch_bytes(n2));

  // X_hat and X_hat^H
  DftGather gx{X, n1 * n2, 1, 1, 0, n1 * n2, nullptr, nullptr, nullptr, 0, n3, Xr, Xi,
               n1 * n2, n1 * n2, nullptr, nullptr, 0};
  if ((rc = launch_rdft(gx, st))) return rc;
  if (!tc) {   // X_hat^H for the CUDA-core products (the split forms take planes)
    KernelScope ks("conj_transpose", st);
    conj_transpose_kernel<<<dim3(unsigned((n1 + 31) / 32), unsigned((n2 + 31) / 32), unsigned(h)),
                            dim3(32, 8), 0, st>>>(Xr, Xi, n1, n2, Hr, Hi);
  }
  if (sketch_mode == TP_SKETCH_SLICES) {
    // l lateral slices drawn with replacement, p_j ~ ||X(:,j,:)||_F^2
    // (Philox stream 2, word 3 = 1), rescaled by 1/sqrt(l p_j)
    if ((rc = launch_slice_norms(X, n1, n2, n3, 0, a2, part, st))) return rc;
    if ((rc = launch_draw(a2, nullptr, n2, l, seed, TP_PROB_A2, 2u, pidx, pscale, pcnt, nullptr,
                          dscr, st, TP_SAMPLE_IID)))
      return rc;
    {
      KernelScope ks("sketch", st);
      slice_sketch_kernel<<<grid_for(n2 * l * h), 256, 0, st>>>(Or, Oi, n2, l, h, pidx, pscale,
                                                                 pcnt);
    }
  } else {
    KernelScope ks("sketch", st);
    sketch_kernel<<<grid_for(n2 * l * h), 256, 0, st>>>(Or, Oi, n2, l, h, n3, seed);
  }
  if (sketch_per_freq) {
    KernelScope ks("sketch", st);
    sketch_cols_kernel<<<unsigned(h), 256, 0, st>>>(Or, Oi, n2, l, sketch_per_freq);
  }
  if ((rc = launch_status("sketch"))) return rc;

  auto gemm = [&](const float* ar, const float* ai, int64_t M, int64_t K, const float* br,
                  const float* bi, int64_t N, float* cr, float* ci) {
    CGemm g{ar, ai, br, bi, cr, ci, M, N, K, nullptr, M, K, M, M * K, K * N, M * N, h, n3,
            TP_FP32, nullptr, nullptr, nullptr, nullptr, K, status};
    return launch_cgemm(g, st);
  };
  const int bf = prec == TP_BF16X3 ? 1 : 0;
  // split planes of the column-major rows x cols matrices (src, ld rows) with
  // K leading dimension ldk
  auto split = [&](const float* sr, const float* si, int64_t rows, int64_t cols, int conj,
                   int64_t ldk, float* const* P) {
    {
      KernelScope ks("rsvd_split", st);
      split_planes_kernel<<<grid_for(ldk * cols * h), 256, 0, st>>>(
          sr, si, rows, cols, rows, rows * cols, h, ldk, ldk * cols, conj, bf, P[0], P[1], P[2],
          P[3]);
    }
    return launch_status("split_planes_kernel");
  };
  // C (M x N, column-major) = A B with A the split planes XA (M = n1, K = n2)
  // or XH (M = n2, K = n1) and B the split planes BP (K x N, column-major)
  auto gemm_tc = [&](bool hermitian, int64_t N, float* cr, float* ci) {
    const int64_t M = hermitian ? n2 : n1, K = hermitian ? n1 : n2;
    const int64_t lk = hermitian ? ln : lm;
    float* const* A = hermitian ? XH : XA;
    CGemm g{A[0], A[2], BP[0], BP[2], cr, ci, M, N, K, nullptr, lk, lk, M, lk * M, lk * N, M * N,
            h, n3, prec, A[1], A[3], BP[1], BP[3], lk, status};
    return launch_cgemm(g, st);
  };
  // Y = X_hat B (hermitian = false) or X_hat^H B on the selected path, with B
  // given as float32 (br, bi: K x N column-major)
  // the tensor-core forms: orth() on the Householder path also writes the
  // next product's B planes (K = rows), so that product() skips its split
  bool planes_ready = false;
  auto product = [&](bool hermitian, const float* br, const float* bi, int64_t N, float* cr,
                     float* ci) {
    const int64_t K = hermitian ? n1 : n2;
    if (!tc) return hermitian ? gemm(Hr, Hi, n2, n1, br, bi, N, cr, ci)
                              : gemm(Xr, Xi, n1, n2, br, bi, N, cr, ci);
    if (!planes_ready) {
      int r2 = split(br, bi, K, N, 0, hermitian ? ln : lm, BP);
      if (r2) return r2;
    }
    planes_ready = false;
    return gemm_tc(hermitian, N, cr, ci);
  };
  const size_t qr_smem = size_t(2) * l * l * sizeof(double);
  TP_SET_SMEM(cholqr2_kernel, qr_smem);
  constexpr size_t kSmemCap = 200 * 1024;
  auto orth = [&](float* yr, float* yi, int64_t rows) {
    if (rows <= 256 && l <= HQR_MAX_L) {
      HqrSplit sp{};
      if (tc) sp = HqrSplit{BP[0], BP[1], BP[2], BP[3], split_ld(rows, prec), bf};
      planes_ready = tc;
      return launch_hqr(yr, yi, rows * l, int(rows), int(l), sketch_per_freq, false, h, st, sp);
    }
    planes_ready = false;
    {
      KernelScope ks("cholqr2", st);
      cholqr2_kernel<<<unsigned(h), QR_THREADS, qr_smem, st>>>(yr, yi, rows * l, int(rows),
                                                               int(l), sketch_per_freq, status);
    }
    return launch_status("cholqr2_kernel");
  };

  if (tc) {
    // X_hat (element (i, j) at j + lm i: the transpose of X_hat^H without
    // its conjugation) and conj(X_hat) (element (j, i) of X_hat^H at i + ln j)
    {
      KernelScope ks("rsvd_split", st);
      transpose_split_kernel<<<dim3(unsigned((n1 + 31) / 32), unsigned((lm + 31) / 32),
                                    unsigned(h)),
                               dim3(32, 8), 0, st>>>(Xr, Xi, n1, n2, lm, bf, XA[0], XA[1], XA[2],
                                                     XA[3]);
    }
    if ((rc = launch_status("transpose_split_kernel"))) return rc;
    if ((rc = split(Xr, Xi, n1, n2, 1, ln, XH))) return rc;
  }
  if ((rc = product(false, Or, Oi, l, Yr, Yi))) return rc;     // Y = X_hat Omega
  if ((rc = orth(Yr, Yi, n1))) return rc;
  for (int it = 0; it < q; ++it) {
    if ((rc = product(true, Yr, Yi, l, Zr, Zi))) return rc;    // Z = X_hat^H Q
    if ((rc = orth(Zr, Zi, n2))) return rc;
    if ((rc = product(false, Zr, Zi, l, Yr, Yi))) return rc;   // Y = X_hat Z
    if ((rc = orth(Yr, Yi, n1))) return rc;
  }
  if ((rc = product(true, Yr, Yi, l, Zr, Zi))) return rc;      // B^H = X_hat^H Q
  const int sweeps = (opts && opts->max_sweeps > 0) ? opts->max_sweeps : 30;
  const size_t tri_smem = core_tridiag_smem(int(l)), fin_smem = core_finish_smem(int(l));
  bool u_formed = false;   // U_hat (ranks applied) already written by the core
  if (tri_smem <= kSmemCap && l <= 128) {
    // d, e in sig's space, Q (then W) in Wr's, P = B^H W in Gr's
    float* dg = reinterpret_cast<float*>(sig);
    float* eg = dg + l * h;
    float2* zg = reinterpret_cast<float2*>(Wr);
    TP_SET_SMEM(core_tridiag_kernel, tri_smem);
    TP_SET_SMEM(core_finish_kernel, fin_smem);
    {
      KernelScope ks("core_tridiag", st);
      core_tridiag_kernel<<<unsigned(h), EIG_THREADS, tri_smem, st>>>(Zr, Zi, int(n2), int(l),
                                                                      dg, eg, zg);
    }
    {
      KernelScope ks("core_ql", st);
      core_ql_kernel<<<unsigned(h), QL_THREADS, size_t(2) * l * sizeof(float), st>>>(
          dg, eg, int(l), qlog, qcnt, sweeps, status);
    }
    {
      KernelScope ks("core_finish", st);
      // the factors' U_hat = Q W_k and the per-frequency ranks in the same
      // kernel (not for the singular values alone)
      core_finish_kernel<<<unsigned(h), EIG_THREADS, fin_smem, st>>>(
          Zr, Zi, int(n2), int(l), k, zg, qlog, qcnt, Wkr, Wki, Vr, Vi, Sr, Si,
          reinterpret_cast<float2*>(Gr), sig_out ? nullptr : rank_per_freq, Yr, Yi, int(n1),
          sig_out ? nullptr : Ur, sig_out ? nullptr : Ui);
    }
    if ((rc = launch_status("core SVD kernels"))) return rc;
    u_formed = !sig_out;
  } else {
  {
    KernelScope ks("to_double", st);
    to_double_kernel<<<grid_for(n2 * l * h), 256, 0, st>>>(Zr, Gr, n2 * l * h);
    to_double_kernel<<<grid_for(n2 * l * h), 256, 0, st>>>(Zi, Gi, n2 * l * h);
    real_flags2_kernel<<<unsigned((h + 255) / 256), 256, 0, st>>>(flags, h, n3);
  }
  note_launches(2);
  if ((rc = launch_status("to_double"))) return rc;
  if ((rc = jacobi_double_launch(Gr, Gi, n2 * l, Wr, Wi, l * l, sig, int(n2), int(l), int(h),
                                 sweeps, flags, status, st)))
    return rc;
  {
    KernelScope ks("pick_topk", st);
    pick_topk_kernel<<<unsigned(h), 256, size_t(l) * sizeof(int), st>>>(
        Gr, Gi, n2 * l, Wr, Wi, l * l, sig, int(n2), int(l), k, Wkr, Wki, Vr, Vi, Sr, Si);
  }
  if ((rc = launch_status("pick_topk_kernel"))) return rc;
  }
  if (sig_out) {
    {
      KernelScope ks("sketch_spectrum", st);
      diag_kernel<<<unsigned((h * k + 255) / 256), 256, 0, st>>>(Sr, k, h, sig_out);
    }
    return launch_status("diag_kernel");
  }
  if (!u_formed) {
    if (rank_per_freq) {
      {
        KernelScope ks("rank_mask", st);
        rank_mask_kernel<<<unsigned(h), 256, 0, st>>>(rank_per_freq, int(l), int(n2), k, Wkr,
                                                      Wki, Vr, Vi, Sr, Si);
      }
      if ((rc = launch_status("rank_mask_kernel"))) return rc;
    }
    if ((rc = gemm(Yr, Yi, n1, l, Wkr, Wki, k, Ur, Ui))) return rc;   // U_hat = Q W_k
  }
  if ((rc = launch_irdft(Ur, Ui, n1 * k, n1 * k, n3, U, st))) return rc;
  if ((rc = launch_irdft(Sr, Si, int64_t(k) * k, int64_t(k) * k, n3, S, st))) return rc;
  return launch_irdft(Vr, Vi, n2 * k, n2 * k, n3, V, st);
}

}  // namespace tp
