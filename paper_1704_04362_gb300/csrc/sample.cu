// Randomized slice selection of Section 3.1: slice Frobenius norms, the
// sampling probabilities (eqs. nearly_optimal_probs and nonoptimal_probs with
// beta = 1), and the picking loop of Algorithm 2 with Philox4x32-10 coins.
//
// Norms stream the tensor once with coalesced loads.  Each lane keeps its
// running sum of squares as an unevaluated float pair (hi + lo, Dekker's
// two-sum with the exact FMA square residual), so that the result carries
// about 44 significant bits at float32 speed; lanes, warps and partial blocks
// are then combined in float64 in a fixed order, making every norm
// deterministic run to run.
#include "tp_internal.cuh"

namespace tp {
namespace {

__device__ __forceinline__ void acc_sq(float& hi, float& lo, float x) {
  const float p = x * x;
  const float e = fmaf(x, x, -p);       // p + e == x*x exactly
  const float s = hi + p;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (p - bp);   // hi + p == s + err exactly
  hi = s;
  lo += err + e;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Lateral: one warp per column s of the n1 x (n2*n3) matrix; column s is the
// contiguous segment (j, t) with s = j + n2*t.  partial[s] = sum_i X(i,s)^2.
__global__ void lateral_partial_kernel(const float* __restrict__ X, int64_t n1, int64_t ncols,
                                       bool vec4, double* __restrict__ partial) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t s = warp; s < ncols; s += nwarps) {
    const float* col = X + s * n1;
    float hi = 0.f, lo = 0.f;
    if (vec4) {
      const float4* c4 = reinterpret_cast<const float4*>(col);
      const int64_t n4 = n1 >> 2;
      for (int64_t i = lane; i < n4; i += 32) {
        const float4 v = __ldg(c4 + i);
        acc_sq(hi, lo, v.x); acc_sq(hi, lo, v.y); acc_sq(hi, lo, v.z); acc_sq(hi, lo, v.w);
      }
    } else {
      for (int64_t i = lane; i < n1; i += 32) acc_sq(hi, lo, __ldg(col + i));
    }
    const double v = warp_sum(double(hi) + double(lo));
    if (lane == 0) partial[s] = v;
  }
}

// out[j] = sum_t partial[j + n2*t], t ascending.
__global__ void lateral_reduce_kernel(const double* __restrict__ partial, int64_t n2, int64_t n3,
                                      double* __restrict__ out) {
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n2;
       j += int64_t(gridDim.x) * blockDim.x) {
    double a = 0.0;
    for (int64_t t = 0; t < n3; ++t) a += partial[j + n2 * t];
    out[j] = a;
  }
}

// Horizontal: thread per row i; block column-chunk g covers columns
// [g*chunk, (g+1)*chunk) of the n1 x (n2*n3) matrix.  partial[g*n1 + i].
__global__ void horizontal_partial_kernel(const float* __restrict__ X, int64_t n1, int64_t ncols,
                                          int64_t chunk, double* __restrict__ partial) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t g = blockIdx.y;
  if (i >= n1) return;
  const int64_t s0 = g * chunk;
  const int64_t s1 = min(ncols, s0 + chunk);
  float hi = 0.f, lo = 0.f;
  int64_t s = s0;
  for (; s + 4 <= s1; s += 4) {
    const float a = __ldg(X + i + n1 * s);
    const float b = __ldg(X + i + n1 * (s + 1));
    const float c = __ldg(X + i + n1 * (s + 2));
    const float d = __ldg(X + i + n1 * (s + 3));
    acc_sq(hi, lo, a); acc_sq(hi, lo, b); acc_sq(hi, lo, c); acc_sq(hi, lo, d);
  }
  for (; s < s1; ++s) acc_sq(hi, lo, __ldg(X + i + n1 * s));
  partial[g * n1 + i] = double(hi) + double(lo);
}

__global__ void horizontal_reduce_kernel(const double* __restrict__ partial, int64_t n1, int64_t G,
                                         double* __restrict__ out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n1;
       i += int64_t(gridDim.x) * blockDim.x) {
    double a = 0.0;
    for (int64_t g = 0; g < G; ++g) a += partial[g * n1 + i];
    out[i] = a;
  }
}

int64_t horizontal_chunks(int64_t n1, int64_t ncols) {
  const int64_t bx = (n1 + 255) / 256;
  int64_t G = (152 * 8 + bx - 1) / bx;
  if (G > ncols) G = ncols;
  if (G < 1) G = 1;
  if (G > 65535) G = 65535;
  return G;
}

// ---------------------------------------------------------------- Philox
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    const uint32_t y0 = hi1 ^ c[1] ^ k0, y2 = hi0 ^ c[3] ^ k1;
    c[0] = y0; c[1] = lo1; c[2] = y2; c[3] = lo0;
  }
}

__device__ __forceinline__ uint64_t uniform53(uint64_t j, uint32_t stream_id, uint64_t seed) {
  uint32_t c[4] = {uint32_t(j), uint32_t(j >> 32), stream_id, 0u};
  philox4x32_10(c, uint32_t(seed), uint32_t(seed >> 32));
  return (uint64_t(c[0] >> 5) << 26) | uint64_t(c[1] >> 6);
}

__device__ __forceinline__ double weight(const double* w, const double* w2, int mode, int64_t j) {
  if (mode == TP_PROB_AB) return sqrt(w[j]) * sqrt(w2[j]);
  return w[j];
}

// One block of 1024 threads.  Deterministic float64 normaliser: each thread
// sums a strided subsequence in order, then a fixed tree over threads.
__global__ void __launch_bounds__(1024) draw_kernel(const double* __restrict__ w,
                                                    const double* __restrict__ w2, int64_t n,
                                                    int64_t c, uint64_t seed, int mode,
                                                    uint32_t stream_id, int32_t* __restrict__ idx,
                                                    float* __restrict__ scale,
                                                    int64_t* __restrict__ count,
                                                    double* __restrict__ q_out) {
  __shared__ double red[1024];
  __shared__ int wsum[32];
  __shared__ int64_t base_s;
  const int tid = threadIdx.x;
  double total = 1.0;
  if (mode != TP_PROB_GIVEN) {
    double a = 0.0;
    for (int64_t j = tid; j < n; j += 1024) a += weight(w, w2, mode, j);
    red[tid] = a;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
      if (tid < s) red[tid] += red[tid + s];
      __syncthreads();
    }
    total = red[0];
  }
  if (tid == 0) base_s = 0;
  __syncthreads();
  const double cd = double(c);
  const int lane = tid & 31, wid = tid >> 5;
  for (int64_t j0 = 0; j0 < n; j0 += 1024) {
    const int64_t j = j0 + tid;
    bool pick = false;
    double q = 0.0;
    if (j < n) {
      double p;
      if (mode == TP_PROB_GIVEN) p = w[j];
      else p = (total > 0.0) ? weight(w, w2, mode, j) / total : 0.0;
      q = fmin(1.0, cd * p);
      if (!(q > 0.0)) q = 0.0;   // also maps NaN to 0
      const uint64_t Q = uint64_t(q * 9007199254740992.0);   // floor(q 2^53), q in [0,1]
      pick = uniform53(uint64_t(j), stream_id, seed) < Q;
      if (q_out) q_out[j] = q;
    }
    const unsigned ball = __ballot_sync(0xffffffffu, pick);
    if (lane == 0) wsum[wid] = __popc(ball);
    __syncthreads();
    if (wid == 0) {
      int v = wsum[lane];
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
      }
      wsum[lane] = incl - v;   // exclusive prefix over warps
    }
    __syncthreads();
    const int64_t base = base_s;
    if (pick) {
      const int64_t pos = base + wsum[wid] + __popc(ball & ((1u << lane) - 1u));
      idx[pos] = int32_t(j);
      if (scale) scale[pos] = float(1.0 / sqrt(q));
    }
    __syncthreads();   // every thread has used base_s and wsum
    // running total = prefix before warp 31 plus warp 31's own picks
    if (wid == 31 && lane == 0) base_s = base + wsum[31] + __popc(ball);
    __syncthreads();
  }
  if (tid == 0) *count = base_s;
}

__device__ __forceinline__ uint64_t uniform53_iid(uint64_t t, uint32_t stream_id, uint64_t seed) {
  uint32_t c[4] = {uint32_t(t), uint32_t(t >> 32), stream_id, 1u};
  philox4x32_10(c, uint32_t(seed), uint32_t(seed >> 32));
  return (uint64_t(c[0] >> 5) << 26) | uint64_t(c[1] >> 6);
}

// p_j of the i.i.d. draws and its integer weight floor(p_j 2^53) (p clipped to
// [0, 1], NaN to 0).  One out-of-line function so that every use rounds alike.
__device__ __noinline__ double iid_p(const double* w, const double* w2, int mode, double total,
                                    int64_t j) {
  double p;
  if (mode == TP_PROB_GIVEN) p = w[j];
  else p = (total > 0.0) ? weight(w, w2, mode, j) / total : 0.0;
  if (!(p > 0.0)) p = 0.0;
  return p < 1.0 ? p : 1.0;
}

// c independent draws with replacement (the with-replacement sampling that
// Algorithm 2 reduces to at n3 = 1, Drineas, Kannan and Mahoney 2006), in
// integers so that the oracle given the same float64 p draws the same
// indices: W_j = floor(p_j 2^53), draw t takes the 53-bit U_t of counter
// (t, stream, 1) and the first j whose inclusive prefix sum of W exceeds
// floor(U_t sum(W) / 2^53).  Thread i owns the contiguous chunk
// [i L, (i + 1) L) of the indices; the exact uint64 chunk sums are scanned in
// shared memory, a draw binary-searches the chunk and walks it.  One block of
// 1024 threads; no workspace.  scale_t = 1/sqrt(c p_j); q_out[j] = c p_j.
__global__ void __launch_bounds__(1024) draw_iid_kernel(const double* __restrict__ w,
                                                        const double* __restrict__ w2, int64_t n,
                                                        int64_t c, uint64_t seed, int mode,
                                                        uint32_t stream_id,
                                                        int32_t* __restrict__ idx,
                                                        float* __restrict__ scale,
                                                        int64_t* __restrict__ count,
                                                        double* __restrict__ q_out) {
  __shared__ double red[1024];
  __shared__ uint64_t csum[1024];
  const int tid = threadIdx.x;
  double total = 1.0;
  if (mode != TP_PROB_GIVEN) {
    double a = 0.0;
    for (int64_t j = tid; j < n; j += 1024) a += weight(w, w2, mode, j);
    red[tid] = a;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
      if (tid < s) red[tid] += red[tid + s];
      __syncthreads();
    }
    total = red[0];
  }
  const int64_t L = (n + 1023) / 1024;
  const int64_t j0 = int64_t(tid) * L, j1 = j0 + L < n ? j0 + L : n;
  uint64_t own = 0;
  for (int64_t j = j0; j < j1; ++j) {
    const double p = iid_p(w, w2, mode, total, j);
    own += uint64_t(p * 9007199254740992.0);
    if (q_out) q_out[j] = double(c) * p;
  }
  csum[tid] = own;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {   // inclusive scan (exact in uint64)
    const uint64_t v = tid >= o ? csum[tid - o] : 0;
    __syncthreads();
    csum[tid] += v;
    __syncthreads();
  }
  const uint64_t W = csum[1023];
  if (W == 0) {
    if (tid == 0) *count = 0;
    return;
  }
  for (int64_t t = tid; t < c; t += 1024) {
    const uint64_t U = uniform53_iid(uint64_t(t), stream_id, seed);
    const uint64_t lo = U * W, hi = __umul64hi(U, W);
    const uint64_t target = (hi << 11) | (lo >> 53);   // floor(U W / 2^53) < W
    int a = 0, b = 1023;                                 // first chunk with csum > target
    while (a < b) {
      const int m = (a + b) >> 1;
      if (csum[m] > target) b = m;
      else a = m + 1;
    }
    uint64_t run = a > 0 ? csum[a - 1] : 0;
    const int64_t k0 = int64_t(a) * L, k1 = k0 + L < n ? k0 + L : n;
    int64_t j = k1 - 1;
    double pj = 0.0;
    for (int64_t k = k0; k < k1; ++k) {
      const double p = iid_p(w, w2, mode, total, k);
      run += uint64_t(p * 9007199254740992.0);
      if (run > target) {
        j = k;
        pj = p;
        break;
      }
    }
    idx[t] = int32_t(j);
    if (scale) scale[t] = float(1.0 / sqrt(double(c) * pj));
  }
  if (tid == 0) *count = c;
}

}  // namespace

size_t norms_partial_count(int64_t n1, int64_t n2, int64_t n3, int which) {
  if (which == 0) return size_t(n2) * size_t(n3);
  return size_t(horizontal_chunks(n1, n2 * n3)) * size_t(n1);
}

int launch_slice_norms(const float* X, int64_t n1, int64_t n2, int64_t n3, int which,
                       double* out, double* partial, cudaStream_t st) {
  const int64_t ncols = n2 * n3;
  if (which == 0) {
    const bool vec4 = (n1 % 4 == 0) && aligned16(X);
    int64_t blocks = (ncols * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    {
      KernelScope ks("norms_lateral", st);
      lateral_partial_kernel<<<unsigned(blocks), 256, 0, st>>>(X, n1, ncols, vec4, partial);
    }
    int64_t rb = (n2 + 255) / 256;
    if (rb > 152 * 8) rb = 152 * 8;
    {
      KernelScope ks("norms_reduce", st);
      lateral_reduce_kernel<<<unsigned(rb), 256, 0, st>>>(partial, n2, n3, out);
    }
  } else {
    const int64_t G = horizontal_chunks(n1, ncols);
    const int64_t chunk = (ncols + G - 1) / G;
    const int64_t bx = (n1 + 255) / 256;
    {
      KernelScope ks("norms_horizontal", st);
      horizontal_partial_kernel<<<dim3(unsigned(bx), unsigned(G)), 256, 0, st>>>(X, n1, ncols,
                                                                                chunk, partial);
    }
    int64_t rb = (n1 + 255) / 256;
    if (rb > 152 * 8) rb = 152 * 8;
    {
      KernelScope ks("norms_reduce", st);
      horizontal_reduce_kernel<<<unsigned(rb), 256, 0, st>>>(partial, n1, G, out);
    }
  }
  return launch_status("slice_norms");
}

int launch_draw(const double* w, const double* w2, int64_t n, int64_t c, uint64_t seed,
                int mode, uint32_t stream_id, int32_t* idx, float* scale, int64_t* count,
                double* q_out, cudaStream_t st, int sample_mode) {
  if (sample_mode == TP_SAMPLE_IID) {
    {
      KernelScope ks("draw_iid", st);
      draw_iid_kernel<<<1, 1024, 0, st>>>(w, w2, n, c, seed, mode, stream_id, idx, scale, count,
                                          q_out);
    }
    return launch_status("draw_iid_kernel");
  }
  {
    KernelScope ks("draw", st);
    draw_kernel<<<1, 1024, 0, st>>>(w, w2, n, c, seed, mode, stream_id, idx, scale, count, q_out);
  }
  return launch_status("draw_kernel");
}

}  // namespace tp
