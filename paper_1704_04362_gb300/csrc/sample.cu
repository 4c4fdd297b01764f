// Randomized slice selection of Section 3.1: slice Frobenius norms, the
// sampling probabilities (eqs. nearly_optimal_probs and nonoptimal_probs with
// beta = 1), and the picking loop of Algorithm 2 with Philox4x32-10 coins.
//
// Norms stream the tensor once with coalesced loads.  Each lane keeps its
// running sum of squares as an unevaluated float pair (hi + lo, Dekker's
// two-sum with the exact FMA square residual), so that the result carries
// about 44 significant bits at float32 speed; the lanes of a column are
// combined as float pairs, partial sums in float64, all in a fixed order,
// making every norm deterministic run to run.
#include "philox.cuh"
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

// (h, l) += (h2, l2) for unevaluated float pairs: Knuth's two-sum of the
// high parts, the low parts added to its error, then renormalised so that
// |l| <= ulp(h) / 2.
__device__ __forceinline__ void pair_add(float& h, float& l, float h2, float l2) {
  const float s = h + h2;
  const float bp = s - h;
  const float e = ((h - (s - bp)) + (h2 - bp)) + (l + l2);
  h = s + e;
  l = e - (h - s);
}

// Lateral: a group of LC lanes per column s of the n1 x (n2*n3) matrix
// (32 / LC columns per warp, so that short columns still keep every lane
// loading); column s is the contiguous segment (j, t) with s = j + n2*t.
// partial[s] = sum_i X(i,s)^2.  Every lane of a warp runs the same number of
// iterations (the shuffles need them all).
template <int LC>
__global__ void lateral_partial_kernel(const float* __restrict__ X, int64_t n1, int64_t ncols,
                                       bool vec4, double* __restrict__ partial) {
  constexpr int G = 32 / LC;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LC - 1), grp = lane / LC;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t s0 = warp * G; s0 < ncols; s0 += nwarps * G) {
    const int64_t s = s0 + grp;
    float hi = 0.f, lo = 0.f;
    if (s < ncols) {
      const float* col = X + s * n1;
      if (vec4) {
        const float4* c4 = reinterpret_cast<const float4*>(col);
        const int64_t n4 = n1 >> 2;
#pragma unroll 4
        for (int64_t i = sub; i < n4; i += LC) {
          const float4 v = __ldg(c4 + i);
          acc_sq(hi, lo, v.x); acc_sq(hi, lo, v.y); acc_sq(hi, lo, v.z); acc_sq(hi, lo, v.w);
        }
      } else {
        for (int64_t i = sub; i < n1; i += LC) acc_sq(hi, lo, __ldg(col + i));
      }
    }
    // combine the lanes' float pairs in float32 (float64 arithmetic runs at a
    // small fraction of the float32 rate on this part); one conversion per column
#pragma unroll
    for (int o = LC / 2; o > 0; o >>= 1)
      pair_add(hi, lo, __shfl_xor_sync(0xffffffffu, hi, o), __shfl_xor_sync(0xffffffffu, lo, o));
    if (sub == 0 && s < ncols) partial[s] = double(hi) + double(lo);
  }
}

// out[j] = sum_t partial[j + n2*t], t ascending.
__global__ void lateral_reduce_kernel(const double* __restrict__ partial, int64_t n2, int64_t n3,
                                      double* __restrict__ out) {
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n2;
       j += int64_t(gridDim.x) * blockDim.x) {
    double a = 0.0;
#pragma unroll 8
    for (int64_t t = 0; t < n3; ++t) a += partial[j + n2 * t];   // loads batched, adds in order
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
  for (; s + 8 <= s1; s += 8) {   // eight loads in flight per thread
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldg(X + i + n1 * (s + u));
#pragma unroll
    for (int u = 0; u < 8; ++u) acc_sq(hi, lo, v[u]);
  }
  for (; s < s1; ++s) acc_sq(hi, lo, __ldg(X + i + n1 * s));
  partial[g * n1 + i] = double(hi) + double(lo);
}

// out[i] = sum over the G chunk partials of row i: a block takes 32 rows,
// its 8 warps each sum a contiguous eighth of the chunks (loads batched,
// adds in chunk order), then warp 0 adds the eight eighths in order; the
// same partition for a given G, so every norm is deterministic.
__global__ void __launch_bounds__(256) horizontal_reduce_kernel(const double* __restrict__ partial,
                                                                int64_t n1, int64_t G,
                                                                double* __restrict__ out) {
  __shared__ double seg_sum[8][33];
  const int lr = threadIdx.x & 31, seg = threadIdx.x >> 5;
  const int64_t S = (G + 7) / 8;
  for (int64_t r0 = int64_t(blockIdx.x) * 32; r0 < n1; r0 += int64_t(gridDim.x) * 32) {
    const int64_t i = r0 + lr;
    double a = 0.0;
    if (i < n1) {
      const int64_t g1 = (seg + 1) * S < G ? (seg + 1) * S : G;
#pragma unroll 8
      for (int64_t g = seg * S; g < g1; ++g) a += partial[g * n1 + i];
    }
    seg_sum[seg][lr] = a;
    __syncthreads();
    if (seg == 0 && i < n1) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k) t += seg_sum[k][lr];
      out[i] = t;
    }
    __syncthreads();
  }
}

int64_t horizontal_chunks(int64_t n1, int64_t ncols) {
  // about four waves of 8 blocks per SM, so that the last wave's tail is
  // short, while the G n1 partial sums stay within 2^20 doubles (8 MiB) unless
  // one wave alone needs more.  The SM count is fixed at GB300's 152 here, not
  // queried: G is the partition of each row's sum, so a fixed G keeps the
  // horizontal norms bit-identical on every device, and the no-allocation
  // entry point's capacity check depends on it.
  const int64_t bx = (n1 + 255) / 256;
  const int64_t one_wave = (152 * 8 + bx - 1) / bx;
  int64_t G = (152 * 8 * 4 + bx - 1) / bx;
  const int64_t fit = (int64_t(1) << 20) / n1;
  if (G > fit) G = fit > one_wave ? fit : one_wave;
  if (G > ncols) G = ncols;
  if (G < 1) G = 1;
  if (G > 65535) G = 65535;
  return G;
}

// ---------------------------------------------------------------- Philox
__device__ __forceinline__ uint64_t uniform53(uint64_t j, uint32_t stream_id, uint64_t seed) {
  uint32_t c[4] = {uint32_t(j), uint32_t(j >> 32), stream_id, 0u};
  philox4x32_10(c, uint32_t(seed), uint32_t(seed >> 32));
  return (uint64_t(c[0] >> 5) << 26) | uint64_t(c[1] >> 6);
}

__device__ __forceinline__ double weight(const double* w, const double* w2, int mode, int64_t j) {
  if (mode == TP_PROB_AB) return sqrt(w[j]) * sqrt(w2[j]);
  return w[j];
}

// The picking loop runs in three launches so that the float64 work (square
// roots, divisions; GB300's float64 rate is a small fraction of its float32
// rate) is spread over every SM and only integer compaction stays in one
// block:
//   1. draw_sum_kernel: per-block sums of the weights (fixed order);
//   2. draw_decide_kernel: every block adds the block sums in block order
//      (the same total everywhere), then per index j the probability p_j,
//      q_j = min{1, c p_j} and the Philox coin; the decision is parked in
//      idx[j] (1 picked, 0 not) and 1/sqrt(q_j) in scale[j];
//   3. draw_compact_kernel (one block): the picked j, ascending, packed to
//      the front of idx and scale in place (a chunk is read completely
//      before any of its positions is written, and positions never pass j).
// The i.i.d. mode replaces 2-3 by iid_weights_kernel (W_j = floor(p_j 2^53)
// and 1/sqrt(c p_j) per j, in parallel) and iid_draw_kernel (one block,
// integer chunk sums, scan and searches).
constexpr int kDrawBlocks = 608;

int draw_blocks(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > kDrawBlocks) g = kDrawBlocks;
  return g < 1 ? 1 : int(g);
}

__device__ __forceinline__ double block_sum256(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (int(threadIdx.x) < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  return red[0];
}

__global__ void __launch_bounds__(256) draw_sum_kernel(const double* __restrict__ w,
                                                       const double* __restrict__ w2, int64_t n,
                                                       int mode, double* __restrict__ bpart) {
  __shared__ double red[256];
  double a = 0.0;
  for (int64_t j = int64_t(blockIdx.x) * 256 + threadIdx.x; j < n; j += int64_t(gridDim.x) * 256)
    a += weight(w, w2, mode, j);
  const double t = block_sum256(a, red);
  if (threadIdx.x == 0) bpart[blockIdx.x] = t;
}

__device__ __forceinline__ double draw_total(const double* bpart, int G, int mode) {
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double s = 0.0;
    if (mode != TP_PROB_GIVEN)
      for (int b = 0; b < G; ++b) s += bpart[b];
    tot = s;
  }
  __syncthreads();
  return tot;
}

// p_j from the weights (mode) and the total.
__device__ __forceinline__ double draw_p(const double* w, const double* w2, int mode,
                                         double total, int64_t j) {
  if (mode == TP_PROB_GIVEN) return w[j];
  return (total > 0.0) ? weight(w, w2, mode, j) / total : 0.0;
}

__global__ void __launch_bounds__(256) draw_decide_kernel(
    const double* __restrict__ w, const double* __restrict__ w2, int64_t n, int64_t c,
    uint64_t seed, int mode, uint32_t stream_id, const double* __restrict__ bpart, int G,
    int32_t* __restrict__ idx, float* __restrict__ scale, double* __restrict__ q_out) {
  const double total = draw_total(bpart, G, mode);
  const double cd = double(c);
  for (int64_t j = int64_t(blockIdx.x) * 256 + threadIdx.x; j < n; j += int64_t(gridDim.x) * 256) {
    double q = fmin(1.0, cd * draw_p(w, w2, mode, total, j));
    if (!(q > 0.0)) q = 0.0;   // also maps NaN to 0
    const uint64_t Q = uint64_t(q * 9007199254740992.0);   // floor(q 2^53), q in [0,1]
    const bool pick = uniform53(uint64_t(j), stream_id, seed) < Q;
    idx[j] = pick ? 1 : 0;
    if (scale) scale[j] = pick ? float(1.0 / sqrt(q)) : 0.f;
    if (q_out) q_out[j] = q;
  }
}

__global__ void __launch_bounds__(1024) draw_compact_kernel(int64_t n, int32_t* __restrict__ idx,
                                                            float* __restrict__ scale,
                                                            int64_t* __restrict__ count) {
  __shared__ int wsum[32];
  __shared__ int64_t base_s;
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  if (tid == 0) base_s = 0;
  __syncthreads();
  for (int64_t j0 = 0; j0 < n; j0 += 1024) {
    const int64_t j = j0 + tid;
    const bool pick = j < n && idx[j] != 0;
    const float sv = (pick && scale) ? scale[j] : 0.f;
    const unsigned ball = __ballot_sync(0xffffffffu, pick);
    if (lane == 0) wsum[wid] = __popc(ball);
    __syncthreads();   // also: the whole chunk has been read
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
      if (scale) scale[pos] = sv;
    }
    __syncthreads();   // every thread has used base_s and wsum
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

// i.i.d. draws, pass 2: p_j clipped to [0, 1] (NaN to 0), its integer weight
// W_j = floor(p_j 2^53), the rescale 1/sqrt(c p_j) and q_out[j] = c p_j.
__global__ void __launch_bounds__(256) iid_weights_kernel(
    const double* __restrict__ w, const double* __restrict__ w2, int64_t n, int64_t c, int mode,
    const double* __restrict__ bpart, int G, uint64_t* __restrict__ W, float* __restrict__ sval,
    double* __restrict__ q_out) {
  const double total = draw_total(bpart, G, mode);
  for (int64_t j = int64_t(blockIdx.x) * 256 + threadIdx.x; j < n; j += int64_t(gridDim.x) * 256) {
    double p = draw_p(w, w2, mode, total, j);
    if (!(p > 0.0)) p = 0.0;
    if (p > 1.0) p = 1.0;
    W[j] = uint64_t(p * 9007199254740992.0);
    sval[j] = p > 0.0 ? float(1.0 / sqrt(double(c) * p)) : 0.f;
    if (q_out) q_out[j] = double(c) * p;
  }
}

// i.i.d. draws, pass 3 (one block of 1024): c independent draws with
// replacement (the with-replacement sampling Algorithm 2 reduces to at
// n3 = 1, Drineas, Kannan and Mahoney 2006) in integers, so that the oracle
// given the same float64 p draws the same indices: draw t takes the 53-bit
// U_t of counter (t, stream, 1) and the first j whose inclusive prefix sum of
// W exceeds floor(U_t sum(W) / 2^53).  Thread i owns the contiguous chunk
// [i L, (i + 1) L) of the indices; the exact uint64 chunk sums are scanned in
// shared memory, a draw binary-searches the chunks and walks one.
__global__ void __launch_bounds__(1024) iid_draw_kernel(int64_t n, int64_t c, uint64_t seed,
                                                        uint32_t stream_id,
                                                        const uint64_t* __restrict__ W,
                                                        const float* __restrict__ sval,
                                                        int32_t* __restrict__ idx,
                                                        float* __restrict__ scale,
                                                        int64_t* __restrict__ count) {
  __shared__ uint64_t csum[1024];
  const int tid = threadIdx.x;
  const int64_t L = (n + 1023) / 1024;
  const int64_t j0 = int64_t(tid) * L, j1 = j0 + L < n ? j0 + L : n;
  uint64_t own = 0;
  for (int64_t j = j0; j < j1; ++j) own += W[j];
  csum[tid] = own;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {   // inclusive scan (exact in uint64)
    const uint64_t v = tid >= o ? csum[tid - o] : 0;
    __syncthreads();
    csum[tid] += v;
    __syncthreads();
  }
  const uint64_t tot = csum[1023];
  if (tot == 0) {
    if (tid == 0) *count = 0;
    return;
  }
  for (int64_t t = tid; t < c; t += 1024) {
    const uint64_t U = uniform53_iid(uint64_t(t), stream_id, seed);
    const uint64_t lo = U * tot, hi = __umul64hi(U, tot);
    const uint64_t target = (hi << 11) | (lo >> 53);   // floor(U tot / 2^53) < tot
    int a = 0, b = 1023;                                 // first chunk with csum > target
    while (a < b) {
      const int m = (a + b) >> 1;
      if (csum[m] > target) b = m;
      else a = m + 1;
    }
    uint64_t run = a > 0 ? csum[a - 1] : 0;
    const int64_t k0 = int64_t(a) * L, k1 = k0 + L < n ? k0 + L : n;
    int64_t j = k1 - 1;
    for (int64_t k = k0; k < k1; ++k) {
      run += W[k];
      if (run > target) {
        j = k;
        break;
      }
    }
    idx[t] = int32_t(j);
    if (scale) scale[t] = sval[j];
  }
  if (tid == 0) *count = c;
}

// Raw Philox4x32-10 words of n caller-given counters (tp_philox4x32_10).
__global__ void philox_words_kernel(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1,
                                    int64_t n, uint32_t* __restrict__ out) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x) {
    uint32_t c[4] = {ctr[4 * e], ctr[4 * e + 1], ctr[4 * e + 2], ctr[4 * e + 3]};
    philox4x32_10(c, k0, k1);
    out[4 * e] = c[0];
    out[4 * e + 1] = c[1];
    out[4 * e + 2] = c[2];
    out[4 * e + 3] = c[3];
  }
}

}  // namespace

int launch_philox_words(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out,
                        cudaStream_t st) {
  if (n == 0) return TP_OK;
  int64_t blocks = (n + 255) / 256;
  if (blocks > int64_t(sm_count()) * 8) blocks = int64_t(sm_count()) * 8;
  {
    KernelScope ks("philox_words", st);
    philox_words_kernel<<<unsigned(blocks), 256, 0, st>>>(ctr, k0, k1, n, out);
  }
  return launch_status("philox_words_kernel");
}

size_t norms_partial_count(int64_t n1, int64_t n2, int64_t n3, int which) {
  if (which == 0) return size_t(n2) * size_t(n3);
  return size_t(horizontal_chunks(n1, n2 * n3)) * size_t(n1);
}

int launch_slice_norms(const float* X, int64_t n1, int64_t n2, int64_t n3, int which,
                       double* out, double* partial, cudaStream_t st,
                       bool tunable) {
  const int64_t ncols = n2 * n3;
  if (which == 0) {
    const bool vec4 = (n1 % 4 == 0) && aligned16(X);
    // lanes per column: about three loads each, a power of two up to 32
    const int64_t loads = vec4 ? n1 / 4 : n1;
    int lc = 32;
    while (lc > 1 && int64_t(lc) * 3 > loads) lc >>= 1;
    const int64_t warps = (ncols + (32 / lc) - 1) / (32 / lc);
    // blocks per SM (the grid-stride walk does not change any column's sum):
    // autotuned among 4, 8, 16 and 32, default 16
    const auto run = [&](int c) {
      int64_t blocks = (warps * 32 + 255) / 256;
      const int64_t cap = int64_t(sm_count()) * (int64_t(4) << c);
      if (blocks > cap) blocks = cap;
      if (blocks < 1) blocks = 1;
      {
        KernelScope ks("norms_lateral", st);
        const unsigned b = unsigned(blocks);
        switch (lc) {
          case 32: lateral_partial_kernel<32><<<b, 256, 0, st>>>(X, n1, ncols, vec4, partial); break;
          case 16: lateral_partial_kernel<16><<<b, 256, 0, st>>>(X, n1, ncols, vec4, partial); break;
          case 8: lateral_partial_kernel<8><<<b, 256, 0, st>>>(X, n1, ncols, vec4, partial); break;
          case 4: lateral_partial_kernel<4><<<b, 256, 0, st>>>(X, n1, ncols, vec4, partial); break;
          case 2: lateral_partial_kernel<2><<<b, 256, 0, st>>>(X, n1, ncols, vec4, partial); break;
          default: lateral_partial_kernel<1><<<b, 256, 0, st>>>(X, n1, ncols, vec4, partial); break;
        }
      }
      return launch_status("lateral_partial_kernel");
    };
    const int64_t key[4] = {n1, size_class(ncols), vec4 ? 1 : 0, lc};
    int c = 2;
    int rc = tunable ? autotune_pick("norms_lateral", key, 4, 4, 2, run, st, &c) : TP_OK;
    if (!rc) rc = run(c);
    if (rc) return rc;
    int64_t rb = (n2 + 255) / 256;
    if (rb > int64_t(sm_count()) * 8) rb = int64_t(sm_count()) * 8;
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
    int64_t rb = (n1 + 31) / 32;
    if (rb > int64_t(sm_count()) * 8) rb = int64_t(sm_count()) * 8;
    {
      KernelScope ks("norms_reduce", st);
      horizontal_reduce_kernel<<<unsigned(rb), 256, 0, st>>>(partial, n1, G, out);
    }
  }
  return launch_status("slice_norms");
}

size_t draw_scratch_bytes(int64_t n) {
  return ws_bytes(kDrawBlocks, 8) + ws_bytes(size_t(n), 8) + ws_bytes(size_t(n), 4);
}

int launch_draw(const double* w, const double* w2, int64_t n, int64_t c, uint64_t seed,
                int mode, uint32_t stream_id, int32_t* idx, float* scale, int64_t* count,
                double* q_out, void* scratch, cudaStream_t st, int sample_mode) {
  const int G = draw_blocks(n);
  char* sp = static_cast<char*>(scratch);
  double* bpart = reinterpret_cast<double*>(sp);
  const bool iid = sample_mode == TP_SAMPLE_IID;
  {
    KernelScope ks(iid ? "draw_iid" : "draw", st);
    if (mode != TP_PROB_GIVEN) draw_sum_kernel<<<G, 256, 0, st>>>(w, w2, n, mode, bpart);
    if (iid) {
      uint64_t* W = reinterpret_cast<uint64_t*>(sp + ws_bytes(kDrawBlocks, 8));
      float* sval = reinterpret_cast<float*>(sp + ws_bytes(kDrawBlocks, 8) + ws_bytes(size_t(n), 8));
      iid_weights_kernel<<<G, 256, 0, st>>>(w, w2, n, c, mode, bpart, G, W, sval, q_out);
      iid_draw_kernel<<<1, 1024, 0, st>>>(n, c, seed, stream_id, W, sval, idx, scale, count);
    } else {
      draw_decide_kernel<<<G, 256, 0, st>>>(w, w2, n, c, seed, mode, stream_id, bpart, G, idx,
                                            scale, q_out);
      draw_compact_kernel<<<1, 1024, 0, st>>>(n, idx, scale, count);
    }
  }
  note_launches(mode != TP_PROB_GIVEN ? 2 : 1);
  return launch_status(iid ? "draw_iid" : "draw");
}

}  // namespace tp
