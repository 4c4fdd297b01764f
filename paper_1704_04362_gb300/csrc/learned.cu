// Per-frequency truncation ranks for the randomized t-SVD: the plain adaptive
// rank rule and the learned rank/oversampling predictor (the paper has neither;
// the multi-rank of Section 2 is the rule's tol -> 0 limit).
//
// Rank rule.  With sketch singular values s_1 >= ... >= s_l of a frequency,
// the rank is the smallest r in [1, cap] whose discarded energy
// sum_{i > r} s_i^2 is at most tol^2 sum_i s_i^2 (cap if none; 0 for a zero
// slice).  Tail sums run from s_l upwards in float64 with separately rounded
// products and sums (no fused multiply-add), so the integer decision is
// reproducible anywhere the same order is used.
//
// Predictor.  Features log10(s_i / s_1), i = 2 .. 17, clipped at -8 and
// scaled by 1/8 (float16); a 16 -> 128 -> 128 -> 2 perceptron with ReLU and
// float16 weights, float32 activations and accumulation; mean-squared-error
// loss; Adam on float32 master weights.  Packed parameters, matrices
// row-major with the output index slowest: W1 (128 x 16), b1, W2 (128 x 128),
// b2, W3 (2 x 128), b3.
//
// Training kernels: a block takes 64 samples with the weights (as float) and
// both hidden layers in shared memory (row pitch 129: conflict-free along
// either index), runs forward and back-propagation and writes its gradient
// sums to its own row of a partial buffer; a second kernel adds the rows in a
// fixed order (deterministic), a third applies Adam and re-rounds the float16
// copy.
#include <cuda_fp16.h>

#include "tp_internal.cuh"

namespace tp {

constexpr int MLP_IN = 16, MLP_HID = 128, MLP_OUT = 2;
constexpr int MLP_NPARAM = MLP_HID * MLP_IN + MLP_HID + MLP_HID * MLP_HID + MLP_HID +
                           MLP_OUT * MLP_HID + MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_HID * MLP_IN, OFF_W2 = OFF_B1 + MLP_HID,
              OFF_B2 = OFF_W2 + MLP_HID * MLP_HID, OFF_W3 = OFF_B2 + MLP_HID,
              OFF_B3 = OFF_W3 + MLP_OUT * MLP_HID;
constexpr int MLP_S = 64;          // samples per block
constexpr int MLP_THREADS = 256;
constexpr int HP = MLP_HID + 1;    // row pitch of the shared matrices

size_t mlp_partial_count(int64_t B) {
  return size_t((B + MLP_S - 1) / MLP_S) * (MLP_NPARAM + 1);
}

namespace {

__global__ void rank_rule_kernel(const float* __restrict__ sig, int64_t h, int l, int cap,
                                 double tol, int32_t* __restrict__ out) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= h) return;
  const float* s = sig + k * l;
  // tail(r) = sum_{i > r} s_i^2; total = tail(0)
  double total = 0.0;
  for (int i = l - 1; i >= 0; --i) total = __dadd_rn(total, __dmul_rn(double(s[i]), double(s[i])));
  if (total == 0.0) {
    out[k] = 0;
    return;
  }
  const double thr = __dmul_rn(__dmul_rn(tol, tol), total);
  const int rmax = cap < l ? cap : l;
  // walk r upwards: the tail after r is the sum of the suffix, recomputed in the
  // same order (from the smallest value) so the comparison is reproducible
  int r = cap;
  for (int rr = 1; rr <= rmax; ++rr) {
    double tail = 0.0;
    for (int i = l - 1; i >= rr; --i) tail = __dadd_rn(tail, __dmul_rn(double(s[i]), double(s[i])));
    if (tail <= thr) {
      r = rr;
      break;
    }
  }
  out[k] = r;
}

__global__ void features_kernel(const float* __restrict__ sig, int64_t h, int l,
                                __half* __restrict__ feat) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= h * MLP_IN) return;
  const int64_t k = e / MLP_IN;
  const int i = int(e - k * MLP_IN) + 1;   // s_{i+1} / s_1, 0-based column i
  const double s1 = sig[k * l];
  double ratio = s1 > 0.0 ? double(sig[k * l + i]) / s1 : 0.0;
  if (ratio < 1e-8) ratio = 1e-8;
  double f = log10(ratio);
  if (f < -8.0) f = -8.0;
  feat[e] = __float2half_rn(float(f / 8.0));
}

struct MlpSmem {
  float w1t[MLP_IN * HP];      // W1 transposed: [input][hidden]
  float w2t[MLP_HID * HP];     // W2 transposed: [input k][output j]
  float w3[MLP_OUT * MLP_HID];
  float b1[MLP_HID], b2[MLP_HID], b3[MLP_OUT];
  float x[MLP_S * MLP_IN];
  float h1[MLP_S * HP];        // then dz1
  float h2[MLP_S * HP];        // then dz2
  float y[MLP_S * MLP_OUT];    // outputs, then dy
  float red[MLP_THREADS / 32];
};

__device__ void mlp_load(MlpSmem& sm, const __half* __restrict__ w, const __half* __restrict__ x,
                         int64_t s0, int ns) {
  const int tid = threadIdx.x;
  for (int e = tid; e < MLP_HID * MLP_IN; e += MLP_THREADS) {
    const int j = e / MLP_IN, i = e % MLP_IN;
    sm.w1t[i * HP + j] = __half2float(w[OFF_W1 + e]);
  }
  for (int e = tid; e < MLP_HID * MLP_HID; e += MLP_THREADS) {
    const int j = e / MLP_HID, k = e % MLP_HID;
    sm.w2t[k * HP + j] = __half2float(w[OFF_W2 + e]);
  }
  for (int e = tid; e < MLP_OUT * MLP_HID; e += MLP_THREADS) sm.w3[e] = __half2float(w[OFF_W3 + e]);
  for (int e = tid; e < MLP_HID; e += MLP_THREADS) {
    sm.b1[e] = __half2float(w[OFF_B1 + e]);
    sm.b2[e] = __half2float(w[OFF_B2 + e]);
  }
  if (tid < MLP_OUT) sm.b3[tid] = __half2float(w[OFF_B3 + tid]);
  for (int e = tid; e < MLP_S * MLP_IN; e += MLP_THREADS) {
    const int s = e / MLP_IN;
    sm.x[e] = s < ns ? __half2float(x[(s0 + s) * MLP_IN + e % MLP_IN]) : 0.f;
  }
  __syncthreads();
}

// h1, h2 and y of the block's samples (rows past ns are computed on zero
// inputs and ignored by the callers).
__device__ void mlp_forward_block(MlpSmem& sm) {
  const int tid = threadIdx.x;
  for (int e = tid; e < MLP_S * MLP_HID; e += MLP_THREADS) {
    const int s = e / MLP_HID, j = e % MLP_HID;
    float z = sm.b1[j];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) z = fmaf(sm.w1t[i * HP + j], sm.x[s * MLP_IN + i], z);
    sm.h1[s * HP + j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  for (int e = tid; e < MLP_S * MLP_HID; e += MLP_THREADS) {
    const int s = e / MLP_HID, j = e % MLP_HID;
    float z = sm.b2[j];
#pragma unroll 8
    for (int k = 0; k < MLP_HID; ++k) z = fmaf(sm.w2t[k * HP + j], sm.h1[s * HP + k], z);
    sm.h2[s * HP + j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  for (int e = tid; e < MLP_S * MLP_OUT; e += MLP_THREADS) {
    const int s = e / MLP_OUT, o = e % MLP_OUT;
    float z = sm.b3[o];
    for (int k = 0; k < MLP_HID; ++k) z = fmaf(sm.w3[o * MLP_HID + k], sm.h2[s * HP + k], z);
    sm.y[e] = z;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(MLP_THREADS) mlp_forward_kernel(const __half* __restrict__ w,
                                                                  const __half* __restrict__ x,
                                                                  int64_t B,
                                                                  float* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char mlp_raw[];
  MlpSmem& sm = *reinterpret_cast<MlpSmem*>(mlp_raw);
  const int64_t s0 = int64_t(blockIdx.x) * MLP_S;
  const int ns = int(B - s0 < MLP_S ? B - s0 : MLP_S);
  mlp_load(sm, w, x, s0, ns);
  mlp_forward_block(sm);
  for (int e = threadIdx.x; e < ns * MLP_OUT; e += MLP_THREADS) y[s0 * MLP_OUT + e] = sm.y[e];
}

__device__ float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < MLP_THREADS / 32; ++w) t += red[w];
  return t;
}

// Gradient sums of one block of samples (scaled by 1/B) into part[block].
__global__ void __launch_bounds__(MLP_THREADS) mlp_grad_kernel(const __half* __restrict__ w,
                                                               const __half* __restrict__ x,
                                                               const float* __restrict__ tgt,
                                                               int64_t B,
                                                               float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char mlp_raw[];
  MlpSmem& sm = *reinterpret_cast<MlpSmem*>(mlp_raw);
  const int tid = threadIdx.x;
  const int64_t s0 = int64_t(blockIdx.x) * MLP_S;
  const int ns = int(B - s0 < MLP_S ? B - s0 : MLP_S);
  float* g = part + int64_t(blockIdx.x) * (MLP_NPARAM + 1);
  const float invB = 1.0f / float(B);
  mlp_load(sm, w, x, s0, ns);
  mlp_forward_block(sm);
  // dy = (y - t) / B on valid rows, 0 past them; loss partial
  float lp = 0.f;
  for (int e = tid; e < MLP_S * MLP_OUT; e += MLP_THREADS) {
    const int s = e / MLP_OUT;
    float d = 0.f;
    if (s < ns) {
      d = sm.y[e] - tgt[s0 * MLP_OUT + e];
      lp += d * d;
    }
    sm.y[e] = d * invB;
  }
  const float loss = block_sum(lp, sm.red);
  if (tid == 0) g[MLP_NPARAM] = 0.5f * loss * invB;
  __syncthreads();
  // W3, b3
  for (int e = tid; e < MLP_OUT * MLP_HID; e += MLP_THREADS) {
    const int o = e / MLP_HID, k = e % MLP_HID;
    float a = 0.f;
    for (int s = 0; s < MLP_S; ++s) a = fmaf(sm.y[s * MLP_OUT + o], sm.h2[s * HP + k], a);
    g[OFF_W3 + e] = a;
  }
  if (tid < MLP_OUT) {
    float a = 0.f;
    for (int s = 0; s < MLP_S; ++s) a += sm.y[s * MLP_OUT + tid];
    g[OFF_B3 + tid] = a;
  }
  __syncthreads();
  // dz2 = (W3^T dy) * [h2 > 0], in place of h2
  for (int e = tid; e < MLP_S * MLP_HID; e += MLP_THREADS) {
    const int s = e / MLP_HID, k = e % MLP_HID;
    float d = 0.f;
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) d = fmaf(sm.w3[o * MLP_HID + k], sm.y[s * MLP_OUT + o], d);
    sm.h2[s * HP + k] = sm.h2[s * HP + k] > 0.f ? d : 0.f;
  }
  __syncthreads();
  // W2 (j, k) = sum_s dz2(s, j) h1(s, k); b2
  for (int e = tid; e < MLP_HID * MLP_HID; e += MLP_THREADS) {
    const int j = e / MLP_HID, k = e % MLP_HID;
    float a = 0.f;
    for (int s = 0; s < MLP_S; ++s) a = fmaf(sm.h2[s * HP + j], sm.h1[s * HP + k], a);
    g[OFF_W2 + e] = a;
  }
  for (int j = tid; j < MLP_HID; j += MLP_THREADS) {
    float a = 0.f;
    for (int s = 0; s < MLP_S; ++s) a += sm.h2[s * HP + j];
    g[OFF_B2 + j] = a;
  }
  __syncthreads();
  // dz1 = (W2^T dz2) * [h1 > 0], in place of h1
  for (int e = tid; e < MLP_S * MLP_HID; e += MLP_THREADS) {
    const int s = e / MLP_HID, k = e % MLP_HID;
    float d = 0.f;
#pragma unroll 8
    for (int j = 0; j < MLP_HID; ++j) d = fmaf(sm.w2t[k * HP + j], sm.h2[s * HP + j], d);
    sm.h1[s * HP + k] = sm.h1[s * HP + k] > 0.f ? d : 0.f;
  }
  __syncthreads();
  // W1 (j, i) = sum_s dz1(s, j) x(s, i); b1
  for (int e = tid; e < MLP_HID * MLP_IN; e += MLP_THREADS) {
    const int j = e / MLP_IN, i = e % MLP_IN;
    float a = 0.f;
    for (int s = 0; s < MLP_S; ++s) a = fmaf(sm.h1[s * HP + j], sm.x[s * MLP_IN + i], a);
    g[OFF_W1 + e] = a;
  }
  for (int j = tid; j < MLP_HID; j += MLP_THREADS) {
    float a = 0.f;
    for (int s = 0; s < MLP_S; ++s) a += sm.h1[s * HP + j];
    g[OFF_B1 + j] = a;
  }
}

// grad[p] = sum over blocks of part[b][p], blocks in order; p = MLP_NPARAM is the loss.
__global__ void mlp_reduce_kernel(const float* __restrict__ part, int64_t nblocks,
                                  float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > MLP_NPARAM) return;
  float a = 0.f;
  for (int64_t b = 0; b < nblocks; ++b) a += part[b * (MLP_NPARAM + 1) + p];
  grad[p] = a;
}

__global__ void mlp_adam_kernel(float* __restrict__ theta, float* __restrict__ m,
                                float* __restrict__ v, const float* __restrict__ grad,
                                __half* __restrict__ w16, float lr, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAM) return;
  const float gp = grad[p];
  const float mp = 0.9f * m[p] + 0.1f * gp;
  const float vp = 0.999f * v[p] + 0.001f * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const float th = theta[p] - lr * (mp / c1) / (sqrtf(vp / c2) + 1e-8f);
  theta[p] = th;
  w16[p] = __float2half_rn(th);
}

__global__ void mlp_round_kernel(const float* __restrict__ theta, __half* __restrict__ w16) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < MLP_NPARAM) w16[p] = __float2half_rn(theta[p]);
}

}  // namespace

int launch_rank_rule(const float* sig, int64_t h, int l, int cap, double tol, int32_t* out,
                     cudaStream_t st) {
  {
    KernelScope ks("rank_rule", st);
    rank_rule_kernel<<<unsigned((h + 127) / 128), 128, 0, st>>>(sig, h, l, cap, tol, out);
  }
  return launch_status("rank_rule_kernel");
}

int launch_rank_features(const float* sig, int64_t h, int l, void* feat, cudaStream_t st) {
  {
    KernelScope ks("rank_features", st);
    features_kernel<<<unsigned((h * MLP_IN + 255) / 256), 256, 0, st>>>(
        sig, h, l, reinterpret_cast<__half*>(feat));
  }
  return launch_status("features_kernel");
}

int launch_mlp_forward(const void* w16, const void* x16, int64_t B, float* y, cudaStream_t st) {
  if (B == 0) return TP_OK;
  const size_t smem = sizeof(MlpSmem);
  TP_SET_SMEM(mlp_forward_kernel, smem);
  {
    KernelScope ks("mlp_forward", st);
    mlp_forward_kernel<<<unsigned((B + MLP_S - 1) / MLP_S), MLP_THREADS, smem, st>>>(
        reinterpret_cast<const __half*>(w16), reinterpret_cast<const __half*>(x16), B, y);
  }
  return launch_status("mlp_forward_kernel");
}

int launch_mlp_round(const float* theta, void* w16, cudaStream_t st) {
  {
    KernelScope ks("mlp_round", st);
    mlp_round_kernel<<<unsigned((MLP_NPARAM + 255) / 256), 256, 0, st>>>(
        theta, reinterpret_cast<__half*>(w16));
  }
  return launch_status("mlp_round_kernel");
}

// grad (MLP_NPARAM + 1 floats, the last the loss) of the float16 weights on
// the batch; part: mlp_partial_count(B) floats of scratch.
int launch_mlp_grad(const void* w16, const void* x16, const float* tgt, int64_t B, float* part,
                    float* grad, cudaStream_t st) {
  const int64_t nb = (B + MLP_S - 1) / MLP_S;
  const size_t smem = sizeof(MlpSmem);
  TP_SET_SMEM(mlp_grad_kernel, smem);
  {
    KernelScope ks("mlp_grad", st);
    mlp_grad_kernel<<<unsigned(nb), MLP_THREADS, smem, st>>>(
        reinterpret_cast<const __half*>(w16), reinterpret_cast<const __half*>(x16), tgt, B, part);
  }
  {
    KernelScope ks("mlp_reduce", st);
    mlp_reduce_kernel<<<unsigned((MLP_NPARAM + 1 + 255) / 256), 256, 0, st>>>(part, nb, grad);
  }
  return launch_status("mlp_grad_kernel");
}

int launch_mlp_adam(float* theta, float* m, float* v, const float* grad, void* w16, int step,
                    float lr, cudaStream_t st) {
  const float c1 = 1.0f - powf(0.9f, float(step)), c2 = 1.0f - powf(0.999f, float(step));
  {
    KernelScope ks("mlp_adam", st);
    mlp_adam_kernel<<<unsigned((MLP_NPARAM + 255) / 256), 256, 0, st>>>(
        theta, m, v, grad, reinterpret_cast<__half*>(w16), lr, c1, c2);
  }
  return launch_status("mlp_adam_kernel");
}

}  // namespace tp
