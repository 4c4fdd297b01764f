// Mode-3 DFT of real tubes kept to the half spectrum, and its inverse
// (Section 2, "Operators": fft(X,[],3) / ifft(X,[],3); Algorithm 1 steps 2-3
// and the final inverse).  Direct DFT per tube with the twiddle table
// exp(-2 pi i m / n3), m < n3, in shared memory; index m = k*t mod n3 is
// advanced incrementally.  Each thread owns one tube; the tube is staged in
// its own column of shared memory so that frequency chunks can re-read it.
#include "tp_internal.cuh"

namespace tp {
namespace {

constexpr int KC = 8;   // frequencies (or output times) per register chunk

__device__ __forceinline__ void build_twiddles(float2* tw, int n3) {
  for (int m = threadIdx.x; m < n3; m += blockDim.x) {
    double s, c;
    sincospi(2.0 * double(m) / double(n3), &s, &c);   // exact at quarter turns
    tw[m] = make_float2(float(c), float(s));
  }
}

__global__ void rdft_kernel(DftGather g) {
  extern __shared__ float sm[];
  const int n3 = int(g.n3);
  const int RB = blockDim.x;
  const int h = n3 / 2 + 1;
  float2* tw = reinterpret_cast<float2*>(sm);
  float* xs = sm + 2 * n3;
  build_twiddles(tw, n3);
  __syncthreads();

  int64_t count = g.dyn_count ? *g.dyn_count : (g.gather_dim == 1 ? g.rows : g.cols);
  int64_t rows_eff = g.rows, cols_eff = g.cols, rows_pad = g.rows, cols_pad = g.cols;
  if (g.gather_dim == 1) {
    rows_eff = count;
    rows_pad = min(g.rows, (count + 31) / 32 * 32);   // zero tail for tiled consumers
  } else if (g.gather_dim == 2) {
    cols_eff = count;
    cols_pad = min(g.cols, (count + 31) / 32 * 32);
  }
  const int64_t r = int64_t(blockIdx.x) * RB + threadIdx.x;
  if (int64_t(blockIdx.x) * RB >= rows_pad) return;
  const int tid = threadIdx.x;

  for (int64_t c = blockIdx.y; c < cols_pad; c += gridDim.y) {
    const bool active = r < rows_pad;
    const bool live = active && r < rows_eff && c < cols_eff;
    if (live) {
      int64_t ro = r, co = c;
      float s = 1.0f;
      if (g.gather_dim == 1) {
        ro = g.idx[r];
        if (g.scale) s = g.scale[r];
      } else if (g.gather_dim == 2) {
        co = g.idx[c];
        if (g.scale) s = g.scale[c];
      }
      const float* p = g.src + ro * g.row_stride + co * g.col_stride;
      for (int t = 0; t < n3; ++t) xs[t * RB + tid] = s * __ldg(p + int64_t(t) * g.slice_stride);
    } else {
      for (int t = 0; t < n3; ++t) xs[t * RB + tid] = 0.0f;
    }
    if (!active) continue;
    float* ore = g.out_re + r + g.out_ld * c;
    float* oim = g.out_im + r + g.out_ld * c;
    for (int k0 = 0; k0 < h; k0 += KC) {
      float ar[KC], ai[KC];
      int m[KC], step[KC];
#pragma unroll
      for (int q = 0; q < KC; ++q) {
        ar[q] = 0.f; ai[q] = 0.f; m[q] = 0; step[q] = (k0 + q) % n3;
      }
      for (int t = 0; t < n3; ++t) {
        const float x = xs[t * RB + tid];
#pragma unroll
        for (int q = 0; q < KC; ++q) {
          const float2 w = tw[m[q]];
          ar[q] = fmaf(x, w.x, ar[q]);
          ai[q] = fmaf(-x, w.y, ai[q]);
          m[q] += step[q];
          if (m[q] >= n3) m[q] -= n3;
        }
      }
#pragma unroll
      for (int q = 0; q < KC; ++q) {
        if (k0 + q < h) {
          ore[int64_t(k0 + q) * g.out_slice] = ar[q];
          oim[int64_t(k0 + q) * g.out_slice] = ai[q];
        }
      }
    }
  }
}

// out[r + rows*t] = (1/n3) sum_k w_k (Re X_k cos(2 pi k t/n3) - Im X_k sin(2 pi k t/n3)),
// w_k = 1 for k = 0 and k = n3/2, else 2 (conjugate partners folded in).
__global__ void irdft_kernel(const float* __restrict__ in_re, const float* __restrict__ in_im,
                             int64_t rows, int64_t in_slice, int n3, float* __restrict__ out) {
  extern __shared__ float sm[];
  const int RB = blockDim.x;
  const int h = n3 / 2 + 1;
  float2* tw = reinterpret_cast<float2*>(sm);
  float* sre = sm + 2 * n3;
  float* sim = sre + h * RB;
  build_twiddles(tw, n3);
  __syncthreads();
  const int tid = threadIdx.x;
  const float inv = 1.0f / float(n3);
  for (int64_t r0 = int64_t(blockIdx.x) * RB; r0 < rows; r0 += int64_t(gridDim.x) * RB) {
    const int64_t r = r0 + tid;
    if (r >= rows) continue;
    for (int k = 0; k < h; ++k) {
      const float wk = (k == 0 || 2 * k == n3) ? inv : 2.0f * inv;
      sre[k * RB + tid] = wk * __ldg(in_re + int64_t(k) * in_slice + r);
      sim[k * RB + tid] = wk * __ldg(in_im + int64_t(k) * in_slice + r);
    }
    for (int t0 = 0; t0 < n3; t0 += KC) {
      float acc[KC];
      int m[KC], step[KC];
#pragma unroll
      for (int q = 0; q < KC; ++q) { acc[q] = 0.f; m[q] = 0; step[q] = (t0 + q) % n3; }
      for (int k = 0; k < h; ++k) {
        const float re = sre[k * RB + tid];
        const float im = sim[k * RB + tid];
#pragma unroll
        for (int q = 0; q < KC; ++q) {
          const float2 w = tw[m[q]];
          acc[q] = fmaf(re, w.x, fmaf(-im, w.y, acc[q]));
          m[q] += step[q];
          if (m[q] >= n3) m[q] -= n3;
        }
      }
#pragma unroll
      for (int q = 0; q < KC; ++q)
        if (t0 + q < n3) out[r + rows * int64_t(t0 + q)] = acc[q];
    }
  }
}

int rows_per_block(int64_t n3) { return n3 <= 128 ? 128 : (n3 <= 256 ? 64 : 32); }

}  // namespace

int launch_rdft(const DftGather& g, cudaStream_t st) {
  if (g.n3 < 1 || g.n3 > 512) {
    set_error("rdft: n3 = %lld outside [1, 512]", (long long)g.n3);
    return TP_EUNSUPPORTED;
  }
  if (g.rows == 0 || g.cols == 0) return TP_OK;
  const int RB = rows_per_block(g.n3);
  const size_t smem = size_t(2 * g.n3) * sizeof(float) + size_t(g.n3) * RB * sizeof(float);
  cudaFuncSetAttribute(rdft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  const int64_t bx = (g.rows + RB - 1) / RB;
  if (bx > 0x7fffffff) { set_error("rdft: too many rows"); return TP_EINVAL; }
  const int64_t by = g.cols < 65535 ? g.cols : 65535;
  {
    KernelScope ks("rdft", st);
    rdft_kernel<<<dim3(unsigned(bx), unsigned(by)), RB, smem, st>>>(g);
  }
  return launch_status("rdft_kernel");
}

int launch_irdft(const float* in_re, const float* in_im, int64_t rows, int64_t in_slice,
                 int64_t n3, float* out, cudaStream_t st) {
  if (n3 < 1 || n3 > 512) {
    set_error("irdft: n3 = %lld outside [1, 512]", (long long)n3);
    return TP_EUNSUPPORTED;
  }
  if (rows == 0) return TP_OK;
  const int RB = rows_per_block(n3);
  const int64_t h = n3 / 2 + 1;
  const size_t smem = size_t(2 * n3) * sizeof(float) + size_t(2 * h) * RB * sizeof(float);
  cudaFuncSetAttribute(irdft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  int64_t blocks = (rows + RB - 1) / RB;
  if (blocks > 152 * 32) blocks = 152 * 32;
  {
    KernelScope ks("irdft", st);
    irdft_kernel<<<unsigned(blocks), RB, smem, st>>>(in_re, in_im, rows, in_slice, int(n3), out);
  }
  return launch_status("irdft_kernel");
}

}  // namespace tp
