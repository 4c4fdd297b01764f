// Mode-3 DFT of real tubes kept to the half spectrum, and its inverse
// (Section 2, "Operators": fft(X,[],3) / ifft(X,[],3); Algorithm 1 steps 2-3
// and the final inverse).
//
// Both directions are small dense contractions per tube (n3 x h complex
// coefficients), computed as register-blocked SIMT products: each thread owns
// TPT tubes and KC output frequencies (or times) at a time, and the KC
// columns of the transform matrix it needs are built once per block and
// chunk in shared memory from the n3-entry twiddle table
// exp(-2 pi i m / n3), m = k*t mod n3.  Tube samples are read straight from
// global memory (coalesced across the warp; L1 serves the re-reads of later
// chunks).
#include "tp_internal.cuh"

namespace tp {
namespace {

constexpr int KC = 16;   // frequencies (forward) or times (inverse) per chunk
constexpr int TPT = 2;   // tubes per thread
constexpr int RB = 128;  // threads per block
constexpr int TU = 8;    // samples (forward) or frequencies (inverse) loaded ahead

// Nearest tf32 value of x (10 explicit mantissa bits), as a float.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void build_twiddles(float2* tw, int n3) {
  for (int m = threadIdx.x; m < n3; m += blockDim.x) {
    double s, c;
    sincospi(2.0 * double(m) / double(n3), &s, &c);   // exact at quarter turns
    tw[m] = make_float2(float(c), float(s));
  }
}

__global__ void __launch_bounds__(RB) rdft_kernel(DftGather g) {
  extern __shared__ float2 sm2[];
  const int n3 = int(g.n3);
  const int h = n3 / 2 + 1;
  const int n3p = (n3 + TU - 1) / TU * TU;
  float2* tw = sm2;
  float2* Wc = sm2 + n3;   // Wc[t*KC + q] = tw[(k0+q)*t mod n3], zero for t >= n3
  build_twiddles(tw, n3);

  const int64_t count = g.dyn_count ? *g.dyn_count : (g.gather_dim == 1 ? g.rows : g.cols);
  int64_t rows_eff = g.rows, cols_eff = g.cols, rows_pad = g.rows, cols_pad = g.cols;
  if (g.gather_dim == 1) {
    rows_eff = count;
    rows_pad = min(g.rows, (count + 31) / 32 * 32);   // zero tail for tiled consumers
  } else if (g.gather_dim == 2) {
    cols_eff = count;
    cols_pad = min(g.cols, (count + 31) / 32 * 32);
  }
  const int64_t base = int64_t(blockIdx.x) * (RB * TPT);
  if (base >= rows_pad) return;   // uniform over the block
  const int tid = threadIdx.x;

  for (int64_t c = blockIdx.y; c < cols_pad; c += gridDim.y) {
    const float* p[TPT];
    float s[TPT];
    bool act[TPT];
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
      const int64_t r = base + j * RB + tid;
      act[j] = r < rows_pad;
      p[j] = nullptr;
      s[j] = 0.f;
      if (act[j] && r < rows_eff && c < cols_eff) {
        int64_t ro = r, co = c;
        s[j] = 1.0f;
        if (g.gather_dim == 1) {
          ro = g.idx[r];
          if (g.scale) s[j] = g.scale[r];
        } else if (g.gather_dim == 2) {
          co = g.idx[c];
          if (g.scale) s[j] = g.scale[c];
        }
        p[j] = g.src + ro * g.row_stride + co * g.col_stride;
      }
    }
    for (int k0 = 0; k0 < h; k0 += KC) {
      __syncthreads();   // previous chunk done with Wc (and tw built)
      for (int e = tid; e < n3p * KC; e += RB) {
        const int t = e / KC, q = e - t * KC;
        Wc[e] = t < n3 ? tw[int((int64_t(k0 + q) * t) % n3)] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      float ar[TPT][KC], ai[TPT][KC];
#pragma unroll
      for (int j = 0; j < TPT; ++j)
#pragma unroll
        for (int q = 0; q < KC; ++q) { ar[j][q] = 0.f; ai[j][q] = 0.f; }
      for (int t0 = 0; t0 < n3; t0 += TU) {
        // all TU samples of both tubes in flight before the arithmetic
        float x[TPT][TU];
#pragma unroll
        for (int u = 0; u < TU; ++u)
#pragma unroll
          for (int j = 0; j < TPT; ++j)
            x[j][u] = (p[j] && t0 + u < n3) ? s[j] * __ldg(p[j] + int64_t(t0 + u) * g.slice_stride)
                                            : 0.f;
#pragma unroll
        for (int u = 0; u < TU; ++u) {
#pragma unroll
          for (int q = 0; q < KC; ++q) {
            const float2 w = Wc[(t0 + u) * KC + q];   // zero rows past n3
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
              ar[j][q] = fmaf(x[j][u], w.x, ar[j][q]);
              ai[j][q] = fmaf(-x[j][u], w.y, ai[j][q]);
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < TPT; ++j) {
        if (!act[j]) continue;
        const int64_t r = base + j * RB + tid;
        const int64_t o = r + g.out_ld * c;
        if (g.out_re_lo) {
#pragma unroll
          for (int q = 0; q < KC; ++q) {
            if (k0 + q < h) {
              const int64_t oo = o + int64_t(k0 + q) * g.out_slice;
              const float hr = tf32_rna(ar[j][q]), hi = tf32_rna(ai[j][q]);
              g.out_re[oo] = hr;
              g.out_re_lo[oo] = ar[j][q] - hr;
              g.out_im[oo] = hi;
              g.out_im_lo[oo] = ai[j][q] - hi;
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < KC; ++q) {
            if (k0 + q < h) {
              g.out_re[o + int64_t(k0 + q) * g.out_slice] = ar[j][q];
              g.out_im[o + int64_t(k0 + q) * g.out_slice] = ai[j][q];
            }
          }
        }
      }
    }
  }
}

// Same transform, written transposed: element (r, c) of slice k goes to
// out[k*out_slice + c + out_ld*r], so that the picked-slice index (the
// facewise product's inner dimension) is contiguous.  A block owns a tile of
// 32 rows x 8 columns (rows fastest, so tube reads stay coalesced); each
// frequency chunk is staged through shared memory and stored as 32-byte runs
// along the column index.
constexpr int TR = 32, TCOL = 8;

__global__ void __launch_bounds__(RB) rdft_t_kernel(DftGather g) {
  extern __shared__ float2 sm2[];
  const int n3 = int(g.n3);
  const int h = n3 / 2 + 1;
  const int n3p = (n3 + TU - 1) / TU * TU;
  float2* tw = sm2;
  float2* Wc = sm2 + n3;
  float* stg = reinterpret_cast<float*>(Wc + n3p * KC);   // [KC][TR][TCOL + 1]
  build_twiddles(tw, n3);

  const int64_t count = g.dyn_count ? *g.dyn_count : (g.gather_dim == 1 ? g.rows : g.cols);
  int64_t rows_eff = g.rows, cols_eff = g.cols, rows_pad = g.rows, cols_pad = g.cols;
  if (g.gather_dim == 1) {
    rows_eff = count;
    rows_pad = min(g.rows, (count + 31) / 32 * 32);
  } else if (g.gather_dim == 2) {
    cols_eff = count;
    cols_pad = min(g.cols, (count + 31) / 32 * 32);
  }
  const int64_t r0 = int64_t(blockIdx.x) * TR;
  if (r0 >= rows_pad) return;   // uniform over the block
  const int tid = threadIdx.x;
  const int lr = tid % TR, lc = tid / TR;   // this thread: row lr, columns lc and lc + 4
  const int64_t r = r0 + lr;

  for (int64_t c0 = int64_t(blockIdx.y) * TCOL; c0 < cols_pad; c0 += int64_t(gridDim.y) * TCOL) {
    const float* p[TPT];
    float s[TPT];
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
      const int64_t c = c0 + lc + 4 * j;
      p[j] = nullptr;
      s[j] = 0.f;
      if (r < rows_eff && c < cols_eff) {
        int64_t ro = r, co = c;
        s[j] = 1.0f;
        if (g.gather_dim == 1) {
          ro = g.idx[r];
          if (g.scale) s[j] = g.scale[r];
        } else if (g.gather_dim == 2) {
          co = g.idx[c];
          if (g.scale) s[j] = g.scale[c];
        }
        p[j] = g.src + ro * g.row_stride + co * g.col_stride;
      }
    }
    for (int k0 = 0; k0 < h; k0 += KC) {
      __syncthreads();
      for (int e = tid; e < n3p * KC; e += RB) {
        const int t = e / KC, q = e - t * KC;
        Wc[e] = t < n3 ? tw[int((int64_t(k0 + q) * t) % n3)] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      float ar[TPT][KC], ai[TPT][KC];
#pragma unroll
      for (int j = 0; j < TPT; ++j)
#pragma unroll
        for (int q = 0; q < KC; ++q) { ar[j][q] = 0.f; ai[j][q] = 0.f; }
      for (int t0 = 0; t0 < n3; t0 += TU) {
        // all TU samples of both tubes in flight before the arithmetic
        float x[TPT][TU];
#pragma unroll
        for (int u = 0; u < TU; ++u)
#pragma unroll
          for (int j = 0; j < TPT; ++j)
            x[j][u] = (p[j] && t0 + u < n3) ? s[j] * __ldg(p[j] + int64_t(t0 + u) * g.slice_stride)
                                            : 0.f;
#pragma unroll
        for (int u = 0; u < TU; ++u) {
#pragma unroll
          for (int q = 0; q < KC; ++q) {
            const float2 w = Wc[(t0 + u) * KC + q];   // zero rows past n3
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
              ar[j][q] = fmaf(x[j][u], w.x, ar[j][q]);
              ai[j][q] = fmaf(-x[j][u], w.y, ai[j][q]);
            }
          }
        }
      }
      // planes: 0 re (hi), 1 im (hi), 2 re lo, 3 im lo
      const int nplanes = g.out_re_lo ? 4 : 2;
      for (int pl = 0; pl < nplanes; ++pl) {
        __syncthreads();   // staging buffer free
#pragma unroll
        for (int j = 0; j < TPT; ++j)
#pragma unroll
          for (int q = 0; q < KC; ++q) {
            const float v = (pl & 1) ? ai[j][q] : ar[j][q];
            float o;
            if (!g.out_re_lo) o = v;
            else if (pl < 2) o = tf32_rna(v);
            else o = v - tf32_rna(v);
            stg[(q * TR + lr) * (TCOL + 1) + lc + 4 * j] = o;
          }
        __syncthreads();
        float* dst = pl == 0 ? g.out_re : pl == 1 ? g.out_im : pl == 2 ? g.out_re_lo : g.out_im_lo;
        // thread -> (column wc, row wr); 16 rows per pass, two passes
        const int wc = tid % TCOL, wr = tid / TCOL;
        const int64_t c = c0 + wc;
        if (c < cols_pad) {
          for (int q = 0; q < KC && k0 + q < h; ++q) {
#pragma unroll
            for (int pass = 0; pass < TR / (RB / TCOL); ++pass) {
              const int rr = wr + pass * (RB / TCOL);
              const int64_t rg = r0 + rr;
              if (rg < rows_pad)
                dst[int64_t(k0 + q) * g.out_slice + c + g.out_ld * rg] =
                    stg[(q * TR + rr) * (TCOL + 1) + wc];
            }
          }
        }
      }
    }
  }
}

// out[r + rows*t] = sum_k (w_k/n3) (Re X_k cos(2 pi k t/n3) - Im X_k sin(2 pi k t/n3)),
// w_k = 1 for k = 0 and k = n3/2, else 2 (conjugate partners folded in).
__global__ void __launch_bounds__(RB) irdft_kernel(const float* __restrict__ in_re,
                                                   const float* __restrict__ in_im, int64_t rows,
                                                   int64_t in_slice, int n3,
                                                   float* __restrict__ out) {
  extern __shared__ float2 sm2[];
  const int h = n3 / 2 + 1;
  const int hp = (h + TU - 1) / TU * TU;
  float2* tw = sm2;
  float2* Vc = sm2 + n3;   // Vc[k*KC + q] = (w_k/n3) tw[k*(t0+q) mod n3], zero for k >= h
  build_twiddles(tw, n3);
  const int tid = threadIdx.x;
  const float inv = 1.0f / float(n3);
  for (int64_t base = int64_t(blockIdx.x) * (RB * TPT); base < rows;
       base += int64_t(gridDim.x) * (RB * TPT)) {
    int64_t r[TPT];
#pragma unroll
    for (int j = 0; j < TPT; ++j) r[j] = base + j * RB + tid;
    for (int t0 = 0; t0 < n3; t0 += KC) {
      __syncthreads();
      for (int e = tid; e < hp * KC; e += RB) {
        const int k = e / KC, q = e - k * KC;
        if (k < h) {
          const float wk = (k == 0 || 2 * k == n3) ? inv : 2.0f * inv;
          const float2 w = tw[int((int64_t(k) * (t0 + q)) % n3)];
          Vc[e] = make_float2(wk * w.x, wk * w.y);
        } else {
          Vc[e] = make_float2(0.f, 0.f);
        }
      }
      __syncthreads();
      float acc[TPT][KC];
#pragma unroll
      for (int j = 0; j < TPT; ++j)
#pragma unroll
        for (int q = 0; q < KC; ++q) acc[j][q] = 0.f;
      for (int k0 = 0; k0 < h; k0 += TU) {
        float re[TPT][TU], im[TPT][TU];
#pragma unroll
        for (int u = 0; u < TU; ++u)
#pragma unroll
          for (int j = 0; j < TPT; ++j) {
            const bool ok = r[j] < rows && k0 + u < h;
            re[j][u] = ok ? __ldg(in_re + int64_t(k0 + u) * in_slice + r[j]) : 0.f;
            im[j][u] = ok ? __ldg(in_im + int64_t(k0 + u) * in_slice + r[j]) : 0.f;
          }
#pragma unroll
        for (int u = 0; u < TU; ++u)
#pragma unroll
          for (int q = 0; q < KC; ++q) {
            const float2 v = Vc[(k0 + u) * KC + q];   // zero rows past h
#pragma unroll
            for (int j = 0; j < TPT; ++j)
              acc[j][q] = fmaf(re[j][u], v.x, fmaf(-im[j][u], v.y, acc[j][q]));
          }
      }
#pragma unroll
      for (int j = 0; j < TPT; ++j) {
        if (r[j] >= rows) continue;
#pragma unroll
        for (int q = 0; q < KC; ++q)
          if (t0 + q < n3) out[r[j] + rows * int64_t(t0 + q)] = acc[j][q];
      }
    }
  }
}

}  // namespace

bool fft_supported(int64_t n3);
int launch_fft_fwd(const float* X, int64_t rows, int64_t n3, float* ore, float* oim,
                   int64_t out_slice, cudaStream_t st);
int launch_fft_inv(const float* ire, const float* iim, int64_t rows, int64_t in_slice, int64_t n3,
                   float* out, cudaStream_t st);

// Tubes longer than this go through the shared-memory FFT when their length
// factors into small radices and no gather or split output is asked for.
constexpr int64_t kFftThreshold = 256;

int launch_rdft(const DftGather& g, cudaStream_t st) {
  const bool plain = g.gather_dim == 0 && !g.out_transposed && !g.out_re_lo &&
                     (g.cols == 1 || g.col_stride == g.rows) && g.out_ld == g.rows &&
                     g.out_slice == g.rows * g.cols && g.slice_stride == g.rows * g.cols &&
                     g.row_stride == 1;
  if (plain && g.n3 > kFftThreshold && fft_supported(g.n3))
    return launch_fft_fwd(g.src, g.rows * g.cols, g.n3, g.out_re, g.out_im, g.out_slice, st);
  if (g.n3 < 1 || g.n3 > 512) {
    set_error("rdft: n3 = %lld: longer than 512 needs a plain (ungathered) transform and "
              "prime factors <= 13", (long long)g.n3);
    return TP_EUNSUPPORTED;
  }
  if (g.rows == 0 || g.cols == 0) return TP_OK;
  if (g.out_transposed) {
    const int64_t n3p = (g.n3 + TU - 1) / TU * TU;
    const size_t smem = size_t(g.n3 + n3p * KC) * sizeof(float2) +
                        size_t(KC) * TR * (TCOL + 1) * sizeof(float);
    cudaFuncSetAttribute(rdft_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    const int64_t bx = (g.rows + TR - 1) / TR;
    if (bx > 0x7fffffff) { set_error("rdft: too many rows"); return TP_EINVAL; }
    int64_t by = (g.cols + TCOL - 1) / TCOL;
    if (by > 65535) by = 65535;
    {
      KernelScope ks("rdft_t", st);
      rdft_t_kernel<<<dim3(unsigned(bx), unsigned(by)), RB, smem, st>>>(g);
    }
    return launch_status("rdft_t_kernel");
  }
  const int64_t n3p = (g.n3 + TU - 1) / TU * TU;
  const size_t smem = size_t(g.n3 + n3p * KC) * sizeof(float2);
  cudaFuncSetAttribute(rdft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  const int64_t bx = (g.rows + RB * TPT - 1) / (RB * TPT);
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
  if (n3 > kFftThreshold && fft_supported(n3))
    return launch_fft_inv(in_re, in_im, rows, in_slice, n3, out, st);
  if (n3 < 1 || n3 > 512) {
    set_error("irdft: n3 = %lld: longer than 512 needs prime factors <= 13", (long long)n3);
    return TP_EUNSUPPORTED;
  }
  if (rows == 0) return TP_OK;
  const int64_t h = n3 / 2 + 1;
  const int64_t hp = (h + TU - 1) / TU * TU;
  const size_t smem = size_t(n3 + hp * KC) * sizeof(float2);
  cudaFuncSetAttribute(irdft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  int64_t blocks = (rows + RB * TPT - 1) / (RB * TPT);
  if (blocks > 152 * 64) blocks = 152 * 64;
  {
    KernelScope ks("irdft", st);
    irdft_kernel<<<unsigned(blocks), RB, smem, st>>>(in_re, in_im, rows, in_slice, int(n3), out);
  }
  return launch_status("irdft_kernel");
}

}  // namespace tp
