// Mode-3 DFT of real tubes (half spectrum) and its inverse for power-of-two
// tube lengths N = 2 .. 128, one tube per thread, held in registers
// (Section 2, "Operators": fft(X,[],3) / ifft(X,[],3); Algorithm 1 steps 2-3
// and the final inverse).
//
// Forward.  The N real samples are packed as M = N/2 complex values
// z_n = x_{2n} + i x_{2n+1}.  An M-point complex FFT (radix-2 decimation in
// frequency, fully unrolled, output in bit-reversed order) gives Z_k, and the
// spectra of the even and of the odd samples are
//     E_k = (Z_k + conj Z_{M-k}) / 2,   O_k = (Z_k - conj Z_{M-k}) / (2i),
// so that with w = exp(-2 pi i / N)
//     X_k = E_k + w^k O_k,   X_{M-k} = conj(E_k - w^k O_k),
//     X_0 = Re Z_0 + Im Z_0,  X_M = Re Z_0 - Im Z_0.
// Inverse.  The same relations read backwards give, from the half spectrum,
//     E_k = (X_k + conj X_{M-k}) / 2,   O_k = (X_k - conj X_{M-k}) conj(w^k) / 2,
//     Z_k = E_k + i O_k,
// and z = IFFT_M(Z) = conj(FFT_M(conj Z)) / M returns x_{2n} = Re z_n,
// x_{2n+1} = Im z_n.  The imaginary parts of the real slices X_0 and X_M
// are ignored, as the Hermitian completion requires.
//
// Each tube costs O(N log N) register arithmetic, so these kernels are bound
// by their HBM traffic (the direct contraction costs O(N^2) and is bound by
// instruction issue).  Twiddles are compile-time constants: a 128-entry
// table exp(-2 pi i m / 128) evaluated by the compiler (Taylor series in
// double, rounded once to float) and placed in constant memory, read at
// indices known after unrolling.
#include "dft_common.cuh"

namespace tp {
namespace {
using namespace dftc;

constexpr int kTw = 128;
constexpr int kThreads = 256;

constexpr double series_sin(double x) {   // |x| <= pi/4
  double term = x, sum = x;
  for (int n = 1; n <= 12; ++n) {
    term *= -(x * x) / double((2 * n) * (2 * n + 1));
    sum += term;
  }
  return sum;
}
constexpr double series_cos(double x) {   // |x| <= pi/4
  double term = 1.0, sum = 1.0;
  for (int n = 1; n <= 12; ++n) {
    term *= -(x * x) / double((2 * n - 1) * (2 * n));
    sum += term;
  }
  return sum;
}

struct TwTable {
  float c[kTw];   // cos(2 pi m / 128)
  float s[kTw];   // sin(2 pi m / 128)
};

// Angle 2 pi m / 128 = q (pi/2) + b with quadrant q and b = (pi/2) r / 128;
// b above pi/4 is taken as the complement so that the series stay on [0, pi/4].
constexpr TwTable make_twiddles() {
  TwTable t{};
  const double half_pi = 1.57079632679489661923;
  for (int m = 0; m < kTw; ++m) {
    const int q = (4 * m) / kTw;
    const int r = 4 * m - q * kTw;
    double cb = 0.0, sb = 0.0;
    if (2 * r <= kTw) {
      const double b = half_pi * double(r) / double(kTw);
      cb = series_cos(b);
      sb = series_sin(b);
    } else {
      const double b = half_pi * double(kTw - r) / double(kTw);
      cb = series_sin(b);
      sb = series_cos(b);
    }
    double c = cb, s = sb;
    if (q == 1) {
      c = -sb;
      s = cb;
    } else if (q == 2) {
      c = -cb;
      s = -sb;
    } else if (q == 3) {
      c = sb;
      s = -cb;
    }
    t.c[m] = float(c);
    t.s[m] = float(s);
  }
  return t;
}

__constant__ TwTable kTwd = make_twiddles();

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

__device__ __forceinline__ constexpr int bitrev(int k, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((k >> b) & 1) << (bits - 1 - b);
  return r;
}

// In-place M-point FFT (exp(-2 pi i nk / M)), natural order in, bit-reversed out.
template <int M>
__device__ __forceinline__ void fft_dif(float2 (&a)[M]) {
  constexpr int S = ilog2(M);
#pragma unroll
  for (int st = 0; st < S; ++st) {
    const int L = M >> (st + 1);   // butterfly half-span
#pragma unroll
    for (int b = 0; b < M; b += 2 * L) {
#pragma unroll
      for (int j = 0; j < L; ++j) {
        const float2 u = a[b + j], v = a[b + j + L];
        a[b + j] = make_float2(u.x + v.x, u.y + v.y);
        const float dx = u.x - v.x, dy = u.y - v.y;
        if (j == 0) {
          a[b + j + L] = make_float2(dx, dy);
        } else if (2 * j == L) {   // times exp(-i pi / 2) = -i
          a[b + j + L] = make_float2(dy, -dx);
        } else {                   // times exp(-2 pi i j / (2L)) = c - i s
          const int m = j * (kTw / (2 * L));
          const float c = kTwd.c[m], s = kTwd.s[m];
          a[b + j + L] = make_float2(fmaf(dx, c, dy * s), fmaf(dy, c, -(dx * s)));
        }
      }
    }
  }
}

// Half spectrum X_0 .. X_M of the packed tube z (destroyed); put(k, re, im).
template <int N, class Put>
__device__ __forceinline__ void forward_tube(float2 (&z)[N / 2], Put&& put) {
  constexpr int M = N / 2, B = ilog2(N / 2);
  fft_dif<M>(z);
  const float2 z0 = z[0];
  put(0, z0.x + z0.y, 0.f);
  put(M, z0.x - z0.y, 0.f);
#pragma unroll
  for (int k = 1; 2 * k <= M; ++k) {
    const float2 A = z[bitrev(k, B)], Bv = z[bitrev(M - k, B)];
    const float ex = 0.5f * (A.x + Bv.x), ey = 0.5f * (A.y - Bv.y);
    const float ox = 0.5f * (A.y + Bv.y), oy = -0.5f * (A.x - Bv.x);   // (Z_k - conj Z_{M-k}) / 2i
    const int m = k * (kTw / N);
    const float c = kTwd.c[m], s = kTwd.s[m];                            // w^k = c - i s
    const float tx = fmaf(ox, c, oy * s), ty = fmaf(oy, c, -(ox * s));
    put(k, ex + tx, ey + ty);
    if (2 * k != M) put(M - k, ex - tx, ty - ey);
  }
}

// Samples of one tube from its half spectrum X[0 .. M]: x_{2n} = z[n].x,
// x_{2n+1} = z[n].y on return (z in natural order).
template <int N>
__device__ __forceinline__ void inverse_tube(const float2 (&X)[N / 2 + 1], float2 (&z)[N / 2]) {
  constexpr int M = N / 2, B = ilog2(N / 2);
  float2 a[M];
  a[0] = make_float2(0.5f * (X[0].x + X[M].x), -0.5f * (X[0].x - X[M].x));   // conj Z_0
#pragma unroll
  for (int k = 1; 2 * k <= M; ++k) {
    const float2 P = X[k], Q = X[M - k];
    const float ex = 0.5f * (P.x + Q.x), ey = 0.5f * (P.y - Q.y);
    const float dx = P.x - Q.x, dy = P.y + Q.y;                        // X_k - conj X_{M-k}
    const int m = k * (kTw / N);
    const float c = kTwd.c[m], s = kTwd.s[m];                          // conj(w^k) = c + i s
    const float ox = 0.5f * fmaf(dx, c, -(dy * s)), oy = 0.5f * fmaf(dx, s, dy * c);
    a[k] = make_float2(ex - oy, -(ey + ox));                           // conj(E + i O)
    if (2 * k != M) a[M - k] = make_float2(ex + oy, ey - ox);          // conj(conj E + i conj O)
  }
  fft_dif<M>(a);
  constexpr float inv = 1.0f / float(M);
#pragma unroll
  for (int n = 0; n < M; ++n) {
    const float2 v = a[bitrev(n, B)];
    z[n] = make_float2(v.x * inv, -v.y * inv);
  }
}

// The value of v, hidden from the optimiser so that the per-frequency output
// offsets are formed inside each tube's iteration instead of being hoisted
// out of the grid-stride loop (which would hold them all in registers).
__device__ __forceinline__ int64_t opaque(int64_t v) {
  asm volatile("" : "+l"(v));
  return v;
}

__device__ __forceinline__ void put_value(const DftGather& g, int64_t o, float re, float im) {
  if (g.out_re_lo) {
    put_split(g.out_re, g.out_re_lo, g.out_bf16 != 0, o, re);
    put_split(g.out_im, g.out_im_lo, g.out_bf16 != 0, o, im);
  } else {
    g.out_re[o] = re;
    g.out_im[o] = im;
  }
}

template <int N>
__device__ __forceinline__ void load_tube(const float* p, float s, int64_t ss, float2 (&z)[N / 2]) {
  if (p) {
#pragma unroll
    for (int n = 0; n < N / 2; ++n)
      z[n] = make_float2(s * __ldg(p + int64_t(2 * n) * ss), s * __ldg(p + int64_t(2 * n + 1) * ss));
  } else {
#pragma unroll
    for (int n = 0; n < N / 2; ++n) z[n] = make_float2(0.f, 0.f);
  }
}

// Output element (r, c) of slice k at k*out_slice + r + out_ld*c.  Threads
// walk the rows fastest, so reads and writes are coalesced along r (for a row
// gather the reads are sector-granular gathers of the picked rows).
template <int N>
__global__ void __launch_bounds__(kThreads) rfft_reg_kernel(const DftGather g) {
  const Extent ex = extent_of(g);
  const int64_t total = ex.rows_pad * ex.cols_pad;
#pragma unroll 1
  for (int64_t e = int64_t(blockIdx.x) * kThreads + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * kThreads) {
    const int64_t c = e / ex.rows_pad, r = e - c * ex.rows_pad;
    float s;
    const float* p = tube_ptr(g, ex, r, c, s);
    float2 z[N / 2];
    load_tube<N>(p, s, g.slice_stride, z);
    const int64_t o = r + g.out_ld * c;
    const int64_t os = opaque(g.out_slice);
    forward_tube<N>(z, [&](int k, float re, float im) { put_value(g, o + int64_t(k) * os, re, im); });
  }
}

// Output element (r, c) of slice k at k*out_slice + c + out_ld*r.  A warp
// covers (32 / LC) rows x LC columns, so a load reads LC runs of 32 / LC
// consecutive rows and a store writes 32 / LC runs of LC consecutive columns;
// a block's 8 warps stack along the rows.
#ifndef TP_RFFT_T_LC
#define TP_RFFT_T_LC 16
#endif
constexpr int LC = TP_RFFT_T_LC;
constexpr int TROWS = (kThreads / 32) * (32 / LC);   // rows of a block tile

template <int N>
__global__ void __launch_bounds__(kThreads) rfft_reg_t_kernel(const DftGather g) {
  const Extent ex = extent_of(g);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lr = warp * (32 / LC) + lane / LC, lc = lane % LC;
  const int64_t tr = (ex.rows_pad + TROWS - 1) / TROWS, tcn = (ex.cols_pad + LC - 1) / LC;
#pragma unroll 1
  for (int64_t t = blockIdx.x; t < tr * tcn; t += gridDim.x) {
    const int64_t tj = t / tr, ti = t - tj * tr;
    const int64_t r = ti * TROWS + lr, c = tj * LC + lc;
    if (r >= ex.rows_pad || c >= ex.cols_pad) continue;
    float s;
    const float* p = tube_ptr(g, ex, r, c, s);
    float2 z[N / 2];
    load_tube<N>(p, s, g.slice_stride, z);
    const int64_t o = c + g.out_ld * r;
    const int64_t os = opaque(g.out_slice);
    forward_tube<N>(z, [&](int k, float re, float im) { put_value(g, o + int64_t(k) * os, re, im); });
  }
}

// Staged form of the transposed transform (unit row stride, no row gather,
// N <= 64).  A block owns tiles of 8 rows x 32 columns.  The tile's samples
// are first copied to shared memory as 32-byte runs (8 consecutive rows of
// one column and one sample; by 16-byte loads staged through registers when
// the columns are 16-byte aligned (VEC), else by 4-byte asynchronous
// copies), then each thread transforms the tube (r, c)
// from shared memory and a warp stores 128-byte runs along the columns.
// Shared layout xs[t][row][col] with a row pitch of 36 floats: the copy
// (8 rows x 4 columns per warp access) and the reads (32 columns of one row)
// are both free of bank conflicts.
constexpr int SROWS = 8, SCOLS = 32, SPITCH = 36;
static_assert(SROWS * SCOLS == kThreads, "one tube per thread");

template <int N, bool VEC>
__global__ void __launch_bounds__(kThreads) rfft_reg_ts_kernel(const DftGather g) {
  extern __shared__ float xs[];   // [N][SROWS][SPITCH]
  __shared__ const float* cbase[SCOLS];
  __shared__ float cscale[SCOLS];
  const Extent ex = extent_of(g);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tr = (ex.rows_pad + SROWS - 1) / SROWS, tcn = (ex.cols_pad + SCOLS - 1) / SCOLS;
#pragma unroll 1
  for (int64_t t = blockIdx.x; t < tr * tcn; t += gridDim.x) {
    const int64_t tj = t / tr, ti = t - tj * tr;
    const int64_t r0 = ti * SROWS, c0 = tj * SCOLS;
    if (tid < SCOLS) {
      float sc;
      const float* p = tube_ptr(g, ex, 0, c0 + tid, sc);   // column base (row 0)
      cbase[tid] = p;
      cscale[tid] = sc;
    }
    __syncthreads();
    if constexpr (VEC) {
      // copy by 16-byte loads (4 rows of one column and sample; columns and
      // samples 16-byte aligned): chunk q = (sample s, column c, half hh), a
      // warp covers 16 columns x both halves of one sample (32-byte runs);
      // eight loads of a thread are issued before they are stored to shared
      // memory.  Stores: row pitch 36 puts the two halves on disjoint banks.
      constexpr int PER = N * SCOLS * 2 / kThreads;
      constexpr int BATCH = PER < 8 ? PER : 8;   // loads in flight per thread (registers)
#pragma unroll 1
      for (int m0 = 0; m0 < PER; m0 += BATCH) {
      float4 v[BATCH];
#pragma unroll
      for (int m = 0; m < BATCH; ++m) {
        const int q = tid + kThreads * (m0 + m);
        const int hh = q & 1, c = (q >> 1) & (SCOLS - 1), smp = q >> 6;
        const float* p = cbase[c];
        const int64_t r = r0 + 4 * hh;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p != nullptr) {
          const float* a = p + r + int64_t(smp) * g.slice_stride;
          if (r + 3 < ex.rows_eff) {
            x = __ldg(reinterpret_cast<const float4*>(a));
          } else {   // ragged last rows
            if (r < ex.rows_eff) x.x = __ldg(a);
            if (r + 1 < ex.rows_eff) x.y = __ldg(a + 1);
            if (r + 2 < ex.rows_eff) x.z = __ldg(a + 2);
          }
        }
        v[m] = x;
      }
#pragma unroll
      for (int m = 0; m < BATCH; ++m) {
        const int q = tid + kThreads * (m0 + m);
        const int hh = q & 1, c = (q >> 1) & (SCOLS - 1), smp = q >> 6;
        float* d = &xs[(smp * SROWS + 4 * hh) * SPITCH + c];
        d[0] = v[m].x;
        d[SPITCH] = v[m].y;
        d[2 * SPITCH] = v[m].z;
        d[3 * SPITCH] = v[m].w;
      }
      }
    } else {
    // copy: run q = (column, sample); a warp access covers 4 runs x 8 rows.
    // Asynchronous 4-byte copies keep every sample of the tile in flight;
    // padding (rows or columns past the data) is zero-filled.
      const int row = lane & 7, col = warp * 4 + (lane >> 3);
      const float* p = cbase[col];
      const bool ok = p != nullptr && r0 + row < ex.rows_eff;
      const float* src = ok ? p + (r0 + row) : g.src;
      const int64_t ss = ok ? opaque(g.slice_stride) : 0;
      const int nbytes = ok ? 4 : 0;
      uint32_t dst = uint32_t(__cvta_generic_to_shared(&xs[row * SPITCH + col]));
#pragma unroll
      for (int it = 0; it < N; ++it) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
                     "r"(nbytes)
                     : "memory");
        src += ss;
        dst += SROWS * SPITCH * sizeof(float);
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncthreads();
    {
      const int row = tid / SCOLS, col = tid % SCOLS;
      const int64_t r = r0 + row, c = c0 + col;
      const float s = cscale[col];
      float2 z[N / 2];
#pragma unroll
      for (int n = 0; n < N / 2; ++n)
        z[n] = make_float2(s * xs[(2 * n * SROWS + row) * SPITCH + col],
                           s * xs[((2 * n + 1) * SROWS + row) * SPITCH + col]);
      if (r < ex.rows_pad && c < ex.cols_pad) {
        const int64_t o = c + g.out_ld * r;
        const int64_t os = opaque(g.out_slice);
        forward_tube<N>(z, [&](int k, float re, float im) { put_value(g, o + int64_t(k) * os, re, im); });
      }
    }
    __syncthreads();   // xs and cbase are rewritten by the next tile
  }
}

template <int N>
__global__ void __launch_bounds__(kThreads) irfft_reg_kernel(const float* __restrict__ in_re,
                                                             const float* __restrict__ in_im,
                                                             int64_t rows, int64_t in_slice,
                                                             float* __restrict__ out) {
  constexpr int M = N / 2;
#pragma unroll 1
  for (int64_t r = int64_t(blockIdx.x) * kThreads + threadIdx.x; r < rows;
       r += int64_t(gridDim.x) * kThreads) {
    float2 X[M + 1];
#pragma unroll
    for (int k = 0; k <= M; ++k) {
      const float re = __ldg(in_re + int64_t(k) * in_slice + r);
      const float im = (k == 0 || k == M) ? 0.f : __ldg(in_im + int64_t(k) * in_slice + r);
      X[k] = make_float2(re, im);
    }
    float2 z[M];
    inverse_tube<N>(X, z);
#pragma unroll
    for (int n = 0; n < M; ++n) {
      out[r + rows * int64_t(2 * n)] = z[n].x;
      out[r + rows * int64_t(2 * n + 1)] = z[n].y;
    }
  }
}

// TP_RFFT_OVERSUB waves of resident blocks (the kernels stride over their
// work), or fewer blocks when the work is smaller.
#ifndef TP_RFFT_OVERSUB
#define TP_RFFT_OVERSUB 4
#endif
template <class Kernel>
unsigned grid_for(Kernel kernel, int64_t work_blocks, size_t smem = 0,
                  int oversub = TP_RFFT_OVERSUB) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t cap = int64_t(sm_count()) * per_sm * oversub;
  const int64_t b = work_blocks < cap ? work_blocks : cap;
  return unsigned(b < 1 ? 1 : b);
}

#ifndef TP_RFFT_T_STAGE
#define TP_RFFT_T_STAGE 1
#endif

template <int N>
int launch_fwd(const DftGather& g, cudaStream_t st, int oversub) {
  if constexpr (N <= 64) {
    if (TP_RFFT_T_STAGE && g.out_transposed && g.gather_dim != 1 && g.row_stride == 1) {
      const size_t smem = size_t(N) * SROWS * SPITCH * sizeof(float);
      const int64_t tiles = (g.rows + SROWS - 1) / SROWS * ((g.cols + SCOLS - 1) / SCOLS);
      // 16-byte loads when every column and sample starts 16-byte aligned
      const bool vec = N >= 4 && g.col_stride % 4 == 0 && g.slice_stride % 4 == 0 &&
                       aligned16(g.src);
      {
        KernelScope ks("rdft_t", st);
        if (vec) {
          auto k = rfft_reg_ts_kernel<N, (N >= 4)>;
          TP_SET_SMEM(k, smem);
          k<<<grid_for(k, tiles, smem, oversub), kThreads, smem, st>>>(g);
        } else {
          auto k = rfft_reg_ts_kernel<N, false>;
          TP_SET_SMEM(k, smem);
          k<<<grid_for(k, tiles, smem, oversub), kThreads, smem, st>>>(g);
        }
      }
      return launch_status("rfft_reg_ts_kernel");
    }
  }
  if (g.out_transposed) {
    const int64_t tiles = (g.rows + TROWS - 1) / TROWS * ((g.cols + LC - 1) / LC);
    {
      KernelScope ks("rdft_t", st);
      rfft_reg_t_kernel<N><<<grid_for(rfft_reg_t_kernel<N>, tiles, 0, oversub), kThreads, 0, st>>>(g);
    }
    return launch_status("rfft_reg_t_kernel");
  }
  {
    KernelScope ks("rdft", st);
    rfft_reg_kernel<N><<<grid_for(rfft_reg_kernel<N>, (g.rows * g.cols + kThreads - 1) / kThreads,
                                  0, oversub),
                         kThreads, 0, st>>>(g);
  }
  return launch_status("rfft_reg_kernel");
}

template <int N>
int launch_inv(const float* in_re, const float* in_im, int64_t rows, int64_t in_slice, float* out,
               cudaStream_t st, int oversub) {
  {
    KernelScope ks("irdft", st);
    irfft_reg_kernel<N><<<grid_for(irfft_reg_kernel<N>, (rows + kThreads - 1) / kThreads, 0,
                                   oversub),
                          kThreads, 0, st>>>(in_re, in_im, rows, in_slice, out);
  }
  return launch_status("irfft_reg_kernel");
}

}  // namespace

bool rfft_reg_supported(int64_t n3) {
  return n3 >= 2 && n3 <= kTw && (n3 & (n3 - 1)) == 0;
}

// Waves of resident blocks per launch, the autotuned choice (every tube is
// transformed alone, so the grid does not change any result).
constexpr int kOversub[4] = {1, 2, 4, 8};
constexpr int kOversubDefault = 2;   // TP_RFFT_OVERSUB = 4

int launch_rfft_reg(const DftGather& g, cudaStream_t st) {
  const auto run = [&](int c) {
    const int os = kOversub[c];
    switch (g.n3) {
      case 2: return launch_fwd<2>(g, st, os);
      case 4: return launch_fwd<4>(g, st, os);
      case 8: return launch_fwd<8>(g, st, os);
      case 16: return launch_fwd<16>(g, st, os);
      case 32: return launch_fwd<32>(g, st, os);
      case 64: return launch_fwd<64>(g, st, os);
      case 128: return launch_fwd<128>(g, st, os);
      default:
        set_error("register FFT: n3 = %lld is not a power of two in [2, 128]", (long long)g.n3);
        return int(TP_EUNSUPPORTED);
    }
  };
  if (!rfft_reg_supported(g.n3)) return run(0);
  const int64_t key[7] = {g.n3, size_class(g.rows), size_class(g.cols), g.gather_dim,
                          g.out_transposed, g.out_re_lo ? 1 : 0, g.out_bf16};
  int c = kOversubDefault;
  const int rc = autotune_pick("rfft_reg", key, 7, 4, kOversubDefault, run, st, &c);
  return rc ? rc : run(c);
}

int launch_irfft_reg(const float* in_re, const float* in_im, int64_t rows, int64_t in_slice,
                     int64_t n3, float* out, cudaStream_t st) {
  const auto run = [&](int c) {
    const int os = kOversub[c];
    switch (n3) {
      case 2: return launch_inv<2>(in_re, in_im, rows, in_slice, out, st, os);
      case 4: return launch_inv<4>(in_re, in_im, rows, in_slice, out, st, os);
      case 8: return launch_inv<8>(in_re, in_im, rows, in_slice, out, st, os);
      case 16: return launch_inv<16>(in_re, in_im, rows, in_slice, out, st, os);
      case 32: return launch_inv<32>(in_re, in_im, rows, in_slice, out, st, os);
      case 64: return launch_inv<64>(in_re, in_im, rows, in_slice, out, st, os);
      case 128: return launch_inv<128>(in_re, in_im, rows, in_slice, out, st, os);
      default:
        set_error("register FFT: n3 = %lld is not a power of two in [2, 128]", (long long)n3);
        return int(TP_EUNSUPPORTED);
    }
  };
  if (!rfft_reg_supported(n3)) return run(0);
  const int64_t key[3] = {n3, size_class(rows), size_class(in_slice)};
  int c = kOversubDefault;
  const int rc = autotune_pick("irfft_reg", key, 3, 4, kOversubDefault, run, st, &c);
  return rc ? rc : run(c);
}

}  // namespace tp
