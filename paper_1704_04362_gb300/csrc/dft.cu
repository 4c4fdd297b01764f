// Mode-3 DFT of real tubes kept to the half spectrum, and its inverse
// (Section 2, "Operators": fft(X,[],3) / ifft(X,[],3); Algorithm 1 steps 2-3
// and the final inverse).
//
// Both directions are small dense contractions per tube, computed as
// register-blocked SIMT products.  The t <-> n3 - t symmetry halves them:
// with e_t = x_t + x_{n3-t} and o_t = x_t - x_{n3-t} (t = 1 .. n3/2; e_0 = x_0
// and, for even n3, e_{n3/2} = x_{n3/2}, o = 0 there),
//     Re X_k = sum_{t <= n3/2} e_t cos(2 pi k t / n3),
//     Im X_k = -sum_{t <= n3/2} o_t sin(2 pi k t / n3);
// and for the inverse, with P_t = sum_k w_k Re X_k cos, Q_t = sum_k w_k Im X_k sin
// (w_k = 1/n3 at k = 0 and k = n3/2, else 2/n3), x_t = P_t - Q_t and
// x_{n3-t} = P_t + Q_t.  Each thread owns TPT tubes and KC frequencies (or
// output times) per chunk; the KC columns of the transform matrix a chunk
// needs are built once per block in shared memory from the n3-entry twiddle
// table exp(-2 pi i m / n3), m = k t mod n3.  KC is chosen per call to
// minimise padding.  The (Re, Im) and (P, Q) accumulator pairs are updated
// with Blackwell's packed two-lane float32 FMA.
#include "dft_common.cuh"

namespace tp {
namespace {
using namespace dftc;

#ifndef TP_DFT_TPT
#define TP_DFT_TPT 2
#endif
constexpr int TPT = TP_DFT_TPT;  // tubes per thread
constexpr int RB = 128;          // threads per block
constexpr int TU = 8;            // samples (forward) or frequencies (inverse) loaded ahead
constexpr int STAGE_BYTES_MAX = 64 * 1024;

// (cos, sin)(2 pi m / n3) for m < n3.  float sincospi (about 1 ulp; exact at
// quarter turns, m/n3 in {0, 1/4, 1/2, 3/4}) keeps the tables off the slow
// float64 pipe.  The argument 2m/n3 is formed exactly enough: 2m and n3 are
// small integers, and the quotient's rounding (2^-24 relative) moves the angle
// by less than the float result's own rounding.
__device__ __forceinline__ void build_twiddles(float2* tw, int n3) {
  for (int m = threadIdx.x; m < n3; m += blockDim.x) {
    float s, c;
    sincospif(float(2 * m) / float(n3), &s, &c);
    tw[m] = make_float2(c, s);
  }
}

// Folded pair (e_t, o_t) of one tube; t <= n3/2.
__device__ __forceinline__ void fold(float x0, float x1, int t, int n3, float& e, float& o) {
  if (t == 0 || 2 * t == n3) {
    e = x0;
    o = 0.f;
  } else {
    e = x0 + x1;
    o = x0 - x1;
  }
}

// Wc[t*KC + q] = (cos, sin)(2 pi (k0+q) t / n3) for t <= nh, zero above.
template <int KC>
__device__ __forceinline__ void build_fwd_cols(float2* Wc, const float2* tw, int n3, int nh,
                                               int nhp, int k0) {
  for (int e = threadIdx.x; e < nhp * KC; e += blockDim.x) {
    const int t = e / KC, q = e - t * KC;
    Wc[e] = t <= nh ? tw[int((int64_t(k0 + q) * t) % n3)] : make_float2(0.f, 0.f);
  }
}

template <int KC>
__global__ void __launch_bounds__(RB) rdft_kernel(DftGather g, int stage) {
  extern __shared__ float2 sm2[];
  const int n3 = int(g.n3);
  const int h = n3 / 2 + 1, nh = n3 / 2;
  const int nhp = (nh + 1 + TU - 1) / TU * TU;
  float2* tw = sm2;
  float2* Wc = sm2 + n3;
  float* xs = reinterpret_cast<float*>(Wc + nhp * KC);   // staging [n3][RB*TPT] when stage
  build_twiddles(tw, n3);
  const Extent ex = extent_of(g);
  const int64_t base = int64_t(blockIdx.x) * (RB * TPT);
  if (base >= ex.rows_pad) return;   // uniform over the block
  const int tid = threadIdx.x;

  for (int64_t c = blockIdx.y; c < ex.cols_pad; c += gridDim.y) {
    const float* p[TPT];
    float s[TPT];
    bool act[TPT];
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
      const int64_t r = base + j * RB + tid;
      act[j] = r < ex.rows_pad;
      p[j] = act[j] ? tube_ptr(g, ex, r, c, s[j]) : nullptr;
    }
    if (stage) {
      // every sample of this thread's tubes, read once (all loads in flight)
      for (int t = 0; t < n3; ++t)
#pragma unroll
        for (int j = 0; j < TPT; ++j)
          xs[t * (RB * TPT) + j * RB + tid] =
              p[j] ? s[j] * __ldg(p[j] + int64_t(t) * g.slice_stride) : 0.f;
    }
    for (int k0 = 0; k0 < h; k0 += KC) {
      __syncthreads();
      build_fwd_cols<KC>(Wc, tw, n3, nh, nhp, k0);
      __syncthreads();
      float2 acc[TPT][KC];   // (Re, Im), updated by packed two-lane FMAs
#pragma unroll
      for (int j = 0; j < TPT; ++j)
#pragma unroll
        for (int q = 0; q < KC; ++q) acc[j][q] = make_float2(0.f, 0.f);
      for (int t0 = 0; t0 <= nh; t0 += TU) {
        float ev[TPT][TU], ov[TPT][TU];
#pragma unroll
        for (int u = 0; u < TU; ++u)
#pragma unroll
          for (int j = 0; j < TPT; ++j) {
            const int t = t0 + u;
            float x0 = 0.f, x1 = 0.f;
            if (t <= nh) {
              if (stage) {
                x0 = xs[t * (RB * TPT) + j * RB + tid];
                x1 = xs[((n3 - t) % n3) * (RB * TPT) + j * RB + tid];
              } else if (p[j]) {
                x0 = s[j] * __ldg(p[j] + int64_t(t) * g.slice_stride);
                if (t > 0 && 2 * t != n3)
                  x1 = s[j] * __ldg(p[j] + int64_t(n3 - t) * g.slice_stride);
              }
            }
            fold(x0, x1, t, n3, ev[j][u], ov[j][u]);
          }
#pragma unroll
        for (int u = 0; u < TU; ++u)
#pragma unroll
          for (int q = 0; q < KC; ++q) {
            const float2 w = Wc[(t0 + u) * KC + q];   // zero rows past nh
#pragma unroll
            for (int j = 0; j < TPT; ++j)
              acc[j][q] = __ffma2_rn(make_float2(ev[j][u], -ov[j][u]), w, acc[j][q]);
          }
      }
#pragma unroll
      for (int j = 0; j < TPT; ++j) {
        if (!act[j]) continue;
        const int64_t o = base + j * RB + tid + g.out_ld * c;
#pragma unroll
        for (int q = 0; q < KC; ++q) {
          if (k0 + q < h) {
            const int64_t oo = o + int64_t(k0 + q) * g.out_slice;
            const float ar = acc[j][q].x, ai = acc[j][q].y;
            if (g.out_re_lo) {
              put_split(g.out_re, g.out_re_lo, g.out_bf16 != 0, oo, ar);
              put_split(g.out_im, g.out_im_lo, g.out_bf16 != 0, oo, ai);
            } else {
              g.out_re[oo] = ar;
              g.out_im[oo] = ai;
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
// along the column index.  This kernel runs the plain (unfolded) contraction:
// the folded form's extra live registers cost more occupancy than the
// arithmetic it saves here.
constexpr int TR = 32, TCOL = 8;
constexpr int TPTT = TCOL / (RB / TR);   // columns per thread in the transposed kernel (2)

template <int KC>
__global__ void __launch_bounds__(RB) rdft_t_kernel(DftGather g) {
  extern __shared__ float2 sm2[];
  const int n3 = int(g.n3);
  const int h = n3 / 2 + 1;
  const int n3p = (n3 + TU - 1) / TU * TU;
  float2* tw = sm2;
  float2* Wc = sm2 + n3;   // Wc[t*KC + q] = tw[(k0+q) t mod n3], zero for t >= n3
  float* stg = reinterpret_cast<float*>(Wc + n3p * KC);   // [KC][TR][TCOL + 1]
  build_twiddles(tw, n3);
  const Extent ex = extent_of(g);
  const int64_t r0 = int64_t(blockIdx.x) * TR;
  if (r0 >= ex.rows_pad) return;   // uniform over the block
  const int tid = threadIdx.x;
  const int lr = tid % TR, lc = tid / TR;   // this thread: row lr, columns lc and lc + 4
  const int64_t r = r0 + lr;

  for (int64_t c0 = int64_t(blockIdx.y) * TCOL; c0 < ex.cols_pad; c0 += int64_t(gridDim.y) * TCOL) {
    const float* p[TPTT];
    float s[TPTT];
#pragma unroll
    for (int j = 0; j < TPTT; ++j) p[j] = tube_ptr(g, ex, r, c0 + lc + 4 * j, s[j]);
    for (int k0 = 0; k0 < h; k0 += KC) {
      __syncthreads();
      for (int e = tid; e < n3p * KC; e += RB) {
        const int t = e / KC, q = e - t * KC;
        Wc[e] = t < n3 ? tw[int((int64_t(k0 + q) * t) % n3)] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      float2 acc[TPTT][KC];   // (Re, Im), updated by packed two-lane FMAs
#pragma unroll
      for (int j = 0; j < TPTT; ++j)
#pragma unroll
        for (int q = 0; q < KC; ++q) acc[j][q] = make_float2(0.f, 0.f);
      for (int t0 = 0; t0 < n3; t0 += TU) {
        float x[TPTT][TU];
#pragma unroll
        for (int u = 0; u < TU; ++u)
#pragma unroll
          for (int j = 0; j < TPTT; ++j)
            x[j][u] = (p[j] && t0 + u < n3) ? s[j] * __ldg(p[j] + int64_t(t0 + u) * g.slice_stride)
                                            : 0.f;
#pragma unroll
        for (int u = 0; u < TU; ++u)
#pragma unroll
          for (int q = 0; q < KC; ++q) {
            const float2 w = Wc[(t0 + u) * KC + q];
#pragma unroll
            for (int j = 0; j < TPTT; ++j)
              acc[j][q] = __ffma2_rn(make_float2(x[j][u], -x[j][u]), w, acc[j][q]);
          }
      }
      // planes: 0 re (hi), 1 im (hi), 2 re lo, 3 im lo
      const int nplanes = g.out_re_lo ? 4 : 2;
      for (int pl = 0; pl < nplanes; ++pl) {
        __syncthreads();   // staging buffer free
#pragma unroll
        for (int j = 0; j < TPTT; ++j)
#pragma unroll
          for (int q = 0; q < KC; ++q) {
            const float v = (pl & 1) ? acc[j][q].y : acc[j][q].x;
            float o;
            if (!g.out_re_lo) {
              o = v;
            } else {   // hi, or lo = v - hi rounded to tf32 (a bf16 lo is rounded when stored)
              const float hi = g.out_bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : tf32_rna(v);
              o = pl < 2 ? hi : (g.out_bf16 ? v - hi : tf32_rna(v - hi));
            }
            stg[(q * TR + lr) * (TCOL + 1) + lc + 4 * j] = o;
          }
        __syncthreads();
        float* dst = pl == 0 ? g.out_re : pl == 1 ? g.out_im : pl == 2 ? g.out_re_lo : g.out_im_lo;
        // thread -> (column wc, row wr); 16 rows per pass, two passes
        const int wc = tid % TCOL, wr = tid / TCOL;
        const int64_t c = c0 + wc;
        if (c < ex.cols_pad) {
          for (int q = 0; q < KC && k0 + q < h; ++q) {
#pragma unroll
            for (int pass = 0; pass < TR / (RB / TCOL); ++pass) {
              const int rr = wr + pass * (RB / TCOL);
              const int64_t rg = r0 + rr;
              if (rg < ex.rows_pad) {
                const int64_t o = int64_t(k0 + q) * g.out_slice + c + g.out_ld * rg;
                const float v = stg[(q * TR + rr) * (TCOL + 1) + wc];
                if (g.out_bf16 && g.out_re_lo)
                  reinterpret_cast<__nv_bfloat16*>(dst)[o] = __float2bfloat16_rn(v);
                else
                  dst[o] = v;
              }
            }
          }
        }
      }
    }
  }
}

// Inverse: x_t = P_t - Q_t, x_{n3-t} = P_t + Q_t over output-time chunks t <= n3/2.
template <int KC>
__global__ void __launch_bounds__(RB) irdft_kernel(const float* __restrict__ in_re,
                                                   const float* __restrict__ in_im, int64_t rows,
                                                   int64_t in_slice, int n3,
                                                   float* __restrict__ out) {
  extern __shared__ float2 sm2[];
  const int h = n3 / 2 + 1, nh = n3 / 2;
  const int hp = (h + TU - 1) / TU * TU;
  float2* tw = sm2;
  float2* Vc = sm2 + n3;   // Vc[k*KC + q] = (w_k/n3) tw[k*(t0+q) mod n3], zero past h or nh
  build_twiddles(tw, n3);
  const int tid = threadIdx.x;
  const float inv = 1.0f / float(n3);
  for (int64_t base = int64_t(blockIdx.x) * (RB * TPT); base < rows;
       base += int64_t(gridDim.x) * (RB * TPT)) {
    int64_t r[TPT];
#pragma unroll
    for (int j = 0; j < TPT; ++j) r[j] = base + j * RB + tid;
    for (int t0 = 0; t0 <= nh; t0 += KC) {
      __syncthreads();
      for (int e = tid; e < hp * KC; e += RB) {
        const int k = e / KC, q = e - k * KC;
        const int t = t0 + q;
        if (k < h && t <= nh) {
          const float wk = (k == 0 || 2 * k == n3) ? inv : 2.0f * inv;
          const float2 w = tw[int((int64_t(k) * t) % n3)];
          Vc[e] = make_float2(wk * w.x, wk * w.y);
        } else {
          Vc[e] = make_float2(0.f, 0.f);
        }
      }
      __syncthreads();
      float2 PQ[TPT][KC];   // (P, Q), updated by packed two-lane FMAs
#pragma unroll
      for (int j = 0; j < TPT; ++j)
#pragma unroll
        for (int q = 0; q < KC; ++q) PQ[j][q] = make_float2(0.f, 0.f);
      for (int k0 = 0; k0 < h; k0 += TU) {
        float re[TPT][TU], im[TPT][TU];
#pragma unroll
        for (int u = 0; u < TU; ++u)
#pragma unroll
          for (int j = 0; j < TPT; ++j) {
            const int k = k0 + u;
            const bool ok = r[j] < rows && k < h;
            re[j][u] = ok ? __ldg(in_re + int64_t(k) * in_slice + r[j]) : 0.f;
            // the imaginary parts of the real slices are ignored
            im[j][u] = (ok && k > 0 && 2 * k != n3) ? __ldg(in_im + int64_t(k) * in_slice + r[j])
                                                    : 0.f;
          }
#pragma unroll
        for (int u = 0; u < TU; ++u)
#pragma unroll
          for (int q = 0; q < KC; ++q) {
            const float2 v = Vc[(k0 + u) * KC + q];
#pragma unroll
            for (int j = 0; j < TPT; ++j)
              PQ[j][q] = __ffma2_rn(make_float2(re[j][u], im[j][u]), v, PQ[j][q]);
          }
      }
#pragma unroll
      for (int j = 0; j < TPT; ++j) {
        if (r[j] >= rows) continue;
#pragma unroll
        for (int q = 0; q < KC; ++q) {
          const int t = t0 + q;
          if (t <= nh) {
            out[r[j] + rows * int64_t(t)] = PQ[j][q].x - PQ[j][q].y;
            if (t > 0 && n3 - t > nh) out[r[j] + rows * int64_t(n3 - t)] = PQ[j][q].x + PQ[j][q].y;
          }
        }
      }
    }
  }
}

// Chunk size among {16, 12, 8} that pads n the least (ties: larger).
int pick_kc(int64_t n) {
  const int cands[3] = {16, 12, 8};
  int best = 16;
  int64_t best_cost = -1;
  for (int kc : cands) {
    const int64_t cost = (n + kc - 1) / kc * kc;
    if (best_cost < 0 || cost < best_cost) {
      best = kc;
      best_cost = cost;
    }
  }
  return best;
}

template <int KC>
int launch_rdft_kc(const DftGather& g, cudaStream_t st) {
  const int64_t nh = g.n3 / 2;
  const int64_t nhp = (nh + 1 + TU - 1) / TU * TU;
  if (g.out_transposed) {
    const int64_t n3p = (g.n3 + TU - 1) / TU * TU;
    const size_t smem = size_t(g.n3 + n3p * KC) * sizeof(float2) +
                        size_t(KC) * TR * (TCOL + 1) * sizeof(float);
    TP_SET_SMEM(rdft_t_kernel<KC>, smem);
    const int64_t bx = (g.rows + TR - 1) / TR;
    if (bx > 0x7fffffff) { set_error("rdft: too many rows"); return TP_EINVAL; }
    // the column tiles are walked grid-stride: with all rows live (no row
    // gather) about 16 blocks per SM suffice, and a column gather's capacity
    // can far exceed the picked count
    int64_t by = (g.cols + TCOL - 1) / TCOL;
    const int64_t by_cap = bx >= int64_t(sm_count()) * 16 ? 1 : int64_t(sm_count()) * 16 / bx;
    if (g.gather_dim != 1 && by > by_cap) by = by_cap;
    if (by > 65535) by = 65535;
    {
      KernelScope ks("rdft_t", st);
      rdft_t_kernel<KC><<<dim3(unsigned(bx), unsigned(by)), RB, smem, st>>>(g);
    }
    return launch_status("rdft_t_kernel");
  }
  // stage the scattered row gathers so that each sample is read once
  const size_t stage_bytes = size_t(g.n3) * RB * TPT * sizeof(float);
  const int stage = (g.gather_dim == 1 && stage_bytes <= size_t(STAGE_BYTES_MAX)) ? 1 : 0;
  const size_t smem = size_t(g.n3 + nhp * KC) * sizeof(float2) + (stage ? stage_bytes : 0);
  TP_SET_SMEM(rdft_kernel<KC>, smem);
  const int64_t bx = (g.rows + RB * TPT - 1) / (RB * TPT);
  if (bx > 0x7fffffff) { set_error("rdft: too many rows"); return TP_EINVAL; }
  int64_t by = g.cols < 65535 ? g.cols : 65535;   // columns walked grid-stride
  const int64_t by_cap = bx >= int64_t(sm_count()) * 16 ? 1 : int64_t(sm_count()) * 16 / bx;
  if (g.gather_dim == 2 && by > by_cap) by = by_cap;   // see the transposed form
  {
    KernelScope ks("rdft", st);
    rdft_kernel<KC><<<dim3(unsigned(bx), unsigned(by)), RB, smem, st>>>(g, stage);
  }
  return launch_status("rdft_kernel");
}

template <int KC>
int launch_irdft_kc(const float* in_re, const float* in_im, int64_t rows, int64_t in_slice,
                    int64_t n3, float* out, cudaStream_t st) {
  const int64_t h = n3 / 2 + 1;
  const int64_t hp = (h + TU - 1) / TU * TU;
  const size_t smem = size_t(n3 + hp * KC) * sizeof(float2);
  TP_SET_SMEM(irdft_kernel<KC>, smem);
  int64_t blocks = (rows + RB * TPT - 1) / (RB * TPT);
  if (blocks > int64_t(sm_count()) * 64) blocks = int64_t(sm_count()) * 64;
  {
    KernelScope ks("irdft", st);
    irdft_kernel<KC><<<unsigned(blocks), RB, smem, st>>>(in_re, in_im, rows, in_slice, int(n3), out);
  }
  return launch_status("irdft_kernel");
}

}  // namespace

bool fft_supported(int64_t n3);
bool rfft_reg_supported(int64_t n3);
int launch_rfft_reg(const DftGather& g, cudaStream_t st);
int launch_irfft_reg(const float* in_re, const float* in_im, int64_t rows, int64_t in_slice,
                     int64_t n3, float* out, cudaStream_t st);
int launch_fft_fwd(const float* X, int64_t rows, int64_t n3, float* ore, float* oim,
                   int64_t out_slice, cudaStream_t st);
int launch_fft_inv(const float* ire, const float* iim, int64_t rows, int64_t in_slice, int64_t n3,
                   float* out, cudaStream_t st);

// Tubes longer than this go through the shared-memory FFT when their length
// factors into small radices and no gather or split output is asked for.
#ifndef TP_FFT_THRESHOLD
#define TP_FFT_THRESHOLD 256
#endif
constexpr int64_t kFftThreshold = TP_FFT_THRESHOLD;
// Power-of-two tubes up to 128 go through the register FFT (rfft_reg.cu);
// building with -DTP_REG_FFT=0 keeps them on the direct contraction.
#ifndef TP_REG_FFT
#define TP_REG_FFT 1
#endif
constexpr bool kRegFft = TP_REG_FFT != 0;

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
  if (kRegFft && rfft_reg_supported(g.n3)) return launch_rfft_reg(g, st);
  // tile width KC among {8, 12, 16} (each frequency sums its samples in the
  // same order whatever the width): autotuned, default the least padding
  const auto run = [&](int c) {
    switch (c) {
      case 0: return launch_rdft_kc<8>(g, st);
      case 1: return launch_rdft_kc<12>(g, st);
      default: return launch_rdft_kc<16>(g, st);
    }
  };
  const int kc = pick_kc(g.n3 / 2 + 1);
  const int64_t key[7] = {g.n3, size_class(g.rows), size_class(g.cols), g.gather_dim,
                          g.out_transposed, g.out_re_lo ? 1 : 0, g.out_bf16};
  int c = 0;
  const int rc = autotune_pick("rdft", key, 7, 3, kc == 8 ? 0 : kc == 12 ? 1 : 2, run, st, &c);
  return rc ? rc : run(c);
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
  if (kRegFft && rfft_reg_supported(n3))
    return launch_irfft_reg(in_re, in_im, rows, in_slice, n3, out, st);
  const auto run = [&](int c) {
    switch (c) {
      case 0: return launch_irdft_kc<8>(in_re, in_im, rows, in_slice, n3, out, st);
      case 1: return launch_irdft_kc<12>(in_re, in_im, rows, in_slice, n3, out, st);
      default: return launch_irdft_kc<16>(in_re, in_im, rows, in_slice, n3, out, st);
    }
  };
  const int kc = pick_kc(n3 / 2 + 1);
  const int64_t key[2] = {n3, size_class(rows)};
  int c = 0;
  const int rc = autotune_pick("irdft", key, 2, 3, kc == 8 ? 0 : kc == 12 ? 1 : 2, run, st, &c);
  return rc ? rc : run(c);
}

}  // namespace tp
