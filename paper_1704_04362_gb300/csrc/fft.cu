// Mode-3 transform for long tubes (Section 2 "Operators", fft/ifft along the
// third dimension) by a shared-memory mixed-radix FFT, used when n3 is too
// long for the direct contraction in dft.cu.
//
// Two real tubes a, b are packed into one complex sequence z = a + i b and
// transformed together (Z = FFT(z)); their half spectra follow from
// A_k = (Z_k + conj(Z_{N-k}))/2, B_k = (Z_k - conj(Z_{N-k}))/(2i).  The FFT
// is the self-sorting Stockham formulation: for each radix R of
// N = R_1 R_2 ... R_s, butterfly j (of N/R) reads R points N/R apart, applies
// the twiddles exp(-2 pi i (j mod Ns) r / (Ns R)), does an R-point DFT and
// writes R points Ns apart at (j div Ns) Ns R + (j mod Ns); Ns grows by R
// per stage, and the result comes out in natural order.  The inverse packs
// the Hermitian-completed spectra the same way and runs the forward FFT on
// the conjugate.  One warp per packed pair; a block of four warps owns 8
// consecutive tubes so that global loads and stores are 32-byte runs.
#include "tp_internal.cuh"

namespace tp {
namespace {

constexpr int FFT_WARPS_MAX = 4;
constexpr int MAX_STAGES = 16;

struct FftPlan {
  int n;
  int nstages;
  int radix[MAX_STAGES];
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One Stockham FFT of length plan.n on buffers owned by the calling warp.
// Returns the buffer holding the result.  Radices 2, 3, 4 and 5 use fixed
// butterflies in registers; other radices (7, 11, 13) an on-the-fly R-point
// DFT read straight from shared memory.
__device__ float2* stockham(const FftPlan& plan, const float2* __restrict__ tw, float2* b0,
                            float2* b1, int lane) {
  const int N = plan.n;
  float2* src = b0;
  float2* dst = b1;
  int Ns = 1;
  for (int s = 0; s < plan.nstages; ++s) {
    const int R = plan.radix[s];
    const int NR = N / R;
    const int step_tw = N / (Ns * R);
    for (int j = lane; j < NR; j += 32) {
      const int k = j % Ns;
      const int base = (j / Ns) * Ns * R + k;
      if (R <= 5) {
        float2 v[5];
#pragma unroll
        for (int r = 0; r < 5; ++r) {
          if (r < R) {
            float2 x = src[j + r * NR];
            if (r > 0 && k > 0) x = cmul(x, tw[k * r * step_tw]);
            v[r] = x;
          }
        }
        float2 out[5];
        if (R == 2) {
          out[0] = make_float2(v[0].x + v[1].x, v[0].y + v[1].y);
          out[1] = make_float2(v[0].x - v[1].x, v[0].y - v[1].y);
        } else if (R == 4) {
          const float2 a = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
          const float2 b = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
          const float2 c = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
          const float2 d = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);   // times -i below
          out[0] = make_float2(a.x + c.x, a.y + c.y);
          out[2] = make_float2(a.x - c.x, a.y - c.y);
          out[1] = make_float2(b.x + d.y, b.y - d.x);
          out[3] = make_float2(b.x - d.y, b.y + d.x);
        } else if (R == 3) {
          // w = exp(-2 pi i / 3) = -1/2 - i sqrt(3)/2
          const float c1 = -0.5f, s1 = -0.86602540378443865f;
          const float2 t = make_float2(v[1].x + v[2].x, v[1].y + v[2].y);
          const float2 d = make_float2(v[1].x - v[2].x, v[1].y - v[2].y);
          out[0] = make_float2(v[0].x + t.x, v[0].y + t.y);
          const float2 m = make_float2(v[0].x + c1 * t.x, v[0].y + c1 * t.y);
          out[1] = make_float2(m.x - s1 * d.y, m.y + s1 * d.x);   // m + i s1 d
          out[2] = make_float2(m.x + s1 * d.y, m.y - s1 * d.x);   // m - i s1 d
        } else {   // R == 5: cos/sin of -72 and -144 degrees
          const float c1 = 0.30901699437494742f, s1 = -0.95105651629515357f;
          const float c2 = -0.80901699437494742f, s2 = -0.58778525229247313f;
          const float2 t1 = make_float2(v[1].x + v[4].x, v[1].y + v[4].y);
          const float2 d1 = make_float2(v[1].x - v[4].x, v[1].y - v[4].y);
          const float2 t2 = make_float2(v[2].x + v[3].x, v[2].y + v[3].y);
          const float2 d2 = make_float2(v[2].x - v[3].x, v[2].y - v[3].y);
          out[0] = make_float2(v[0].x + t1.x + t2.x, v[0].y + t1.y + t2.y);
          const float2 m1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
          const float2 m2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
          const float2 n1 = make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
          const float2 n2 = make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
          out[1] = make_float2(m1.x - n1.y, m1.y + n1.x);
          out[4] = make_float2(m1.x + n1.y, m1.y - n1.x);
          out[2] = make_float2(m2.x - n2.y, m2.y + n2.x);
          out[3] = make_float2(m2.x + n2.y, m2.y - n2.x);
        }
#pragma unroll
        for (int r = 0; r < 5; ++r)
          if (r < R) dst[base + r * Ns] = out[r];
      } else {
        // R-point DFT of the twiddled inputs: exp(-2 pi i r q / R) = tw[(r q mod R) N/R]
        for (int q = 0; q < R; ++q) {
          float2 acc = src[j];
          for (int r = 1; r < R; ++r) {
            float2 x = src[j + r * NR];
            if (k > 0) x = cmul(x, tw[k * r * step_tw]);
            const float2 w = tw[(r * q % R) * NR];
            acc.x += x.x * w.x - x.y * w.y;
            acc.y += x.x * w.y + x.y * w.x;
          }
          dst[base + q * Ns] = acc;
        }
      }
    }
    __syncwarp();
    float2* t = src;
    src = dst;
    dst = t;
    Ns *= R;
  }
  return src;
}

// exp(-2 pi i m / n) for m < n, by float sincospi (off the float64 pipe).
__device__ __forceinline__ void build_tw(float2* tw, int n) {
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    float s, c;
    sincospif(-float(2 * m) / float(n), &s, &c);
    tw[m] = make_float2(c, s);
  }
}

// Each warp owns two buffers of N + 2 complex values (the spare two hold the
// packed half spectra, 2h <= N + 2).
__device__ __forceinline__ float2* warp_buf(float2* fsm, int N, int w) {
  return fsm + N + size_t(2 * (N + 2)) * w;
}

// Forward: tubes r (rows of a rows x n3 array, element (r, t) at r + rows*t)
// to the half spectrum out{re,im}[k*out_slice + r].
__global__ void __launch_bounds__(FFT_WARPS_MAX * 32) fft_fwd_kernel(const float* __restrict__ X,
                                                                 int64_t rows, FftPlan plan,
                                                                 float* __restrict__ ore,
                                                                 float* __restrict__ oim,
                                                                 int64_t out_slice) {
  extern __shared__ float2 fsm[];
  const int N = plan.n;
  const int h = N / 2 + 1;
  float2* tw = fsm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int FFT_WARPS = blockDim.x >> 5;
  float2* b0 = warp_buf(fsm, N, warp);
  float2* b1 = b0 + N + 2;
  build_tw(tw, N);
  __syncthreads();
  for (int64_t r0 = int64_t(blockIdx.x) * (2 * FFT_WARPS); r0 < rows;
       r0 += int64_t(gridDim.x) * (2 * FFT_WARPS)) {
    // load all 8 tubes of the block sample by sample (32-byte runs);
    // tube c goes to the real (c even) or imaginary (c odd) part of warp c/2
    for (int e = threadIdx.x; e < 2 * FFT_WARPS * N; e += blockDim.x) {
      const int t = e / (2 * FFT_WARPS), c = e % (2 * FFT_WARPS);
      const int64_t r = r0 + c;
      const float x = r < rows ? __ldg(X + r + rows * int64_t(t)) : 0.f;
      float2* bw = warp_buf(fsm, N, c >> 1);
      if (c & 1) bw[t].y = x; else bw[t].x = x;
    }
    __syncthreads();
    const float2* Z = stockham(plan, tw, b0, b1, lane);
    const int64_t ra = r0 + 2 * warp, rb = ra + 1;
    for (int k = lane; k < h; k += 32) {
      const float2 z = Z[k];
      const float2 w = Z[(N - k) % N];
      if (ra < rows) {
        ore[int64_t(k) * out_slice + ra] = 0.5f * (z.x + w.x);
        oim[int64_t(k) * out_slice + ra] = 0.5f * (z.y - w.y);
      }
      if (rb < rows) {
        ore[int64_t(k) * out_slice + rb] = 0.5f * (z.y + w.y);
        oim[int64_t(k) * out_slice + rb] = -0.5f * (z.x - w.x);
      }
    }
    __syncthreads();
  }
}

// Inverse: half spectra in{re,im}[k*in_slice + r] to real tubes
// out[r + rows*t] (imaginary parts of the k = 0 and k = n3/2 slices ignored).
__global__ void __launch_bounds__(FFT_WARPS_MAX * 32) fft_inv_kernel(const float* __restrict__ ire,
                                                                 const float* __restrict__ iim,
                                                                 int64_t rows, int64_t in_slice,
                                                                 FftPlan plan,
                                                                 float* __restrict__ out) {
  extern __shared__ float2 fsm[];
  const int N = plan.n;
  const int h = N / 2 + 1;
  float2* tw = fsm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int FFT_WARPS = blockDim.x >> 5;
  float2* b0 = warp_buf(fsm, N, warp);
  float2* b1 = b0 + N + 2;
  build_tw(tw, N);
  __syncthreads();
  const float inv = 1.0f / float(N);
  for (int64_t r0 = int64_t(blockIdx.x) * (2 * FFT_WARPS); r0 < rows;
       r0 += int64_t(gridDim.x) * (2 * FFT_WARPS)) {
    // stage the half spectra: tube c into the second buffer of warp c/2,
    // A (c even) at [0, h), B (c odd) at [h, 2h)
    for (int e = threadIdx.x; e < 2 * FFT_WARPS * h; e += blockDim.x) {
      const int k = e / (2 * FFT_WARPS), c = e % (2 * FFT_WARPS);
      const int64_t r = r0 + c;
      float2 v = make_float2(0.f, 0.f);
      if (r < rows) {
        v.x = __ldg(ire + int64_t(k) * in_slice + r);
        v.y = (k == 0 || 2 * k == N) ? 0.f : __ldg(iim + int64_t(k) * in_slice + r);
      }
      float2* bw = warp_buf(fsm, N, c >> 1) + N + 2;
      bw[(c & 1) * h + k] = v;
    }
    __syncthreads();
    // conj(Z), Z_k = A_k + i B_k over the whole circle (A_{N-k} = conj A_k)
    for (int k = lane; k < N; k += 32) {
      const bool lo = k < h;
      const int kk = lo ? k : N - k;
      float2 A = b1[kk], B = b1[h + kk];
      if (!lo) { A.y = -A.y; B.y = -B.y; }
      b0[k] = make_float2(A.x - B.y, -(A.y + B.x));
    }
    __syncwarp();
    stockham(plan, tw, b0, b1, lane);
    __syncthreads();
    // ifft(Z) = conj(FFT(conj Z)) / N: tube a = Re, tube b = -Im
    for (int e = threadIdx.x; e < 2 * FFT_WARPS * N; e += blockDim.x) {
      const int t = e / (2 * FFT_WARPS), c = e % (2 * FFT_WARPS);
      const int64_t r = r0 + c;
      if (r >= rows) continue;
      float2* bw = warp_buf(fsm, N, c >> 1);
      const float2* res = (plan.nstages & 1) ? bw + N + 2 : bw;
      const float2 v = res[t];
      out[r + rows * int64_t(t)] = (c & 1) ? -v.y * inv : v.x * inv;
    }
    __syncthreads();
  }
}

bool make_plan(int64_t n, FftPlan* p) {
  if (n < 2 || n > 65536) return false;
  p->n = int(n);
  p->nstages = 0;
  int64_t m = n;
  const int prefs[] = {4, 2, 3, 5, 7, 11, 13};
  for (int r : prefs) {
    while (m % r == 0) {
      if (p->nstages >= MAX_STAGES) return false;
      p->radix[p->nstages++] = r;
      m /= r;
    }
  }
  return m == 1;
}

size_t fft_smem(int64_t n, int warps) { return size_t(n + 2 * warps * (n + 2)) * sizeof(float2); }
constexpr size_t kFftSmemCap = 200 * 1024;
int fft_warps(int64_t n) {
  for (int w = FFT_WARPS_MAX; w >= 1; w >>= 1)
    if (fft_smem(n, w) <= kFftSmemCap) return w;
  return 0;
}

}  // namespace

bool fft_supported(int64_t n3) {
  FftPlan p;
  return make_plan(n3, &p) && fft_warps(n3) > 0;
}

int launch_fft_fwd(const float* X, int64_t rows, int64_t n3, float* ore, float* oim,
                   int64_t out_slice, cudaStream_t st) {
  FftPlan plan;
  const int nw = fft_warps(n3);
  if (!make_plan(n3, &plan) || nw == 0) {
    set_error("fft: n3 = %lld is not a product of radices 2,3,5,7,11,13 that fits in shared memory",
              (long long)n3);
    return TP_EUNSUPPORTED;
  }
  if (rows == 0) return TP_OK;
  const size_t smem = fft_smem(n3, nw);
  TP_SET_SMEM(fft_fwd_kernel, smem);
  int64_t blocks = (rows + 2 * nw - 1) / (2 * nw);
  if (blocks > int64_t(sm_count()) * 64) blocks = int64_t(sm_count()) * 64;
  {
    KernelScope ks("fft_fwd", st);
    fft_fwd_kernel<<<unsigned(blocks), nw * 32, smem, st>>>(X, rows, plan, ore, oim, out_slice);
  }
  return launch_status("fft_fwd_kernel");
}

int launch_fft_inv(const float* ire, const float* iim, int64_t rows, int64_t in_slice, int64_t n3,
                   float* out, cudaStream_t st) {
  FftPlan plan;
  const int nw = fft_warps(n3);
  if (!make_plan(n3, &plan) || nw == 0) {
    set_error("fft: n3 = %lld is not a product of radices 2,3,5,7,11,13 that fits in shared memory",
              (long long)n3);
    return TP_EUNSUPPORTED;
  }
  if (rows == 0) return TP_OK;
  const size_t smem = fft_smem(n3, nw);
  TP_SET_SMEM(fft_inv_kernel, smem);
  int64_t blocks = (rows + 2 * nw - 1) / (2 * nw);
  if (blocks > int64_t(sm_count()) * 64) blocks = int64_t(sm_count()) * 64;
  {
    KernelScope ks("fft_inv", st);
    fft_inv_kernel<<<unsigned(blocks), nw * 32, smem, st>>>(ire, iim, rows, in_slice, plan, out);
  }
  return launch_status("fft_inv_kernel");
}

}  // namespace tp
