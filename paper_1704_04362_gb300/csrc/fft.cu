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
// the conjugate.
//
// A block of 512 (forward) or 1024 (inverse) threads owns 2P consecutive tubes (P packed sequences,
// P = 4 for n3 up to about 3000): the loads and stores move 8P-byte runs of
// consecutive tubes, and every stage spreads the P N / R butterflies of all
// sequences over all threads (out of place between two shared buffers, one
// barrier per stage), so that a block keeps 16 or 32 warps busy instead of
// one warp per sequence.  The grid is persistent over groups of tubes; the
// forward transform loads the next group into registers (32 values a
// thread) before transforming the current one, which hides the loads when
// a long tube leaves room for one block per SM.
#include "tp_internal.cuh"

namespace tp {
namespace {

constexpr int FFT_THREADS = 512;        // forward: room for the prefetch registers
constexpr int FFT_INV_THREADS = 1024;
constexpr int FFT_P_MAX = 4;
constexpr int FFT_PF = 32;   // prefetched input values per thread
constexpr int MAX_STAGES = 16;

struct FftPlan {
  int n;
  int nstages;
  int radix[MAX_STAGES];
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One Stockham stage of radix R for the P sequences (length N, stride N)
// in src, written to dst.  Radices 2, 3, 4 and 5 use fixed butterflies in
// registers; other radices (7, 11, 13) an on-the-fly R-point DFT read
// straight from shared memory.
__device__ void stockham_stage(const float2* __restrict__ src, float2* __restrict__ dst, int P,
                               int N, int R, int Ns, const float2* __restrict__ tw) {
  const int NR = N / R;
  const int B = P * NR;
  const int step_tw = N / (Ns * R);
  for (int bfly = threadIdx.x; bfly < B; bfly += blockDim.x) {
    const int sq = bfly / NR;
    const int j = bfly - sq * NR;
    const float2* in = src + sq * N;
    float2* out_p = dst + sq * N;
    const int k = j % Ns;
    const int base = (j / Ns) * Ns * R + k;
    if (R <= 5) {
      float2 v[5];
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        if (r < R) {
          float2 x = in[j + r * NR];
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
        if (r < R) out_p[base + r * Ns] = out[r];
    } else {
      // R-point DFT of the twiddled inputs: exp(-2 pi i r q / R) = tw[(r q mod R) N/R]
      for (int q = 0; q < R; ++q) {
        float2 acc = in[j];
        for (int r = 1; r < R; ++r) {
          float2 x = in[j + r * NR];
          if (k > 0) x = cmul(x, tw[k * r * step_tw]);
          const float2 w = tw[(r * q % R) * NR];
          acc.x += x.x * w.x - x.y * w.y;
          acc.y += x.x * w.y + x.y * w.x;
        }
        out_p[base + q * Ns] = acc;
      }
    }
  }
}

// The whole FFT of the P sequences in b0 (b1 is scratch); returns the
// buffer holding the result.  Ends with a block barrier.
__device__ float2* stockham_all(const FftPlan& plan, const float2* tw, float2* b0, float2* b1,
                                int P) {
  float2* src = b0;
  float2* dst = b1;
  int Ns = 1;
  for (int s = 0; s < plan.nstages; ++s) {
    const int R = plan.radix[s];
    stockham_stage(src, dst, P, plan.n, R, Ns, tw);
    __syncthreads();
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

// Forward: tubes r (rows of a rows x n3 array, element (r, t) at r + rows*t)
// to the half spectrum out{re,im}[k*out_slice + r].
__global__ void __launch_bounds__(FFT_THREADS) fft_fwd_kernel(const float* __restrict__ X,
                                                              int64_t rows, FftPlan plan, int P,
                                                              float* __restrict__ ore,
                                                              float* __restrict__ oim,
                                                              int64_t out_slice) {
  extern __shared__ float2 fsm[];
  const int N = plan.n;
  const int h = N / 2 + 1;
  const int G = 2 * P;   // tubes per group
  float2* tw = fsm;
  float2* b0 = fsm + N;
  float2* b1 = b0 + P * N;
  build_tw(tw, N);
  __syncthreads();
  // a group that fits FFT_PF values per thread is loaded into registers one
  // group ahead (issued before the current group's transform, so that the
  // loads' latency hides behind it: one block per SM when n3 is long)
  const bool pf = G * N <= FFT_PF * FFT_THREADS;
  const int64_t gstride = int64_t(gridDim.x) * G;
  float nxt[FFT_PF];
  auto fetch = [&](int64_t rg) {
#pragma unroll
    for (int u = 0; u < FFT_PF; ++u) {
      const int e = int(threadIdx.x) + u * FFT_THREADS;
      const int t = e / G, c = e - t * G;
      const int64_t r = rg + c;
      nxt[u] = (e < G * N && r < rows) ? __ldg(X + r + rows * int64_t(t)) : 0.f;
    }
  };
  if (pf && int64_t(blockIdx.x) * G < rows) fetch(int64_t(blockIdx.x) * G);
  for (int64_t r0 = int64_t(blockIdx.x) * G; r0 < rows; r0 += gstride) {
    // tube c of the group goes to the real (c even) or imaginary (c odd)
    // part of sequence c/2; consecutive threads read consecutive tubes
    if (pf) {
#pragma unroll
      for (int u = 0; u < FFT_PF; ++u) {
        const int e = int(threadIdx.x) + u * FFT_THREADS;
        if (e < G * N) {
          const int t = e / G, c = e - t * G;
          reinterpret_cast<float*>(b0 + (c >> 1) * N + t)[c & 1] = nxt[u];
        }
      }
      __syncthreads();
      if (r0 + gstride < rows) fetch(r0 + gstride);
    } else {
      for (int e = threadIdx.x; e < G * N; e += blockDim.x) {
        const int t = e / G, c = e - t * G;
        const int64_t r = r0 + c;
        const float x = r < rows ? __ldg(X + r + rows * int64_t(t)) : 0.f;
        reinterpret_cast<float*>(b0 + (c >> 1) * N + t)[c & 1] = x;
      }
      __syncthreads();
    }
    const float2* Z = stockham_all(plan, tw, b0, b1, P);
    for (int e = threadIdx.x; e < G * h; e += blockDim.x) {
      const int k = e / G, c = e - k * G;
      const int64_t r = r0 + c;
      if (r >= rows) continue;
      const float2* Zs = Z + (c >> 1) * N;
      const float2 z = Zs[k];
      const float2 w = Zs[(N - k) % N];
      float re, im;
      if (c & 1) {
        re = 0.5f * (z.y + w.y);
        im = -0.5f * (z.x - w.x);
      } else {
        re = 0.5f * (z.x + w.x);
        im = 0.5f * (z.y - w.y);
      }
      ore[int64_t(k) * out_slice + r] = re;
      oim[int64_t(k) * out_slice + r] = im;
    }
    __syncthreads();
  }
}

// Inverse: half spectra in{re,im}[k*in_slice + r] to real tubes
// out[r + rows*t] (imaginary parts of the k = 0 and k = n3/2 slices ignored).
__global__ void __launch_bounds__(FFT_INV_THREADS) fft_inv_kernel(const float* __restrict__ ire,
                                                              const float* __restrict__ iim,
                                                              int64_t rows, int64_t in_slice,
                                                              FftPlan plan, int P,
                                                              float* __restrict__ out) {
  extern __shared__ float2 fsm[];
  const int N = plan.n;
  const int h = N / 2 + 1;
  const int G = 2 * P;
  float2* tw = fsm;
  float2* b0 = fsm + N;
  float2* b1 = b0 + P * N;
  build_tw(tw, N);
  __syncthreads();
  const float inv = 1.0f / float(N);
  for (int64_t r0 = int64_t(blockIdx.x) * G; r0 < rows; r0 += int64_t(gridDim.x) * G) {
    // conj(Z), Z_k = A_k + i B_k over the whole circle (A_{N-k} = conj A_k),
    // A the spectrum of tube 2s, B of tube 2s + 1
    for (int e = threadIdx.x; e < P * N; e += blockDim.x) {
      const int k = e / P, sq = e - k * P;
      const bool lo = k < h;
      const int kk = lo ? k : N - k;
      const bool real_k = kk == 0 || 2 * kk == N;
      const int64_t ra = r0 + 2 * sq, rb = ra + 1;
      float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
      if (ra < rows) {
        A.x = __ldg(ire + int64_t(kk) * in_slice + ra);
        A.y = real_k ? 0.f : __ldg(iim + int64_t(kk) * in_slice + ra);
      }
      if (rb < rows) {
        B.x = __ldg(ire + int64_t(kk) * in_slice + rb);
        B.y = real_k ? 0.f : __ldg(iim + int64_t(kk) * in_slice + rb);
      }
      if (!lo) {
        A.y = -A.y;
        B.y = -B.y;
      }
      b0[sq * N + k] = make_float2(A.x - B.y, -(A.y + B.x));
    }
    __syncthreads();
    const float2* res = stockham_all(plan, tw, b0, b1, P);
    // ifft(Z) = conj(FFT(conj Z)) / N: tube a = Re, tube b = -Im
    for (int e = threadIdx.x; e < G * N; e += blockDim.x) {
      const int t = e / G, c = e - t * G;
      const int64_t r = r0 + c;
      if (r >= rows) continue;
      const float2 v = res[(c >> 1) * N + t];
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

// Sequences per block: four when they fit in the shared-memory budget
// (twiddles + two buffers of P sequences), fewer for long tubes.
constexpr size_t kFftSmemCap = 200 * 1024;
size_t fft_smem(int64_t n, int P) { return size_t(n) * (1 + 2 * size_t(P)) * sizeof(float2); }
int fft_seqs(int64_t n) {
  for (int P = FFT_P_MAX; P >= 1; --P)
    if (fft_smem(n, P) <= kFftSmemCap) return P;
  return 0;
}

unsigned fft_grid(int64_t rows, int P, size_t smem) {
  const int64_t groups = (rows + 2 * P - 1) / (2 * P);
  const int per_sm = int(227 * 1024 / (smem + 1024));
  int64_t b = int64_t(sm_count()) * (per_sm < 1 ? 1 : per_sm);
  if (b > groups) b = groups;
  return unsigned(b < 1 ? 1 : b);
}

}  // namespace

bool fft_supported(int64_t n3) {
  FftPlan p;
  return make_plan(n3, &p) && fft_seqs(n3) > 0;
}

int launch_fft_fwd(const float* X, int64_t rows, int64_t n3, float* ore, float* oim,
                   int64_t out_slice, cudaStream_t st) {
  FftPlan plan;
  const int P = fft_seqs(n3);
  if (!make_plan(n3, &plan) || P == 0) {
    set_error("fft: n3 = %lld is not a product of radices 2,3,5,7,11,13 that fits in shared memory",
              (long long)n3);
    return TP_EUNSUPPORTED;
  }
  if (rows == 0) return TP_OK;
  const size_t smem = fft_smem(n3, P);
  TP_SET_SMEM(fft_fwd_kernel, smem);
  {
    KernelScope ks("fft_fwd", st);
    fft_fwd_kernel<<<fft_grid(rows, P, smem), FFT_THREADS, smem, st>>>(X, rows, plan, P, ore, oim,
                                                                      out_slice);
  }
  return launch_status("fft_fwd_kernel");
}

int launch_fft_inv(const float* ire, const float* iim, int64_t rows, int64_t in_slice, int64_t n3,
                   float* out, cudaStream_t st) {
  FftPlan plan;
  const int P = fft_seqs(n3);
  if (!make_plan(n3, &plan) || P == 0) {
    set_error("fft: n3 = %lld is not a product of radices 2,3,5,7,11,13 that fits in shared memory",
              (long long)n3);
    return TP_EUNSUPPORTED;
  }
  if (rows == 0) return TP_OK;
  const size_t smem = fft_smem(n3, P);
  TP_SET_SMEM(fft_inv_kernel, smem);
  {
    KernelScope ks("fft_inv", st);
    fft_inv_kernel<<<fft_grid(rows, P, smem), FFT_INV_THREADS, smem, st>>>(ire, iim, rows, in_slice,
                                                                      plan, P, out);
  }
  return launch_status("fft_inv_kernel");
}

}  // namespace tp
