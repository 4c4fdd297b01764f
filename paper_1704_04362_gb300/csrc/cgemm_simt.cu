// Facewise complex GEMM of the half spectrum in plain FP32 (Algorithm 1 and
// Algorithm 2 loops over k: C_hat_k = A_hat_k B_hat_k).  Planar split-complex
// operands, four real products per complex multiply-add.  The real slices
// (k = 0 and, for even n3, k = n3/2) skip the imaginary planes.
//
// Tiling: 128 x 64 output tile per 256-thread block, BK = 16, each thread an
// 8 x 4 complex micro-tile (64 float accumulators); the next K tile is
// prefetched into registers while the current one is consumed from shared
// memory.
#include "tp_internal.cuh"

namespace tp {
namespace {

constexpr int BM = 128, BN = 64, BK = 16, NT = 256;

template <bool REAL>
__device__ __forceinline__ void cgemm_tile(const CGemm& g, int64_t f, int64_t K,
                                           float (&As)[2][BK][BM], float (&Bs)[2][BK][BN]) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = int64_t(blockIdx.x) * BM;
  const int64_t n0 = int64_t(blockIdx.y) * BN;
  const float* ar = g.ar + f * g.sA;
  const float* ai = g.ai + f * g.sA;
  const float* br = g.br + f * g.sB;
  const float* bi = g.bi + f * g.sB;

  float cr[8][4], ci[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { cr[i][j] = 0.f; ci[i][j] = 0.f; }

  // global -> register staging indices
  const int a_m = tid & 127, a_k = tid >> 7;      // kk = a_k + 2u, u < 8
  const int b_k = tid & 15, b_n = tid >> 4;       // n = b_n + 16u, u < 4
  float ra[2][8], rb[2][4];

  auto load = [&](int64_t kt) {
    const int64_t m = m0 + a_m;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t kk = kt + a_k + 2 * u;
      const bool ok = (m < g.M) && (kk < K);
      ra[0][u] = ok ? __ldg(ar + m + g.lda * kk) : 0.f;
      if (!REAL) ra[1][u] = ok ? __ldg(ai + m + g.lda * kk) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t n = n0 + b_n + 16 * u;
      const int64_t kk = kt + b_k;
      const bool ok = (n < g.N) && (kk < K);
      const int64_t off = g.b_conj_trans ? n + g.ldb * kk : kk + g.ldb * n;
      rb[0][u] = ok ? __ldg(br + off) : 0.f;
      if (!REAL) {
        const float v = ok ? __ldg(bi + off) : 0.f;
        rb[1][u] = g.b_conj_trans ? -v : v;
      }
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      As[0][a_k + 2 * u][a_m] = ra[0][u];
      if (!REAL) As[1][a_k + 2 * u][a_m] = ra[1][u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      Bs[0][b_k][b_n + 16 * u] = rb[0][u];
      if (!REAL) Bs[1][b_k][b_n + 16 * u] = rb[1][u];
    }
  };

  if (K > 0) load(0);
  for (int64_t kt = 0; kt < K; kt += BK) {
    __syncthreads();
    store();
    __syncthreads();
    if (kt + BK < K) load(kt + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a_r[8], a_i[8], b_r[4], b_i[4];
      const float4 x0 = *reinterpret_cast<const float4*>(&As[0][kk][tx * 4]);
      const float4 x1 = *reinterpret_cast<const float4*>(&As[0][kk][64 + tx * 4]);
      a_r[0] = x0.x; a_r[1] = x0.y; a_r[2] = x0.z; a_r[3] = x0.w;
      a_r[4] = x1.x; a_r[5] = x1.y; a_r[6] = x1.z; a_r[7] = x1.w;
      const float4 y0 = *reinterpret_cast<const float4*>(&Bs[0][kk][ty * 4]);
      b_r[0] = y0.x; b_r[1] = y0.y; b_r[2] = y0.z; b_r[3] = y0.w;
      if (!REAL) {
        const float4 x2 = *reinterpret_cast<const float4*>(&As[1][kk][tx * 4]);
        const float4 x3 = *reinterpret_cast<const float4*>(&As[1][kk][64 + tx * 4]);
        a_i[0] = x2.x; a_i[1] = x2.y; a_i[2] = x2.z; a_i[3] = x2.w;
        a_i[4] = x3.x; a_i[5] = x3.y; a_i[6] = x3.z; a_i[7] = x3.w;
        const float4 y1 = *reinterpret_cast<const float4*>(&Bs[1][kk][ty * 4]);
        b_i[0] = y1.x; b_i[1] = y1.y; b_i[2] = y1.z; b_i[3] = y1.w;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          cr[i][j] = fmaf(a_r[i], b_r[j], cr[i][j]);
          if (!REAL) {
            cr[i][j] = fmaf(-a_i[i], b_i[j], cr[i][j]);
            ci[i][j] = fmaf(a_r[i], b_i[j], ci[i][j]);
            ci[i][j] = fmaf(a_i[i], b_r[j], ci[i][j]);
          }
        }
    }
  }

  float* Cr = g.cr + f * g.sC;
  float* Ci = g.ci + f * g.sC;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t n = n0 + ty * 4 + j;
    if (n >= g.N) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t m = m0 + (i < 4 ? tx * 4 + i : 64 + tx * 4 + (i - 4));
      if (m < g.M) {
        Cr[m + g.ldc * n] = cr[i][j];
        Ci[m + g.ldc * n] = REAL ? 0.f : ci[i][j];
      }
    }
  }
}

__global__ void __launch_bounds__(NT) cgemm_simt_kernel(CGemm g) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int64_t K = g.dynK ? *g.dynK : g.K;
  for (int64_t f = blockIdx.z; f < g.h; f += gridDim.z) {
    const bool real = (f == 0) || ((g.n3 % 2 == 0) && f == g.h - 1);
    if (real) cgemm_tile<true>(g, f, K, As, Bs);
    else cgemm_tile<false>(g, f, K, As, Bs);
    __syncthreads();
  }
}

}  // namespace

int launch_cgemm_simt(const CGemm& g, cudaStream_t st) {
  if (g.M == 0 || g.N == 0 || g.h == 0) return TP_OK;
  const int64_t gx = (g.M + BM - 1) / BM, gy = (g.N + BN - 1) / BN;
  if (gx > 0x7fffffff || gy > 65535) {
    set_error("cgemm: output %lld x %lld too large for one launch", (long long)g.M, (long long)g.N);
    return TP_EUNSUPPORTED;
  }
  const int64_t gz = g.h < 65535 ? g.h : 65535;
  {
    KernelScope ks("cgemm_fp32", st);
    cgemm_simt_kernel<<<dim3(unsigned(gx), unsigned(gy), unsigned(gz)), NT, 0, st>>>(g);
  }
  return launch_status("cgemm_simt_kernel");
}

}  // namespace tp
