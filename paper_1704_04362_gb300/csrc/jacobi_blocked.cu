// Blocked one-sided Jacobi (float32) for the singular-value thresholding of
// the completion ADMM (Algorithm 7) on slices too large for the
// shared-memory form of svd.cu.
//
// The columns of the p x q work matrix G are cut into blocks of B = 16.  For
// every pair of blocks (I, J) the CTA copies the (at most 32) columns of both
// blocks into shared memory, rotates there the 16 x 16 pairs across the two
// blocks (and, once per sweep, each block's internal pairs) in rounds of
// disjoint pairs, one pair per warp per round (the same rotation formula as
// svd.cu), accumulates those rotations in a small 32 x 32 matrix Q, writes
// the columns back and applies Q to the matching 32 columns of V
// (V_blk <- V_blk Q, staged through the same shared memory).  Visiting every
// block pair rotates every column pair once: one sweep of a cyclic Jacobi
// ordering by blocks; sweeps repeat until one makes no rotation (or the
// sweep cap, TP_DEV_NOCONV).  Each column pair
// thereby costs shared-memory traffic; global memory sees each column once
// per block pair instead of twice per rotation.  The convergence threshold
// is the one of svd.cu, so the result is an SVD to the same tolerance (the
// rotation order differs).
#include "jacobi_rot.cuh"

namespace tp {
namespace {
using jrot::rotation;

constexpr int JB_THREADS = 512;   // 16 warps: one column pair each per round
constexpr int JB_B = 16;          // columns per block; a block pair holds <= 32
constexpr int JB_C = 2 * JB_B;
constexpr size_t JB_SMEM_MAX = size_t(212) * 1024;   // dynamic; the static arrays take ~9 KB
constexpr int JB_MAX_NB = 64;     // blocks of a slice whose block pairs keep records

__device__ __forceinline__ float jb_warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Global column of local column c of the block pair (I, J): the bI columns
// of block I first, then those of block J.
__device__ __forceinline__ int jb_col(int c, int I, int J, int bI) {
  return c < bI ? I * JB_B + c : J * JB_B + (c - bI);
}


// One CTA per slice b: G (p x q, ld p) at g_re/g_im + b*sG, V (q x q) at
// v_re/v_im + b*sV, q <= p.  On exit G is rotated (not normalised), V holds
// the accumulated rotations and sig[b*q + j] = ||G_j||.
// RPL > 0 (p <= 32 RPL): in the cross rounds warp i keeps local column i of
// block I in registers (RPL rows a lane) -- it is that column's partner in
// every cross round -- and only the columns of block J move, through shared
// memory: per row and pair 16 bytes of shared-memory traffic instead of 48
// for 16 FMA.  RPL = 0: every pair is read from and written to shared memory.
template <int RPL>
__global__ void __launch_bounds__(JB_THREADS) jacobi_blocked_kernel(
    float* __restrict__ g_re, float* __restrict__ g_im, int64_t sG, float* __restrict__ v_re,
    float* __restrict__ v_im, int64_t sV, float* __restrict__ sig, int p, int q, int max_sweeps,
    const int* __restrict__ real_flags, int32_t* __restrict__ status, int init_v) {
  extern __shared__ __align__(16) float jb_smem[];
  // staged columns of G at stride ld (the register path's 32 RPL >= p rows:
  // its lanes move 4 consecutive rows with one 16-byte access and the zero
  // rows past p need no guard), later those of V at stride q
  const int ld = RPL > 0 ? 32 * RPL : p;
  float* const Sr = jb_smem;                      // [JB_C][ld]
  float* const Si = jb_smem + size_t(JB_C) * ld;
  float* const Qr = jb_smem + size_t(2) * JB_C * ld;   // Q(r, c) at c * JB_C + r
  float* const Qi = Qr + JB_C * JB_C;
  __shared__ int any_rot, blk_rot;
  // Skipping converged block pairs: bver[I] counts the block pairs that
  // rotated block I's columns; pquiet[bp] holds the two blocks' counts when
  // block pair bp last made no rotation.  While both counts are unchanged its
  // columns are bit-identical to then, so its inner products are too and it
  // would again rotate nothing: it is skipped (the result is the same as
  // visiting it; a converged warm sweep mostly consists of such pairs).
  __shared__ int bver[JB_MAX_NB];
  __shared__ int pquiet[JB_MAX_NB * (JB_MAX_NB - 1) / 2];
  __shared__ float nrm[JB_C];   // squared norms of the staged columns
  const int64_t b = blockIdx.x;
  float* const Gr = g_re + b * sG;
  float* const Gi = g_im + b * sG;
  float* const Vr = v_re + b * sV;
  float* const Vi = v_im + b * sV;
  const bool real = real_flags ? real_flags[b] != 0 : false;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = JB_THREADS / 32;
  const int64_t pq = int64_t(p) * q, qq = int64_t(q) * q;
  if (init_v)
    for (int64_t e = tid; e < qq; e += JB_THREADS) {
      Vr[e] = (e % (q + 1) == 0) ? 1.f : 0.f;
      Vi[e] = 0.f;
    }
  if (real) {
    for (int64_t e = tid; e < pq; e += JB_THREADS) Gi[e] = 0.f;
    for (int64_t e = tid; e < qq; e += JB_THREADS) Vi[e] = 0.f;
  }
  __syncthreads();

  float tol = 8.f * 5.96e-8f * sqrtf(float(p));
  if (tol < 1e-6f) tol = 1e-6f;
  const int nb = (q + JB_B - 1) / JB_B;
  const int npair = nb == 1 ? 1 : nb * (nb - 1) / 2;
  const bool rec = nb <= JB_MAX_NB;
  for (int e = tid; e < JB_MAX_NB * (JB_MAX_NB - 1) / 2; e += JB_THREADS) pquiet[e] = -1;
  for (int e = tid; e < JB_MAX_NB; e += JB_THREADS) bver[e] = 0;
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) any_rot = 0;
    for (int bp = 0; bp < npair; ++bp) {
      int I = 0, J = -1;   // block pair bp, I < J, row by row
      if (nb > 1) {
        int rem = bp;
        while (rem >= nb - 1 - I) {
          rem -= nb - 1 - I;
          ++I;
        }
        J = I + 1 + rem;
      }
      const int key = rec ? (bver[I] & 0xffff) | ((J < 0 ? 0 : bver[J] & 0x7fff) << 16) : -2;
      if (rec && pquiet[bp] == key) continue;   // uniform: written before the last barrier
      const int bI = min(JB_B, q - I * JB_B);
      const int bJ = J < 0 ? 0 : min(JB_B, q - J * JB_B);
      const int nc = bI + bJ;
      if (tid == 0) blk_rot = 0;
      // stage the nc columns (a warp per column, lanes along it) and their
      // squared norms; the rotations below update the norms exactly
      // (||a'||^2 = alpha - t |gamma|, ||b'||^2 = beta + t |gamma|), so each
      // pair needs only its inner product
      for (int c = warp; c < nc; c += NW) {
        const float* gr_c = Gr + int64_t(jb_col(c, I, J, bI)) * p;
        const float* gi_c = Gi + int64_t(jb_col(c, I, J, bI)) * p;
        float* sr_c = Sr + size_t(c) * ld;
        float* si_c = Si + size_t(c) * ld;
        float acc = 0.f;
        for (int r = lane; r < p; r += 32) {
          const float xr = gr_c[r], xi = gi_c[r];
          sr_c[r] = xr;
          si_c[r] = xi;
          acc = fmaf(xr, xr, fmaf(xi, xi, acc));
        }
        for (int r = p + lane; r < ld; r += 32) {   // the padding rows (V's staging overwrote them)
          sr_c[r] = 0.f;
          si_c[r] = 0.f;
        }
        acc = jb_warp_sum(acc);
        if (lane == 0) nrm[c] = acc;
      }
      for (int e = tid; e < JB_C * JB_C; e += JB_THREADS) {
        Qr[e] = (e % (JB_C + 1) == 0) ? 1.f : 0.f;
        Qi[e] = 0.f;
      }
      __syncthreads();
      // The rotations of this block pair, in rounds of disjoint column pairs
      // (one pair per warp): the bI x bJ cross pairs (round t pairs local
      // column i of I with column (i + t) mod bI of J), and each block's
      // internal pairs once per sweep -- block I's in the block pair
      // (I, I + 1), the last block's also in (nb - 2, nb - 1) -- by the
      // round-robin order; a lone block has internal pairs only.
      const bool within_I = J < 0 || J == I + 1;
      const bool within_J = J >= 0 && J == nb - 1 && I == nb - 2;
      const int ncI = bI + (bI & 1), ncJ = bJ + (bJ & 1);
      const int wrounds = max(within_I ? ncI - 1 : 0, within_J ? ncJ - 1 : 0);
      const int crounds = J < 0 || RPL > 0 ? 0 : bI;
      for (int round = 0; round < wrounds + crounds; ++round) {
        const bool cross = round >= wrounds;
        const int t = cross ? round - wrounds : round;
        const int npr = cross ? bI : (within_I ? ncI / 2 : 0) + (within_J ? ncJ / 2 : 0);
        for (int i = warp; i < npr; i += NW) {
          int a, c2;
          if (cross) {
            const int jj = (i + t) % bI;
            if (jj >= bJ) continue;
            a = i;
            c2 = bI + jj;
          } else {
            int base = 0, n = bI, nn = ncI, k = i;
            if (!within_I || k >= ncI / 2) {
              k -= within_I ? ncI / 2 : 0;
              base = bI;
              n = bJ;
              nn = ncJ;
            }
            if (t >= nn - 1) continue;
            int x, y;
            if (k == 0) {
              x = nn - 1;
              y = t;
            } else {
              x = (t + k) % (nn - 1);
              y = (t - k + (nn - 1)) % (nn - 1);
            }
            if (x >= n || y >= n) continue;
            a = base + min(x, y);
            c2 = base + max(x, y);
          }
          float* const ar = Sr + size_t(a) * ld;
          float* const ai = Si + size_t(a) * ld;
          float* const br = Sr + size_t(c2) * ld;
          float* const bi = Si + size_t(c2) * ld;
          const float alpha = nrm[a], beta = nrm[c2];
          float gr = 0.f, gi = 0.f;
          for (int r = lane; r < p; r += 32) {
            const float xr = ar[r], xi = ai[r], yr = br[r], yi = bi[r];
            gr = fmaf(xr, yr, fmaf(xi, yi, gr));    // Re(conj(x) y)
            gi = fmaf(xr, yi, fmaf(-xi, yr, gi));   // Im(conj(x) y)
          }
          gr = jb_warp_sum(gr);
          gi = jb_warp_sum(gi);
          const float g2 = gr * gr + gi * gi;
          if (!(g2 > tol * tol * alpha * beta) || g2 == 0.f) continue;
          if (lane == 0) blk_rot = 1;
          float cs, sn, er, ei;   // cos, sin and e^{-i phi}
          rotation(alpha, beta, gr, gi, g2, cs, sn, er, ei);
          if (lane == 0) {
            const float tg = (sn / cs) * sqrtf(g2);
            nrm[a] = alpha - tg;
            nrm[c2] = beta + tg;
          }
          for (int r = lane; r < p; r += 32) {
            const float xr = ar[r], xi = ai[r];
            const float yr = br[r] * er - bi[r] * ei, yi = br[r] * ei + bi[r] * er;
            ar[r] = cs * xr - sn * yr;
            ai[r] = cs * xi - sn * yi;
            br[r] = sn * xr + cs * yr;
            bi[r] = sn * xi + cs * yi;
          }
          // the same column operation on Q (rows 0 .. nc-1; lane r < 32)
          {
            float* const qa_r = Qr + a * JB_C;
            float* const qa_i = Qi + a * JB_C;
            float* const qb_r = Qr + c2 * JB_C;
            float* const qb_i = Qi + c2 * JB_C;
            const int r = lane;
            if (r < nc) {
              const float xr = qa_r[r], xi = qa_i[r];
              const float yr = qb_r[r] * er - qb_i[r] * ei, yi = qb_r[r] * ei + qb_i[r] * er;
              qa_r[r] = cs * xr - sn * yr;
              qa_i[r] = cs * xi - sn * yi;
              qb_r[r] = sn * xr + cs * yr;
              qb_i[r] = sn * xi + cs * yi;
            }
          }
        }
        __syncthreads();
      }
      if (RPL > 0 && J >= 0) {
        // cross rounds with block I's columns resident: round t pairs local
        // column i (warp i) with column bI + (i + t) mod bI of block J
        const bool own = warp < bI;
        float xr[RPL > 0 ? RPL : 1], xi[RPL > 0 ? RPL : 1];
        float alpha = 0.f;
        // lane's rows: 128 m + 4 lane + j (register k = 4 m + j)
        if (own) {
          const float4* ar = reinterpret_cast<const float4*>(Sr + size_t(warp) * ld);
          const float4* ai = reinterpret_cast<const float4*>(Si + size_t(warp) * ld);
#pragma unroll
          for (int m = 0; m < RPL / 4; ++m) {
            const float4 u = ar[32 * m + lane], v = ai[32 * m + lane];
            xr[4 * m] = u.x; xr[4 * m + 1] = u.y; xr[4 * m + 2] = u.z; xr[4 * m + 3] = u.w;
            xi[4 * m] = v.x; xi[4 * m + 1] = v.y; xi[4 * m + 2] = v.z; xi[4 * m + 3] = v.w;
          }
          alpha = nrm[warp];
        }
        for (int t = 0; t < bI; ++t) {
          const int jj = own ? (warp + t) % bI : 0;
          if (own && jj < bJ) {
            const int c2 = bI + jj;
            float4* const br = reinterpret_cast<float4*>(Sr + size_t(c2) * ld);
            float4* const bi = reinterpret_cast<float4*>(Si + size_t(c2) * ld);
            float yr[RPL > 0 ? RPL : 1], yi[RPL > 0 ? RPL : 1];
#pragma unroll
            for (int m = 0; m < RPL / 4; ++m) {
              const float4 u = br[32 * m + lane], v = bi[32 * m + lane];
              yr[4 * m] = u.x; yr[4 * m + 1] = u.y; yr[4 * m + 2] = u.z; yr[4 * m + 3] = u.w;
              yi[4 * m] = v.x; yi[4 * m + 1] = v.y; yi[4 * m + 2] = v.z; yi[4 * m + 3] = v.w;
            }
            float gr = 0.f, gi = 0.f;
#pragma unroll
            for (int k = 0; k < RPL; ++k) {
              gr = fmaf(xr[k], yr[k], fmaf(xi[k], yi[k], gr));    // Re(conj(x) y)
              gi = fmaf(xr[k], yi[k], fmaf(-xi[k], yr[k], gi));   // Im(conj(x) y)
            }
            gr = jb_warp_sum(gr);
            gi = jb_warp_sum(gi);
            const float beta = nrm[c2];
            const float g2 = gr * gr + gi * gi;
            if (g2 > tol * tol * alpha * beta && g2 != 0.f) {
              if (lane == 0) blk_rot = 1;
              float cs, sn, er, ei, tg;   // cos, sin, e^{-i phi} and t |gamma|
              rotation(alpha, beta, gr, gi, g2, cs, sn, er, ei, tg);
              alpha -= tg;
              if (lane == 0) nrm[c2] = beta + tg;
#pragma unroll
              for (int k = 0; k < RPL; ++k) {
                const float ur = yr[k] * er - yi[k] * ei, ui = yr[k] * ei + yi[k] * er;
                const float x0 = xr[k], x1 = xi[k];
                xr[k] = cs * x0 - sn * ur;
                xi[k] = cs * x1 - sn * ui;
                yr[k] = sn * x0 + cs * ur;
                yi[k] = sn * x1 + cs * ui;
              }
#pragma unroll
              for (int m = 0; m < RPL / 4; ++m) {
                br[32 * m + lane] = make_float4(yr[4 * m], yr[4 * m + 1], yr[4 * m + 2],
                                                yr[4 * m + 3]);
                bi[32 * m + lane] = make_float4(yi[4 * m], yi[4 * m + 1], yi[4 * m + 2],
                                                yi[4 * m + 3]);
              }
              // the same column operation on Q (rows 0 .. nc-1; lane r < 32)
              float* const qa_r = Qr + warp * JB_C;
              float* const qa_i = Qi + warp * JB_C;
              float* const qb_r = Qr + c2 * JB_C;
              float* const qb_i = Qi + c2 * JB_C;
              if (lane < nc) {
                const float x0 = qa_r[lane], x1 = qa_i[lane];
                const float ur = qb_r[lane] * er - qb_i[lane] * ei,
                            ui = qb_r[lane] * ei + qb_i[lane] * er;
                qa_r[lane] = cs * x0 - sn * ur;
                qa_i[lane] = cs * x1 - sn * ui;
                qb_r[lane] = sn * x0 + cs * ur;
                qb_i[lane] = sn * x1 + cs * ui;
              }
            }
          }
          __syncthreads();   // block J's columns change hands
        }
        if (own) {
          float4* const ar = reinterpret_cast<float4*>(Sr + size_t(warp) * ld);
          float4* const ai = reinterpret_cast<float4*>(Si + size_t(warp) * ld);
#pragma unroll
          for (int m = 0; m < RPL / 4; ++m) {
            ar[32 * m + lane] = make_float4(xr[4 * m], xr[4 * m + 1], xr[4 * m + 2], xr[4 * m + 3]);
            ai[32 * m + lane] = make_float4(xi[4 * m], xi[4 * m + 1], xi[4 * m + 2], xi[4 * m + 3]);
          }
          if (lane == 0) nrm[warp] = alpha;
        }
        __syncthreads();
      }
      if (blk_rot) {   // uniform: every write of it precedes the last barrier
        for (int c = warp; c < nc; c += NW) {
          float* gr_c = Gr + int64_t(jb_col(c, I, J, bI)) * p;
          float* gi_c = Gi + int64_t(jb_col(c, I, J, bI)) * p;
          const float* sr_c = Sr + size_t(c) * ld;
          const float* si_c = Si + size_t(c) * ld;
          for (int r = lane; r < p; r += 32) {
            gr_c[r] = sr_c[r];
            gi_c[r] = si_c[r];
          }
        }
        __syncthreads();   // the staging area now takes V's columns
        for (int c = warp; c < nc; c += NW) {
          const float* vr_c = Vr + int64_t(jb_col(c, I, J, bI)) * q;
          const float* vi_c = Vi + int64_t(jb_col(c, I, J, bI)) * q;
          float* sr_c = Sr + size_t(c) * q;
          float* si_c = Si + size_t(c) * q;
          for (int r = lane; r < q; r += 32) {
            sr_c[r] = vr_c[r];
            si_c[r] = vi_c[r];
          }
        }
        __syncthreads();
        // V_blk <- V_blk Q, register-tiled: a warp task is 128 rows (4 per
        // lane, 32 apart, so the lanes read consecutive words) by 4 columns;
        // per k a lane loads 4 entries of V_blk and 4 of Q (the same for the
        // whole warp) for 16 complex multiply-adds
        {
          const int rgroups = (q + 127) / 128, cgroups = (nc + 3) / 4;
          for (int task = warp; task < rgroups * cgroups; task += NW) {
            const int r0 = (task % rgroups) * 128 + lane, c0 = (task / rgroups) * 4;
            float ar[4][4], ai[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                ar[i][j] = 0.f;
                ai[i][j] = 0.f;
              }
            for (int k = 0; k < nc; ++k) {
              float xr[4], xi[4], yr[4], yi[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const int r = r0 + 32 * i;
                xr[i] = r < q ? Sr[k * q + r] : 0.f;
                xi[i] = r < q ? Si[k * q + r] : 0.f;
              }
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int c = c0 + j;
                yr[j] = c < nc ? Qr[c * JB_C + k] : 0.f;
                yi[j] = c < nc ? Qi[c * JB_C + k] : 0.f;
              }
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  ar[i][j] = fmaf(xr[i], yr[j], fmaf(-xi[i], yi[j], ar[i][j]));
                  ai[i][j] = fmaf(xr[i], yi[j], fmaf(xi[i], yr[j], ai[i][j]));
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int c = c0 + j;
              if (c >= nc) continue;
              const int64_t col = int64_t(jb_col(c, I, J, bI)) * q;
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const int r = r0 + 32 * i;
                if (r < q) {
                  Vr[col + r] = ar[i][j];
                  Vi[col + r] = ai[i][j];
                }
              }
            }
          }
        }
        if (tid == 0) any_rot = 1;
      }
      if (tid == 0 && rec) {
        if (blk_rot) {
          ++bver[I];
          if (J >= 0) ++bver[J];
        } else {
          pquiet[bp] = key;
        }
      }
      __syncthreads();   // the staging area, blk_rot and the records are reused by the next pair
    }
    const int any = any_rot;
    __syncthreads();
    if (!any) break;
  }
  if (sweep >= max_sweeps && tid == 0 && status) atomicOr(status, TP_DEV_NOCONV);
  for (int j = warp; j < q; j += NW) {
    const float* xr = Gr + int64_t(j) * p;
    const float* xi = Gi + int64_t(j) * p;
    float nrm = 0.f;
    for (int r = lane; r < p; r += 32) nrm += xr[r] * xr[r] + xi[r] * xi[r];
    nrm = sqrtf(jb_warp_sum(nrm));
    if (lane == 0) sig[b * q + j] = nrm;
  }
}

size_t jb_smem_bytes(int p) {
  return (size_t(2) * JB_C * p + size_t(2) * JB_C * JB_C) * sizeof(float);
}

template <int RPL>
int jb_launch(float* gr, float* gi, int64_t sG, float* vr, float* vi, int64_t sV, float* sig,
              int p, int q, int batch, int max_sweeps, const int* real_flags, int32_t* status,
              bool init_v, cudaStream_t st) {
  const size_t smem = jb_smem_bytes(RPL > 0 ? 32 * RPL : p);
  TP_SET_SMEM(jacobi_blocked_kernel<RPL>, smem);
  {
    KernelScope ks("jacobi_blocked", st);
    jacobi_blocked_kernel<RPL><<<unsigned(batch), JB_THREADS, smem, st>>>(
        gr, gi, sG, vr, vi, sV, sig, p, q, max_sweeps, real_flags, status, init_v ? 1 : 0);
  }
  return launch_status("jacobi_blocked_kernel");
}

}  // namespace

// The blocked form serves slices whose G and V do not fit the shared-memory
// form of svd.cu (200 KB) while 32 of G's columns do.
bool jacobi_blocked_applies(int p, int q) {
  const size_t whole = (size_t(2) * p * q + size_t(2) * q * q) * sizeof(float);
  return q <= p && whole > size_t(200) * 1024 && jb_smem_bytes(p) <= JB_SMEM_MAX;
}

// float32 blocked one-sided Jacobi from V = I (init_v) or from the given V
// (then G must be the work matrix times that V); G is left rotated.
int jacobi_float_blocked_launch(float* gr, float* gi, int64_t sG, float* vr, float* vi,
                                int64_t sV, float* sig, int p, int q, int batch, int max_sweeps,
                                const int* real_flags, int32_t* status, bool init_v,
                                cudaStream_t st) {
  if (batch <= 0 || q <= 0) return TP_OK;
  // the register form's rows come in steps of 128 (the zero rows past p
  // cost the same arithmetic as data rows)
  if (p <= 128)
    return jb_launch<4>(gr, gi, sG, vr, vi, sV, sig, p, q, batch, max_sweeps, real_flags, status,
                        init_v, st);
  if (p <= 256)
    return jb_launch<8>(gr, gi, sG, vr, vi, sV, sig, p, q, batch, max_sweeps, real_flags, status,
                        init_v, st);
  if (p <= 384)
    return jb_launch<12>(gr, gi, sG, vr, vi, sV, sig, p, q, batch, max_sweeps, real_flags, status,
                         init_v, st);
  if (p <= 512)
    return jb_launch<16>(gr, gi, sG, vr, vi, sV, sig, p, q, batch, max_sweeps, real_flags, status,
                         init_v, st);
  return jb_launch<0>(gr, gi, sG, vr, vi, sV, sig, p, q, batch, max_sweeps, real_flags, status,
                      init_v, st);
}

}  // namespace tp
