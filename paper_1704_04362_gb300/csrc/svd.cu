// Facewise SVD of the half spectrum for the t-SVD (Theorem 2.6 computed as in
// Eq. circ1): every Fourier slice X_hat_k = U_k diag(s_k) V_k^H.
//
// One CTA per slice runs the one-sided (Hestenes) Jacobi method on the
// columns of a p x q work matrix G (p >= q): pairs of columns (a, b) are
// rotated by a 2 x 2 unitary until every pair is orthogonal to a relative
// tolerance; the same rotations accumulate in V (q x q).  Then s_j = ||G_j||,
// U_j = G_j / s_j.  Pairs are scheduled by the round-robin (circle) ordering
// so that the q/2 pairs of a step are disjoint and run on separate warps.
// The complex rotation: with gamma = a^H b = |gamma| e^{i phi}, b~ = e^{-i phi} b
// makes the pair real; zeta = (||b||^2 - ||a||^2) / (2|gamma|),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t,
// a' = c a - s b~, b' = s a + c b~.  Sweeps are capped (opts->max_sweeps); a
// slice that reaches the cap sets TP_DEV_NOCONV.  G and V live in shared
// memory when they fit, else in global memory.  With fewer slices than SMs a
// cluster of CTAs shares each slice instead (jacobi_cluster_kernel: the
// round-robin ordering on blocks of columns, one block pair per CTA).
//
// GB300 runs float64 at 1/64 of the float32 rate, so the t-SVD takes the
// sweeps in float32 and finishes in float64:
//   1. float32 Jacobi on G = X (or X^H) from V = I, to float32 convergence;
//   2. V <- V (3 I - V^H V) / 2 in float64 (one Newton-Schulz step: the
//      accumulated float32 rotations are orthonormal to ~1e-6, after it to
//      ~1e-12);
//   3. G = X V in float64;
//   4. float64 Jacobi on that G, starting from V, to float64 convergence:
//      the columns are already orthogonal to float32 accuracy, so two or
//      three sweeps (quadratic convergence) suffice, more only for a cluster
//      of singular values at the float32 rounding floor (rank-deficient
//      input), which float32 cannot resolve.
// Steps 2-3 are batched float64 GEMMs spread over all SMs.
#include <atomic>

#include "jacobi_rot.cuh"

namespace tp {
int householder_orth_launch(float* yr, float* yi, int64_t sY, int p, int l, int64_t batch,
                            bool keep_phase, cudaStream_t st);
namespace {
using jrot::rotation;

#ifndef TP_SVD_THREADS
#define TP_SVD_THREADS 1024
#endif
constexpr int SVD_THREADS = TP_SVD_THREADS;

template <class T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class T> struct Eps;
template <> struct Eps<float> { static constexpr float v = 5.96e-8f; };
template <> struct Eps<double> { static constexpr double v = 1.12e-16; };

// Batched one-sided Jacobi.  Item b: G (p x q, column-major, ld p) at
// g_re/g_im + b*sG, V (q x q) at v_re/v_im + b*sV.  On exit G holds U
// (unit columns, unsorted), sig[b*q + j] the singular values (unsorted).
// Flags of jacobi_kernel.
constexpr int JAC_INIT_V = 1;      // start from V = I (else from the given V)
constexpr int JAC_NORMALIZE = 2;   // on exit scale G's columns to unit length
constexpr int JAC_SMEM = 4;        // work on shared-memory copies of G and V
constexpr int JAC_MAX_Q = 512;     // columns of a slice (min(n1, n2) <= 512 at the entry points)

template <class T>
__global__ void __launch_bounds__(SVD_THREADS) jacobi_kernel(T* g_re, T* g_im, int64_t sG, T* v_re,
                                                             T* v_im, int64_t sV, T* sig, int p,
                                                             int q, int max_sweeps,
                                                             const int* real_flags,
                                                             int32_t* status, int flags) {
  extern __shared__ __align__(16) unsigned char jac_smem[];
  const int64_t b = blockIdx.x;
  T* const gGr = g_re + b * sG;
  T* const gGi = g_im + b * sG;
  T* const gVr = v_re + b * sV;
  T* const gVi = v_im + b * sV;
  T* Gr = gGr;
  T* Gi = gGi;
  T* Vr = gVr;
  T* Vi = gVi;
  const bool real = real_flags ? real_flags[b] != 0 : false;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = SVD_THREADS / 32;
  const int64_t pq = int64_t(p) * q;
  __shared__ int rotated;

  if (flags & JAC_SMEM) {
    T* sm = reinterpret_cast<T*>(jac_smem);
    Gr = sm;
    Gi = sm + pq;
    Vr = sm + 2 * pq;
    Vi = sm + 2 * pq + q * q;
    for (int64_t e = tid; e < pq; e += SVD_THREADS) {
      Gr[e] = gGr[e];
      Gi[e] = gGi[e];
    }
    if (!(flags & JAC_INIT_V))
      for (int e = tid; e < q * q; e += SVD_THREADS) {
        Vr[e] = gVr[e];
        Vi[e] = gVi[e];
      }
  }
  if (flags & JAC_INIT_V)
    for (int e = tid; e < q * q; e += SVD_THREADS) {
      Vr[e] = (e % (q + 1) == 0) ? T(1) : T(0);
      Vi[e] = T(0);
    }
  if (real) {
    for (int64_t e = tid; e < pq; e += SVD_THREADS) Gi[e] = T(0);
    for (int e = tid; e < q * q; e += SVD_THREADS) Vi[e] = T(0);
  }
  __syncthreads();

  T tol = T(8) * Eps<T>::v * sqrt(T(p));
  if (tol < T(sizeof(T) == 4 ? 1e-6 : 1e-13)) tol = T(sizeof(T) == 4 ? 1e-6 : 1e-13);
  const int qq = q + (q & 1);
  // float64: squared column norms computed at the start of every sweep,
  // then kept by each rotation (||a'||^2 = alpha - t |gamma|, ||b'||^2 =
  // beta + t |gamma|), so that a pair needs only its inner product (float64
  // runs at 1/64 of the float32 rate; float32 sweeps are latency-bound and
  // compute the norms with the inner product instead)
  constexpr bool keep = sizeof(T) == 8;
  __shared__ T nrm[keep ? JAC_MAX_Q : 1];
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    if (keep) {
      for (int j = warp; j < q; j += nw) {
        const T* xr = Gr + int64_t(j) * p;
        const T* xi = Gi + int64_t(j) * p;
        T acc = 0;
        for (int r = lane; r < p; r += 32) acc += xr[r] * xr[r] + xi[r] * xi[r];
        acc = warp_sum_t(acc);
        if (lane == 0) nrm[j] = acc;
      }
    }
    __syncthreads();
    for (int step = 0; step < qq - 1; ++step) {
      for (int i = warp; i < qq / 2; i += nw) {
        int a, c2;
        if (i == 0) {
          a = qq - 1;
          c2 = step;
        } else {
          a = (step + i) % (qq - 1);
          c2 = (step - i + (qq - 1)) % (qq - 1);
        }
        if (a >= q || c2 >= q) continue;
        if (a > c2) { const int t = a; a = c2; c2 = t; }
        T* ar = Gr + int64_t(a) * p;
        T* ai = Gi + int64_t(a) * p;
        T* br = Gr + int64_t(c2) * p;
        T* bi = Gi + int64_t(c2) * p;
        T alpha = 0, beta = 0, gr = 0, gi = 0;
        if (keep) {
          alpha = nrm[a] > T(0) ? nrm[a] : T(0);
          beta = nrm[c2] > T(0) ? nrm[c2] : T(0);
          for (int r = lane; r < p; r += 32) {
            const T xr = ar[r], xi = ai[r], yr = br[r], yi = bi[r];
            gr += xr * yr + xi * yi;    // Re(conj(x) y)
            gi += xr * yi - xi * yr;    // Im(conj(x) y)
          }
        } else {
          for (int r = lane; r < p; r += 32) {
            const T xr = ar[r], xi = ai[r], yr = br[r], yi = bi[r];
            alpha += xr * xr + xi * xi;
            beta += yr * yr + yi * yi;
            gr += xr * yr + xi * yi;
            gi += xr * yi - xi * yr;
          }
          alpha = warp_sum_t(alpha);
          beta = warp_sum_t(beta);
        }
        gr = warp_sum_t(gr);
        gi = warp_sum_t(gi);
        const T g2 = gr * gr + gi * gi;
        if (!(g2 > tol * tol * alpha * beta) || g2 == T(0)) continue;
        if (lane == 0) rotated = 1;
        T cs, sn, er, ei, tg;   // cos, sin, e^{-i phi} and t |gamma|
        rotation(alpha, beta, gr, gi, g2, cs, sn, er, ei, tg);
        if (keep && lane == 0) {
          nrm[a] = alpha - tg;
          nrm[c2] = beta + tg;
        }
        for (int r = lane; r < p; r += 32) {
          const T xr = ar[r], xi = ai[r];
          const T yr = br[r] * er - bi[r] * ei, yi = br[r] * ei + bi[r] * er;   // b~
          ar[r] = cs * xr - sn * yr;
          ai[r] = cs * xi - sn * yi;
          br[r] = sn * xr + cs * yr;
          bi[r] = sn * xi + cs * yi;
        }
        T* var = Vr + int64_t(a) * q;
        T* vai = Vi + int64_t(a) * q;
        T* vbr = Vr + int64_t(c2) * q;
        T* vbi = Vi + int64_t(c2) * q;
        for (int r = lane; r < q; r += 32) {
          const T xr = var[r], xi = vai[r];
          const T yr = vbr[r] * er - vbi[r] * ei, yi = vbr[r] * ei + vbi[r] * er;
          var[r] = cs * xr - sn * yr;
          vai[r] = cs * xi - sn * yi;
          vbr[r] = sn * xr + cs * yr;
          vbi[r] = sn * xi + cs * yi;
        }
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  if (sweep >= max_sweeps && tid == 0 && status) atomicOr(status, TP_DEV_NOCONV);
  // singular values and (optionally) unit left vectors
  for (int j = warp; j < q; j += nw) {
    T* xr = Gr + int64_t(j) * p;
    T* xi = Gi + int64_t(j) * p;
    T nrm = 0;
    for (int r = lane; r < p; r += 32) nrm += xr[r] * xr[r] + xi[r] * xi[r];
    nrm = sqrt(warp_sum_t(nrm));
    if (lane == 0) sig[b * q + j] = nrm;
    if (flags & JAC_NORMALIZE) {
      const T inv = nrm > T(0) ? T(1) / nrm : T(0);
      for (int r = lane; r < p; r += 32) {
        xr[r] *= inv;
        xi[r] *= inv;
      }
    }
  }
  if (flags & JAC_SMEM) {
    __syncthreads();
    for (int64_t e = tid; e < pq; e += SVD_THREADS) {
      gGr[e] = Gr[e];
      gGi[e] = Gi[e];
    }
    for (int e = tid; e < q * q; e += SVD_THREADS) {
      gVr[e] = Vr[e];
      gVi[e] = Vi[e];
    }
  }
}

// ---- sweeps of a few slices: one thread-block cluster per slice ----
//
// One CTA per slice leaves most SMs idle when there are few slices (t-CX /
// t-CUR and the t-SVD of a short tube: 17 slices), and float64 runs at only
// 2 FMA per clock per SM.  Here a cluster of JPC CTAs shares one slice: its q
// columns are cut into 2 JPC blocks of bs = ceil(q / 2 JPC), and a sweep runs
// the round-robin (circle) ordering on the blocks.  In each of its 2 JPC - 1
// rounds every CTA owns one block pair and rotates its bs x bs cross pairs (bs
// steps of bs disjoint pairs, one pair per warp); in round 0, where every
// block appears once, it also rotates the internal pairs of its two blocks.
// Each column pair thus meets once per sweep, as in the cyclic sweep.  G, V
// and the kept squared norms live in global memory between rounds (L2
// resident: the slices of this path are small) and are read through L2
// (ld.global.cg), so that what another SM wrote in the previous round is seen
// after the cluster barrier (release / acquire at cluster scope).  When the
// block pair fits, a CTA copies it to shared memory for the round (SMEM).
constexpr int JPC = 8;                 // CTAs per slice (portable cluster size)
constexpr int JPC_BLOCKS = 2 * JPC;    // column blocks per slice
constexpr int JPC_THREADS = 512;

__device__ __forceinline__ void jpc_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned jpc_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// an int in CTA `rank`'s shared memory at the address of `local`
__device__ __forceinline__ int jpc_peek(const int* local, unsigned rank) {
  const unsigned a = unsigned(__cvta_generic_to_shared(local));
  unsigned remote;
  int v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(a), "r"(rank));
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(remote) : "memory");
  return v;
}

template <bool S, class T>
__device__ __forceinline__ T jld(const T* x) {
  if constexpr (S) return *x;
  else return __ldcg(x);
}
template <bool S, class T>
__device__ __forceinline__ void jst(T* x, T v) {
  if constexpr (S) *x = v;
  else __stcg(x, v);
}

// One warp rotates columns (a, b) of G (p rows) and V (q rows) unless they
// are orthogonal to tol.  float64 reads and keeps the squared norms na, nb;
// float32 computes them with the inner product.
template <bool S, class T>
__device__ __forceinline__ bool jpc_pair(T* ar, T* ai, T* br, T* bi, T* var, T* vai, T* vbr,
                                         T* vbi, T* na, T* nb, int p, int q, int lane, T tol) {
  constexpr bool keep = sizeof(T) == 8;
  T alpha = 0, beta = 0, gr = 0, gi = 0;
  if (keep) {
    alpha = jld<S>(na);
    beta = jld<S>(nb);
    alpha = alpha > T(0) ? alpha : T(0);
    beta = beta > T(0) ? beta : T(0);
  }
  for (int r = lane; r < p; r += 32) {
    const T xr = jld<S>(ar + r), xi = jld<S>(ai + r), yr = jld<S>(br + r), yi = jld<S>(bi + r);
    if (!keep) {
      alpha += xr * xr + xi * xi;
      beta += yr * yr + yi * yi;
    }
    gr += xr * yr + xi * yi;
    gi += xr * yi - xi * yr;
  }
  if (!keep) {
    alpha = warp_sum_t(alpha);
    beta = warp_sum_t(beta);
  }
  gr = warp_sum_t(gr);
  gi = warp_sum_t(gi);
  const T g2 = gr * gr + gi * gi;
  if (!(g2 > tol * tol * alpha * beta) || g2 == T(0)) return false;
  T cs, sn, er, ei, tg;
  rotation(alpha, beta, gr, gi, g2, cs, sn, er, ei, tg);
  if (keep && lane == 0) {
    jst<S>(na, alpha - tg);
    jst<S>(nb, beta + tg);
  }
#pragma unroll 4
  for (int r = lane; r < p; r += 32) {
    const T xr = jld<S>(ar + r), xi = jld<S>(ai + r);
    const T ur = jld<S>(br + r), ui = jld<S>(bi + r);
    const T yr = ur * er - ui * ei, yi = ur * ei + ui * er;
    jst<S>(ar + r, cs * xr - sn * yr);
    jst<S>(ai + r, cs * xi - sn * yi);
    jst<S>(br + r, sn * xr + cs * yr);
    jst<S>(bi + r, sn * xi + cs * yi);
  }
#pragma unroll 4
  for (int r = lane; r < q; r += 32) {
    const T xr = jld<S>(var + r), xi = jld<S>(vai + r);
    const T ur = jld<S>(vbr + r), ui = jld<S>(vbi + r);
    const T yr = ur * er - ui * ei, yi = ur * ei + ui * er;
    jst<S>(var + r, cs * xr - sn * yr);
    jst<S>(vai + r, cs * xi - sn * yi);
    jst<S>(vbr + r, sn * xr + cs * yr);
    jst<S>(vbi + r, sn * xi + cs * yi);
  }
  return true;
}

// Shared memory of a SMEM cluster CTA (the round's 2 bs columns of G and V
// and their norms), or 0 when it does not fit.
template <class T>
size_t jacobi_cluster_smem(int p, int q) {
  const size_t bs = size_t((q + JPC_BLOCKS - 1) / JPC_BLOCKS);
  const size_t bytes = (4 * bs * size_t(p) + 4 * bs * size_t(q) + 2 * bs) * sizeof(T);
  return bytes <= size_t(200) * 1024 ? bytes : 0;
}

// One-sided Jacobi of slice blockIdx.x / JPC with the flags of jacobi_kernel
// (JAC_INIT_V, JAC_NORMALIZE): the result of jacobi_kernel<T>, one cluster per
// slice.  nrm_ws: q values per slice of scratch (float64 only).
template <class T, bool S>
__global__ void __cluster_dims__(JPC, 1, 1) __launch_bounds__(JPC_THREADS)
    jacobi_cluster_kernel(T* g_re, T* g_im, int64_t sG, T* v_re, T* v_im, int64_t sV, T* nrm_ws,
                          T* sig, int p, int q, int max_sweeps, const int* real_flags,
                          int32_t* status, int flags) {
  extern __shared__ __align__(16) unsigned char jpc_smem[];
  constexpr bool keep = sizeof(T) == 8;
  const int c = int(jpc_rank());
  const int64_t b = blockIdx.x / JPC;
  T* const Gr = g_re + b * sG;
  T* const Gi = g_im + b * sG;
  T* const Vr = v_re + b * sV;
  T* const Vi = v_im + b * sV;
  T* const nrm = keep ? nrm_ws + b * q : nullptr;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = JPC_THREADS / 32;
  const int bs = (q + JPC_BLOCKS - 1) / JPC_BLOCKS;
  const int bs2 = bs + (bs & 1);   // positions of the internal round-robin
  // the round's block pair in shared memory: local column l < bs is column
  // i0 + l of the slice, l >= bs column j0 + l - bs
  T* const sGr = reinterpret_cast<T*>(jpc_smem);
  T* const sGi = sGr + 2 * bs * p;
  T* const sVr = sGi + 2 * bs * p;
  T* const sVi = sVr + 2 * bs * q;
  T* const sN = sVi + 2 * bs * q;
  __shared__ int rotated, any_s;

  const bool real = real_flags ? real_flags[b] != 0 : false;
  for (int j = c; j < q; j += JPC) {
    if (flags & JAC_INIT_V) {
      for (int r = tid; r < q; r += JPC_THREADS) {
        Vr[int64_t(j) * q + r] = r == j ? T(1) : T(0);
        Vi[int64_t(j) * q + r] = T(0);
      }
    } else if (real) {
      for (int r = tid; r < q; r += JPC_THREADS) Vi[int64_t(j) * q + r] = T(0);
    }
    if (real)
      for (int r = tid; r < p; r += JPC_THREADS) Gi[int64_t(j) * p + r] = T(0);
  }
  T tol = T(8) * Eps<T>::v * sqrt(T(p));
  if (tol < T(keep ? 1e-13 : 1e-6)) tol = T(keep ? 1e-13 : 1e-6);
  __threadfence();
  jpc_cluster_sync();

  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    if (keep) {
      for (int j = c + JPC * warp; j < q; j += JPC * nw) {
        const T* xr = Gr + int64_t(j) * p;
        const T* xi = Gi + int64_t(j) * p;
        T acc = 0;
        for (int r = lane; r < p; r += 32) {
          const T u = __ldcg(xr + r), v = __ldcg(xi + r);
          acc += u * u + v * v;
        }
        acc = warp_sum_t(acc);
        if (lane == 0) __stcg(nrm + j, acc);
      }
      __threadfence();
    }
    jpc_cluster_sync();
    bool rot = false;
    for (int round = 0; round < JPC_BLOCKS - 1; ++round) {
      int I, J;
      if (c == 0) {
        I = JPC_BLOCKS - 1;
        J = round;
      } else {
        I = (round + c) % (JPC_BLOCKS - 1);
        J = (round - c + JPC_BLOCKS - 1) % (JPC_BLOCKS - 1);
      }
      const int i0 = I * bs, j0 = J * bs;
      auto gcol = [&](int l) { return l < bs ? i0 + l : j0 + l - bs; };
      if (S) {
        for (int e = tid; e < 2 * bs * p; e += JPC_THREADS) {
          const int l = e / p, g = gcol(l);
          if (g < q) {
            const int64_t o = int64_t(g) * p + (e - l * p);
            sGr[e] = __ldcg(Gr + o);
            sGi[e] = __ldcg(Gi + o);
          }
        }
        for (int e = tid; e < 2 * bs * q; e += JPC_THREADS) {
          const int l = e / q, g = gcol(l);
          if (g < q) {
            const int64_t o = int64_t(g) * q + (e - l * q);
            sVr[e] = __ldcg(Vr + o);
            sVi[e] = __ldcg(Vi + o);
          }
        }
        if (keep)
          for (int l = tid; l < 2 * bs; l += JPC_THREADS)
            if (gcol(l) < q) sN[l] = __ldcg(nrm + gcol(l));
        __syncthreads();
      }
      // rotates local columns (la, lb) of the block pair
      auto pair = [&](int la, int lb) {
        int ga = gcol(la), gb = gcol(lb);
        if (ga >= q || gb >= q) return;
        if (ga > gb) {
          const int t = la; la = lb; lb = t;
          const int u = ga; ga = gb; gb = u;
        }
        if (S)
          rot |= jpc_pair<true, T>(sGr + la * p, sGi + la * p, sGr + lb * p, sGi + lb * p,
                                   sVr + la * q, sVi + la * q, sVr + lb * q, sVi + lb * q,
                                   sN + la, sN + lb, p, q, lane, tol);
        else
          rot |= jpc_pair<false, T>(Gr + int64_t(ga) * p, Gi + int64_t(ga) * p,
                                    Gr + int64_t(gb) * p, Gi + int64_t(gb) * p,
                                    Vr + int64_t(ga) * q, Vi + int64_t(ga) * q,
                                    Vr + int64_t(gb) * q, Vi + int64_t(gb) * q,
                                    keep ? nrm + ga : nullptr, keep ? nrm + gb : nullptr, p, q,
                                    lane, tol);
      };
      if (round == 0) {
        // internal pairs of both blocks: bs2 - 1 steps of bs2 / 2 pairs each
        for (int step = 0; step < bs2 - 1; ++step) {
          for (int k = warp; k < bs2; k += nw) {
            const int off = k < bs2 / 2 ? 0 : bs;
            const int i = k < bs2 / 2 ? k : k - bs2 / 2;
            int x, y;
            if (i == 0) {
              x = bs2 - 1;
              y = step;
            } else {
              x = (step + i) % (bs2 - 1);
              y = (step - i + bs2 - 1) % (bs2 - 1);
            }
            if (x < bs && y < bs) pair(off + x, off + y);
          }
          __syncthreads();
        }
      }
      // cross pairs: step t pairs column i of block I with (i + t) mod bs of J
      for (int t = 0; t < bs; ++t) {
        for (int i = warp; i < bs; i += nw) pair(i, bs + (i + t) % bs);
        __syncthreads();
      }
      if (S) {
        for (int e = tid; e < 2 * bs * p; e += JPC_THREADS) {
          const int l = e / p, g = gcol(l);
          if (g < q) {
            const int64_t o = int64_t(g) * p + (e - l * p);
            __stcg(Gr + o, sGr[e]);
            __stcg(Gi + o, sGi[e]);
          }
        }
        for (int e = tid; e < 2 * bs * q; e += JPC_THREADS) {
          const int l = e / q, g = gcol(l);
          if (g < q) {
            const int64_t o = int64_t(g) * q + (e - l * q);
            __stcg(Vr + o, sVr[e]);
            __stcg(Vi + o, sVi[e]);
          }
        }
        if (keep)
          for (int l = tid; l < 2 * bs; l += JPC_THREADS)
            if (gcol(l) < q) __stcg(nrm + gcol(l), sN[l]);
        __syncthreads();   // the next round's loads overwrite the copies
      }
      if (rot && lane == 0) rotated = 1;
      __threadfence();
      jpc_cluster_sync();
    }
    if (tid == 0) {
      int any = 0;
      for (int r = 0; r < JPC; ++r) any |= jpc_peek(&rotated, unsigned(r));
      any_s = any;
    }
    jpc_cluster_sync();   // every CTA has read every flag before any resets its own
    if (!any_s) break;
  }
  if (sweep >= max_sweeps && c == 0 && tid == 0 && status) atomicOr(status, TP_DEV_NOCONV);
  // singular values and (optionally) unit left vectors
  for (int j = c + JPC * warp; j < q; j += JPC * nw) {
    T* xr = Gr + int64_t(j) * p;
    T* xi = Gi + int64_t(j) * p;
    T acc = 0;
    for (int r = lane; r < p; r += 32) {
      const T u = __ldcg(xr + r), v = __ldcg(xi + r);
      acc += u * u + v * v;
    }
    const T s = sqrt(warp_sum_t(acc));
    if (lane == 0) sig[b * q + j] = s;
    if (flags & JAC_NORMALIZE) {
      const T inv = s > T(0) ? T(1) / s : T(0);
      for (int r = lane; r < p; r += 32) {
        xr[r] = __ldcg(xr + r) * inv;
        xi[r] = __ldcg(xi + r) * inv;
      }
    }
  }
}

// Gathers slice b of the half spectrum into the work matrix:
// G = X_hat_k (n1 x n2) when n1 >= n2, else G = X_hat_k^H (n2 x n1).
template <class T>
__global__ void load_work_kernel(const float* __restrict__ xr, const float* __restrict__ xi,
                                 int64_t n1, int64_t n2, int64_t h, bool transpose,
                                 T* __restrict__ gr, T* __restrict__ gi) {
  const int64_t per = n1 * n2;
  const int64_t total = per * h;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = e / per, r = e - k * per;
    const int64_t i = r % n1, j = r / n1;
    const float vr = xr[e], vi = xi[e];
    if (!transpose) {
      gr[e] = T(vr);
      gi[e] = T(vi);
    } else {   // G(j, i) = conj(X(i, j)), G is n2 x n1
      const int64_t o = k * per + j + n2 * i;
      gr[o] = T(vr);
      gi[o] = -T(vi);
    }
  }
}

// Sorts each slice's singular triplets by descending value and writes the
// half-spectrum factors: Uh (n1 x m), Sh (m x m, diagonal), Vh (n2 x m).
// `left` is the matrix holding the n1-side vectors (G or V of the Jacobi),
// `right` the n2-side one; `left_ld`/`right_ld` their leading dimensions.
__global__ void write_factors_kernel(const double* __restrict__ lr, const double* __restrict__ li,
                                     int64_t sL, int64_t left_ld,
                                     const double* __restrict__ rr, const double* __restrict__ ri,
                                     int64_t sR, int64_t right_ld, const double* __restrict__ sig,
                                     int q, int64_t n1, int64_t n2, int m,
                                     float* __restrict__ ur, float* __restrict__ ui,
                                     float* __restrict__ sr, float* __restrict__ si,
                                     float* __restrict__ vr, float* __restrict__ vi) {
  extern __shared__ int order[];   // order[rank] = column
  const int64_t k = blockIdx.x;
  const double* s = sig + k * q;
  for (int j = threadIdx.x; j < q; j += blockDim.x) {
    const double sj = s[j];
    int rank = 0;
    for (int l = 0; l < q; ++l) {
      const double sl = s[l];
      rank += (sl > sj) || (sl == sj && l < j);
    }
    order[rank] = j;
  }
  __syncthreads();
  const double* Lr = lr + k * sL;
  const double* Li = li + k * sL;
  const double* Rr = rr + k * sR;
  const double* Ri = ri + k * sR;
  for (int64_t e = threadIdx.x; e < n1 * m; e += blockDim.x) {
    const int64_t i = e % n1, c = e / n1;
    const int j = order[c];
    ur[k * n1 * m + e] = float(Lr[i + left_ld * j]);
    ui[k * n1 * m + e] = float(Li[i + left_ld * j]);
  }
  for (int64_t e = threadIdx.x; e < n2 * m; e += blockDim.x) {
    const int64_t i = e % n2, c = e / n2;
    const int j = order[c];
    vr[k * n2 * m + e] = float(Rr[i + right_ld * j]);
    vi[k * n2 * m + e] = float(Ri[i + right_ld * j]);
  }
  for (int64_t e = threadIdx.x; e < int64_t(m) * m; e += blockDim.x) {
    const int64_t i = e % m, c = e / m;
    sr[k * m * m + e] = (i == c) ? float(s[order[c]]) : 0.f;
    si[k * m * m + e] = 0.f;
  }
}

__global__ void real_flags_kernel(int* flags, int64_t h, int64_t n3) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < h) flags[k] = (k == 0 || (n3 % 2 == 0 && k == h - 1)) ? 1 : 0;
}

// Batched complex GEMM in float64 (inputs float or double, planar):
// C_b (M x N) = op(A_b) B_b with op(A) = A (M x K, element (m, k) at m + lda k)
// or A^H (A stored K x M, element (k, m) at k + lda m); B (K x N) at k + ldb n;
// C at m + ldc n.  16 x 16 output tiles, one element per thread, K staged
// through shared memory in chunks of 16.
constexpr int ZT = 16;
template <class TA, class TB>
__global__ void __launch_bounds__(ZT * ZT) zgemm64_kernel(
    const TA* __restrict__ ar, const TA* __restrict__ ai, int64_t sA, int64_t lda, int conj_a,
    const TB* __restrict__ br, const TB* __restrict__ bi, int64_t sB, int64_t ldb,
    double* __restrict__ cr, double* __restrict__ ci, int64_t sC, int64_t ldc, int M, int N,
    int K) {
  __shared__ double As_r[ZT][ZT + 1], As_i[ZT][ZT + 1], Bs_r[ZT][ZT + 1], Bs_i[ZT][ZT + 1];
  const int64_t b = blockIdx.z;
  const int tx = threadIdx.x % ZT, ty = threadIdx.x / ZT;   // tx: row m, ty: column n
  const int m0 = blockIdx.x * ZT, n0 = blockIdx.y * ZT;
  ar += b * sA;
  ai += b * sA;
  br += b * sB;
  bi += b * sB;
  double accr = 0.0, acci = 0.0;
  for (int k0 = 0; k0 < K; k0 += ZT) {
    {   // A tile: As[m][k] = op(A)(m0 + m, k0 + k); thread (tx, ty) loads m = tx, k = ty
      const int m = m0 + tx, k = k0 + ty;
      double vr = 0.0, vi = 0.0;
      if (m < M && k < K) {
        if (conj_a) {
          vr = double(ar[k + lda * m]);
          vi = -double(ai[k + lda * m]);
        } else {
          vr = double(ar[m + lda * k]);
          vi = double(ai[m + lda * k]);
        }
      }
      As_r[tx][ty] = vr;
      As_i[tx][ty] = vi;
    }
    {   // B tile: Bs[k][n]; thread loads k = tx, n = ty
      const int k = k0 + tx, n = n0 + ty;
      double vr = 0.0, vi = 0.0;
      if (k < K && n < N) {
        vr = double(br[k + ldb * n]);
        vi = double(bi[k + ldb * n]);
      }
      Bs_r[tx][ty] = vr;
      Bs_i[tx][ty] = vi;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ZT; ++k) {
      const double xr = As_r[tx][k], xi = As_i[tx][k], yr = Bs_r[k][ty], yi = Bs_i[k][ty];
      accr = fma(xr, yr, fma(-xi, yi, accr));
      acci = fma(xr, yi, fma(xi, yr, acci));
    }
    __syncthreads();
  }
  const int m = m0 + tx, n = n0 + ty;
  if (m < M && n < N) {
    cr[b * sC + m + ldc * n] = accr;
    ci[b * sC + m + ldc * n] = acci;
  }
}

template <class TA, class TB>
void zgemm64(const TA* ar, const TA* ai, int64_t sA, int64_t lda, bool conj_a, const TB* br,
             const TB* bi, int64_t sB, int64_t ldb, double* cr, double* ci, int64_t sC,
             int64_t ldc, int M, int N, int K, int batch, cudaStream_t st) {
  const dim3 grid(unsigned((M + ZT - 1) / ZT), unsigned((N + ZT - 1) / ZT), unsigned(batch));
  zgemm64_kernel<TA, TB><<<grid, ZT * ZT, 0, st>>>(ar, ai, sA, lda, conj_a ? 1 : 0, br, bi, sB,
                                                   ldb, cr, ci, sC, ldc, M, N, K);
}

// T <- (3 I - T) / 2 for q x q matrices (the Newton-Schulz factor).
__global__ void ns_factor_kernel(double* tr, double* ti, int q, int64_t total) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e % (int64_t(q) * q);
    const bool diag = (r % q) == (r / q);
    tr[e] = (diag ? 1.5 : 0.0) - 0.5 * tr[e];
    ti[e] = -0.5 * ti[e];
  }
}

unsigned grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > int64_t(sm_count()) * 16) b = int64_t(sm_count()) * 16;
  if (b < 1) b = 1;
  return unsigned(b);
}

// Shared memory a Jacobi CTA needs to hold G and V, or 0 when they do not fit.
template <class T>
size_t jacobi_smem(int p, int q) {
  const size_t bytes = (2 * size_t(p) * q + 2 * size_t(q) * q) * sizeof(T);
  return bytes <= size_t(200) * 1024 ? bytes : 0;
}

template <class T>
int jacobi_launch(T* gr, T* gi, int64_t sG, T* vr, T* vi, int64_t sV, T* sig, int p, int q,
                  int batch, int max_sweeps, const int* real_flags, int32_t* status, int flags,
                  cudaStream_t st) {
  if (batch <= 0 || q <= 0) return TP_OK;
  if (q > JAC_MAX_Q) {
    set_error("jacobi: %d columns, more than %d", q, JAC_MAX_Q);
    return TP_EUNSUPPORTED;
  }
  const size_t smem = jacobi_smem<T>(p, q);
  if (smem) {
    flags |= JAC_SMEM;
    TP_SET_SMEM(jacobi_kernel<T>, smem);
  }
  {
    KernelScope ks(sizeof(T) == 4 ? "jacobi_f32" : "jacobi_svd", st);
    jacobi_kernel<T><<<unsigned(batch), SVD_THREADS, smem, st>>>(
        gr, gi, sG, vr, vi, sV, sig, p, q, max_sweeps, real_flags, status, flags);
  }
  return launch_status("jacobi_kernel");
}

// Whether the device can place a cluster of JPC CTAs at all (a partitioned
// GPU may not): asked once per device; an error of the query itself leaves
// the cluster form on (the query, not the launch, is what failed).
bool cluster_fits() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];   // 0 unknown, 1 fits, 2 does not
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return true;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(JPC, 1, 1);
    cfg.blockDim = dim3(JPC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;   // the cluster size comes from the kernel's __cluster_dims__
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(
        &n, (const void*)jacobi_cluster_kernel<double, false>, &cfg);
    if (e != cudaSuccess) cudaGetLastError();
    v = (e == cudaSuccess && n < 1) ? 2 : 1;
    cache[dev].store(v, std::memory_order_relaxed);
  }
  return v == 1;
}

// A cluster of CTAs per slice pays when the slices are fewer than the SMs and
// wide enough to give every CTA of the cluster a block pair of columns.
bool use_cluster(int q, int batch) {
  return q >= 2 * JPC_BLOCKS && q <= JAC_MAX_Q && batch < sm_count() && cluster_fits();
}

template <class T>
int jacobi_cluster_launch(T* gr, T* gi, int64_t sG, T* vr, T* vi, int64_t sV, T* nrm, T* sig,
                          int p, int q, int batch, int max_sweeps, const int* real_flags,
                          int32_t* status, int flags, cudaStream_t st) {
  if (batch <= 0 || q <= 0) return TP_OK;
  const size_t smem = jacobi_cluster_smem<T>(p, q);
  const unsigned grid = unsigned(batch) * JPC;
  {
    KernelScope ks(sizeof(T) == 4 ? "jacobi_f32" : "jacobi_svd", st);
    if (smem) {
      if (int rc = set_smem_attr((const void*)jacobi_cluster_kernel<T, true>, smem,
                                 "jacobi_cluster_kernel"))
        return rc;
      jacobi_cluster_kernel<T, true><<<grid, JPC_THREADS, smem, st>>>(
          gr, gi, sG, vr, vi, sV, nrm, sig, p, q, max_sweeps, real_flags, status, flags);
    } else {
      jacobi_cluster_kernel<T, false><<<grid, JPC_THREADS, 0, st>>>(
          gr, gi, sG, vr, vi, sV, nrm, sig, p, q, max_sweeps, real_flags, status, flags);
    }
  }
  return launch_status("jacobi_cluster_kernel");
}

}  // namespace

// float32 one-sided Jacobi from V = I (init_v) or from the given V (then G
// must be the work matrix times that V); G is left rotated, not normalised.
int jacobi_float_launch(float* gr, float* gi, int64_t sG, float* vr, float* vi, int64_t sV,
                        float* sig, int p, int q, int batch, int max_sweeps,
                        const int* real_flags, int32_t* status, bool init_v, cudaStream_t st) {
  return jacobi_launch<float>(gr, gi, sG, vr, vi, sV, sig, p, q, batch, max_sweeps, real_flags,
                              status, init_v ? JAC_INIT_V : 0, st);
}

// Whether jacobi_float_cluster_launch takes a batch of p x q slices (fewer
// slices than SMs, q >= 32).
bool jacobi_cluster_applies(int q, int batch) { return use_cluster(q, batch); }

// jacobi_float_launch with a thread-block cluster per slice.
int jacobi_float_cluster_launch(float* gr, float* gi, int64_t sG, float* vr, float* vi,
                                int64_t sV, float* sig, int p, int q, int batch, int max_sweeps,
                                const int* real_flags, int32_t* status, bool init_v,
                                cudaStream_t st) {
  return jacobi_cluster_launch<float>(gr, gi, sG, vr, vi, sV, nullptr, sig, p, q, batch,
                                      max_sweeps, real_flags, status, init_v ? JAC_INIT_V : 0, st);
}

// C_b = op(A_b) B_b in float64 from float32 planes (see zgemm64_kernel).
int zgemm64_from_float(const float* ar, const float* ai, int64_t sA, int64_t lda, bool conj_a,
                       const float* br, const float* bi, int64_t sB, int64_t ldb, double* cr,
                       double* ci, int64_t sC, int64_t ldc, int M, int N, int K, int batch,
                       cudaStream_t st) {
  if (batch <= 0 || M <= 0 || N <= 0) return TP_OK;
  {
    KernelScope ks("zgemm64", st);
    zgemm64<float, float>(ar, ai, sA, lda, conj_a, br, bi, sB, ldb, cr, ci, sC, ldc, M, N, K,
                          batch, st);
  }
  return launch_status("zgemm64_kernel");
}

int jacobi_double_launch(double* gr, double* gi, int64_t sG, double* vr, double* vi, int64_t sV,
                         double* sig, int p, int q, int batch, int max_sweeps,
                         const int* real_flags, int32_t* status, cudaStream_t st) {
  return jacobi_launch<double>(gr, gi, sG, vr, vi, sV, sig, p, q, batch, max_sweeps, real_flags,
                               status, JAC_INIT_V | JAC_NORMALIZE, st);
}


// Float64-quality SVD of every p x q work matrix op(X_b) (op = identity or
// the conjugate transpose of the float32 slice X_b, leading dimension ldx,
// slice stride sX): steps 1-4 of the header.  F (p x q float32) must hold the
// work matrix on entry and is overwritten.  On exit G (p x q) holds the unit
// left singular vectors, W (q x q) the right ones, sig the singular values
// (unsorted).  Q (q x q float32), qsig (q float32) and T (q x q float64) are
// scratch.
int hybrid_svd(const float* xr, const float* xi, int64_t sX, int64_t ldx, bool conj, int p, int q,
               int batch, float* fr, float* fi, float* qr, float* qi, float* qsig, double* tr,
               double* ti, double* gr, double* gi, double* wr, double* wi, double* sig,
               const int* real_flags, int max_sweeps, int32_t* status, cudaStream_t st,
               bool polish) {
  int rc;
  const int64_t pq = int64_t(p) * q, qq = int64_t(q) * q;
  // 1. float32 sweeps (with the polish, a cluster of singular values at the
  //    float32 rounding floor may stall here and step 4 decides convergence;
  //    without it this step does)
  //    (fewer slices than SMs: a cluster of CTAs per slice)
  if ((rc = use_cluster(q, batch)
                ? jacobi_cluster_launch<float>(fr, fi, pq, qr, qi, qq, nullptr, qsig, p, q, batch,
                                               max_sweeps, real_flags, polish ? nullptr : status,
                                               JAC_INIT_V, st)
                : jacobi_launch<float>(fr, fi, pq, qr, qi, qq, qsig, p, q, batch, max_sweeps,
                                       real_flags, polish ? nullptr : status, JAC_INIT_V, st)))
    return rc;
  {
    KernelScope ks("svd_refine", st);
    // 2. W = Q (3 I - Q^H Q) / 2
    zgemm64<float, float>(qr, qi, qq, q, true, qr, qi, qq, q, tr, ti, qq, q, q, q, q, batch, st);
    ns_factor_kernel<<<grid_of(qq * batch), 256, 0, st>>>(tr, ti, q, qq * batch);
    zgemm64<float, double>(qr, qi, qq, q, false, tr, ti, qq, q, wr, wi, qq, q, q, q, q, batch, st);
    // 3. G = op(X) W
    zgemm64<float, double>(xr, xi, sX, ldx, conj, wr, wi, qq, q, gr, gi, pq, p, p, q, q, batch, st);
  }
  note_launches(3);
  if ((rc = launch_status("svd_refine"))) return rc;
  // 4. float64 sweeps from W to float64 convergence: from columns already
  //    orthogonal to float32 accuracy each sweep squares the residual, so two
  //    or three sweeps suffice, more only for clusters of singular values at
  //    the float32 rounding floor (rank-deficient input); the sweep cap and
  //    TP_DEV_NOCONV apply here.  Without the polish: no sweeps, only the
  //    column norms (singular values) and unit columns of G.  Fewer slices
  //    than SMs: a cluster of CTAs per slice (T is free scratch by now).
  if (polish && use_cluster(q, batch))
    return jacobi_cluster_launch<double>(gr, gi, pq, wr, wi, qq, tr, sig, p, q, batch, max_sweeps,
                                         real_flags, status, JAC_NORMALIZE, st);
  return jacobi_launch<double>(gr, gi, pq, wr, wi, qq, sig, p, q, batch, polish ? max_sweeps : 0,
                               real_flags, polish ? status : nullptr, JAC_NORMALIZE, st);
}

size_t tsvd_ws(int64_t n1, int64_t n2, int64_t n3) {
  const size_t h = size_t(half_len(n3));
  const size_t m = size_t(n1 < n2 ? n1 : n2);
  const size_t p = size_t(n1 < n2 ? n2 : n1);
  return 2 * ws_bytes(size_t(n1) * n2 * h, 4)      // X_hat
         + 2 * ws_bytes(p * m * h, 4)              // float32 work matrix
         + 2 * ws_bytes(m * m * h, 4)              // float32 rotations
         + ws_bytes(m * h, 4)                      // float32 column norms
         + 2 * ws_bytes(m * m * h, 8)              // Newton-Schulz factor
         + 2 * ws_bytes(p * m * h, 8)              // G (float64)
         + 2 * ws_bytes(m * m * h, 8)              // V of the Jacobi (float64)
         + ws_bytes(m * h, 8)                      // singular values
         + ws_bytes(h, 4)                          // real-slice flags
         + 2 * ws_bytes(size_t(n1) * m * h, 4)     // U_hat
         + 2 * ws_bytes(m * m * h, 4)              // S_hat
         + 2 * ws_bytes(size_t(n2) * m * h, 4);    // V_hat
}

int tsvd_run(const float* X, int64_t n1, int64_t n2, int64_t n3, float* U, float* S, float* V,
             const tp_opts* opts, cudaStream_t st) {
  const int64_t h = half_len(n3);
  const int64_t m = n1 < n2 ? n1 : n2;
  const int64_t p = n1 < n2 ? n2 : n1;
  const bool transpose = n1 < n2;
  Arena ws;
  int rc = acquire_workspace(opts, tsvd_ws(n1, n2, n3), &ws);
  if (rc) return rc;
  int32_t* status = opts ? opts->status : nullptr;
  float* Xr = ws.take<float>(size_t(n1) * n2 * h);
  float* Xi = ws.take<float>(size_t(n1) * n2 * h);
  float* Fr = ws.take<float>(size_t(p) * m * h);
  float* Fi = ws.take<float>(size_t(p) * m * h);
  float* Qr = ws.take<float>(size_t(m) * m * h);
  float* Qi = ws.take<float>(size_t(m) * m * h);
  float* fsig = ws.take<float>(size_t(m) * h);
  double* Tr = ws.take<double>(size_t(m) * m * h);
  double* Ti = ws.take<double>(size_t(m) * m * h);
  double* Gr = ws.take<double>(size_t(p) * m * h);
  double* Gi = ws.take<double>(size_t(p) * m * h);
  double* Wr = ws.take<double>(size_t(m) * m * h);
  double* Wi = ws.take<double>(size_t(m) * m * h);
  double* sig = ws.take<double>(size_t(m) * h);
  int* flags = ws.take<int>(size_t(h));
  float* Ur = ws.take<float>(size_t(n1) * m * h);
  float* Ui = ws.take<float>(size_t(n1) * m * h);
  float* Sr = ws.take<float>(size_t(m) * m * h);
  float* Si = ws.take<float>(size_t(m) * m * h);
  float* Vr = ws.take<float>(size_t(n2) * m * h);
  float* Vi = ws.take<float>(size_t(n2) * m * h);

  DftGather gx{X, n1 * n2, 1, 1, 0, n1 * n2, nullptr, nullptr, nullptr, 0, n3, Xr, Xi,
               n1 * n2, n1 * n2, nullptr, nullptr, 0};
  if ((rc = launch_rdft(gx, st))) return rc;
  {
    KernelScope ks("svd_prep", st);
    load_work_kernel<float><<<grid_of(n1 * n2 * h), 256, 0, st>>>(Xr, Xi, n1, n2, h, transpose,
                                                                  Fr, Fi);
    real_flags_kernel<<<unsigned((h + 255) / 256), 256, 0, st>>>(flags, h, n3);
  }
  note_launches(1);
  if ((rc = launch_status("svd_prep"))) return rc;
  const int sweeps = (opts && opts->max_sweeps > 0) ? opts->max_sweeps : 30;
  // slices of at most 4096 entries (and 256 x 96): no float64 sweeps; the
  // vectors of G are re-orthonormalised by a float32 Householder QR in
  // descending order instead.  The QR's own rounding grows as
  // u32 sqrt(p m) (1.2e-5 of reconstruction at 256 x 96 against 3e-6 at
  // 64 x 48), so larger slices keep the float64 sweeps.
  const bool fast = p <= 256 && m <= 96 && p * m <= 4096;
  if ((rc = hybrid_svd(Xr, Xi, n1 * n2, n1, transpose, int(p), int(m), int(h), Fr, Fi, Qr, Qi, fsig,
                       Tr, Ti, Gr, Gi, Wr, Wi, sig, flags, sweeps, status, st, !fast)))
    return rc;
  {
    KernelScope ks("svd_factors", st);
    // n1 >= n2: G holds U (n1 x m), Jacobi V holds V (n2 x m).  n1 < n2: the
    // roles swap (the Jacobi ran on X_hat^H).
    if (!transpose)
      write_factors_kernel<<<unsigned(h), 256, size_t(m) * sizeof(int), st>>>(
          Gr, Gi, p * m, p, Wr, Wi, m * m, m, sig, int(m), n1, n2, int(m), Ur, Ui, Sr, Si, Vr, Vi);
    else
      write_factors_kernel<<<unsigned(h), 256, size_t(m) * sizeof(int), st>>>(
          Wr, Wi, m * m, m, Gr, Gi, p * m, p, sig, int(m), n1, n2, int(m), Ur, Ui, Sr, Si, Vr, Vi);
  }
  if ((rc = launch_status("write_factors_kernel"))) return rc;
  if (fast) {
    // the G side (U when n1 >= n2, else V), sorted by descending singular
    // value: its float32-converged columns are orthogonal to about
    // u32 s_1 / (s_a s_b) -- loose only where s is small, and arbitrary for a
    // cluster at the rounding floor (rank-deficient input); the QR keeps the
    // leading columns and completes the rest to an orthonormal set
    const int64_t rows = transpose ? n2 : n1;
    if ((rc = householder_orth_launch(transpose ? Vr : Ur, transpose ? Vi : Ui, rows * m,
                                      int(rows), int(m), h, true, st)))
      return rc;
  }
  if ((rc = launch_irdft(Ur, Ui, n1 * m, n1 * m, n3, U, st))) return rc;
  if ((rc = launch_irdft(Sr, Si, m * m, m * m, n3, S, st))) return rc;
  return launch_irdft(Vr, Vi, n2 * m, n2 * m, n3, V, st);
}

}  // namespace tp
