// Jacobi rotation parameters shared by the one-sided (svd.cu) and two-sided
// (rsvd.cu) Jacobi kernels.
#pragma once

#include "tp_internal.cuh"

namespace tp {
namespace jrot {

// Jacobi rotation of a pair from its two diagonal terms alpha, beta (the
// squared column norms of a one-sided sweep, or the diagonal entries of a
// Hermitian matrix) and its off-diagonal term gamma = gr + i gi, g2 =
// gr^2 + gi^2 > 0: with zeta = (beta - alpha) / (2 |gamma|),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t,
// and e^{-i phi} = conj(gamma) / |gamma|.
// tg = t |gamma|: the change of the two squared norms, ||a'||^2 = alpha - tg
// and ||b'||^2 = beta + tg.
__device__ __forceinline__ void rotation(float alpha, float beta, float gr, float gi, float g2,
                                         float& cs, float& sn, float& er, float& ei, float& tg) {
  const float g = sqrtf(g2);
  const float zeta = (beta - alpha) / (2.f * g);
  const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  cs = 1.f / sqrtf(1.f + t * t);
  sn = cs * t;
  er = gr / g;
  ei = -gi / g;
  tg = t * g;
}
__device__ __forceinline__ void rotation(float alpha, float beta, float gr, float gi, float g2,
                                         float& cs, float& sn, float& er, float& ei) {
  float tg;
  rotation(alpha, beta, gr, gi, g2, cs, sn, er, ei, tg);
}

// float64: the tangent only steers convergence, so it is formed in float32
// (after scaling by a power of two into float range); what must hold to
// float64 accuracy is that the rotation is unitary, c^2 + s^2 = 1 and
// |e^{-i phi}| = 1, which one Newton step x (3 - v x^2) / 2 on a float32
// reciprocal square root gives (relative error ~(2^-23)^2).  This keeps the
// slow float64 divide and square root out of the sweep.
__device__ __forceinline__ double rsqrt_nr(double v, double seed) {
  return seed * (1.5 - 0.5 * v * seed * seed);
}
__device__ __forceinline__ void rotation(double alpha, double beta, double gr, double gi,
                                         double g2, double& cs, double& sn, double& er,
                                         double& ei, double& tg) {
  int e;
  const double big = fabs(alpha) > fabs(beta) ? fabs(alpha) : fabs(beta);
  frexp(big, &e);
  e += (e & 1);                          // even, so that 2^(e/2) is exact
  const double sc = ldexp(1.0, -e);      // alpha, beta scaled to <= 1, g2 by sc^2
  const float af = float(alpha * sc), bf = float(beta * sc), g2f = float(g2 * sc * sc);
  if (!(g2f > 1e-30f)) {   // |gamma| below float range after scaling: exact float64 path
    const double g = sqrt(g2);
    const double zeta = (beta - alpha) / (2.0 * g);
    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    cs = 1.0 / sqrt(1.0 + t * t);
    sn = cs * t;
    er = gr / g;
    ei = -gi / g;
    tg = t * g;
    return;
  }
  const float gf = sqrtf(g2f);
  const float zeta = (bf - af) / (2.f * gf);
  const float tf = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  const double t = double(tf);
  const double one_t2 = 1.0 + t * t;
  cs = rsqrt_nr(one_t2, double(rsqrtf(float(one_t2))));
  sn = cs * t;
  // g2 = g2s / sc^2, so 1/|gamma| = rsqrt(g2s) * sc
  const double g2s = g2 * sc * sc;
  const double rinv = rsqrt_nr(g2s, double(rsqrtf(float(g2s)))) * sc;
  er = gr * rinv;
  ei = -gi * rinv;
  tg = t * (g2 * rinv);   // |gamma| = g2 / |gamma|: no float64 divide or square root
}
__device__ __forceinline__ void rotation(double alpha, double beta, double gr, double gi,
                                         double g2, double& cs, double& sn, double& er,
                                         double& ei) {
  double tg;
  rotation(alpha, beta, gr, gi, g2, cs, sn, er, ei, tg);
}

}  // namespace jrot
}  // namespace tp
