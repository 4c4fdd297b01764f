// Helpers shared by the mode-3 DFT kernels (dft.cu, rfft_reg.cu): tube
// addressing with the optional rescaled gather, and the hi/lo operand split
// (3xTF32 or BF16x3).
#pragma once

#include <cuda_bf16.h>

#include "tp_internal.cuh"

namespace tp {
namespace dftc {

// Nearest tf32 value of x (10 explicit mantissa bits), as a float.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Element o of a split operand pair v ~ hi + lo: hi = tf32(v) and
// lo = tf32(v - hi) in float planes, or hi = bf16(v) and lo = bf16(v - hi) in
// 16-bit planes, all rounded to nearest.  (The tensor cores read only the
// tf32 bits of a float operand; a lo plane left at full float precision would
// be truncated there, a biased error.)
__device__ __forceinline__ void put_split(float* hi_plane, float* lo_plane, bool bf16, int64_t o,
                                          float v) {
  if (bf16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    reinterpret_cast<__nv_bfloat16*>(hi_plane)[o] = h;
    reinterpret_cast<__nv_bfloat16*>(lo_plane)[o] = __float2bfloat16_rn(v - __bfloat162float(h));
  } else {
    const float h = tf32_rna(v);
    hi_plane[o] = h;
    lo_plane[o] = tf32_rna(v - h);
  }
}

struct Extent {
  int64_t rows_eff, cols_eff, rows_pad, cols_pad;
};
__device__ __forceinline__ Extent extent_of(const DftGather& g) {
  const int64_t count = g.dyn_count ? *g.dyn_count : (g.gather_dim == 1 ? g.rows : g.cols);
  Extent x{g.rows, g.cols, g.rows, g.cols};
  if (g.gather_dim == 1) {
    x.rows_eff = count;
    x.rows_pad = min(g.rows, (count + 31) / 32 * 32);   // zero tail for tiled consumers
  } else if (g.gather_dim == 2) {
    x.cols_eff = count;
    x.cols_pad = min(g.cols, (count + 31) / 32 * 32);
  }
  return x;
}

__device__ __forceinline__ const float* tube_ptr(const DftGather& g, const Extent& x, int64_t r,
                                                 int64_t c, float& s) {
  s = 0.f;
  if (r >= x.rows_eff || c >= x.cols_eff) return nullptr;
  int64_t ro = r, co = c;
  s = 1.0f;
  if (g.gather_dim == 1) {
    ro = g.idx[r];
    if (g.scale) s = g.scale[r];
  } else if (g.gather_dim == 2) {
    co = g.idx[c];
    if (g.scale) s = g.scale[c];
  }
  return g.src + ro * g.row_stride + co * g.col_stride;
}

}  // namespace dftc
}  // namespace tp
