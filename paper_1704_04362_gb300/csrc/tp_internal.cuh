// Internal declarations shared by the translation units of libtprod.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <functional>

#include "../../include/tprod.h"

namespace tp {

// ---------------------------------------------------------------- host runtime
void set_error(const char* fmt, ...);
int launch_status(const char* what);      // cudaGetLastError -> TP_OK / TP_ECUDA
void note_launches(uint64_t n);           // kernel launch counter
int sm_count();                           // SMs of the current device (cached per device)

// Brackets one kernel launch: counts it and, while tp_profile_start() is in
// effect, records a CUDA event pair around it on the launch stream.
// count = false: a timed region that is not one kernel (e.g. a graph
// replay), profiled under its name but not counted as a launch.
struct KernelScope {
  KernelScope(const char* name, cudaStream_t st, bool count = true);
  ~KernelScope();
  const char* name;
  cudaStream_t st;
  int slot;
  bool count;
};
// Raises a kernel's dynamic shared memory limit to `bytes`; a failure is
// reported (TP_ECUDA with the kernel's name and the size) instead of
// surfacing later as a launch error under another name.
int set_smem_attr(const void* func, size_t bytes, const char* name);
#define TP_SET_SMEM(kernel, bytes)                                                   \
  do {                                                                             \
    if (int rc_smem_ = ::tp::set_smem_attr((const void*)(kernel), (bytes), #kernel)) \
      return rc_smem_;                                                             \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Bump allocator over a workspace buffer; every block 256-byte aligned.
struct Arena {
  char* base = nullptr;
  size_t size = 0;
  size_t off = 0;
  template <class T> T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};
inline size_t ws_bytes(size_t count, size_t elem) { return (count * elem + 255) & ~size_t(255); }

// Resolves the workspace of a call: opts->workspace when given (checked
// against `need`), else the library-managed per-device buffer.
int acquire_workspace(const tp_opts* opts, size_t need, Arena* out);

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
inline int64_t half_len(int64_t n3) { return n3 / 2 + 1; }

// ---------------------------------------------------------------- kernels
// Generic half-spectrum DFT along mode 3 with an optional gather.  Output
// element (r, c) of slice k goes to out{re,im}[k*out_slice + r + out_ld*c];
// its input tube is src[row_off(r) + col_off(c) + t*slice_stride], scaled.
struct DftGather {
  const float* src;
  int64_t rows, cols;          // logical output rows (fastest) and columns
  int64_t row_stride, col_stride, slice_stride;
  const int32_t* idx;          // gather indices (device) or null
  const float* scale;          // per gathered position (device) or null
  const int64_t* dyn_count;    // device count of the gathered dimension or null
  int gather_dim;              // 0 none, 1 rows, 2 columns
  int64_t n3;
  float* out_re;
  float* out_im;
  int64_t out_ld, out_slice;
  float* out_re_lo;            // non-null: write the 3xTF32 split, hi to out_re/out_im
  float* out_im_lo;            //   (tf32 round-to-nearest) and lo = x - hi here
  int out_transposed;          // 1: element (r, c) of slice k at k*out_slice + c + out_ld*r
  int out_bf16;                // with the split: the four planes hold bf16 (hi, lo) pairs
};
int launch_rdft(const DftGather& g, cudaStream_t st);

// Inverse: out[r + rows*t] = (1/n3) sum over the Hermitian-completed spectrum.
// Input spectrum in{re,im}[k*in_slice + r], k < h.
int launch_irdft(const float* in_re, const float* in_im, int64_t rows, int64_t in_slice,
                 int64_t n3, float* out, cudaStream_t st);

// Facewise planar complex GEMM over the half spectrum:
// C_k = A_k B_k for k < h; A_k (m,kk) at a[k*sA + m + lda*kk], B_k (kk,n) at
// b[k*sB + kk + ldb*n], C_k (m,n) at c[k*sC + m + ldc*n].  K is `K` or, when
// dynK is non-null, read on the device.  Slices k = 0 and (n3 even) k = h-1
// are real: their imaginary parts are ignored on input and written as 0.
struct CGemm {
  const float *ar, *ai, *br, *bi;
  float *cr, *ci;
  int64_t M, N, K;
  const int64_t* dynK;
  int64_t lda, ldb, ldc, sA, sB, sC;
  int64_t h, n3;
  int precision;
  // tensor-core path only: lo planes of the 3xTF32 split, K capacity of the
  // operand planes, device status word (may be null)
  const float *ar_lo, *ai_lo, *br_lo, *bi_lo;
  int64_t kcap;
  int32_t* status;
  // tensor-core path: bound of the MMA warp's wait for a loaded stage, in
  // clock64 ticks (0 = the default of about two seconds)
  long long wait_limit = 0;
  // FP32 path only: B_k(kk, n) = conj(b[k*sB + n + ldb*kk]) (B given as its
  // conjugate transpose)
  int b_conj_trans = 0;
};
int launch_cgemm(const CGemm& g, cudaStream_t st);

// Slice norms (squared, float64).  Lateral: out[j] = sum over (i,t) of X(i,j,t)^2.
// Horizontal: out[i] = sum over (j,t) of X(i,j,t)^2.  `partial` is scratch of
// norms_partial_count() doubles.  tunable = false keeps the launch shape at
// its default (no autotuning: no timing, no stream synchronisation).
size_t norms_partial_count(int64_t n1, int64_t n2, int64_t n3, int which);
int launch_slice_norms(const float* X, int64_t n1, int64_t n2, int64_t n3, int which,
                       double* out, double* partial, cudaStream_t st,
                       bool tunable = true);

// Picking loop of Algorithm 2 (see tp_sample_draw in tprod.h).
// sample_mode TP_SAMPLE_IID: c independent draws with replacement instead.
// idx must hold n entries (the decisions are parked there before packing);
// scratch: draw_scratch_bytes(n) bytes of device memory, 256-byte aligned.
size_t draw_scratch_bytes(int64_t n);
int launch_draw(const double* w, const double* w2, int64_t n, int64_t c, uint64_t seed,
                int mode, uint32_t stream_id, int32_t* idx, float* scale, int64_t* count,
                double* q_out, void* scratch, cudaStream_t st,
                int sample_mode = TP_SAMPLE_BERNOULLI);

// Raw Philox4x32-10 words: out[4e..4e+3] = philox(ctr[4e..4e+3], key (k0, k1)).
int launch_philox_words(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out,
                        cudaStream_t st);

// Bit length of v (0 for v <= 0): the size class of a tuning key, so that
// problems within a factor of two share one tuned choice.
inline int64_t size_class(int64_t v) {
  int64_t b = 0;
  while (v > 0) {
    ++b;
    v >>= 1;
  }
  return b;
}

// Launch-shape autotuner (autotune.cu): `launch(c)` enqueues candidate c of a
// tunable launch on st (every candidate computes bit-identical results); the
// chosen candidate for this op and key is returned in *choice (timed on the
// first call, cached after; `dflt` when tuning is off or st is capturing).
int autotune_pick(const char* op, const int64_t* key, int nkey, int ncand, int dflt,
                  const std::function<int(int)>& launch, cudaStream_t st, int* choice);

}  // namespace tp
