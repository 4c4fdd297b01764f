/*
 * tprod.h -- C ABI of libtprod.so, a GB300 (sm_103a) implementation of the
 * t-product tensor methods of Tarzanagh & Michailidis, "Fast Randomized
 * Algorithms for t-Product Based Tensor Operations and Decompositions with
 * Applications to Imaging Data" (arXiv 1704.04362).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Tensors.  A real n1 x n2 x n3 tensor X (Section 2, "Tensor indexing") is a
 *   float32 device array with X(i,j,t) at X[i + n1*(j + n2*t)]: column-major,
 *   frontal slices contiguous (the storage order of MATLAB, which the paper
 *   uses).  The base address must be 16-byte aligned unless noted.
 * Fourier domain.  The transform along mode 3 is MATLAB's fft(X,[],3)
 *   (unnormalised, kernel exp(-2*pi*i*k*t/n3)); the inverse carries 1/n3.
 *   Only the half spectrum k = 0..h-1, h = n3/2 + 1 (integer division), is
 *   ever formed; slice n3-k is the conjugate of slice k for real data.  A
 *   half-spectrum tensor is stored planar: real and imaginary float32 arrays,
 *   each [k][column][row] with rows fastest.
 * Pointers.  Unless said otherwise every array argument is a DEVICE pointer
 *   on the current CUDA device, owned by the caller.  The library never
 *   frees or keeps caller memory.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *   default stream).  Every entry point validates its arguments on the host,
 *   enqueues kernels on `stream` and returns without synchronising.
 * Errors.  Every entry point returns a tp_status.  Argument errors are found
 *   before anything is enqueued and leave outputs untouched.  A CUDA launch
 *   error returns TP_ECUDA.  Conditions found on the device (an iteration
 *   cap reached, a Cholesky breakdown) are OR-ed as TP_DEV_* bits into
 *   opts->status when the caller supplies that word; the call itself still
 *   returns TP_OK.  tp_last_error() gives a message for the calling thread.
 * Workspace.  Scratch memory comes from opts->workspace (caller-owned device
 *   buffer of opts->workspace_bytes, 256-byte aligned) when given.  With no
 *   workspace the library allocates once per device and keeps the buffer,
 *   growing it when a larger call needs it (that growth synchronises the
 *   device); tp_release() frees it.  tp_workspace_query() gives the size a
 *   call needs.  Calls that share a workspace must be ordered on one stream.
 */
#ifndef TPROD_H
#define TPROD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TP_OK = 0,
  TP_EINVAL = -1,        /* a size or mode is out of range */
  TP_ENULL = -2,         /* a required pointer is NULL */
  TP_EALIGN = -3,        /* a pointer is not aligned as required */
  TP_ENOMEM = -4,        /* the library could not allocate its workspace */
  TP_ECUDA = -5,         /* a CUDA runtime call or kernel launch failed */
  TP_EWORKSPACE = -9,    /* opts->workspace is smaller than tp_workspace_query() */
  TP_EUNSUPPORTED = -10  /* valid but not supported by this library (see message) */
} tp_status;

/* Device status bits OR-ed into opts->status. */
#define TP_DEV_NOCONV     0x1  /* Jacobi sweeps reached opts->max_sweeps */
#define TP_DEV_BREAKDOWN  0x2  /* CholeskyQR (slices > 256 rows): Gram not positive definite after shift */
#define TP_DEV_TIMEOUT    0x4  /* a pipeline wait inside a kernel gave up (results invalid) */

typedef enum {
  TP_FP32 = 0,   /* plain FP32 SIMT arithmetic */
  TP_TF32X3 = 1, /* facewise GEMMs on tcgen05 tensor cores, 3xTF32 split, FP32 accumulate */
  TP_BF16X3 = 2  /* facewise GEMMs on tcgen05 tensor cores, BF16 hi/lo split (3 products), FP32
                    accumulate: twice the 3xTF32 rate; each real product is exact to about
                    3 * 2^-16 relative (bf16 hi + lo keeps 16 significand bits), so results
                    carry a relative error of a few 1e-6, against about 1e-7 for 3xTF32 */
} tp_precision;

typedef enum {
  TP_PROB_AB = 0,    /* p_j proportional to ||A(:,j,:)||_F ||B(j,:,:)||_F (eq. nearly_optimal_probs, beta=1) */
  TP_PROB_A2 = 1,    /* p_j proportional to ||A(:,j,:)||_F^2          (eq. nonoptimal_probs, beta=1) */
  TP_PROB_GIVEN = 2  /* p_j supplied by the caller (device float64[n2]) */
} tp_prob_mode;

/* How slices are drawn. */
typedef enum {
  TP_SAMPLE_BERNOULLI = 0, /* Algorithm 2: slice j kept with probability min{1, c p_j} */
  TP_SAMPLE_IID = 1        /* c independent draws with replacement, j with probability
                              p_j (the matrix case Algorithm 2 reduces to at n3 = 1,
                              Drineas, Kannan and Mahoney 2006), rescale 1/sqrt(c p_j) */
} tp_sample_mode;

typedef struct {
  int precision;          /* tp_precision of the facewise GEMMs (default TP_FP32) */
  int max_sweeps;         /* Jacobi sweep cap, 0 = default (30) */
  void* workspace;        /* device scratch or NULL (library-managed) */
  size_t workspace_bytes; /* size of `workspace` */
  int32_t* status;        /* device int32 receiving TP_DEV_* bits, or NULL */
  int64_t pipeline_wait_limit; /* failure-detection test hook: bound, in clock64 ticks, of the
                              tensor-core GEMM's wait for a loaded operand stage (0 = the
                              default, about two seconds).  A tiny value makes that wait
                              run out: the kernel then sets TP_DEV_TIMEOUT, stops, waits
                              for the copies and products it already issued and returns;
                              the outputs of that call are invalid, the context stays
                              usable. */
} tp_opts;

/* Operation codes for tp_workspace_query(). */
typedef enum {
  TP_OP_TPROD = 1,           /* dims: n1, n2, n4, n3 */
  TP_OP_TPROD_SAMPLED = 2,   /* dims: n1, n2, n4, n3 */
  TP_OP_TSVD = 3,            /* dims: n1, n2, n3 */
  TP_OP_TSVD_RANDOMIZED = 4, /* dims: n1, n2, n3, k, p */
  TP_OP_TCOMPLETE_SVT = 5,   /* dims: n1, n2, n3 */
  TP_OP_SLICE_NORMS = 6,     /* dims: n1, n2, n3 */
  TP_OP_TCX = 7,             /* dims: n1, n2, n3 */
  TP_OP_TCOMPLETE_SVT_BATCHED = 8, /* dims: n1, n2, n3 of every tensor (nd = 3 ntens) */
  TP_OP_SKETCH_SPECTRUM = 9,        /* dims: n1, n2, n3, l */
  TP_OP_MLP_TRAIN = 10,             /* dims: batch */
  TP_OP_TRPCA = 11,                 /* dims: n1, n2, n3 */
  TP_OP_TCUR = 12,                  /* dims: n1, n2, n3 */
  TP_OP_CUR_TNN = 13                /* dims: n1, n2, n3 */
} tp_op;

/* ---------------------------------------------------------------- t-product
 * tprod: C = A * B, the t-product of Def. 2.1 computed as Algorithm 1 (DFT
 * along mode 3, facewise complex products of the half spectrum, inverse DFT).
 *   A  n1 x n2 x n3 (input), B  n2 x n4 x n3 (input), C  n1 x n4 x n3 (output).
 * Sizes must be >= 1 (n3 <= 4096).  C must not overlap A or B.            */
int tprod(const float* A, const float* B, float* C,
          int64_t n1, int64_t n2, int64_t n4, int64_t n3,
          const tp_opts* opts, void* stream);

/* tprod_sampled: the rt-product of Algorithm 2, Z = C * R ~ A * B.
 * Slice j of n2 is kept with probability q_j = min{1, c p_j} (Bernoulli,
 * decided in index order), p from `prob_mode` (see tp_prob_mode; p_given is
 * a device float64[n2] summing to 1 when prob_mode == TP_PROB_GIVEN, else
 * ignored).  Kept lateral slices A(:,j,:) and horizontal slices B(j,:,:)
 * are scaled by 1/sqrt(q_j) (the rescale 1/min{1, sqrt(c p_j)} of
 * Algorithm 2), transformed and multiplied facewise; S and D are never
 * formed.  The coin for slice j is Philox4x32-10 (Salmon et al., SC'11) with
 * counter (j mod 2^32, j >> 32, 0, 0) and key (seed mod 2^32, seed >> 32):
 * j is kept iff ((x0 >> 5) * 2^26 + (x1 >> 6)) < floor(q_j * 2^53).
 * sample_mode TP_SAMPLE_IID instead draws c indices independently with
 * replacement (1 <= c <= n2): with W_j = floor(p_j 2^53) and U_t the 53-bit
 * integer of counter (t mod 2^32, t >> 32, 0, 1), draw t is the first j whose
 * prefix sum W_0 + ... + W_j exceeds floor(U_t sum(W) / 2^53); each drawn
 * slice pair is scaled by 1/sqrt(c p_j) and the c' = c draws (duplicates
 * allowed) are multiplied in draw order.
 *   idx_out    device int32[n2] or NULL: kept indices, ascending (Bernoulli)
 *              or in draw order (i.i.d.), first c' valid
 *   count_out  device int64 or NULL: c', the number kept
 *   Z          n1 x n4 x n3 output (zero when nothing is kept)
 * c >= 1.  The count stays on the device: no host synchronisation.          */
int tprod_sampled(const float* A, const float* B, float* Z,
                  int64_t n1, int64_t n2, int64_t n4, int64_t n3,
                  int64_t c, uint64_t seed, int prob_mode, int sample_mode,
                  const double* p_given, int32_t* idx_out, int64_t* count_out,
                  const tp_opts* opts, void* stream);

/* ---------------------------------------------------------------- t-SVD
 * tsvd: X = U * S * V^T (Theorem 2.6), computed as in Eq. circ1: an SVD of
 * every half-spectrum Fourier slice (one-sided Jacobi, singular values
 * descending), the conjugate slices implied, then the inverse DFT.
 * Economy form with m = min(n1, n2):
 *   U  n1 x m x n3,  S  m x m x n3 (f-diagonal),  V  n2 x m x n3 (outputs).
 * Singular vectors are unique only up to a unit phase per column (and a
 * rotation inside repeated singular values).  The per-slice one-sided
 * Jacobi sweeps in float32; V is re-orthonormalised in float64 (one
 * Newton-Schulz step) and G = X_hat V formed in float64.  Slices of at most
 * 4096 entries (p <= 256, m <= 96) then re-orthonormalise the vectors of G
 * by a float32 Householder QR in descending order (float32-level
 * orthogonality; an orthonormal completion for a cluster at the rounding
 * floor); larger slices finish with float64 sweeps.  The forward DFT is float32, so singular values are
 * determined to about u32 s_1 either way.  Limits: m <= 512; n3 <= 512 or a
 * product of the radices 2..13.  */
int tsvd(const float* X, int64_t n1, int64_t n2, int64_t n3,
         float* U, float* S, float* V, const tp_opts* opts, void* stream);

/* Test matrix of the randomized t-SVD. */
#define TP_SKETCH_SIGNS 0   /* random signs (below) */
#define TP_SKETCH_SLICES 1  /* picked lateral slices of X (t-CX sketch) */

/* tsvd_randomized: rank-k approximation X ~ U * S * V^T of tubal rank k.
 * Per half-spectrum slice: Y = X_hat Omega with an n2 x (k+p) test matrix:
 * TP_SKETCH_SIGNS, random signs from Philox stream 2 (entries
 * (s0 + i s1)/sqrt(2), real signs on the real slices; entry (r,c,f) uses
 * counter r + n2*(c + (k+p)*f)); TP_SKETCH_SLICES, the k + p lateral slices
 * of X drawn with replacement as tprod_sampled's TP_SAMPLE_IID does (p_j =
 * ||X(:,j,:)||_F^2 / ||X||_F^2, Philox stream 2), each rescaled by
 * 1/sqrt((k+p) p_j), so that Y holds picked columns of X_hat;
 * q power iterations Q <- orth(X_hat^H Q), Q <- orth(X_hat Q), each orth a
 * float32 Householder QR in shared memory (slices of at most 256 rows; it
 * cannot break down) or, for taller slices, CholeskyQR2 with a float64 Gram
 * (shifted CholeskyQR3 on failure, then TP_DEV_BREAKDOWN), then B = Q^H X_hat, the SVD of B through its l x l Gram (float32
 * two-sided Jacobi, singular values as the Rayleigh quotients ||B^H w_j||
 * with float64 sums) and U = Q U_B truncated to k.
 *   opts->precision  TP_FP32: the products with X_hat on the CUDA cores;
 *                  TP_TF32X3 / TP_BF16X3: those products on the tcgen05
 *                  tensor cores with split (hi + lo) operands, float32
 *                  accumulation drained every K chunk (float32-level error).
 *   rank_per_freq  device int32[n3/2 + 1] or NULL: per-frequency ranks (the
 *                  multi-rank of Section 2): half-spectrum slice f keeps its
 *                  top min(max(r_f, 0), k) triplets and zeroes the rest (its
 *                  conjugate slice alike); NULL keeps k everywhere.
 *   sketch_per_freq device int32[n3/2 + 1] or NULL: per-frequency sketch
 *                  sizes: slice f sketches with the first
 *                  l_f = min(max(s_f, 1), k + p) columns of the test matrix
 *                  (its range finder, power iterations and core SVD work on
 *                  l_f columns) and keeps at most min(k, l_f) triplets; NULL
 *                  uses k + p everywhere.  The products run over k + p
 *                  columns for every slice (the others held at zero).
 *   U  n1 x k x n3,  S  k x k x n3,  V  n2 x k x n3 (outputs).
 * Requires 1 <= k, p >= 0, q >= 0, k + p <= min(n1, n2, 96); n3 <= 512 or
 * n3 a product of the radices 2, 3, 5, 7, 11, 13.                           */
int tsvd_randomized(const float* X, int64_t n1, int64_t n2, int64_t n3,
                    int k, int p, int q, uint64_t seed, int sketch_mode,
                    const int32_t* rank_per_freq, const int32_t* sketch_per_freq,
                    float* U, float* S, float* V, const tp_opts* opts, void* stream);

/* tcx: t-CX of Algorithm 4 with the t-project of Algorithm 3.  Lateral
 * slice j of A (n1 x n2 x n3) is picked with probability min{1, c p_j}
 * (p from TP_PROB_A2: ||A(:,j,:)||_F^2 / ||A||_F^2, or TP_PROB_GIVEN), by
 * the same Philox coins as tprod_sampled; C = picked slices / sqrt(q_j).
 * Z = C * C^dagger * A (n1 x n2 x n3 output), computed per half-spectrum
 * slice as P_k A_hat_k with P_k the projector onto range(C_hat_k), whose
 * basis is the left singular vectors of C_hat_k (float64 Jacobi) above
 * MATLAB's pinv cut-off max(n1, c') eps(s_max).
 *   idx_out / count_out: as tprod_sampled.
 * Reads the pick count back to the host once (synchronises `stream`).
 * Limits: min(n1, n2) <= 512, n2 <= 4096, n3 <= 512.                        */
int tcx(const float* A, int64_t n1, int64_t n2, int64_t n3, int64_t c, uint64_t seed,
        int prob_mode, const double* p_given, float* Z, int32_t* idx_out, int64_t* count_out,
        const tp_opts* opts, void* stream);

/* tcur: t-CUR of Algorithm 5.  Lateral slices C as in tcx (probability
 * min{1, c p_j}, p from prob_mode / p_cols, Philox stream 0, rescaled by
 * 1/sqrt(q_j)).  Horizontal slice i is picked with probability
 * min{1, l p_i} by the Philox coins of stream 1 and rescaled by 1/sqrt(q_i)
 * (D); p_i is p_rows[i] when p_rows (device float64[n1]) is given, else the
 * row leverage of C (eq. colprob_rows_exact with beta = 1): the squared row
 * norms of the left singular vectors of every Fourier slice C_hat_k above
 * the pinv cut-off max(n1, c') eps(s_max) -- with rank > 0 (Algorithm 5's
 * rank parameter) only the `rank` largest of each slice -- summed over all
 * n3 frequencies and normalised to sum 1.  Per half-spectrum slice
 *   Z_hat_k = C_hat_k (D S^T C_hat_k)^dagger (D S^T A_hat_k),
 * the pseudo-inverse with MATLAB's cut-off max(l', c') eps(s_max).
 *   A        n1 x n2 x n3 input (device);  Z  n1 x n2 x n3 output (device).
 *   col_idx / col_count: int32[n2] / int64[1] (device, may be NULL): the
 *            picked lateral slices, as tcx.
 *   row_idx / row_count: int32[n1] / int64[1] (device, may be NULL): the
 *            picked horizontal slices, ascending.
 *   row_prob float64[n1] (device, may be NULL): the row probabilities used
 *            (zeros when no lateral slice was picked).
 * No pick in either draw gives Z = 0.  Reads both pick counts back to the
 * host (synchronises `stream` twice).  Workspace: TP_OP_TCUR {n1, n2, n3}.
 * Limits: min(n1, n2) <= 512, max(n1, n2) <= 4096, n3 <= 512.               */
int tcur(const float* A, int64_t n1, int64_t n2, int64_t n3, int64_t c, int64_t l, int rank,
         uint64_t seed, int prob_mode, const double* p_cols, const double* p_rows, float* Z,
         int32_t* col_idx, int64_t* col_count, int32_t* row_idx, int64_t* row_count,
         double* row_prob, const tp_opts* opts, void* stream);

/* cur_tnn: CUR t-NN of Algorithm 6.  Lateral slices C of X are picked with
 * probability min{1, c p_j} (Philox stream 0; p from the lateral norms of
 * the observed data P_Omega(X), TP_PROB_A2, or p_cols, TP_PROB_GIVEN) and
 * horizontal slices R with probability min{1, l p_i} (stream 1; p_i from
 * p_rows, else the top-`rank` row leverage of C as in tcur); the picks are
 * not rescaled.  C~ and R~ are the results of `iters` iterations of the ADMM
 * of Algorithm 7 from (L, E, Y) = 0, mu = mu0: with mask == NULL the robust
 * form of problem tlow7 (lambda > 0, or 0 for 1/sqrt(max(rows, cols) n3) of
 * each sub-tensor), with a mask the completion form of problem tlow6 on the
 * observed entries (lambda unused).  The two ADMM runs go concurrently on
 * side streams.  Then per half-spectrum slice
 *   L~_hat_k = C~_hat_k (S^T C~_hat_k)^dagger R~_hat_k,
 * the pseudo-inverse over the singular values above pinv_rtol * s_max
 * (MATLAB's pinv(W, tol); pinv_rtol = 0 takes the default cut-off
 * max(l', c') eps(s_max)).
 *   X, L      n1 x n2 x n3 input / output (device);  mask  uint8 n1 x n2 x n3
 *             (device, 1 = observed) or NULL.
 *   Ct, Rt    device float32[n1 n2 n3] or NULL: receive C~ (n1 x c' x n3)
 *             and R~ (l' x n2 x n3), column-major, compact.
 *   col_idx, col_count, row_idx, row_count, row_prob: as tcur.
 * No pick in either draw gives L = 0.  Synchronises `stream` (pick counts,
 * the concurrent ADMM runs).  Workspace: TP_OP_CUR_TNN {n1, n2, n3}.
 * Limits: min(n1, n2) <= 512, max(n1, n2) <= 4096; n3 <= 512 or a product of
 * the radices 2..13.                                                         */
int cur_tnn(const float* X, const uint8_t* mask, int64_t n1, int64_t n2, int64_t n3, int64_t c,
            int64_t l, int rank, uint64_t seed, int prob_mode, const double* p_cols,
            const double* p_rows, int iters, double lambda, double mu0, double rho, double mu_max,
            double pinv_rtol, float* L, float* Ct, float* Rt, int32_t* col_idx,
            int64_t* col_count, int32_t* row_idx, int64_t* row_count, double* row_prob,
            const tp_opts* opts, void* stream);

/* ---------------------------------------------------------------- completion
 * tcomplete_svt: `iters` iterations of the ADMM of Algorithm 7 in the
 * completion form of problem (tlow6): minimise ||L||_TNN subject to
 * L + E = X, E = 0 on the observed set.  Per iteration, with tau = 1/mu:
 *   L <- SVT_tau(X - E - Y/mu)  (tensor singular value thresholding: every
 *                                Fourier slice's singular values shrunk by tau)
 *   E <- (X - L - Y/mu) where mask == 0, 0 where mask != 0
 *   Y <- Y + mu (L + E - X);    mu <- min(rho mu, mu_max)
 *   X     n1 x n2 x n3 observed data (entries off the mask are ignored)
 *   mask  uint8 n1 x n2 x n3, nonzero = observed
 *   L, E, Y  n1 x n2 x n3 state, read as the starting point and overwritten
 *            (zeros and *mu = mu0 start Algorithm 7 afresh; passing the
 *            previous outputs resumes it)
 *   mu    device float64 scalar, read and updated in place
 * Paper constants: mu0 = 1e-3, rho = 1.1, mu_max = 1e10.  The slice SVT
 * takes V from a float32 one-sided Jacobi (warm-started from the previous
 * iteration's V within a call) and the singular values as Rayleigh quotients
 * ||W v_j|| / ||v_j||.  Resuming from the returned state agrees with one
 * longer call to float32 rounding (the Jacobi's starting rotations are not
 * part of the state).  Limits as tsvd.                                      */
int tcomplete_svt(const float* X, const uint8_t* mask,
                  int64_t n1, int64_t n2, int64_t n3, int iters,
                  double rho, double mu_max,
                  float* L, float* E, float* Y, double* mu,
                  const tp_opts* opts, void* stream);

/* trpca_admm: `iters` iterations of Algorithm 7 as printed, for the robust
 * problem (tlow7): minimise ||L||_TNN + lambda ||E||_1 subject to X = L + E.
 * Per iteration, with tau = 1/mu:
 *   L <- SVT_tau(X - E - Y/mu)
 *   E <- soft(X - L - Y/mu, lambda/mu)   (sign(v) max(|v| - lambda/mu, 0))
 *   Y <- Y + mu (L + E - X);    mu <- min(rho mu, mu_max)
 * lambda <= 0 takes 1/sqrt(max(n1, n2) n3) (the paper leaves it open; Lu et
 * al.'s choice).  State (L, E, Y, *mu) as tcomplete_svt; same SVT, limits
 * and workspace (TP_OP_TRPCA).                                              */
int trpca_admm(const float* X, int64_t n1, int64_t n2, int64_t n3, int iters, double lambda,
               double rho, double mu_max, float* L, float* E, float* Y, double* mu,
               const tp_opts* opts, void* stream);

/* One tensor of a batched completion: X and mask are read; L, E, Y and *mu
 * (device float64) are the state, read and updated as in tcomplete_svt.  All
 * pointers are device pointers owned by the caller.                        */
typedef struct {
  const float* X;
  const uint8_t* mask;
  float* L;
  float* E;
  float* Y;
  double* mu;
  int64_t n1, n2, n3;
} tp_tensor_desc;

/* tcomplete_svt_batched: tcomplete_svt over ntens independent tensors of
 * possibly different sizes (the batched form of the completion workload,
 * e.g. many videos), `iters` iterations each.
 *   descs  HOST array of ntens descriptors
 * The tensors run concurrently on side streams forked from `stream`; the
 * first iteration is launched directly and the remaining iters - 1 replay
 * one captured CUDA graph of an iteration over all tensors.  Results are
 * identical to ntens separate tcomplete_svt calls with the same arguments
 * for tensors with min(n1, n2) < 32 or at least as many half-spectrum slices
 * as the GPU has SMs; otherwise a lone call spreads each slice's Jacobi over
 * a thread-block cluster (another rotation order) and the two agree to
 * float32 rounding (the batch keeps one CTA per slice: with the GPU full, it
 * costs less SM time per slice).
 * Workspace: tp_workspace_query(TP_OP_TCOMPLETE_SVT_BATCHED, {n1, n2, n3 of
 * each tensor}, 3 ntens) (the sum of the tensors' own).  Synchronises
 * `stream` before returning (the graph and side streams are released).
 * Errors: TP_ENULL for a NULL descs or tensor pointer, TP_EINVAL for
 * ntens < 1 or invalid sizes; limits as tcomplete_svt.                      */
int tcomplete_svt_batched(int ntens, const tp_tensor_desc* descs, int iters,
                          double rho, double mu_max, const tp_opts* opts, void* stream);

/* ---------------------------------------------------------------- truncation ranks
 * Per-frequency truncation ranks for the randomized t-SVD.  The paper sets
 * no rank rule (its multi-rank, Section 2, r_i = rank of the i-th Fourier
 * frontal slice, is the rule's tol -> 0 limit) and has no learned part; these
 * calls are the plain adaptive rule and a small learned predictor of the
 * rank and of the oversampling a sketch needs to resolve it.
 *
 * tp_sketch_spectrum: the randomized range finder of tsvd_randomized with l
 *   columns and q power iterations (same seed use), then the singular values
 *   of Q^H X_hat_k at every half-spectrum frequency, descending:
 *   sig_out[k*l + i], device float32, h x l (h = n3/2 + 1).  Limits
 *   l <= min(n1, n2, 96); workspace TP_OP_SKETCH_SPECTRUM {n1, n2, n3, l}.
 * tp_rank_rule: rank_out[k] (device int32, h) = the smallest r in [1, cap]
 *   with sum_{i>r} sig[k,i]^2 <= tol^2 sum_i sig[k,i]^2 (cap if none; 0 for
 *   an all-zero row); sig is h x l device float32, rows descending.  Sums
 *   are float64, accumulated from the smallest value, unfused.
 * tp_rank_features: the predictor's inputs, feat_out[k*16 + i] (device
 *   float16) = max(log10(sig[k,i+1] / sig[k,0]), -8) / 8, i = 0..15; l >= 17.
 * tp_mlp_*: the predictor, a 16 -> 128 -> 128 -> 2 perceptron with ReLU.
 *   theta: tp_mlp_param_count() float32 master parameters, packed W1 (128 x
 *   16), b1, W2 (128 x 128), b2, W3 (2 x 128), b3, matrices row-major (output
 *   index slowest); w16: the same as float16 (the values every kernel uses;
 *   tp_mlp_round sets it from theta).
 *   tp_mlp_forward: y[b*2 + o] (device float32) for float16 inputs x (batch
 *   x 16), float32 accumulation.
 *   tp_mlp_train_step: with loss (1/2B) sum (y - target)^2 over the batch
 *   (target batch x 2, float32), writes grad_out[0 .. P-1] = the gradient
 *   at w16 and grad_out[P] = the loss (P = tp_mlp_param_count(), device
 *   float32), then, if lr > 0, one Adam step (beta 0.9, 0.999, eps 1e-8;
 *   step >= 1 counts updates) on theta with moments adam_m, adam_v (zero
 *   before the first step) and re-rounds w16.  Gradient sums are reduced in
 *   a fixed order (deterministic).  Workspace TP_OP_MLP_TRAIN {batch}.     */
int tp_sketch_spectrum(const float* X, int64_t n1, int64_t n2, int64_t n3, int l, int q,
                       uint64_t seed, float* sig_out, const tp_opts* opts, void* stream);
int tp_rank_rule(const float* sig, int64_t h, int l, int cap, double tol, int32_t* rank_out,
                 void* stream);
int tp_rank_features(const float* sig, int64_t h, int l, void* feat_out, void* stream);
int tp_mlp_param_count(void);
int tp_mlp_round(const float* theta, void* w16, void* stream);
int tp_mlp_forward(const void* w16, const void* x16, int64_t batch, float* y, void* stream);
int tp_mlp_train_step(float* theta, void* w16, float* adam_m, float* adam_v, int step, float lr,
                      const void* x16, const float* target, int64_t batch, float* grad_out,
                      const tp_opts* opts, void* stream);

/* ---------------------------------------------------------------- stages
 * The steps of the paths above, exposed for callers that compose their own.
 *
 * tp_rdft3: half-spectrum DFT along mode 3 of a real rows x n3 array
 *   (X[r + rows*t]) into planar Xr, Xi [k][r], k < h (Section 2, fft(X,[],3)).
 * tp_irdft3: its inverse (ifft(.,[],3) of the conjugate-symmetric spectrum
 *   whose half is given); writes real Out[r + rows*t].                     */
int tp_rdft3(const float* X, int64_t rows, int64_t n3, float* Xr, float* Xi, void* stream);
int tp_irdft3(const float* Xr, const float* Xi, int64_t rows, int64_t n3, float* Out, void* stream);

/* tp_slice_norms: squared Frobenius norms of slices, accumulated in (at
 * least) float64 precision in a fixed order (deterministic), as used by the
 * sampling probabilities of Section 3.1.
 *   which = 0: out[j] = ||X(:,j,:)||_F^2, j < n2 (lateral slices)
 *   which = 1: out[i] = ||X(i,:,:)||_F^2, i < n1 (horizontal slices)
 *   out   device float64 array.                                            */
int tp_slice_norms(const float* X, int64_t n1, int64_t n2, int64_t n3, int which,
                   double* out, const tp_opts* opts, void* stream);

/* tp_slice_norms_noalloc: the same norms as tp_slice_norms, computed by the
 * same kernels, for callers that cannot allocate device memory (a framework
 * that owns the whole memory pool, a real-time caller that forbids
 * allocation after start-up, or one that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree may cause).  The paper has no
 * counterpart: this is a deployment variant, not a step of the method.
 *   No allocation: the partial sums live in a fixed 8 MiB array of device
 *   global memory inside the library (tp_slice_norms_noalloc_capacity()
 *   doubles), which every GPU that loads the library holds until exit.
 *   Limit: the call needs n2*n3 partial sums for which == 0 and about
 *   min(n1, 1216*256) for which == 1; a call needing more than the capacity
 *   returns TP_EINVAL with a message and enqueues nothing.
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Every call shares the one array: calls that may run at the same time on
 *   the GPU (different streams, different host threads) race and give wrong
 *   norms; order them on one stream.  Nothing in the array needs clearing:
 *   each call writes every slot it reads.
 *   X, out: as tp_slice_norms (device pointers; out float64).             */
int tp_slice_norms_noalloc(const float* X, int64_t n1, int64_t n2, int64_t n3, int which,
                           double* out, void* stream);
size_t tp_slice_norms_noalloc_capacity(void);

/* tp_sample_draw: Algorithm 2's picking loop on the device.  From weights
 * w (device float64[n]; mode TP_PROB_AB: w = a2, w2 = b2 and
 * p_j = sqrt(a2_j b2_j)/sum; TP_PROB_A2: p_j = a2_j / sum a2; TP_PROB_GIVEN:
 * p = w) computes q_j = min{1, c p_j}, draws with Philox as in tprod_sampled
 * (counter word 2 = `stream_id`), and writes the kept indices ascending to
 * idx (int32[n]), 1/sqrt(q) of each kept index to scale (float32[n]) and
 * the count to count (int64).  q_out (float64[n]) receives q when non-NULL.
 * sample_mode TP_SAMPLE_IID: the c (<= n) i.i.d. draws of tprod_sampled
 * (counter word 2 = `stream_id`, word 3 = 1) in draw order, scale
 * 1/sqrt(c p_j), count = c (0 when every weight is zero), q_out = c p.    */
int tp_sample_draw(const double* w, const double* w2, int64_t n, int64_t c,
                   uint64_t seed, int prob_mode, int sample_mode, uint32_t stream_id,
                   int32_t* idx, float* scale, int64_t* count, double* q_out,
                   void* stream);

/* ---------------------------------------------------------------- runtime */
/* tp_philox4x32_10: the library's counter-based generator, exposed so that
 * its words can be checked against the published known-answer vectors of
 * Philox4x32-10 (Salmon et al., SC'11).  Every random choice of the library
 * (Algorithm 2's coins, the with-replacement draws, Algorithm 4-5's picks,
 * the randomized t-SVD's test matrix) is a function of these words; the
 * paper does not say how its draws are made (see tprod_sampled).
 *   counters  device uint32[4 n]: counter e is words 4e .. 4e+3 (word 0 first)
 *   k0, k1    the key (k0 = the low key word)
 *   out       device uint32[4 n]: the four output words of counter e
 * n = 0 enqueues nothing.  Returns TP_EINVAL for n < 0, TP_ENULL for a NULL
 * buffer with n > 0.                                                       */
int tp_philox4x32_10(const uint32_t* counters, uint32_t k0, uint32_t k1, int64_t n,
                     uint32_t* out, void* stream);

size_t tp_workspace_query(int op, const int64_t* dims, int ndims, const tp_opts* opts);
const char* tp_status_string(int status);
const char* tp_last_error(void);
/* Frees the library-managed workspace of the current device (synchronises it). */
int tp_release(void);
/* tp_sync_status: waits for `stream`, then reports what went wrong on the
 * device since: TP_ECUDA (message in tp_last_error) for a CUDA error raised
 * by an earlier asynchronous launch, else TP_OK.  With status_dev (a device
 * int32 the calls' tp_opts.status pointed at) non-NULL its TP_DEV_* bits are
 * copied to *status_host (and the device word is left as it is).            */
int tp_sync_status(void* stream, const int32_t* status_dev, int32_t* status_host);
/* Number of kernels this library has launched in this process. */
uint64_t tp_launch_count(void);
int tp_version(void);

/* Launch-shape autotuner.  Tunable launches (the tile width of the direct
 * DFT contractions, the blocks per SM of the register FFTs and of the
 * lateral norm pass) offer candidate shapes that compute bit-identical
 * results.  With tuning on (the default; environment variable TP_AUTOTUNE=0
 * at load switches it off) the first call with a given problem shape times
 * every candidate on the caller's stream (CUDA events; the call synchronises
 * that stream once) and keeps the fastest; later calls reuse it.  A stream
 * being captured into a CUDA graph is never timed (cached choice or the
 * default).
 *   tp_autotune_mode     TP_TUNE_OFF / TP_TUNE_ON; any other value only
 *                        queries.  Returns the previous mode.
 *   tp_autotune_force    every tunable launch takes candidate `candidate`
 *                        (clamped to its count); -1 ends forcing.  For tests.
 *                        Returns the previous setting.
 *   tp_autotune_count / tp_autotune_entry  list the table: key text
 *                        ("op:dims"), chosen and candidate count, its time
 *                        and the default's (ms per launch; -1 if loaded).
 *   tp_autotune_save / tp_autotune_load  one "key choice" line per entry.
 *   tp_autotune_reset    empties the table.                                  */
#define TP_TUNE_OFF 0
#define TP_TUNE_ON 1
int tp_autotune_mode(int mode);
int tp_autotune_force(int candidate);
int tp_autotune_count(void);
int tp_autotune_entry(int i, char* key, int key_len, int* choice, int* ncand, double* best_ms,
                      double* default_ms);
int tp_autotune_save(const char* path);
int tp_autotune_load(const char* path);
int tp_autotune_reset(void);

/* Per-kernel timing.  Between tp_profile_start() and tp_profile_stop() every
 * kernel launch of this library is bracketed by a CUDA event pair recorded on
 * the launch stream.  tp_profile_stop() synchronises the device and adds the
 * elapsed times into per-kernel totals; tp_profile_entry(i, ...) reads total
 * i (name into name[name_len], total milliseconds, launch count) and returns
 * TP_EINVAL past the last one; tp_profile_reset() clears the totals.      */
int tp_profile_start(void);
int tp_profile_stop(void);
int tp_profile_entry(int i, char* name, int name_len, double* total_ms, int64_t* launches);
int tp_profile_reset(void);

#ifdef __cplusplus
}
#endif
#endif /* TPROD_H */
