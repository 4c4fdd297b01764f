// Facewise complex GEMM of the half spectrum on the tcgen05 tensor cores
// (Algorithm 1 / Algorithm 2 loop over k: C_hat_k = A_hat_k B_hat_k) with a
// split operand: every float operand x is held as a pair x_hi + x_lo, and a*b
// is formed as a_hi b_hi + a_hi b_lo + a_lo b_hi with float32 accumulation in
// tensor memory.  3xTF32 (kind::tf32): x_hi = tf32(x) (round to nearest),
// x_lo = x - x_hi in float planes.  BF16x3 (kind::f16 with bf16 operands, twice
// the tf32 rate, half the operand bytes): x_hi = bf16(x), x_lo = bf16(x - x_hi).
// Complex products take four real products (Re = ArBr - AiBi, Im = ArBi +
// AiBr); the minus sign is the instruction descriptor's negate-A bit.
//
// Persistent kernel: one CTA per SM walks the list of 128 x 128 output tiles
// (frequency slowest, so the CTAs in flight share a slice's operands in L2).
//   warp 0 lane 0   TMA producer: 8 operand planes per K block (16 tf32 or
//                   32 bf16 deep: 64-byte rows) into a 3-stage shared-memory
//                   ring (mbarrier complete_tx)
//   warp 1 lane 0   MMA issuer: 12 tcgen05.mma (K = 8 tf32 or 16 bf16: 32
//                   bytes of each row) per K step into
//                   one of two TMEM accumulator sets (Re at +0, Im at +128
//                   columns; sets at columns 0 and 256); tcgen05.commit frees a
//                   stage, and after a tile's last K block marks its set full
//   warps 2-9       epilogue: two warps per TMEM lane quarter, each owning
//                   64 of the tile's 128 columns; wait for a full set,
//                   tcgen05.ld 32x32b, add into float32 registers, mark the
//                   set empty; after a tile's last chunk, bounds-checked
//                   coalesced stores
// K is cut into chunks of KCB K blocks (256 bf16 or 128 tf32 elements): every
// chunk accumulates into a fresh TMEM set (the sets alternate, so the next
// chunk's MMAs run while the epilogue drains the previous one) and the
// epilogue adds the chunk sums in float32 registers with round-to-nearest.
// The tensor cores' own float32 accumulation error grows with the number of
// updates it absorbs; draining every chunk bounds that growth by the chunk
// length, so the split forms keep float32-level error at any K.
// Both operands are K-major (kind::tf32 takes no transposed operand): A
// planes hold element (m, kk) at kk + lda*m, B planes (kk, n) at kk + ldb*n,
// read as 64-byte-swizzled tiles of 128 rows.  Every mbarrier wait is bounded:
// on timeout the CTA records TP_DEV_TIMEOUT, stops issuing, waits (bounded)
// for its own copies in flight, frees its tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "tp_internal.cuh"

namespace tp {
namespace {

constexpr int TM = 128, TN = 128, ROWB = 64, STAGES = 3;   // ROWB: K-block row bytes
constexpr int EPI_WARPS = 8, NTHR = 32 * (2 + EPI_WARPS);
constexpr int KCB = 8;                                   // K blocks per accumulation chunk
constexpr int EPI_COLS = TN / 2;                         // columns per epilogue warp
constexpr uint32_t A_PLANE_BYTES = TM * ROWB;           // 8 KB
constexpr uint32_t B_PLANE_BYTES = TN * ROWB;           // 8 KB
constexpr uint32_t STAGE_BYTES = 4 * A_PLANE_BYTES + 4 * B_PLANE_BYTES;   // 64 KB
constexpr uint32_t TMEM_COLS = 4 * TN;   // two accumulator sets of (Re, Im)
constexpr size_t SMEM_BYTES = size_t(STAGES) * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr long long WAIT_LIMIT = 4000000000LL;           // clock64 ticks (~2 s)

struct TcParams {
  CUtensorMap a[4];   // A planes: re_hi, re_lo, im_hi, im_lo
  CUtensorMap b[4];   // B planes: re_hi, re_lo, im_hi, im_lo
  float* zr;
  float* zi;
  int64_t M, N, ldz, sZ;
  const int64_t* dynK;
  int64_t K;
  int64_t h, n3;
  int32_t* status;
  int mt, nt;   // output tiles along M and N
  long long mma_wait_limit;   // the MMA warp's wait for loaded stages (clock64 ticks)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long limit = WAIT_LIMIT) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// Bounded wait that also gives up once another warp has raised the abort
// flag: 0 = phase completed, 1 = timeout, 2 = aborted.
__device__ __forceinline__ int mbar_wait_or_abort(uint32_t bar, uint32_t parity,
                                                  const int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return 0;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*(const volatile int*)abort_flag) return 2;
    if (clock64() - t0 > WAIT_LIMIT) return 1;
  }
  return 0;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (16-byte units), descriptor version 1, swizzle mode.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo,
                                              uint32_t layout) {
  uint64_t d = uint64_t((saddr & 0x3FFFFu) >> 4);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(layout & 7u) << 61;
  return d;
}
constexpr uint32_t LAYOUT_SW64 = 4;

// Instruction descriptor, kind::tf32: F32 accumulate, TF32 A and B, both
// K-major, N = TN, M = TM; bit 13 negates A.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(TN >> 3) << 17) |
                           (uint32_t(TM >> 4) << 24);
constexpr uint32_t IDESC_NEG = IDESC | (1u << 13);
// kind::f16: F32 accumulate, BF16 A and B, both K-major, N = TN, M = TM.
constexpr uint32_t IDESC_BF16 = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(TN >> 3) << 17) |
                                (uint32_t(TM >> 4) << 24);
constexpr uint32_t IDESC_BF16_NEG = IDESC_BF16 | (1u << 13);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

// One K step (32 bytes of every row) of one accumulator.
template <bool BF16>
__device__ __forceinline__ void mma_step(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  if constexpr (BF16)
    mma_bf16(d, a, b, idesc, accum);
  else
    mma_tf32(d, a, b, idesc, accum);
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

// 8 consecutive TMEM columns of this warp's 32 lanes (no wait).
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Ten warps: two of the four SM sub-partitions hold three of them, and a
// sub-partition's 16K registers then allow 170 per thread; the epilogue's
// 128 float32 accumulators fit with 8-column TMEM loads.
template <bool BF16>
__global__ void __launch_bounds__(NTHR, 1) cgemm_tc_kernel(const __grid_constant__ TcParams p) {
  constexpr int TBK = BF16 ? ROWB / 2 : ROWB / 4;   // K elements per K block
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + size_t(STAGES) * STAGE_BYTES);
  // full[S], empty[S], acc_full[2], acc_empty[2], then the TMEM slot
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* acc_full = bars + 2 * STAGES;
  uint64_t* acc_empty = bars + 2 * STAGES + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t K = p.dynK ? *p.dynK : p.K;
  const int nkb = int((K + TBK - 1) / TBK);
  constexpr int SUBK = BF16 ? 16 : 8;   // K elements per 32-byte MMA step
  const int klast = int(K - int64_t(nkb - 1) * TBK);
  const int nsub_last = (klast + SUBK - 1) / SUBK;
  const int tiles_per_f = p.mt * p.nt;
  const int64_t ntiles = int64_t(tiles_per_f) * p.h;
  const int nch = (nkb + KCB - 1) / KCB;   // accumulation chunks per tile

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), EPI_WARPS);   // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int i = 0; i < 4; ++i) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&p.a[i])) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&p.b[i])) : "memory");
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0 && nkb > 0) {
    // ---------------- TMA producer: stage ring continues across tiles
    int64_t it = 0;   // global K-block counter of this CTA
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int f = int(t / tiles_per_f);
      const int rem = int(t - int64_t(f) * tiles_per_f);
      const int m0 = (rem / p.nt) * TM, n0 = (rem % p.nt) * TN;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = int(it % STAGES);
        const int64_t r = it / STAGES;
        if (r > 0) {
          const int w = mbar_wait_or_abort(smem_u32(&empty[s]), uint32_t((r - 1) & 1), &abort_flag);
          if (w) {
            if (w == 1) atomicExch(&abort_flag, 1);
            ok = false;
            break;
          }
        }
        if (*(volatile int*)&abort_flag) { ok = false; break; }
        const uint32_t fb = smem_u32(&full[s]);
        const uint32_t st = smem_u32(smem + size_t(s) * STAGE_BYTES);
        mbar_expect_tx(fb, STAGE_BYTES);
        const int k0 = kb * TBK;
        for (int pl = 0; pl < 4; ++pl) {
          tma_load_3d(st + pl * A_PLANE_BYTES, &p.a[pl], k0, m0, f, fb);
          tma_load_3d(st + 4 * A_PLANE_BYTES + pl * B_PLANE_BYTES, &p.b[pl], k0, n0, f, fb);
        }
      }
    }
    // drain: the last issued stages must land before the CTA may exit
    const int64_t last = it;
    for (int64_t q = (last > STAGES ? last - STAGES : 0); q < last; ++q) {
      if (!mbar_wait(smem_u32(&full[int(q % STAGES)]), uint32_t((q / STAGES) & 1))) break;
    }
  } else if (warp == 1 && lane == 0 && nkb > 0) {
    // ---------------- MMA issuer
    int64_t it = 0;   // global K-block counter (stage ring)
    int64_t ch = 0;   // global chunk counter (accumulator sets alternate per chunk)
    bool ok = true;
    const uint32_t id = BF16 ? IDESC_BF16 : IDESC, idn = BF16 ? IDESC_BF16_NEG : IDESC_NEG;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int f = int(t / tiles_per_f);
      const bool real_slice = (f == 0) || ((p.n3 % 2 == 0) && f == p.h - 1);
      for (int c = 0; c < nch && ok; ++c, ++ch) {
        const int b = int(ch & 1);
        const int64_t use = ch >> 1;
        if (use > 0 && !mbar_wait(smem_u32(&acc_empty[b]), uint32_t((use - 1) & 1))) {
          atomicExch(&abort_flag, 1);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dre = tmem + uint32_t(b) * (2 * TN), dim = dre + TN;
        // full-width MMAs on every tile (a narrower MMA for the ragged last
        // column of tiles measured slower than multiplying its zero padding)
        const int kb0 = c * KCB, kb1 = min(nkb, kb0 + KCB);
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = int(it % STAGES);
          if (!mbar_wait(smem_u32(&full[s]), uint32_t((it / STAGES) & 1), p.mma_wait_limit)) {
            // raise the flag before the commit below, so that the epilogue
            // sees it once this chunk's MMAs have completed
            atomicExch(&abort_flag, 1);
            ok = false;
            break;
          }
          if (*(volatile int*)&abort_flag) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = smem_u32(smem + size_t(s) * STAGE_BYTES);
          // the last K block runs only the 32-byte steps that hold data
          const int nsub = kb == nkb - 1 ? nsub_last : ROWB / 32;
#pragma unroll
          for (int sub = 0; sub < ROWB / 32; ++sub) {
            if (sub >= nsub) break;
            uint64_t a[4], bb[4];
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) {
              a[pl] = smem_desc(st + pl * A_PLANE_BYTES + sub * 32, 16, 512, LAYOUT_SW64);
              bb[pl] = smem_desc(st + 4 * A_PLANE_BYTES + pl * B_PLANE_BYTES + sub * 32, 16, 512,
                                 LAYOUT_SW64);
            }
            const uint32_t first = (kb == kb0 && sub == 0) ? 0u : 1u;
            // planes: 0 re_hi, 1 re_lo, 2 im_hi, 3 im_lo
            mma_step<BF16>(dre, a[0], bb[0], id, first);
            mma_step<BF16>(dre, a[0], bb[1], id, 1);
            mma_step<BF16>(dre, a[1], bb[0], id, 1);
            if (!real_slice) {
              mma_step<BF16>(dre, a[2], bb[2], idn, 1);
              mma_step<BF16>(dre, a[2], bb[3], idn, 1);
              mma_step<BF16>(dre, a[3], bb[2], idn, 1);
              mma_step<BF16>(dim, a[0], bb[2], id, first);
              mma_step<BF16>(dim, a[0], bb[3], id, 1);
              mma_step<BF16>(dim, a[1], bb[2], id, 1);
              mma_step<BF16>(dim, a[2], bb[0], id, 1);
              mma_step<BF16>(dim, a[2], bb[1], id, 1);
              mma_step<BF16>(dim, a[3], bb[0], id, 1);
            }
          }
          mma_commit(smem_u32(&empty[s]));   // stage s free once these MMAs finish
        }
        mma_commit(smem_u32(&acc_full[b]));  // chunk's accumulator set final (or abandoned)
      }
    }
    if (!ok) atomicExch(&abort_flag, 1);
  } else if (warp >= 2) {
    // ---------------- epilogue warps: TMEM lane quarter = warp % 4, column
    // half = which of the two warps of that quarter
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    int64_t ch = 0;
    bool stop = false;
    for (int64_t t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
      const int f = int(t / tiles_per_f);
      const int rem = int(t - int64_t(f) * tiles_per_f);
      const int64_t m0 = int64_t(rem / p.nt) * TM;
      const int64_t n0 = int64_t(rem % p.nt) * TN + half * EPI_COLS;
      const bool real_slice = (f == 0) || ((p.n3 % 2 == 0) && f == p.h - 1);
      float accr[EPI_COLS], acci[EPI_COLS];
#pragma unroll
      for (int j = 0; j < EPI_COLS; ++j) {
        accr[j] = 0.f;
        acci[j] = 0.f;
      }
      for (int c = 0; c < nch; ++c, ++ch) {
        const int b = int(ch & 1);
        const int64_t use = ch >> 1;
        bool have = mbar_wait(smem_u32(&acc_full[b]), uint32_t(use & 1));
        if (!have) atomicExch(&abort_flag, 1);
        have = __all_sync(0xffffffffu, have);   // tcgen05.ld below is warp-collective
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (have) {
          const uint32_t base = tmem + (uint32_t(q * 32) << 16) + uint32_t(b) * (2 * TN) +
                                uint32_t(half * EPI_COLS);
#pragma unroll
          for (int c0 = 0; c0 < EPI_COLS; c0 += 8) {
            uint32_t vr[8], vi[8];
            tmem_ld8_nowait(base + uint32_t(c0), vr);
            if (!real_slice) tmem_ld8_nowait(base + uint32_t(TN + c0), vi);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              // chunk sums added in float32, round to nearest
              accr[c0 + j] = c == 0 ? __uint_as_float(vr[j]) : accr[c0 + j] + __uint_as_float(vr[j]);
              if (!real_slice)
                acci[c0 + j] =
                    c == 0 ? __uint_as_float(vi[j]) : acci[c0 + j] + __uint_as_float(vi[j]);
            }
          }
        }
        // hand set b back to the MMA warp
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
        if (!have || *(volatile int*)&abort_flag) {
          stop = true;
          break;
        }
      }
      if (stop) break;
      const int64_t m = m0 + q * 32 + lane;
      if (m < p.M) {
        float* zr = p.zr + int64_t(f) * p.sZ;
        float* zi = p.zi + int64_t(f) * p.sZ;
#pragma unroll
        for (int j = 0; j < EPI_COLS; ++j) {
          const int64_t n = n0 + j;
          if (n < p.N) {
            zr[m + p.ldz * n] = accr[j];
            zi[m + p.ldz * n] = real_slice ? 0.f : acci[j];
          }
        }
      }
    }
  }
  __syncwarp();

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag && p.status) atomicOr(p.status, TP_DEV_TIMEOUT);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- host side
// The CUDA driver API's tensor-map encoder, looked up through the runtime so that the
// library has no link-time dependency on libcuda (it loads on GPU-less hosts).
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

int encode_map(CUtensorMap* map, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
               uint64_t s1_bytes, uint64_t s2_bytes, uint32_t b0, uint32_t b1,
               CUtensorMapSwizzle sw,
               CUtensorMapDataType dtype = CU_TENSOR_MAP_DATA_TYPE_FLOAT32) {
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {s1_bytes, s2_bytes};
  const cuuint32_t box[3] = {b0, b1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return TP_ECUDA;
  }
  const CUresult r = enc(map, dtype, 3, const_cast<void*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with CUresult %d", int(r));
    return TP_ECUDA;
  }
  return TP_OK;
}

}  // namespace

// Operands for the tensor-core path come as split planes: g.ar/g.ai are the
// hi planes and g.ar_lo/g.ai_lo (likewise b) the lo planes, float (3xTF32) or
// bf16 (BF16x3) elements; A planes have element (m, kk) at kk + lda*m, B
// planes (kk, n) at kk + ldb*n (lda, ldb multiples of 16 bytes); K capacity
// g.kcap (zero-padded past K up to a multiple of 32 or to the capacity).
int launch_cgemm_tc(const CGemm& g, cudaStream_t st) {
  if (g.M == 0 || g.N == 0 || g.h == 0) return TP_OK;
  if (!g.ar_lo || !g.ai_lo || !g.br_lo || !g.bi_lo) {
    set_error("cgemm_tc: split operand planes missing");
    return TP_EINVAL;
  }
  const bool bf16 = g.precision == TP_BF16X3;
  const int64_t ealign = bf16 ? 8 : 4;   // elements per 16 bytes
  if ((g.lda % ealign) || (g.ldb % ealign) || (g.sA % ealign) || (g.sB % ealign)) {
    set_error("cgemm_tc: leading dimensions must be multiples of 16 bytes");
    return TP_EALIGN;
  }
  const uint64_t esz = bf16 ? 2 : 4;
  const uint32_t tbk = uint32_t(ROWB / esz);
  const CUtensorMapDataType dt =
      bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  if (g.M > 0x7fffffff || g.N > 0x7fffffff || g.kcap > 0x7fffffff || g.h > 65535 ||
      (g.M + TM - 1) / TM * ((g.N + TN - 1) / TN) > 0x7fffffff / 65536) {
    set_error("cgemm_tc: sizes too large for one launch");
    return TP_EUNSUPPORTED;
  }
  TcParams p;
  const float* ap[4] = {g.ar, g.ar_lo, g.ai, g.ai_lo};
  const float* bp[4] = {g.br, g.br_lo, g.bi, g.bi_lo};
  for (int i = 0; i < 4; ++i) {
    if (!aligned16(ap[i]) || !aligned16(bp[i])) {
      set_error("cgemm_tc: operand planes must be 16-byte aligned");
      return TP_EALIGN;
    }
    int rc = encode_map(&p.a[i], ap[i], uint64_t(g.kcap), uint64_t(g.M), uint64_t(g.h),
                        uint64_t(g.lda) * esz, uint64_t(g.sA) * esz, tbk, TM,
                        CU_TENSOR_MAP_SWIZZLE_64B, dt);
    if (rc) return rc;
    rc = encode_map(&p.b[i], bp[i], uint64_t(g.kcap), uint64_t(g.N), uint64_t(g.h),
                    uint64_t(g.ldb) * esz, uint64_t(g.sB) * esz, tbk, TN, CU_TENSOR_MAP_SWIZZLE_64B,
                    dt);
    if (rc) return rc;
  }
  p.zr = g.cr;
  p.zi = g.ci;
  p.M = g.M;
  p.N = g.N;
  p.ldz = g.ldc;
  p.sZ = g.sC;
  p.dynK = g.dynK;
  p.K = g.K;
  p.h = g.h;
  p.n3 = g.n3;
  p.status = g.status;
  p.mt = int((g.M + TM - 1) / TM);
  p.nt = int((g.N + TN - 1) / TN);
  p.mma_wait_limit = g.wait_limit > 0 ? g.wait_limit : WAIT_LIMIT;
  auto kernel = bf16 ? cgemm_tc_kernel<true> : cgemm_tc_kernel<false>;
  TP_SET_SMEM(kernel, SMEM_BYTES);
  const int sms = sm_count();
  const int64_t ntiles = int64_t(p.mt) * p.nt * g.h;
  const dim3 grid(unsigned(ntiles < sms ? ntiles : sms));
  {
    KernelScope ks("cgemm_tc", st);
    kernel<<<grid, NTHR, SMEM_BYTES, st>>>(p);
  }
  return launch_status("cgemm_tc_kernel");
}

}  // namespace tp
