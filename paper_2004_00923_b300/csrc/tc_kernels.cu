// Eq. 4 and Eqs. 6-7 on the 5th-generation tensor cores (tcgen05, kind::f16, FP32
// accumulation in tensor memory), for holograms stored as 16-bit planes.
//
// Layout: the 16-bit hologram store holds, for each block of 64 consecutive pixels, all
// 2*frames rows of it (row 2f = Re H_f, row 2f+1 = Im H_f) as [block][row][64]; a window's
// X = [Re H_0; Im H_0; ...] for one pixel block is 2T consecutive rows, i.e. one contiguous
// 128 x 2T-byte run. One 3-D TMA tensor map with 64-pixel x 2T-row x 1-block boxes
// (128-byte swizzle) feeds both contractions:
//   * covariance (Eq. 4): G = X X^T over pixels, X K-major. 128/(2T) pixel chunks are
//     stacked into one 128-row operand used as both A and B of a 128x128 MMA; the
//     diagonal 2T x 2T blocks are the chunk Gram matrices (the off-diagonal blocks are
//     discarded). Products of stored 16-bit values are exact in FP32; TMEM accumulators
//     are drained every stage into per-thread FP32 block sums that are merged into
//     compensated (Kahan) sums every 8 stages, and
//     the per-unit partials are reduced in FP64 by the covariance reduction kernel.
//   * projection (Eqs. 6-7): P = X^T B^T per 128-pixel tile (A = X, MN-major), with B the
//     real embedding of the retained eigenvectors split into hi + lo 16-bit parts (two
//     MMAs into the same accumulator). The epilogue squares and sums the accumulator row
//     of each pixel straight into the image; P is never stored.
// Roles: warp 0 issues TMA, warp 1 issues MMAs (one thread of it; the warp takes no
// shared-memory step inside its loop, see named_sync), the next warps drain TMEM, and the last
// warp waits on each stage's mbarriers and releases the MMA warp through the stage's named
// barrier. Every mbarrier wait is bounded (tc::kWaitBudget); on expiry the CTA raises
// DH_FLAG_WAIT_TIMEOUT, stops issuing work, waits for its own TMA copies in flight,
// frees its tensor memory and exits.
#include <cudaTypedefs.h>

#include "dh_internal.cuh"
#include "tc_sm100.cuh"

namespace dh {
namespace {

using namespace tc;

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
  return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// Split-K units per window for the tensor-core covariance (a function of the frame size only).
int gram_tc_units(long long npix) {
  long long u = npix / 16384;
  if (u < 1) u = 1;
  if (u > 64) u = 64;
  return (int)u;
}
// The plan's split-K units: its choice (DH_OPT_GRAM_UNITS, the autotuner), else the default.
int gram_tc_units_of(const Plan &p) { return p.gram_units > 0 ? p.gram_units : gram_tc_units(p.npix); }

// ======================================================================= covariance
template <int T>
struct GramCfg {
  static constexpr int M2 = 2 * T;                 // rows per window
  static constexpr int R = 128 / M2;               // pixel chunks stacked per stage
  static constexpr int PIX = 64 * R;               // pixels per stage
  static constexpr int STAGE_BYTES = 128 * 128;    // 128 rows x 64 pixels x 2 bytes
  // One TMEM drain per stage of 4 MMAs: the tensor cores' FP32 accumulation rounds toward
  // zero (measured: about -7e-8 relative per MMA instruction), so short accumulations bound
  // that bias near 3e-7.
  static constexpr int GROUP = 1;
  // Epilogue: each thread owns NCOL columns of one accumulator row; T = 16 runs two CTAs per
  // SM, T = 32 / 64 one CTA per SM (8 stages, 4 TMEM accumulators of 128 columns).
  static constexpr int NCOL = T == 64 ? 64 : 32;
  static constexpr int EPI_WARPS = 4 * (M2 / NCOL);
  static constexpr int WAITER = 2 + EPI_WARPS;     // the warp that watches the mbarriers
  static constexpr int THREADS = 64 + 32 * EPI_WARPS + 32;
  static constexpr bool KAHAN = T <= 32;
  static constexpr int CTAS_PER_SM = T == 16 ? 2 : 1;
  static constexpr int STAGES = CTAS_PER_SM == 2 ? 6 : 8;
  static constexpr int NB = CTAS_PER_SM == 2 ? 2 : 4;   // accumulator buffers
  static constexpr int TMEM_COLS = 128 * NB;
  static constexpr size_t SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};

template <int T, bool BF16>
__global__ void __launch_bounds__(GramCfg<T>::THREADS, 1)
k_gram_tc(const __grid_constant__ CUtensorMap tmH, int first_slot, int slot_stride, int n_windows,
          int units_pw, int stages_per_unit, double *__restrict__ part, uint32_t *__restrict__ status,
          int stall_cycles) {
  using C = GramCfg<T>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *stages = smem;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t *empty = full + C::STAGES;
  uint64_t *acc_full = empty + C::STAGES;
  uint64_t *acc_empty = acc_full + C::NB;
  uint64_t *mma_done = acc_empty + C::NB;
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(mma_done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < C::NB; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 32 * C::EPI_WARPS); }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_barrier_init();
    prefetch_tmap(&tmH);
  }
  if (warp == 1) { tmem_alloc(tmem_holder, C::TMEM_COLS); tmem_relinquish(); }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  const int total_units = n_windows * units_pw;
  auto fail = [&]() { atomicOr(status, DH_FLAG_WAIT_TIMEOUT); *abort_flag = 1; };

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer
      int slot = 0; uint32_t ph = 0;
      long long issued = 0;
      for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x) {
        const int w = u / units_pw, uu = u % units_pw;
        const int row = 2 * (first_slot + w * slot_stride);
        const int p0 = uu * stages_per_unit * C::PIX;
        for (int st = 0; st < stages_per_unit; ++st) {
          if (!mbar_wait(&empty[slot], ph ^ 1)) { fail(); break; }
          mbar_arrive_expect_tx(&full[slot], C::STAGE_BYTES);
          uint8_t *dst = stages + slot * C::STAGE_BYTES;
#pragma unroll
          for (int c = 0; c < C::R; ++c)
            tma_load_3d(dst + c * C::M2 * 128, &tmH, &full[slot], 0, row, (p0 + st * C::PIX + c * 64) >> 6);
          ++issued;
          if (++slot == C::STAGES) { slot = 0; ph ^= 1; }
        }
      }
      if (*abort_flag) {  // let copies still in flight land before the CTA exits
        for (int k = 0; k < C::STAGES && k < issued; ++k) {
          if (--slot < 0) { slot = C::STAGES - 1; ph ^= 1; }
          mbar_wait(&full[slot], ph);
        }
      }
    }
  } else if (warp == 1) {  // ---------------- MMA issuer
    // The whole warp runs the loop (named barriers are per warp) and lane 0 issues. Stage k
    // waits on named barrier 1 + k % STAGES, which the waiter passes once the stage's data has
    // landed and, for a group's first stage, its accumulator buffer is free; the loop has no
    // exit of its own, so its barrier steps pair one to one with the waiter's.
    constexpr uint32_t idesc = idesc_f16(BF16, false, false, 128, 128);
    int slot = 0, grp = 0;
    for (int u = blockIdx.x; u < total_units; u += gridDim.x) {
      for (int g0 = 0; g0 < stages_per_unit; g0 += C::GROUP, ++grp) {
        const int n = stages_per_unit - g0 < C::GROUP ? stages_per_unit - g0 : C::GROUP;
        const uint32_t d = tmem + (grp % C::NB) * 128;
        for (int i = 0; i < n; ++i) {
          named_sync(1 + slot, 64);
          fence_after_sync();
          if (lane == 0) {
            const uint32_t base = smem_u32(stages + slot * C::STAGE_BYTES);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint64_t desc = smem_desc(base + 32 * k, 16, 1024, kSwizzle128);
              mma_f16(d, desc, desc, idesc, (i > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit(&empty[slot]);
          }
          __syncwarp();
          if (++slot == C::STAGES) slot = 0;
        }
        if (lane == 0) mma_commit(&acc_full[grp % C::NB]);
        __syncwarp();
      }
    }
    // every MMA has completed before the tensor memory is freed (also after an abort)
    if (lane == 0) mma_commit(mma_done);
    __syncwarp();
    mbar_wait(mma_done, 0);
  } else if (warp == C::WAITER) {  // ---------------- waiter
    // Stage k's release needs its TMA data (full) and, for a group's first stage, the
    // accumulator buffer back from the epilogue (acc_empty). Normally it runs ahead of the MMA
    // warp by fewer than STAGES stages (a stage's data needs its slot released by the MMAs of
    // the stage STAGES before), so each named barrier has at most one pending arrival. After a
    // failed wait or an abort elsewhere it stops waiting for data and arrives for stage k once
    // the MMAs of stage k - STAGES have completed (empty: the MMA warp passed that stage's
    // barrier before issuing them), which keeps the one-pending-arrival rule, so the MMA warp
    // still completes its loop. (A bar.sync there instead could meet the waiter's own earlier
    // arrival on the same barrier and leave the MMA warp's last bar.sync without a partner.)
    int slot = 0, grp = 0, released = 0;
    uint32_t ph = 0;
    bool ok = true;
    // stall test (DH_OPT_TEST_STALL): a bounded wait on the barrier that completes only after
    // the MMA warp's last stage runs out, and the launch takes its abort path from stage 0
    if (stall_cycles > 0) ok = __all_sync(0xffffffffu, mbar_wait(mma_done, 0, stall_cycles));
    for (int u = blockIdx.x; u < total_units; u += gridDim.x) {
      for (int g0 = 0; g0 < stages_per_unit; g0 += C::GROUP, ++grp) {
        const int n = stages_per_unit - g0 < C::GROUP ? stages_per_unit - g0 : C::GROUP;
        if (ok) ok = !__any_sync(0xffffffffu, *abort_flag != 0) &&
                     __all_sync(0xffffffffu, mbar_wait(&acc_empty[grp % C::NB], ((grp / C::NB) & 1) ^ 1));
        for (int i = 0; i < n; ++i) {
          if (ok) ok = !__any_sync(0xffffffffu, *abort_flag != 0) && __all_sync(0xffffffffu, mbar_wait(&full[slot], ph));
          if (!ok) {
            if (lane == 0 && !*abort_flag) fail();
            // without the data wait, keep at most one pending arrival on this named barrier:
            // wait (bounded) for the MMAs of the stage C::STAGES before, which the MMA warp
            // issued after passing the barrier for that stage
            if (released >= C::STAGES) (void)__all_sync(0xffffffffu, mbar_wait(&empty[slot], ph ^ 1));
          }
          named_arrive(1 + slot, 64);
          ++released;
          if (++slot == C::STAGES) { slot = 0; ph ^= 1; }
        }
      }
    }
  } else {  // ------------------------------ epilogue warps
    const int e = warp - 2;
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int ch = e >> 2;                  // which NCOL-column part of the chunk
    const int L = 32 * q + lane;            // accumulator row = TMEM lane
    const int c = L / C::M2, r = L % C::M2; // stacked chunk, row within the chunk
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    int grp = 0;
    // loop exits and waits are decided warp-uniformly (tcgen05.ld is .sync.aligned)
    for (int u = blockIdx.x; u < total_units && !__any_sync(0xffffffffu, *abort_flag); u += gridDim.x) {
      const int w = u / units_pw, uu = u % units_pw;
      // Per-stage values are added plainly into a block sum; every kBlock drains the block is
      // merged into the unit sum -- compensated (Kahan) where registers allow (T <= 32), plain
      // for T = 64. (Kahan on every drain was measured to halve the kernel's bandwidth.)
      constexpr int kBlock = 8;
      constexpr bool kKahan = C::KAHAN;
      float s[C::NCOL], blk[C::NCOL], comp[kKahan ? C::NCOL : 1];
#pragma unroll
      for (int j = 0; j < C::NCOL; ++j) s[j] = 0.f, blk[j] = 0.f;
#pragma unroll
      for (int j = 0; j < (kKahan ? C::NCOL : 1); ++j) comp[j] = 0.f;
      auto merge = [&]() {
#pragma unroll
        for (int i = 0; i < C::NCOL; ++i) {
          if constexpr (kKahan) {
            const float y = blk[i] - comp[i];
            const float t = s[i] + y;
            comp[i] = (t - s[i]) - y;
            s[i] = t;
          } else {
            s[i] += blk[i];
          }
          blk[i] = 0.f;
        }
      };
      int nd = 0;
      bool ok = true;
      for (int g0 = 0; g0 < stages_per_unit; g0 += C::GROUP, ++grp) {
        const int buf = grp % C::NB;
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (grp / C::NB) & 1))) {
          fail(); ok = false; break;
        }
        fence_after_sync();
        const uint32_t ta = tmem + lane_addr + buf * 128 + c * C::M2 + ch * C::NCOL;
#pragma unroll
        for (int h = 0; h < C::NCOL / 32; ++h) {
          float v[32];
          tmem_ld32(ta + 32 * h, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) blk[32 * h + i] += v[i];
        }
        fence_before_sync();
        mbar_arrive(&acc_empty[buf]);
        if (++nd == kBlock) { nd = 0; merge(); }
      }
      if (!ok) break;
      merge();
      double *dst = part + ((long long)(w * units_pw + uu) * C::R + c) * C::M2 * C::M2 +
                    (long long)r * C::M2 + ch * C::NCOL;
#pragma unroll
      for (int j = 0; j < C::NCOL; ++j) {
        if constexpr (kKahan) dst[j] = (double)s[j] - (double)comp[j];
        else dst[j] = (double)s[j];
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// ======================================================================= raw-domain covariance
// The Fresnel transform of Eq. 1 is unitary per frame, so C = H^{t*} H = I^T I exactly: the
// covariance can be formed from the uint16 frames themselves, exactly, at half the bytes of
// the 16-bit holograms. Each value is split I = 256 hi + lo (hi, lo < 256, exact in FP16); a
// converter warpgroup turns each TMA-loaded uint16 tile (T frames x 256 pixels: each frame
// read as one 512-byte run) into the operand rows [hi_0; lo_0; hi_1; lo_1; ...] of 64-pixel
// chunks (2T rows, K-major, 128-byte swizzle: the layout the hologram Gram reads), and the
// same stacked 128 x 128 MMA forms the 2T x 2T Gram G of those rows. Products are < 2^16 and
// a drain sums 128 of them per element (two operand stages), so every drained accumulator
// value is an exact integer below 2^23; the epilogue adds each drained value to
// a 32-bit integer sum (through the FP32 mantissa: bits(v + 2^23) = 0x4B000000 + v), which is
// exact while a unit's sum stays below 2^32 (<= 65536 pixels per unit). The reduction then
// forms C = 65536 G_hh + 256 (G_hl + G_lh) + G_ll in FP64, exact while sum I^2 < 2^53.
template <int T>
struct RawCfg {
  static constexpr int M2 = 2 * T;
  static constexpr int R = 128 / M2;               // 64-pixel chunks stacked per stage
  static constexpr int PIX = 64 * R;               // pixels per operand stage
  static constexpr int OP_BYTES = 128 * 128;       // operand stage: 128 rows x 64 pixels, FP16
  // uint16 stage: one TMA box of T frames x BOXP pixels (rows 512 bytes apart, no swizzle), so
  // each frame is read in 512-byte runs; it feeds OPS_PER_RAW operand stages
  static constexpr int BOXP = 256;
  static constexpr int RAW_BYTES = BOXP * T * 2;
  static constexpr int OPS_PER_RAW = BOXP / PIX;
  // operand stages accumulated per TMEM drain: a drained value sums GROUP * 64 byte products
  // (< 2^16 each), which must stay below 2^23 for the epilogue's exact integer sums
  static constexpr int GROUP = 2;
  static_assert(GROUP * 64 * 255 * 255 < (1 << 23), "drained sums must stay exact");
  static constexpr int NCOL = T == 64 ? 64 : 32;
  static constexpr int EPI_WARPS = 4 * (M2 / NCOL);
  // converter threads: two warps per SM sub-partition where the registers allow (T = 32; T = 16
  // runs two CTAs per SM, T = 64 needs more registers a thread)
  static constexpr int CONV_THREADS = T == 32 ? 256 : 128;
  static constexpr int WAITER = 2 + CONV_THREADS / 32 + EPI_WARPS;  // watches the mbarriers
  static constexpr int THREADS = 64 + CONV_THREADS + 32 * EPI_WARPS + 32;
  static constexpr int CTAS_PER_SM = T == 16 ? 2 : 1;
  static constexpr int OP_STAGES = CTAS_PER_SM == 2 ? 3 : 6;
  static constexpr int RAW_STAGES = CTAS_PER_SM == 2 ? 4 : 98304 / RAW_BYTES;  // 6 (T = 32), 3 (T = 64)
  static constexpr int NB = CTAS_PER_SM == 2 ? 2 : 4;
  static constexpr int TMEM_COLS = 128 * NB;
  static constexpr size_t SMEM = OP_STAGES * OP_BYTES + RAW_STAGES * RAW_BYTES + 1024 + 512;
};

// Split-K units per window for the raw-domain covariance: the tensor-core units, more where
// needed to keep <= 65536 pixels a unit (exact 32-bit sums).
int gram_raw_units(long long npix) {
  long long u = gram_tc_units(npix);
  const long long need = (npix + 65535) / 65536;
  return (int)(u > need ? u : need);
}

// Bytes SEL picks of w (one per 16-bit lane; 0x4341: bytes 1 and 3, 0x4240: bytes 0 and 2) as
// FP16 values: each byte b goes under the exponent byte 0x64 (one byte permute), which is
// FP16 1024 + b exactly, and 1024 is subtracted.
template <uint32_t SEL>
__device__ __forceinline__ uint32_t bytes_to_half2(uint32_t w) {
  const uint32_t h = __byte_perm(w, 0x64646464u, SEL);
  __half2 x = *reinterpret_cast<const __half2 *>(&h);
  x = __hsub2(x, __half2(__float2half(1024.f), __float2half(1024.f)));
  return *reinterpret_cast<uint32_t *>(&x);
}

template <int T>
__global__ void __launch_bounds__(RawCfg<T>::THREADS, 1)
k_gram_raw_tc(const __grid_constant__ CUtensorMap tmI, int first_frame, int window_stride, int n_windows,
              int units_pw, int stages_per_unit, double *__restrict__ part, uint32_t *__restrict__ status) {
  using C = RawCfg<T>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *ops = smem;
  uint8_t *raws = smem + C::OP_STAGES * C::OP_BYTES;
  uint64_t *bars = reinterpret_cast<uint64_t *>(raws + C::RAW_STAGES * C::RAW_BYTES);
  uint64_t *raw_full = bars, *raw_empty = raw_full + C::RAW_STAGES;
  uint64_t *op_full = raw_empty + C::RAW_STAGES, *op_empty = op_full + C::OP_STAGES;
  uint64_t *acc_full = op_empty + C::OP_STAGES, *acc_empty = acc_full + C::NB;
  uint64_t *mma_done = acc_empty + C::NB;
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(mma_done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::RAW_STAGES; ++s) { mbar_init(&raw_full[s], 1); mbar_init(&raw_empty[s], C::CONV_THREADS); }
    for (int s = 0; s < C::OP_STAGES; ++s) { mbar_init(&op_full[s], C::CONV_THREADS); mbar_init(&op_empty[s], 1); }
    for (int b = 0; b < C::NB; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 32 * C::EPI_WARPS); }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_barrier_init();
    prefetch_tmap(&tmI);
  }
  if (warp == 1) { tmem_alloc(tmem_holder, C::TMEM_COLS); tmem_relinquish(); }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  const int total_units = n_windows * units_pw;
  auto fail = [&]() { atomicOr(status, DH_FLAG_WAIT_TIMEOUT); *abort_flag = 1; };
  constexpr int CONV_W0 = 2, EPI_W0 = 2 + C::CONV_THREADS / 32;

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer: uint16 tiles
      int slot = 0; uint32_t ph = 0;
      long long issued = 0;
      for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x) {
        const int w = u / units_pw, uu = u % units_pw;
        const int f0 = first_frame + w * window_stride;
        const long long p0 = (long long)uu * stages_per_unit * C::PIX;
        for (int st = 0; st < stages_per_unit / C::OPS_PER_RAW; ++st) {
          if (!mbar_wait(&raw_empty[slot], ph ^ 1)) { fail(); break; }
          mbar_arrive_expect_tx(&raw_full[slot], C::RAW_BYTES);
          tma_load_2d(raws + slot * C::RAW_BYTES, &tmI, &raw_full[slot], (int)(p0 + st * C::BOXP), f0);
          ++issued;
          if (++slot == C::RAW_STAGES) { slot = 0; ph ^= 1; }
        }
      }
      if (*abort_flag) {  // let copies still in flight land before the CTA exits
        for (int k = 0; k < C::RAW_STAGES && k < issued; ++k) {
          if (--slot < 0) { slot = C::RAW_STAGES - 1; ph ^= 1; }
          mbar_wait(&raw_full[slot], ph);
        }
      }
    }
  } else if (warp == 1) {  // ---------------- MMA issuer (the whole warp; lane 0 issues)
    // Operand stage k waits on named barrier 1 + k % OP_STAGES, passed by the waiter once the
    // converters have filled it and, for a group's first stage, the accumulator is free; no
    // shared-memory step inside the loop (see named_sync) and no exit of its own.
    constexpr uint32_t idesc = idesc_f16(false, false, false, 128, 128);
    int slot = 0, grp = 0;
    for (int u = blockIdx.x; u < total_units; u += gridDim.x) {
      for (int g0 = 0; g0 < stages_per_unit; g0 += C::GROUP, ++grp) {
        const int n = stages_per_unit - g0 < C::GROUP ? stages_per_unit - g0 : C::GROUP;
        const uint32_t d = tmem + (grp % C::NB) * 128;
        for (int i = 0; i < n; ++i) {
          named_sync(1 + slot, 64);
          fence_after_sync();
          if (lane == 0) {
            const uint32_t base = smem_u32(ops + slot * C::OP_BYTES);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint64_t desc = smem_desc(base + 32 * k, 16, 1024, kSwizzle128);
              mma_f16(d, desc, desc, idesc, (i > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit(&op_empty[slot]);
          }
          __syncwarp();
          if (++slot == C::OP_STAGES) slot = 0;
        }
        if (lane == 0) mma_commit(&acc_full[grp % C::NB]);
        __syncwarp();
      }
    }
    if (lane == 0) mma_commit(mma_done);  // every MMA completes before the tensor memory is freed
    __syncwarp();
    mbar_wait(mma_done, 0);
  } else if (warp == C::WAITER) {  // ---------------- waiter (see k_gram_tc)
    int slot = 0, grp = 0, released = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < total_units; u += gridDim.x) {
      for (int g0 = 0; g0 < stages_per_unit; g0 += C::GROUP, ++grp) {
        const int n = stages_per_unit - g0 < C::GROUP ? stages_per_unit - g0 : C::GROUP;
        if (ok) ok = !__any_sync(0xffffffffu, *abort_flag != 0) &&
                     __all_sync(0xffffffffu, mbar_wait(&acc_empty[grp % C::NB], ((grp / C::NB) & 1) ^ 1));
        for (int i = 0; i < n; ++i) {
          if (ok) ok = !__any_sync(0xffffffffu, *abort_flag != 0) && __all_sync(0xffffffffu, mbar_wait(&op_full[slot], ph));
          if (!ok) {
            if (lane == 0 && !*abort_flag) fail();
            // without the data wait, keep at most one pending arrival on this named barrier:
            // wait (bounded) for the MMAs of the stage C::OP_STAGES before, which the MMA warp
            // issued after passing the barrier for that stage
            if (released >= C::OP_STAGES) (void)__all_sync(0xffffffffu, mbar_wait(&op_empty[slot], ph ^ 1));
          }
          named_arrive(1 + slot, 64);
          ++released;
          if (++slot == C::OP_STAGES) { slot = 0; ph ^= 1; }
        }
      }
    }
  } else if (warp < EPI_W0) {  // ---------------- converters: uint16 -> FP16 hi / lo rows
    const int ct = threadIdx.x - 32 * CONV_W0;
    int rslot = 0, oslot = 0; uint32_t rph = 0, oph = 0;
    for (int u = blockIdx.x; u < total_units && !__any_sync(0xffffffffu, *abort_flag); u += gridDim.x) {
      bool ok = true;
      for (int st = 0; st < stages_per_unit / C::OPS_PER_RAW && ok; ++st) {
        if (!__all_sync(0xffffffffu, mbar_wait(&raw_full[rslot], rph))) { fail(); ok = false; break; }
        for (int o = 0; o < C::OPS_PER_RAW; ++o) {
        if (!__all_sync(0xffffffffu, mbar_wait(&op_empty[oslot], oph ^ 1))) { fail(); ok = false; break; }
        // frame t's pixels of this operand stage: 512-byte rows, operand stage o at o * PIX pixels
        const uint8_t *src = raws + rslot * C::RAW_BYTES + o * C::PIX * 2;
        uint8_t *dst = ops + oslot * C::OP_BYTES;
#pragma unroll
        for (int it = 0; it < C::R * T * 8 / C::CONV_THREADS; ++it) {
          const int item = ct + it * C::CONV_THREADS;   // (chunk c, frame t, 16-byte column j)
          const int j = item & 7, t = (item >> 3) % T, c = (item >> 3) / T;
          const uint4 v = *reinterpret_cast<const uint4 *>(src + t * (C::BOXP * 2) + c * 128 + (j << 4));
          uint4 hi, lo;
          hi.x = bytes_to_half2<0x4341u>(v.x); lo.x = bytes_to_half2<0x4240u>(v.x);
          hi.y = bytes_to_half2<0x4341u>(v.y); lo.y = bytes_to_half2<0x4240u>(v.y);
          hi.z = bytes_to_half2<0x4341u>(v.z); lo.z = bytes_to_half2<0x4240u>(v.z);
          hi.w = bytes_to_half2<0x4341u>(v.w); lo.w = bytes_to_half2<0x4240u>(v.w);
          const int rh = c * C::M2 + 2 * t, rl = rh + 1;  // operand rows of hi_t and lo_t
          *reinterpret_cast<uint4 *>(dst + rh * 128 + ((j ^ (rh & 7)) << 4)) = hi;
          *reinterpret_cast<uint4 *>(dst + rl * 128 + ((j ^ (rl & 7)) << 4)) = lo;
        }
        // the tensor cores read the operand through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&op_full[oslot]);
        if (++oslot == C::OP_STAGES) { oslot = 0; oph ^= 1; }
        }
        if (!ok) break;
        mbar_arrive(&raw_empty[rslot]);
        if (++rslot == C::RAW_STAGES) { rslot = 0; rph ^= 1; }
      }
      if (!ok) break;
    }
  } else {  // ------------------------------ epilogue warps
    const int e = warp - EPI_W0;
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int ch = e >> 2;                  // which NCOL-column part of the chunk
    const int L = 32 * q + lane;            // accumulator row = TMEM lane
    const int c = L / C::M2, r = L % C::M2;
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    int grp = 0;
    for (int u = blockIdx.x; u < total_units && !__any_sync(0xffffffffu, *abort_flag); u += gridDim.x) {
      const int w = u / units_pw, uu = u % units_pw;
      uint32_t acc[C::NCOL];
#pragma unroll
      for (int j = 0; j < C::NCOL; ++j) acc[j] = 0u;
      bool ok = true;
      uint32_t drains = 0;
      for (int g0 = 0; g0 < stages_per_unit; g0 += C::GROUP, ++grp, ++drains) {
        const int buf = grp % C::NB;
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (grp / C::NB) & 1))) {
          fail(); ok = false; break;
        }
        fence_after_sync();
        const uint32_t ta = tmem + lane_addr + buf * 128 + c * C::M2 + ch * C::NCOL;
#pragma unroll
        for (int h = 0; h < C::NCOL / 32; ++h) {
          float v[32];
          tmem_ld32(ta + 32 * h, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[32 * h + i] += (uint32_t)__float_as_int(v[i] + 8388608.f);
        }
        fence_before_sync();
        mbar_arrive(&acc_empty[buf]);
      }
      if (!ok) break;
      // remove the 0x4B000000 of every drained value (mod 2^32)
      const uint32_t bias = drains * 0x4B000000u;
      double *dst = part + ((long long)(w * units_pw + uu) * C::R + c) * C::M2 * C::M2 +
                    (long long)r * C::M2 + ch * C::NCOL;
#pragma unroll
      for (int j = 0; j < C::NCOL; ++j) dst[j] = (double)(acc[j] - bias);
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// ======================================================================= projection
template <int T>
struct ProjCfg {
  static constexpr int M2 = 2 * T;                         // K of the MMA
  static constexpr int A_BYTES = 128 * M2 * 2;             // 128 pixels x 2T rows
  static constexpr int BOX_BYTES = 64 * M2 * 2;            // one 64-pixel TMA box
  static constexpr int STAGES = T == 64 ? 3 : (T == 32 ? 5 : 8);  // two CTAs per SM
  static constexpr int KB = M2 < 64 ? M2 : 64;             // B row width per swizzle atom
  static constexpr int B_ROW = KB * 2;                     // bytes
  static constexpr int B_MAX = 2 * M2 * M2 * 2;            // hi + lo, Npad <= 2T
  static constexpr int TMEM_COLS = M2 <= 32 ? 64 : 2 * M2; // two accumulators
  static constexpr int WAITER = 6;                         // after the 4 epilogue warps
  static constexpr int THREADS = 64 + 128 + 32;
  static constexpr size_t SMEM = STAGES * A_BYTES + B_MAX + 1024 + 256;
};

// RESID (mean-residual storage: the holograms hold D = H - mu 1^T; mu FP32 planes
// [window][re|im][npix]):
//   1  each accumulator column j of pixel p gets mu_r(p) a_j + mu_i(p) b_j added before it is
//      squared (a, b per window from k_mu_coef, 4T floats apart);
//   2  the u-column form (residual.cu): columns Npad - 2 and Npad - 1 hold D u, and the power
//      is the plain sum over the other columns + 2 Re(conj(mu) D u) + |mu|^2 sigma (sigma the
//      window's first coefficient).
template <int T, bool BF16, int RESID>
__global__ void __launch_bounds__(ProjCfg<T>::THREADS, 1)
k_project_tc(const __grid_constant__ CUtensorMap tmH, const __grid_constant__ CUtensorMap tmB,
             int first_slot, int slot_stride, int n_windows, int tiles_pw, int Npad, int B_rows_pw,
             int b_row0, float *__restrict__ images, int nx, int ny, uint32_t *__restrict__ status,
             const float *__restrict__ mu, const float *__restrict__ coef) {
  using C = ProjCfg<T>;
  const long long npix = (long long)nx * ny;
  // Holograms are stored with column-major pixels p = kx n_y + ky, so a 128-pixel tile is
  // (part of) one image column. When n_y >= 128, tiles come in groups of 8 adjacent
  // columns over the same 128 rows: the epilogue stages the group's powers in shared
  // memory and writes 32 contiguous bytes per image row instead of 4 scattered bytes.
  const bool grouped = ny >= 128 && (nx % 8) == 0;
  auto tile_p = [&](int t) -> int {
    if (!grouped) return t * 128;
    const int g = t >> 3, k = t & 7, gx = nx >> 3;
    return ((g % gx) * 8 + k) * ny + (g / gx) * 128;
  };
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *stages = smem;
  uint8_t *bsm = smem + C::STAGES * C::A_BYTES;
  uint64_t *full = reinterpret_cast<uint64_t *>(bsm + C::B_MAX);
  uint64_t *empty = full + C::STAGES;
  uint64_t *acc_full = empty + C::STAGES;
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *bfull = acc_empty + 2;
  uint64_t *bempty = bfull + 1;
  uint64_t *mma_done = bempty + 1;
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(mma_done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long total = (long long)n_windows * tiles_pw;
  // CTAs take contiguous ranges of whole units: 8-tile groups when grouped (tiles_pw is
  // then a multiple of 8), single tiles otherwise
  const int unit = grouped ? 8 : 1;
  const long long units = total / unit;
  const long long uper = units / gridDim.x, urem = units % gridDim.x;
  const long long t_begin = unit * (blockIdx.x * uper + (blockIdx.x < urem ? blockIdx.x : urem));
  const long long t_end = t_begin + unit * (uper + (blockIdx.x < urem ? 1 : 0));

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 128); }
    mbar_init(bfull, 1);
    mbar_init(bempty, 1);
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_barrier_init();
    prefetch_tmap(&tmH);
    prefetch_tmap(&tmB);
  }
  if (warp == 1) { tmem_alloc(tmem_holder, C::TMEM_COLS); tmem_relinquish(); }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  auto fail = [&]() { atomicOr(status, DH_FLAG_WAIT_TIMEOUT); *abort_flag = 1; };
  const int b_half_bytes = Npad * C::B_ROW * (C::M2 / C::KB);  // one of hi / lo

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer
      int slot = 0; uint32_t ph = 0, bph = 0;
      int cur_w = -1;
      long long issued = 0;
      bool b_pending = false;
      for (long long t = t_begin; t < t_end && !*abort_flag; ++t) {
        const int w = (int)(t / tiles_pw);
        const int p = tile_p((int)(t % tiles_pw));
        if (w != cur_w) {  // eigenvector operand of this window
          if (!mbar_wait(bempty, bph ^ 1)) { fail(); break; }
          mbar_arrive_expect_tx(bfull, 2 * b_half_bytes);
          for (int half = 0; half < 2; ++half)
            for (int kh = 0; kh < C::M2 / C::KB; ++kh)
              tma_load_2d(bsm + half * b_half_bytes + kh * Npad * C::B_ROW, &tmB, bfull, kh * C::KB,
                          b_row0 + w * B_rows_pw + half * Npad);
          b_pending = true;
          bph ^= 1;
          cur_w = w;
        }
        if (!mbar_wait(&empty[slot], ph ^ 1)) { fail(); break; }
        mbar_arrive_expect_tx(&full[slot], C::A_BYTES);
        const int row = 2 * (first_slot + w * slot_stride);
        uint8_t *dst = stages + slot * C::A_BYTES;
        tma_load_3d(dst, &tmH, &full[slot], 0, row, p >> 6);
        tma_load_3d(dst + C::BOX_BYTES, &tmH, &full[slot], 0, row, (p >> 6) + 1);
        ++issued;
        if (++slot == C::STAGES) { slot = 0; ph ^= 1; }
      }
      if (*abort_flag) {
        for (int k = 0; k < C::STAGES && k < issued; ++k) {
          if (--slot < 0) { slot = C::STAGES - 1; ph ^= 1; }
          mbar_wait(&full[slot], ph);
        }
        if (b_pending) mbar_wait(bfull, bph ^ 1);
      }
    }
  } else if (warp == 1) {  // ---------------- MMA issuer (whole warp, lane 0 issues)
    // Tile k waits on named barrier 1 + k % STAGES, passed by the waiter once the tile has
    // landed, its accumulator buffer is free and (first tile of a window) the window's operand
    // is in place; no shared-memory step inside the loop (see named_sync).
    const uint32_t idesc = idesc_f16(BF16, true, false, 128, Npad);
    int slot = 0, it = 0;
    for (long long t = t_begin; t < t_end; ++t, ++it) {
      const int w = (int)(t / tiles_pw);
      const int buf = it & 1;
      named_sync(1 + slot, 64);
      fence_after_sync();
      if (lane == 0) {
        const uint32_t d = tmem + buf * C::M2;
        const uint32_t a0 = smem_u32(stages + slot * C::A_BYTES);
        const uint32_t b0 = smem_u32(bsm);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
#pragma unroll
          for (int k = 0; k < C::M2 / 16; ++k) {
            const uint64_t adesc = smem_desc(a0 + k * 16 * 128, C::BOX_BYTES, 1024, kSwizzle128);
            uint64_t bdesc;
            if constexpr (T == 16) {
              bdesc = smem_desc(b0 + half * b_half_bytes + k * 32, 16, 512, kSwizzle64);
            } else {
              const uint32_t sub = (uint32_t)((k * 16) / C::KB);
              bdesc = smem_desc(b0 + half * b_half_bytes + sub * Npad * C::B_ROW + ((k * 32) % 128), 16,
                                1024, kSwizzle128);
            }
            mma_f16(d, adesc, bdesc, idesc, (half > 0 || k > 0) ? 1u : 0u);
          }
        }
        mma_commit(&empty[slot]);
        mma_commit(&acc_full[buf]);
        const bool last_of_window = (t + 1 == t_end) || ((int)((t + 1) / tiles_pw) != w);
        if (last_of_window) mma_commit(bempty);
      }
      __syncwarp();
      if (++slot == C::STAGES) slot = 0;
    }
    if (lane == 0) mma_commit(mma_done);  // every MMA completes before the tensor memory is freed
    __syncwarp();
    mbar_wait(mma_done, 0);
  } else if (warp == C::WAITER) {  // ---------------- waiter
    // Fewer than STAGES tiles ahead of the MMA warp (a tile's data needs its slot released by
    // the MMAs of the tile STAGES before): one pending arrival per named barrier at most. After
    // a failed wait or an abort it stops waiting for data and arrives once the MMAs of the
    // tile STAGES before have completed (see k_gram_tc).
    int slot = 0, it = 0, cur_w = -1, released = 0;
    uint32_t ph = 0, bph = 0;
    bool ok = true;
    for (long long t = t_begin; t < t_end; ++t, ++it) {
      const int w = (int)(t / tiles_pw);
      const int buf = it & 1;
      if (ok && w != cur_w) {
        ok = !__any_sync(0xffffffffu, *abort_flag != 0) && __all_sync(0xffffffffu, mbar_wait(bfull, bph));
        bph ^= 1;
        cur_w = w;
      }
      if (ok) ok = !__any_sync(0xffffffffu, *abort_flag != 0) &&
                   __all_sync(0xffffffffu, mbar_wait(&acc_empty[buf], ((it >> 1) & 1) ^ 1)) &&
                   __all_sync(0xffffffffu, mbar_wait(&full[slot], ph));
      if (!ok) {
        if (lane == 0 && !*abort_flag) fail();
        // without the data wait, keep at most one pending arrival on this named barrier:
        // wait (bounded) for the MMAs of the stage C::STAGES before, which the MMA warp
        // issued after passing the barrier for that stage
        if (released >= C::STAGES) (void)__all_sync(0xffffffffu, mbar_wait(&empty[slot], ph ^ 1));
      }
      named_arrive(1 + slot, 64);
      ++released;
      if (++slot == C::STAGES) { slot = 0; ph ^= 1; }
    }
  } else {  // ------------------------------ epilogue: 4 warps, one pixel per TMEM lane
    const int q = warp & 3;
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    float g8[8];
    int it = 0;
    for (long long t = t_begin; t < t_end && !__any_sync(0xffffffffu, *abort_flag); ++t, ++it) {
      const int w = (int)(t / tiles_pw);
      const int p = tile_p((int)(t % tiles_pw)) + 32 * q + lane;
      const int kx = p / ny, ky = p % ny;
      const int buf = it & 1;
      // u-column form: mu and sigma are loaded before the accumulator wait, which hides their
      // latency
      float mr = 0.f, mi = 0.f, sig = 0.f;
      if constexpr (RESID == 2) {
        const float *mw = mu + (long long)w * 2 * npix;
        mr = __ldg(mw + p);
        mi = __ldg(mw + npix + p);
        sig = __ldg(coef + (long long)w * 4 * T);  // the same on every lane
      }
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (it >> 1) & 1))) { fail(); break; }
      fence_after_sync();
      float m = 0.f;
      const uint32_t ta = tmem + lane_addr + buf * C::M2;
      int col = 0;
      if constexpr (RESID == 0) {
        for (; col + 64 <= Npad; col += 64) {
          float v[64];
          tmem_ld64(ta + col, v);
#pragma unroll
          for (int i = 0; i < 64; ++i) m = fmaf(v[i], v[i], m);
        }
        for (; col < Npad; col += 16) {
          float v[16];
          tmem_ld16(ta + col, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) m = fmaf(v[i], v[i], m);
        }
      } else if constexpr (RESID == 2) {
        // up to 64 columns a pass, their loads issued together and waited on once; the 16-column
        // chunk that ends at Npad holds Re and Im of D u in its last two columns (Npad is a
        // multiple of 16, and every condition below is the same on every lane)
        float du_r = 0.f, du_i = 0.f;
        for (int base = 0; base < Npad; base += 64) {
          float v[64];
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (base + 16 * c < Npad) tmem_ld16_nowait(ta + base + 16 * c, *reinterpret_cast<float(*)[16]>(&v[16 * c]));
          tmem_wait_ld(v);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (base + 16 * c < Npad) {
#pragma unroll
              for (int i = 0; i < 14; ++i) m = fmaf(v[16 * c + i], v[16 * c + i], m);
              if (base + 16 * c + 16 == Npad) {
                du_r = v[16 * c + 14];
                du_i = v[16 * c + 15];
              } else {
                m = fmaf(v[16 * c + 14], v[16 * c + 14], m);
                m = fmaf(v[16 * c + 15], v[16 * c + 15], m);
              }
            }
          }
        }
        m = fmaf(2.f, fmaf(mr, du_r, mi * du_i), m);
        m = fmaf(sig, fmaf(mr, mr, mi * mi), m);
        m = fmaxf(m, 0.f);
      } else {  // coefficients: the same address on every lane (one broadcast load each)
        const float *mw = mu + (long long)w * 2 * npix;
        const float mr = __ldg(mw + p), mi = __ldg(mw + npix + p);
        const float4 *ca = reinterpret_cast<const float4 *>(coef + (long long)w * 4 * T);
        const float4 *cb = reinterpret_cast<const float4 *>(coef + (long long)w * 4 * T + 2 * T);
        for (; col < Npad; col += 16) {
          float v[16];
          tmem_ld16(ta + col, v);
#pragma unroll
          for (int i = 0; i < 16; i += 4) {
            const float4 a = __ldg(ca + (col + i) / 4), b = __ldg(cb + (col + i) / 4);
            const float x0 = fmaf(mr, a.x, fmaf(mi, b.x, v[i]));
            const float x1 = fmaf(mr, a.y, fmaf(mi, b.y, v[i + 1]));
            const float x2 = fmaf(mr, a.z, fmaf(mi, b.z, v[i + 2]));
            const float x3 = fmaf(mr, a.w, fmaf(mi, b.w, v[i + 3]));
            m = fmaf(x0, x0, m);
            m = fmaf(x1, x1, m);
            m = fmaf(x2, x2, m);
            m = fmaf(x3, x3, m);
          }
        }
      }
      fence_before_sync();
      mbar_arrive(&acc_empty[buf]);
      if (!grouped) {
        images[(long long)w * npix + (long long)ky * nx + kx] = m;
      } else {  // shift this pixel's power into the row of 8 adjacent columns
        g8[7] = g8[6]; g8[6] = g8[5]; g8[5] = g8[4]; g8[4] = g8[3];
        g8[3] = g8[2]; g8[2] = g8[1]; g8[1] = g8[0]; g8[0] = m;
        if ((t & 7) == 7) {  // columns kx-7 .. kx of image row ky
          float4 *dst = reinterpret_cast<float4 *>(images + (long long)w * npix + (long long)ky * nx + (kx - 7));
          dst[0] = make_float4(g8[7], g8[6], g8[5], g8[4]);
          dst[1] = make_float4(g8[3], g8[2], g8[1], g8[0]);
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// ======================================================================= host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

dh_status encode_2d(CUtensorMap *map, void *base, bool bf16, uint64_t inner, uint64_t outer,
                    uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz) {
  auto fn = encode_fn();
  if (!fn) return DH_ERR_CUDA;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base,
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? DH_OK : DH_ERR_CUDA;
}


// CTAs of `kern` that fit on one SM by shared memory (with the maximum carveout, which these
// kernels request) and by registers. The runtime's occupancy query assumes the default
// carveout and under-reports these kernels.
template <typename K>
dh_status resident_ctas(K kern, int threads, size_t smem, int *out) {
  int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0;
  DH_CUDA_TRY(cudaGetDevice(&dev));
  DH_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  DH_CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  DH_CUDA_TRY(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
  cudaFuncAttributes fa;
  DH_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
  const int by_smem = smem_sm / (int)(smem + reserved);
  const int regs_cta = ((fa.numRegs + 7) / 8 * 8) * ((threads + 31) / 32 * 32);
  const int by_regs = regs_cta > 0 ? regs_sm / regs_cta : 1;
  *out = by_smem < by_regs ? by_smem : by_regs;
  return DH_OK;
}

// SMs a persistent covariance or projection launch spreads over: all, or the plan's budget
// when an eigensolver runs beside it
int sm_share(const Plan &p) {
  return p.sm_budget > 0 && p.sm_budget < p.num_sms ? p.sm_budget : p.num_sms;
}

template <int T, bool BF16>
dh_status gram_t(Plan &p, int first_slot, int slot_stride, int n_windows, cudaStream_t s) {
  using C = GramCfg<T>;
  auto kern = k_gram_tc<T, BF16>;
  static bool attr = false;
  if (!attr) {
    DH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    DH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared));
    attr = true;
  }
  const int units_pw = gram_tc_units_of(p);
  const int stages_per_unit = (int)(p.npix / units_pw / C::PIX);
  const int total = n_windows * units_pw;
  int per_sm = 0;
  dh_status rs = resident_ctas(kern, C::THREADS, C::SMEM, &per_sm);
  if (rs != DH_OK) return rs;
  if (per_sm > C::CTAS_PER_SM) per_sm = C::CTAS_PER_SM;  // tensor memory: 512 columns per SM
  if (per_sm < 1) per_sm = 1;
  int grid = sm_share(p) * per_sm;
  if (grid > total) grid = total;
  ProfScope ps(p, K_GRAM_TC, s);
  kern<<<grid, C::THREADS, C::SMEM, s>>>(p.tmap_H, first_slot, slot_stride, n_windows, units_pw,
                                          stages_per_unit, p.d_part, p.d_status, p.test_stall);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

template <int T, bool BF16, int RESID>
dh_status project_t(Plan &p, int first_slot, int slot_stride, int n_windows, int Npad, float *images,
                    int woff, cudaStream_t s, const void *shared_op) {
  using C = ProjCfg<T>;
  auto kern = k_project_tc<T, BF16, RESID>;
  static bool attr = false;
  if (!attr) {
    DH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    DH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared));
    attr = true;
  }
  // eigenvector operand map: rows of 2T elements, box = KB x Npad
  const int M2 = 2 * T;
  const long long B_rows_pw = (long long)(p.B_window_bytes / (M2 * 2));
  // a shared operand is one window's rows, read by every window (row stride 0 per window)
  CUtensorMap tmB;
  dh_status st = encode_2d(&tmB, shared_op ? const_cast<void *>(shared_op) : p.d_B, BF16, (uint64_t)M2,
                           (uint64_t)(B_rows_pw * (shared_op ? 1 : p.max_windows)),
                           (uint64_t)M2 * 2, (uint32_t)C::KB, (uint32_t)Npad,
                           T == 16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
  if (st != DH_OK) return st;
  const int tiles_pw = (int)(p.npix / 128);
  const long long total = (long long)n_windows * tiles_pw;
  int per_sm = 0;
  dh_status rs = resident_ctas(kern, C::THREADS, C::SMEM, &per_sm);
  if (rs != DH_OK) return rs;
  if (per_sm < 1) per_sm = 1;
  if (per_sm * C::TMEM_COLS > 512) per_sm = 512 / C::TMEM_COLS;  // tensor memory per SM
  int grid = sm_share(p) * per_sm;
  if (grid > total) grid = (int)total;
  ProfScope ps(p, K_PROJECT_TC, s);
  kern<<<grid, C::THREADS, C::SMEM, s>>>(p.tmap_H, tmB, first_slot, slot_stride, n_windows, tiles_pw, Npad,
                                          shared_op ? 0 : (int)B_rows_pw,
                                          shared_op ? 0 : (int)(woff * B_rows_pw), images, p.nx, p.ny,
                                          p.d_status, RESID ? p.d_mu + 2ll * woff * p.npix : nullptr,
                                          RESID ? p.d_mucoef + 4ll * woff * p.T : nullptr);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}
template <int T>
dh_status gram_raw_t(Plan &p, const uint16_t *frames, long long frame_stride, int n_frames, int first_frame,
                     int window_stride, int n_windows, cudaStream_t s) {
  using C = RawCfg<T>;
  auto kern = k_gram_raw_tc<T>;
  static bool attr = false;
  if (!attr) {
    DH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    DH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared));
    attr = true;
  }
  // uint16 frames as a 2-D tensor: npix x n_frames, box BOXP pixels x T frames, no swizzle
  auto fn = encode_fn();
  if (!fn) return DH_ERR_CUDA;
  CUtensorMap tm;
  const cuuint64_t dims[2] = {(cuuint64_t)p.npix, (cuuint64_t)n_frames};
  const cuuint64_t strides[1] = {(cuuint64_t)frame_stride * 2};
  const cuuint32_t box[2] = {(cuuint32_t)C::BOXP, (cuuint32_t)T};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<uint16_t *>(frames), dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return DH_ERR_CUDA;
  const int units_pw = gram_raw_units(p.npix);
  // a unit's pixels: a whole number of uint16 boxes (npix >= 256, both powers of two)
  if ((p.npix / units_pw) % C::BOXP != 0) return DH_ERR_UNSUPPORTED_SIZE;
  const int stages_per_unit = (int)(p.npix / units_pw / C::PIX);
  const int total = n_windows * units_pw;
  int per_sm = 0;
  dh_status rs = resident_ctas(kern, C::THREADS, C::SMEM, &per_sm);
  if (rs != DH_OK) return rs;
  if (per_sm > C::CTAS_PER_SM) per_sm = C::CTAS_PER_SM;
  if (per_sm < 1) per_sm = 1;
  int grid = sm_share(p) * per_sm;
  if (grid > total) grid = total;
  ProfScope ps(p, K_GRAM_RAW, s);
  kern<<<grid, C::THREADS, C::SMEM, s>>>(tm, first_frame, window_stride, n_windows, units_pw, stages_per_unit,
                                          p.d_part, p.d_status);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}


}  // namespace

dh_status encode_3d(CUtensorMap *map, void *base, bool bf16, const uint64_t dims[3],
                    const uint64_t strides_bytes[2], const uint32_t box[3]) {
  auto fn = encode_fn();
  if (!fn) return DH_ERR_CUDA;
  const cuuint64_t d[3] = {dims[0], dims[1], dims[2]};
  const cuuint64_t st[2] = {strides_bytes[0], strides_bytes[1]};
  const cuuint32_t b[3] = {box[0], box[1], box[2]};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, base, d,
                  st, b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? DH_OK : DH_ERR_CUDA;
}

int gram_tc_parts(const Plan &p) { return gram_tc_units_of(p) * (128 / (2 * p.T)); }
int gram_tc_default_units(long long npix) { return gram_tc_units(npix); }

dh_status make_tensor_maps(Plan &p) {
  p.tmaps_ok = false;
  if (p.prec == DH_PREC_FP32) return DH_OK;
  const bool bf16 = p.prec == DH_PREC_BF16;
  const uint64_t rows = 2ull * p.max_frames;
  const uint64_t dims[3] = {64, rows, (uint64_t)p.npix / 64};
  const uint64_t strides[2] = {64 * 2, rows * 64 * 2};
  const uint32_t box[3] = {64, (uint32_t)(2 * p.T), 1};
  dh_status st = encode_3d(&p.tmap_H, p.d_H, bf16, dims, strides, box);
  if (st != DH_OK) return st;
  const uint32_t box_band[3] = {64, 128, 1};  // one 64-frame block of the banded Gram
  if ((st = encode_3d(&p.tmap_band, p.d_H, bf16, dims, strides, box_band)) != DH_OK) return st;
  p.tmaps_ok = true;
  return DH_OK;
}

dh_status launch_gram_tc(Plan &p, int first_slot, int slot_stride, int n_windows, int *parts_per_window,
                         cudaStream_t s) {
  if (!p.tmaps_ok) return DH_ERR_STATE;
  *parts_per_window = gram_tc_parts(p);
  const bool bf16 = p.prec == DH_PREC_BF16;
  switch (p.T) {
    case 16: return bf16 ? gram_t<16, true>(p, first_slot, slot_stride, n_windows, s)
                         : gram_t<16, false>(p, first_slot, slot_stride, n_windows, s);
    case 32: return bf16 ? gram_t<32, true>(p, first_slot, slot_stride, n_windows, s)
                         : gram_t<32, false>(p, first_slot, slot_stride, n_windows, s);
    case 64: return bf16 ? gram_t<64, true>(p, first_slot, slot_stride, n_windows, s)
                         : gram_t<64, false>(p, first_slot, slot_stride, n_windows, s);
  }
  return DH_ERR_UNSUPPORTED_SIZE;
}

int gram_raw_parts(const Plan &p) { return gram_raw_units(p.npix) * (128 / (2 * p.T)); }

dh_status launch_gram_raw(Plan &p, const uint16_t *frames, long long frame_stride, int n_frames,
                          int first_frame, int window_stride, int n_windows, int *parts_per_window,
                          cudaStream_t s) {
  *parts_per_window = gram_raw_parts(p);
  switch (p.T) {
    case 16: return gram_raw_t<16>(p, frames, frame_stride, n_frames, first_frame, window_stride, n_windows, s);
    case 32: return gram_raw_t<32>(p, frames, frame_stride, n_frames, first_frame, window_stride, n_windows, s);
    case 64: return gram_raw_t<64>(p, frames, frame_stride, n_frames, first_frame, window_stride, n_windows, s);
  }
  return DH_ERR_UNSUPPORTED_SIZE;
}

dh_status launch_project_tc(Plan &p, int first_slot, int slot_stride, int n_windows, int Npad,
                            float *images, int woff, cudaStream_t s, const void *shared_op) {
  if (!p.tmaps_ok) return DH_ERR_STATE;
  const bool bf16 = p.prec == DH_PREC_BF16;
  const int resid = p.residual && !shared_op ? (p.resid_ucol ? 2 : 1) : 0;
#define DH_PROJ_R(TT, BB)                                                                                    \
  return resid == 2 ? project_t<TT, BB, 2>(p, first_slot, slot_stride, n_windows, Npad, images, woff, s, shared_op) \
       : resid == 1 ? project_t<TT, BB, 1>(p, first_slot, slot_stride, n_windows, Npad, images, woff, s, shared_op) \
                    : project_t<TT, BB, 0>(p, first_slot, slot_stride, n_windows, Npad, images, woff, s, shared_op);
#define DH_PROJ(TT)                                                                                          \
  if (bf16) { DH_PROJ_R(TT, true) } else { DH_PROJ_R(TT, false) }
  switch (p.T) {
    case 16: DH_PROJ(16)
    case 32: DH_PROJ(32)
    case 64: DH_PROJ(64)
  }
#undef DH_PROJ
#undef DH_PROJ_R
  return DH_ERR_UNSUPPORTED_SIZE;
}

}  // namespace dh
