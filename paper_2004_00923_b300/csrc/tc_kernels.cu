// Eq. 4 and Eqs. 6-7 on the 5th-generation tensor cores (tcgen05, kind::f16, FP32
// accumulation in tensor memory), for holograms stored as 16-bit planes.
//
// Layout: the hologram store is one 2-D array of 2*frames rows by n_x n_y pixels; row
// 2f is Re H_f and row 2f+1 is Im H_f, so a window's X = [Re H_0; Im H_0; ...] is 2T
// consecutive rows. One TMA tensor map with 64-pixel x 2T-row boxes (128-byte swizzle)
// feeds both contractions:
//   * covariance (Eq. 4): G = X X^T over pixels, X K-major. 128/(2T) pixel chunks are
//     stacked into one 128-row operand used as both A and B of a 128x128 MMA; the
//     diagonal 2T x 2T blocks are the chunk Gram matrices (the off-diagonal blocks are
//     discarded). Products of stored 16-bit values are exact in FP32; TMEM accumulators
//     are flushed every stage into per-thread compensated (Kahan) FP32 sums, and
//     the per-unit partials are reduced in FP64 by the covariance reduction kernel.
//   * projection (Eqs. 6-7): P = X^T B^T per 128-pixel tile (A = X, MN-major), with B the
//     real embedding of the retained eigenvectors split into hi + lo 16-bit parts (two
//     MMAs into the same accumulator). The epilogue squares and sums the accumulator row
//     of each pixel straight into the image; P is never stored.
// Roles: warp 0 issues TMA, warp 1 issues MMAs (one thread), the remaining warps drain
// TMEM. Every mbarrier wait is bounded (tc::kWaitBudget); on expiry the CTA raises
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

// ======================================================================= covariance
template <int T>
struct GramCfg {
  static constexpr int M2 = 2 * T;                 // rows per window
  static constexpr int R = 128 / M2;               // pixel chunks stacked per stage
  static constexpr int PIX = 64 * R;               // pixels per stage
  static constexpr int STAGE_BYTES = 128 * 128;    // 128 rows x 64 pixels x 2 bytes
  static constexpr int STAGES = 6;
  // Stages per TMEM flush. The tensor cores' FP32 accumulation rounds toward zero (measured:
  // about -7e-8 relative per MMA instruction), so accumulators are drained into compensated
  // sums after every stage of 4 MMAs, bounding that bias near 3e-7.
  static constexpr int GROUP = 1;
  static constexpr int NCOL = M2 < 64 ? M2 : 64;   // columns each epilogue thread keeps
  static constexpr int EPI_WARPS = 4 * (M2 / NCOL);
  static constexpr int THREADS = 64 + 32 * EPI_WARPS;
  static constexpr int TMEM_COLS = 256;            // two 128-column accumulators
  static constexpr size_t SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};

template <int T, bool BF16>
__global__ void __launch_bounds__(GramCfg<T>::THREADS, 1)
k_gram_tc(const __grid_constant__ CUtensorMap tmH, int first_slot, int slot_stride, int n_windows,
          int units_pw, int stages_per_unit, double *__restrict__ part, uint32_t *__restrict__ status) {
  using C = GramCfg<T>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *stages = smem;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t *empty = full + C::STAGES;
  uint64_t *acc_full = empty + C::STAGES;
  uint64_t *acc_empty = acc_full + 2;
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(acc_empty + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 32 * C::EPI_WARPS); }
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
            tma_load_2d(dst + c * C::M2 * 128, &tmH, &full[slot], p0 + st * C::PIX + c * 64, row);
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
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer
      constexpr uint32_t idesc = idesc_f16(BF16, false, false, 128, 128);
      int slot = 0; uint32_t ph = 0; int grp = 0;
      for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x) {
        for (int g0 = 0; g0 < stages_per_unit && !*abort_flag; g0 += C::GROUP, ++grp) {
          const int n = stages_per_unit - g0 < C::GROUP ? stages_per_unit - g0 : C::GROUP;
          const int buf = grp & 1;
          if (!mbar_wait(&acc_empty[buf], ((grp >> 1) & 1) ^ 1)) { fail(); break; }
          fence_after_sync();
          const uint32_t d = tmem + buf * 128;
          for (int i = 0; i < n; ++i) {
            if (!mbar_wait(&full[slot], ph)) { fail(); break; }
            fence_after_sync();
            const uint32_t base = smem_u32(stages + slot * C::STAGE_BYTES);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint64_t desc = smem_desc(base + 32 * k, 16, 1024, kSwizzle128);
              mma_f16(d, desc, desc, idesc, (i > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit(&empty[slot]);
            if (++slot == C::STAGES) { slot = 0; ph ^= 1; }
          }
          mma_commit(&acc_full[buf]);
        }
      }
    }
  } else {  // ------------------------------ epilogue warps
    const int e = warp - 2;
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int ch = e >> 2;                  // column half (T = 64 only)
    const int L = 32 * q + lane;            // accumulator row = TMEM lane
    const int c = L / C::M2, r = L % C::M2; // stacked chunk, row within the chunk
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    int grp = 0;
    // loop exits and waits are decided warp-uniformly (tcgen05.ld is .sync.aligned)
    for (int u = blockIdx.x; u < total_units && !__any_sync(0xffffffffu, *abort_flag); u += gridDim.x) {
      const int w = u / units_pw, uu = u % units_pw;
      float s[C::NCOL], comp[C::NCOL];
#pragma unroll
      for (int j = 0; j < C::NCOL; ++j) s[j] = 0.f, comp[j] = 0.f;
      bool ok = true;
      for (int g0 = 0; g0 < stages_per_unit; g0 += C::GROUP, ++grp) {
        const int buf = grp & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (grp >> 1) & 1))) {
          fail(); ok = false; break;
        }
        fence_after_sync();
        const uint32_t ta = tmem + lane_addr + buf * 128 + c * C::M2 + ch * 64;
#pragma unroll
        for (int j16 = 0; j16 < C::NCOL / 16; ++j16) {
          float v[16];
          tmem_ld16(ta + 16 * j16, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) {  // compensated summation
            const float y = v[i] - comp[16 * j16 + i];
            const float t = s[16 * j16 + i] + y;
            comp[16 * j16 + i] = (t - s[16 * j16 + i]) - y;
            s[16 * j16 + i] = t;
          }
        }
        fence_before_sync();
        mbar_arrive(&acc_empty[buf]);
      }
      if (!ok) break;
      double *dst = part + ((long long)(w * units_pw + uu) * C::R + c) * C::M2 * C::M2 +
                    (long long)r * C::M2 + ch * 64;
#pragma unroll
      for (int j = 0; j < C::NCOL; ++j) dst[j] = (double)s[j] - (double)comp[j];
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
  static constexpr int THREADS = 64 + 128;
  static constexpr size_t SMEM = STAGES * A_BYTES + B_MAX + 1024 + 256;
};

template <int T, bool BF16>
__global__ void __launch_bounds__(ProjCfg<T>::THREADS, 1)
k_project_tc(const __grid_constant__ CUtensorMap tmH, const __grid_constant__ CUtensorMap tmB,
             int first_slot, int slot_stride, int n_windows, int tiles_pw, int Npad, int B_rows_pw,
             float *__restrict__ images, int nx, int ny, uint32_t *__restrict__ status) {
  using C = ProjCfg<T>;
  const long long npix = (long long)nx * ny;
  // Holograms are stored with column-major pixels p = kx n_y + ky; tiles walk p
  // contiguously (long sequential reads per plane row), and each pixel's power goes to its
  // row-major image position; the scattered 4-byte stores of neighbouring columns meet in L2.
  auto tile_p = [&](int t) -> int { return t * 128; };
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
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bempty + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long total = (long long)n_windows * tiles_pw;
  const long long per = total / gridDim.x, rem = total % gridDim.x;
  const long long t_begin = blockIdx.x * per + (blockIdx.x < rem ? blockIdx.x : rem);
  const long long t_end = t_begin + per + (blockIdx.x < rem ? 1 : 0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 128); }
    mbar_init(bfull, 1);
    mbar_init(bempty, 1);
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
                          w * B_rows_pw + half * Npad);
          b_pending = true;
          bph ^= 1;
          cur_w = w;
        }
        if (!mbar_wait(&empty[slot], ph ^ 1)) { fail(); break; }
        mbar_arrive_expect_tx(&full[slot], C::A_BYTES);
        const int row = 2 * (first_slot + w * slot_stride);
        uint8_t *dst = stages + slot * C::A_BYTES;
        tma_load_2d(dst, &tmH, &full[slot], p, row);
        tma_load_2d(dst + C::BOX_BYTES, &tmH, &full[slot], p + 64, row);
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
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer
      const uint32_t idesc = idesc_f16(BF16, true, false, 128, Npad);
      int slot = 0; uint32_t ph = 0, bph = 0;
      int cur_w = -1, it = 0;
      for (long long t = t_begin; t < t_end && !*abort_flag; ++t, ++it) {
        const int w = (int)(t / tiles_pw);
        if (w != cur_w) {
          if (!mbar_wait(bfull, bph)) { fail(); break; }
          bph ^= 1;
          cur_w = w;
        }
        const int buf = it & 1;
        if (!mbar_wait(&acc_empty[buf], ((it >> 1) & 1) ^ 1)) { fail(); break; }
        if (!mbar_wait(&full[slot], ph)) { fail(); break; }
        fence_after_sync();
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
        if (++slot == C::STAGES) { slot = 0; ph ^= 1; }
        const bool last_of_window = (t + 1 == t_end) || ((int)((t + 1) / tiles_pw) != w);
        if (last_of_window) mma_commit(bempty);
      }
    }
  } else {  // ------------------------------ epilogue: 4 warps, one pixel per TMEM lane
    const int q = warp & 3;
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    int it = 0;
    for (long long t = t_begin; t < t_end && !__any_sync(0xffffffffu, *abort_flag); ++t, ++it) {
      const int w = (int)(t / tiles_pw);
      const int p = tile_p((int)(t % tiles_pw)) + 32 * q + lane;
      const int kx = p / ny, ky = p % ny;
      const int buf = it & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (it >> 1) & 1))) { fail(); break; }
      fence_after_sync();
      float m = 0.f;
      for (int j16 = 0; j16 < Npad / 16; ++j16) {
        float v[16];
        tmem_ld16(tmem + lane_addr + buf * C::M2 + 16 * j16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) m = fmaf(v[i], v[i], m);
      }
      fence_before_sync();
      mbar_arrive(&acc_empty[buf]);
      images[(long long)w * npix + (long long)ky * nx + kx] = m;
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
  const int units_pw = gram_tc_units(p.npix);
  const int stages_per_unit = (int)(p.npix / units_pw / C::PIX);
  const int total = n_windows * units_pw;
  int per_sm = 0;
  DH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::THREADS, C::SMEM));
  if (per_sm > 2) per_sm = 2;  // tensor memory: two CTAs of 256 columns per SM
  if (per_sm < 1) per_sm = 1;
  int grid = p.num_sms * per_sm;
  if (grid > total) grid = total;
  ProfScope ps(p, K_GRAM_TC, s);
  kern<<<grid, C::THREADS, C::SMEM, s>>>(p.tmap_H, first_slot, slot_stride, n_windows, units_pw,
                                          stages_per_unit, p.d_part, p.d_status);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

template <int T, bool BF16>
dh_status project_t(Plan &p, int first_slot, int slot_stride, int n_windows, int Npad, float *images,
                    cudaStream_t s) {
  using C = ProjCfg<T>;
  auto kern = k_project_tc<T, BF16>;
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
  CUtensorMap tmB;
  dh_status st = encode_2d(&tmB, p.d_B, BF16, (uint64_t)M2, (uint64_t)(B_rows_pw * p.max_windows),
                           (uint64_t)M2 * 2, (uint32_t)C::KB, (uint32_t)Npad,
                           T == 16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
  if (st != DH_OK) return st;
  const int tiles_pw = (int)(p.npix / 128);
  const long long total = (long long)n_windows * tiles_pw;
  int per_sm = 0;
  DH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::THREADS, C::SMEM));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2) per_sm = 2;  // tensor memory: at most 2 x 256 columns per SM
  int grid = p.num_sms * per_sm;
  if (grid > total) grid = (int)total;
  ProfScope ps(p, K_PROJECT_TC, s);
  kern<<<grid, C::THREADS, C::SMEM, s>>>(p.tmap_H, tmB, first_slot, slot_stride, n_windows, tiles_pw, Npad,
                                          (int)B_rows_pw, images, p.nx, p.ny, p.d_status);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

}  // namespace

int gram_tc_parts(const Plan &p) { return gram_tc_units(p.npix) * (128 / (2 * p.T)); }

dh_status make_tensor_maps(Plan &p) {
  p.tmaps_ok = false;
  if (p.prec == DH_PREC_FP32) return DH_OK;
  const bool bf16 = p.prec == DH_PREC_BF16;
  dh_status st = encode_2d(&p.tmap_H, p.d_H, bf16, (uint64_t)p.npix, (uint64_t)2 * p.max_frames,
                           (uint64_t)p.npix * 2, 64u, (uint32_t)(2 * p.T), CU_TENSOR_MAP_SWIZZLE_128B);
  if (st != DH_OK) return st;
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

dh_status launch_project_tc(Plan &p, int first_slot, int slot_stride, int n_windows, int Npad,
                            float *images, cudaStream_t s) {
  if (!p.tmaps_ok) return DH_ERR_STATE;
  const bool bf16 = p.prec == DH_PREC_BF16;
  switch (p.T) {
    case 16: return bf16 ? project_t<16, true>(p, first_slot, slot_stride, n_windows, Npad, images, s)
                         : project_t<16, false>(p, first_slot, slot_stride, n_windows, Npad, images, s);
    case 32: return bf16 ? project_t<32, true>(p, first_slot, slot_stride, n_windows, Npad, images, s)
                         : project_t<32, false>(p, first_slot, slot_stride, n_windows, Npad, images, s);
    case 64: return bf16 ? project_t<64, true>(p, first_slot, slot_stride, n_windows, Npad, images, s)
                         : project_t<64, false>(p, first_slot, slot_stride, n_windows, Npad, images, s);
  }
  return DH_ERR_UNSUPPORTED_SIZE;
}

}  // namespace dh
