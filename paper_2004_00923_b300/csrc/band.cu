// Banded whole-sequence covariance (Eq. 4 for many overlapping windows at once).
//
// C of a window is made of the inner products of its frames' holograms, G[f][f'] =
// sum_p Re/Im H_f[p] Re/Im H_f'[p], so every window of T <= 64 frames, at any start and any
// stride, takes its C from the band |f - f'| < 64 of the whole sequence's real Gram. The
// sequence is cut into 64-frame blocks (128 rows Re/Im each); for block b the tensor cores form
// G_bb = X_b X_b^T and G_b,b+1 = X_b X_{b+1}^T
// (the band; the last block's G_b,b+1 is not needed). A pair of frames less than 64 apart lies in
// one block or in two adjacent ones, so the band holds every pair any window needs.
//
// The two products of a block are separate work units, each an M = N = 128 MMA (A = X_b, B =
// X_b or X_{b+1}; 64 running sums per epilogue thread, no spills), so a frame is read three
// times in all rather than once per window containing it.
//
// Pipeline (one CTA per SM): warp 0 issues TMA loads of the 128-row x 64-pixel boxes of a
// stage (a box past the last slot reads zeros), warp 1 issues the MMAs (released stage by
// stage through named barriers by a waiter warp, so that it takes no shared-memory step in its
// loop: see named_sync), eight epilogue warps
// (TMEM lane quarter x column half) drain the accumulator every GROUP stages into FP32 unit
// sums (short TMEM accumulations keep the tensor cores' truncation bias near 5e-7) and write
// FP64 partials per (block, product, split-K unit); a reduction sums the units in FP64 and an
// assembly kernel gathers each window's C from the band. Waits are bounded as in the other tensor-core
// kernels (DH_FLAG_WAIT_TIMEOUT).
#include "dh_internal.cuh"
#include "tc_sm100.cuh"

namespace dh {
namespace {

using namespace tc;

__device__ __forceinline__ uint8_t *align1024b(uint8_t *p) {
  return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

struct BandCfg {
  static constexpr int BOX_BYTES = 128 * 128;        // 128 rows x 64 pixels x 2 bytes
  static constexpr int STAGE_BYTES = 2 * BOX_BYTES;  // block b, and block b + 1 for G_b,b+1
  static constexpr int STAGES = 6;
  static constexpr int GROUP = 2;                    // stages per TMEM drain
  static constexpr int NB = 4;                       // accumulators of 128 columns
  static constexpr int EPI_WARPS = 8;                // lane quarter x column half (64 columns)
  static constexpr int WAITER = 2 + EPI_WARPS;       // watches the mbarriers for the MMA warp
  static constexpr int THREADS = 64 + 32 * EPI_WARPS + 32;
  static constexpr size_t SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};

// Work unit wu = ((b * 2 + h) * units + u), wu < (2 n_blocks - 1) units: block b, product h (0: G_bb = X_b X_b^T, 1: G_b,b+1 =
// X_b X_{b+1}^T), split-K unit u of the pixels. One M = N = 128 MMA per 16 pixels.
template <bool BF16>
__global__ void __launch_bounds__(BandCfg::THREADS, 1)
k_band_gram(const __grid_constant__ CUtensorMap tm, int row0, int n_blocks, int units, int stages_per_unit,
            double *__restrict__ part, uint32_t *__restrict__ status) {
  using C = BandCfg;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024b(smem_raw);
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
    prefetch_tmap(&tm);
  }
  if (warp == 1) { tmem_alloc(tmem_holder, 128 * C::NB); tmem_relinquish(); }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  // the last block's G_b,b+1 reaches past the band: its units (the last ones) are skipped
  const int total_units = (2 * n_blocks - 1) * units;
  auto fail = [&]() { atomicOr(status, DH_FLAG_WAIT_TIMEOUT); *abort_flag = 1; };

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer
      int slot = 0; uint32_t ph = 0;
      long long issued = 0;
      for (int wu = blockIdx.x; wu < total_units && !*abort_flag; wu += gridDim.x) {
        const int u = wu % units, bh = wu / units, h = bh & 1, b = bh >> 1;
        const int row = row0 + 128 * b;
        for (int st = 0; st < stages_per_unit; ++st) {
          if (!mbar_wait(&empty[slot], ph ^ 1)) { fail(); break; }
          mbar_arrive_expect_tx(&full[slot], (1 + h) * C::BOX_BYTES);
          uint8_t *dst = stages + slot * C::STAGE_BYTES;
          const int pblk = u * stages_per_unit + st;  // 64-pixel block
          tma_load_3d(dst, &tm, &full[slot], 0, row, pblk);
          if (h) tma_load_3d(dst + C::BOX_BYTES, &tm, &full[slot], 0, row + 128, pblk);
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
  } else if (warp == 1) {  // ---------------- MMA issuer: D[128 x 128] += X_b x (X_b or X_b+1)^T
    // whole warp, lane 0 issues; stage k waits on named barrier 1 + k % STAGES (the waiter)
    constexpr uint32_t idesc = idesc_f16(BF16, false, false, 128, 128);
    int slot = 0, grp = 0;
    for (int wu = blockIdx.x; wu < total_units; wu += gridDim.x) {
      const int h = (wu / units) & 1;
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
              const uint64_t da = smem_desc(base + 32 * k, 16, 1024, kSwizzle128);
              const uint64_t db = smem_desc(base + h * C::BOX_BYTES + 32 * k, 16, 1024, kSwizzle128);
              mma_f16(d, da, db, idesc, (i > 0 || k > 0) ? 1u : 0u);
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
    if (lane == 0) mma_commit(mma_done);  // every MMA completes before the tensor memory is freed
    __syncwarp();
    mbar_wait(mma_done, 0);
  } else if (warp == C::WAITER) {  // ---------------- waiter
    // Fewer than STAGES stages ahead of the MMA warp (a stage's data needs its slot released by
    // the MMAs of the stage STAGES before): one pending arrival per named barrier at most. After
    // a failed wait or an abort it stops waiting for data and arrives once the MMAs of the
    // stage STAGES before have completed, so the MMA warp still completes its loop.
    int slot = 0, grp = 0, released = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int wu = blockIdx.x; wu < total_units; wu += gridDim.x) {
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
    const int q = warp & 3;          // TMEM lane quarter this warp may access
    const int ch = e >> 2;           // column half (64 columns)
    const int L = 32 * q + lane;     // accumulator row = row of block b
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    int grp = 0;
    for (int wu = blockIdx.x; wu < total_units && !__any_sync(0xffffffffu, *abort_flag); wu += gridDim.x) {
      float s[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) s[j] = 0.f;
      bool ok = true;
      for (int g0 = 0; g0 < stages_per_unit; g0 += C::GROUP, ++grp) {
        const int buf = grp % C::NB;
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (grp / C::NB) & 1))) {
          fail(); ok = false; break;
        }
        fence_after_sync();
        const uint32_t ta = tmem + lane_addr + buf * 128 + ch * 64;
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
          float v[32];
          tmem_ld32(ta + 32 * c2, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) s[32 * c2 + i] += v[i];
        }
        fence_before_sync();
        mbar_arrive(&acc_empty[buf]);
      }
      if (!ok) break;
      // partials [b][h][u][128][128]
      double *dst = part + (long long)wu * 128 * 128 + (long long)L * 128 + ch * 64;
#pragma unroll
      for (int j = 0; j < 64; ++j) dst[j] = (double)s[j];
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, 128 * C::NB);
  }
}

// band[b][h][i][j] = sum over the split-K units (FP64); partials are [b][h][u][128][128]
__global__ void k_band_reduce(const double *__restrict__ part, int n_blocks, int units, double *__restrict__ band) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long cell = 128ll * 128;
  if (idx >= (2ll * n_blocks - 1) * cell) return;
  const long long bh = idx / cell, e = idx % cell;
  double acc = 0.0;
  for (int u = 0; u < units; ++u) acc += part[(bh * units + u) * cell + e];
  band[idx] = acc;
}

// C of window w (frames f = first + w * stride + t, t < T, counted from the band's first
// frame): C[t][u] = G(2f, 2f') + G(2f+1, 2f'+1) + i (G(2f, 2f'+1) - G(2f+1, 2f')), with G the
// real Gram of the rows Re H_f, Im H_f, taken from the block pair holding (f, f').
template <int T>
__global__ void k_band_cov(const double *__restrict__ band, int first, int stride, int n_windows,
                           double *__restrict__ Cout, uint32_t *__restrict__ status) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_windows * T * T) return;
  const int w = idx / (T * T), e = idx % (T * T), t = e / T, u = e % T;
  const int f = first + w * stride + t, g = first + w * stride + u;
  auto G = [&](int fa, int ca, int fb, int cb) -> double {
    const int ba = fa >> 6, bb = fb >> 6;
    const int ra = 2 * (fa & 63) + ca, rb = 2 * (fb & 63) + cb;
    if (ba == bb) return band[((long long)ba * 2 + 0) * 16384 + ra * 128 + rb];
    if (bb == ba + 1) return band[((long long)ba * 2 + 1) * 16384 + ra * 128 + rb];
    return band[((long long)bb * 2 + 1) * 16384 + rb * 128 + ra];  // ba == bb + 1: G symmetric
  };
  const double re = G(f, 0, g, 0) + G(f, 1, g, 1);
  const double im = G(f, 0, g, 1) - G(f, 1, g, 0);
  Cout[2 * ((long long)w * T * T + e)] = re;
  Cout[2 * ((long long)w * T * T + e) + 1] = im;
  if (!isfinite(re) || !isfinite(im)) atomicOr(status, DH_FLAG_NONFINITE_C);
}

}  // namespace

int band_units(long long npix) {
  long long u = npix / 32768;
  if (u < 1) u = 1;
  if (u > 32) u = 32;
  return (int)u;
}

dh_status launch_band_gram(Plan &p, int first_slot, int n_frames, cudaStream_t s) {
  if (!p.tmaps_ok || p.prec == DH_PREC_FP32) return DH_ERR_STATE;
  const int n_blocks = (n_frames + 63) / 64;
  const int units = band_units(p.npix);
  const int stages_per_unit = (int)(p.npix / 64 / units);
  using C = BandCfg;
  auto kern = p.prec == DH_PREC_BF16 ? k_band_gram<true> : k_band_gram<false>;
  static bool attr[2] = {false, false};
  const int ai = p.prec == DH_PREC_BF16 ? 1 : 0;
  if (!attr[ai]) {
    DH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    attr[ai] = true;
  }
  const int total = (2 * n_blocks - 1) * units;
  const int grid = p.num_sms < total ? p.num_sms : total;
  {
    ProfScope ps(p, K_BAND_GRAM, s);
    kern<<<grid, C::THREADS, C::SMEM, s>>>(p.tmap_band, 2 * first_slot, n_blocks, units, stages_per_unit,
                                           p.d_band_part, p.d_status);
    DH_CUDA_TRY(cudaGetLastError());
  }
  const long long cells = (2ll * n_blocks - 1) * 128 * 128;
  {
    ProfScope ps(p, K_BAND_REDUCE, s);
    k_band_reduce<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(p.d_band_part, n_blocks, units, p.d_band);
    DH_CUDA_TRY(cudaGetLastError());
  }
  return DH_OK;
}

dh_status launch_band_cov(Plan &p, const Plan &owner, int first_slot, int slot_stride, int n_windows, int woff,
                          cudaStream_t s) {
  const int first = first_slot - owner.band_first;
  const int total = n_windows * p.T * p.T;
  double *C = p.d_C + 2ll * woff * p.T * p.T;
  ProfScope ps(p, K_BAND_COV, s);
  switch (p.T) {
    case 16: k_band_cov<16><<<(total + 255) / 256, 256, 0, s>>>(owner.d_band, first, slot_stride, n_windows, C, p.d_status); break;
    case 32: k_band_cov<32><<<(total + 255) / 256, 256, 0, s>>>(owner.d_band, first, slot_stride, n_windows, C, p.d_status); break;
    case 64: k_band_cov<64><<<(total + 255) / 256, 256, 0, s>>>(owner.d_band, first, slot_stride, n_windows, C, p.d_status); break;
    default: return DH_ERR_UNSUPPORTED_SIZE;
  }
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

}  // namespace dh
