// Eqs. 8-9 for overlapping windows (slot stride s < T) on the tensor cores, 7 windows per span.
//
// The DFT basis W of Eq. 8 is the same for every window, so the operand of a group of 7
// consecutive windows is the same for every group: window g's columns hold the real
// embedding of W's kept columns at span rows 2 (s g + t) + c (zeros elsewhere). Each CTA
// loads it once. Per 128-pixel tile the span of the group's frames (T + 6 s) is loaded once
// (TMA) and one MMA chain over the span rows (M = 128 pixels, N = 7 x 2 nS columns, K = span
// rows; W rounded once to FP16) gives every window's kept DFT bins; the epilogue sums
// their squares per window (Eq. 9) and writes the images, 8 adjacent image columns per pass.
// Columns are bin-major (n = j G + g: real column j of window g), so the window of every
// column is a compile-time constant in the unrolled epilogue. Unlike the eigenvector
// projection there is no subtraction: the power is Eq. 7's sum over the kept columns.
// W is one FP16 operand, not a hi + lo pair: its rounding (2^-11 relative) moves the image by
// a few 1e-5 relative, under a tenth of the 16-bit storage's own 3e-4 (measured by emulating
// both roundings on the oracle's holograms), and one product instead of two halves the tensor
// work this kernel was bound by.
//
// Roles: warp 0 issues TMA, warp 1 the MMAs, warps 2-5 (one per TMEM lane quarter) drain
// TMEM, warp 6 waits on the mbarriers and releases the MMA warp tile by tile through named
// barriers (so the MMA warp takes no shared-memory step in its loop: see named_sync). Waits are
// bounded (DH_FLAG_WAIT_TIMEOUT).
#include "dh_internal.cuh"
#include "tc_sm100.cuh"

namespace dh {
namespace {

using namespace tc;

constexpr int kFsG = 7;                     // windows per group
constexpr int kFsCpw = 34;                  // real columns per window (17 bins, Re and Im)
constexpr int kFsNpad = 240;                // kFsG x kFsCpw = 238, rounded up to 16
constexpr int kFsWaiter = 6;                // warp that watches the mbarriers (after 4 epilogue warps)
constexpr int kFsThreads = 64 + 128 + 32;
constexpr int kFsMaxStages = 4;
constexpr size_t kFsSmemLimit = 232448;
constexpr double kFsScale = 1024.0;         // W scaled by 2^10 (exact: a power of two)

// The group operand: one FP16 image of kFsNpad x k_pad, K-major, 128-byte swizzled
// (64-element sub-blocks; the 16-byte chunk index XOR row % 8). Column n = j G + g: window g,
// real column j = 2 b + c of kept bin k0 + b (c = 0: Re, 1: Im of sum_t H_t w_{t,k}); row
// r = 2 (s g + t) + cc (cc = 0: Re H_t, 1: Im H_t), w_{t,k} = exp(-2 pi i t k / T) / sqrt(T).
__global__ void k_fs_operand(int T, int k0, int nS, int s, int k_pad, __half *__restrict__ hi) {
  const int per = kFsNpad * k_pad;
  const double rs = 1.0 / sqrt((double)T);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < per; e += gridDim.x * blockDim.x) {
    const int n = e / k_pad, r = e % k_pad;
    const int j = n / kFsG, g = n % kFsG;
    const int b = j >> 1, c = j & 1;
    const int t = (r >> 1) - s * g, cc = r & 1;
    double v = 0.0;
    if (j < 2 * nS && t >= 0 && t < T) {
      const int k = k0 + b;
      double sn, cs;
      sincospi(-2.0 * (double)((t * k) % T) / (double)T, &sn, &cs);
      const double re = cs * rs, im = sn * rs;
      // Re(h w) = hr wr - hi wi ; Im(h w) = hr wi + hi wr
      v = (c == 0 ? (cc == 0 ? re : -im) : (cc == 0 ? im : re)) * kFsScale;
    }
    const int sub = r >> 6, kk = r & 63;
    const long long i =
        ((long long)sub * kFsNpad * 128 + n * 128 + (((kk >> 3) ^ (n & 7)) << 4) + ((kk & 7) << 1)) >> 1;
    hi[i] = __float2half_rn((float)v);
  }
}

__global__ void __launch_bounds__(kFsThreads, 1)
k_fourier_span(const __grid_constant__ CUtensorMap tmA, const uint8_t *__restrict__ Bimg, int img_bytes,
               int first_slot, int s, int n_windows, int rows, int stages, int cpg, float *__restrict__ images,
               int nx, int ny, uint32_t *__restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int stage_bytes = rows * 256;
  uint8_t *stage0 = smem;
  uint8_t *bsm = smem + stages * stage_bytes;
  uint64_t *full = reinterpret_cast<uint64_t *>(bsm + img_bytes);
  uint64_t *empty = full + kFsMaxStages;
  uint64_t *acc_full = empty + kFsMaxStages;
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *bfull = acc_empty + 2;
  uint64_t *mma_done = bfull + 1;
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(mma_done + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long npix = (long long)nx * ny;
  const int n_groups = (n_windows + kFsG - 1) / kFsG;
  const long long units = (long long)n_groups * cpg;
  const long long uper = units / gridDim.x, urem = units % gridDim.x;
  const long long u_begin = blockIdx.x * uper + (blockIdx.x < urem ? blockIdx.x : urem);
  const long long u_end = u_begin + uper + (blockIdx.x < urem ? 1 : 0);
  const int gx = nx >> 3;

  if (threadIdx.x == 0) {
    for (int i = 0; i < stages; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 128); }
    mbar_init(bfull, 1);
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_barrier_init();
    prefetch_tmap(&tmA);
  }
  if (warp == 1) { tmem_alloc(tmem_holder, 512); tmem_relinquish(); }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  auto fail = [&]() { atomicOr(status, DH_FLAG_WAIT_TIMEOUT); *abort_flag = 1; };

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer
      int slot = 0; uint32_t ph = 0;
      long long issued = 0;
      bool ok = true;
      mbar_arrive_expect_tx(bfull, (uint32_t)img_bytes);  // the operand, once
      bulk_load(bsm, Bimg, (uint32_t)img_bytes, bfull);
      for (long long u = u_begin; u < u_end && ok && !*abort_flag; ++u) {
        const int grp = (int)(u / cpg), cg = (int)(u % cpg);
        const int row = 2 * (first_slot + grp * kFsG * s);
        const int kx0 = (cg % gx) * 8, ky0 = (cg / gx) * 128;
        for (int i = 0; i < 8; ++i) {
          const long long p = (long long)(kx0 + i) * ny + ky0;
          if (!mbar_wait(&empty[slot], ph ^ 1)) { fail(); ok = false; break; }
          mbar_arrive_expect_tx(&full[slot], (uint32_t)stage_bytes);
          uint8_t *dst = stage0 + slot * stage_bytes;
          tma_load_3d(dst, &tmA, &full[slot], 0, row, (int)(p >> 6));
          tma_load_3d(dst + rows * 128, &tmA, &full[slot], 0, row, (int)(p >> 6) + 1);
          ++issued;
          if (++slot == stages) { slot = 0; ph ^= 1; }
        }
      }
      if (*abort_flag) {  // let copies still in flight land before the CTA exits
        for (int k = 0; k < stages && k < issued; ++k) {
          if (--slot < 0) { slot = stages - 1; ph ^= 1; }
          mbar_wait(&full[slot], ph);
        }
        mbar_wait(bfull, 0);
      }
    }
  } else if (warp == 1) {  // ---------------- MMA issuer: D[128 px x kFsNpad] = span^T x operand^T
    // The whole warp runs the loop and lane 0 issues; tile k waits on named barrier
    // 1 + k % stages, which the waiter passes once the tile has landed and its accumulator
    // buffer is free (no shared-memory step inside the loop: see named_sync).
    const uint32_t idesc = idesc_f16(false, true, false, 128, kFsNpad);
    const int k_steps = rows / 16;
    int slot = 0, it = 0;
    for (long long u = u_begin; u < u_end; ++u) {
      for (int i = 0; i < 8; ++i, ++it) {
        const int buf = it & 1;
        named_sync(1 + slot, 64);
        fence_after_sync();
        if (lane == 0) {
          const uint32_t d = tmem + buf * 256;
          const uint64_t adesc0 = smem_desc(smem_u32(stage0 + slot * stage_bytes), rows * 128, 1024, kSwizzle128);
          const uint64_t bdesc0 = smem_desc(smem_u32(bsm), 16, 1024, kSwizzle128);
          for (int kk = 0; kk < k_steps; ++kk) {
            const uint64_t adesc = adesc0 + (uint64_t)(kk * 128);
            const uint64_t bdesc = bdesc0 + (uint64_t)(((kk >> 2) * kFsNpad * 128 + (kk & 3) * 32) >> 4);
            mma_f16(d, adesc, bdesc, idesc, kk == 0 ? 0u : 1u);
          }
          mma_commit(&empty[slot]);
          mma_commit(&acc_full[buf]);
        }
        __syncwarp();
        if (++slot == stages) slot = 0;
      }
    }
    if (lane == 0) mma_commit(mma_done);  // every MMA completes before the tensor memory is freed
    __syncwarp();
    mbar_wait(mma_done, 0);
  } else if (warp == kFsWaiter) {  // ---------------- waiter
    // Runs ahead of the MMA warp by fewer than `stages` tiles (a tile's data needs its slot
    // released by the MMAs of the tile `stages` before), so each named barrier has at most one
    // pending arrival; after a failed wait or an abort it stops waiting for data and arrives
    // once the MMAs of the tile `stages` before have completed.
    int slot = 0, it = 0, released = 0;
    uint32_t ph = 0;
    bool ok = __all_sync(0xffffffffu, mbar_wait(bfull, 0));  // the operand, once
    for (long long u = u_begin; u < u_end; ++u) {
      for (int i = 0; i < 8; ++i, ++it) {
        const int buf = it & 1;
        if (ok) ok = !__any_sync(0xffffffffu, *abort_flag != 0) &&
                     __all_sync(0xffffffffu, mbar_wait(&acc_empty[buf], ((it >> 1) & 1) ^ 1)) &&
                     __all_sync(0xffffffffu, mbar_wait(&full[slot], ph));
        if (!ok) {
          if (lane == 0 && !*abort_flag) fail();
          // without the data wait, keep at most one pending arrival on this named barrier:
          // wait (bounded) for the MMAs of the stage stages before, which the MMA warp
          // issued after passing the barrier for that stage
          if (released >= stages) (void)__all_sync(0xffffffffu, mbar_wait(&empty[slot], ph ^ 1));
        }
        named_arrive(1 + slot, 64);
        ++released;
        if (++slot == stages) { slot = 0; ph ^= 1; }
      }
    }
  } else {  // ------------------------------ epilogue: lane quarter q, all 7 windows
    const int q = warp & 3;
    const int L = 32 * q + lane;
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    constexpr float kInv = (float)(1.0 / (kFsScale * kFsScale));
    int it = 0;
    for (long long u = u_begin; u < u_end && !__any_sync(0xffffffffu, *abort_flag); ++u) {
      const int grp = (int)(u / cpg), cg = (int)(u % cpg);
      const int gw = grp * kFsG;
      const int g_here = n_windows - gw < kFsG ? n_windows - gw : kFsG;
      float out[kFsG][8];
      bool ok = true;
      for (int i = 0; i < 8; ++i, ++it) {
        const int buf = it & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (it >> 1) & 1))) { fail(); ok = false; break; }
        fence_after_sync();
        float m[kFsG];
#pragma unroll
        for (int g = 0; g < kFsG; ++g) m[g] = 0.f;
        const uint32_t ta = tmem + lane_addr + buf * 256;
#pragma unroll
        for (int c0 = 0; c0 < 224; c0 += 32) {
          float v[32];
          tmem_ld32(ta + c0, v);
#pragma unroll
          for (int x = 0; x < 32; ++x) m[(c0 + x) % kFsG] = fmaf(v[x], v[x], m[(c0 + x) % kFsG]);
        }
        {
          float v[16];
          tmem_ld16(ta + 224, v);
#pragma unroll
          for (int x = 0; x < 14; ++x) m[(224 + x) % kFsG] = fmaf(v[x], v[x], m[(224 + x) % kFsG]);
        }
        fence_before_sync();
        mbar_arrive(&acc_empty[buf]);
#pragma unroll
        for (int g = 0; g < kFsG; ++g) {
#pragma unroll
          for (int k = 7; k > 0; --k) out[g][k] = out[g][k - 1];
          out[g][0] = m[g] * kInv;
        }
      }
      if (!ok) break;
      const int kx0 = (cg % gx) * 8, ky = (cg / gx) * 128 + L;
#pragma unroll
      for (int g = 0; g < kFsG; ++g) {
        if (g < g_here) {
          float4 *dst = reinterpret_cast<float4 *>(images + (long long)(gw + g) * npix + (long long)ky * nx + kx0);
          dst[0] = make_float4(out[g][7], out[g][6], out[g][5], out[g][4]);
          dst[1] = make_float4(out[g][3], out[g][2], out[g][1], out[g][0]);
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace

bool fourier_span_applies(const Plan &p, int slot_stride, int n_windows, int nS) {
  if (p.prec != DH_PREC_FP16 || !p.tmaps_ok || nS != kFsCpw / 2) return false;
  if (slot_stride < 1 || slot_stride >= p.T || n_windows < 2) return false;
  if (p.ny < 128 || p.nx % 8 != 0) return false;
  const int rows = (2 * (p.T + (kFsG - 1) * slot_stride) + 15) / 16 * 16;
  if (rows > 256) return false;
  const int k_pad = (rows + 63) / 64 * 64;
  const size_t img = (size_t)kFsNpad * k_pad * 2;
  if (img > p.W_bytes) return false;
  return (size_t)2 * rows * 256 + img + 1024 + 256 <= kFsSmemLimit;
}

dh_status launch_fourier_span(Plan &p, int first_slot, int slot_stride, int n_windows, int k0, int nS,
                              float *images, cudaStream_t s) {
  const int rows = (2 * (p.T + (kFsG - 1) * slot_stride) + 15) / 16 * 16;
  const int k_pad = (rows + 63) / 64 * 64;
  const int img = kFsNpad * k_pad * 2;
  const size_t fixed = (size_t)img + 1024 + 256;
  int stages = (int)((kFsSmemLimit - fixed) / ((size_t)rows * 256));
  if (stages > kFsMaxStages) stages = kFsMaxStages;
  if (stages < 2) return DH_ERR_STATE;
  static bool attr = false;
  if (!attr) {
    DH_CUDA_TRY(cudaFuncSetAttribute(k_fourier_span, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFsSmemLimit));
    attr = true;
  }
  {
    ProfScope ps(p, K_FOURIER_OP, s);
    const int per = kFsNpad * k_pad;
    k_fs_operand<<<(per + 255) / 256, 256, 0, s>>>(p.T, k0, nS, slot_stride, k_pad, static_cast<__half *>(p.d_W));
    DH_CUDA_TRY(cudaGetLastError());
  }
  const uint64_t rows_all = 2ull * p.max_frames;
  const uint64_t dims[3] = {64, rows_all, (uint64_t)p.npix / 64};
  const uint64_t strides[2] = {64 * 2, rows_all * 64 * 2};
  const uint32_t box[3] = {64, (uint32_t)rows, 1};
  CUtensorMap tmA;
  dh_status st = encode_3d(&tmA, p.d_H, false, dims, strides, box);
  if (st != DH_OK) return st;
  const size_t smem = (size_t)stages * rows * 256 + fixed;
  const int cpg = (int)(p.npix / 1024);
  const long long units = (long long)((n_windows + kFsG - 1) / kFsG) * cpg;
  const int grid = (int)(units < p.num_sms ? units : p.num_sms);
  ProfScope ps(p, K_FOURIER_SPAN, s);
  k_fourier_span<<<grid, kFsThreads, smem, s>>>(tmA, static_cast<const uint8_t *>(p.d_W), img, first_slot,
                                                slot_stride, n_windows, rows, stages, cpg, images, p.nx, p.ny,
                                                p.d_status);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

}  // namespace dh
