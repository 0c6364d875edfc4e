// Eqs. 6-7 for overlapping windows, several windows per pass (tensor cores, 16-bit storage).
//
// Windows g = 0..G-1 of a group start at slots f0 + s g (slot stride s < T, s a multiple of 4):
// together they cover a span of T + (G - 1) s frames. For each 128-pixel tile a CTA loads the
// span's rows once (TMA) and forms the power images of all G windows from it, so a frame is
// read once per group holding it rather than once per window holding it.
//
// The power is taken through the complement of the kept components. V is unitary, so for
// the window vector h of a pixel (h_t = H_{f+t}[p]) the projections onto all T components
// carry all of its energy, sum_k |sum_t h_t V_tk|^2 = sum_t |h_t|^2, and
//   M = sum_{k0 <= k <= k1} |sum_t h_t V_tk|^2 = sum_t |h_t|^2 - sum_{k in D} |sum_t h_t V_tk|^2
// with D = {k < k0} u {k > k1} the discarded components. When D is small (the paper drops
// only the first components) this needs CPW = 2|D| operand columns per window (padded to 4
// or 8) instead of 2 (k1 - k0 + 1). The group's operand is banded: the eigensolver writes
// window g's columns with its V at span rows 2 (s g + t) + c and zeros elsewhere (real
// embedding scaled by 2^10, hi + lo 16-bit parts, already in the 128-byte-swizzled
// shared-memory image), so
// one MMA chain over the span rows (M = 128 pixels, N = G CPW padded to 16, K = span rows)
// gives every window's discarded projections. The epilogue forms each window's sum_t |h_t|^2
// from the tile still in shared memory (a running sum along the span: s frames enter and s
// frames leave per window) and subtracts. The result clamps at 0.
//
// Roles: warp 0 issues TMA (span tiles, and the group operand as one bulk copy), warp 1
// issues the MMAs (released tile by tile through named barriers by a waiter warp, the last
// one, so that it takes no shared-memory step in its loop), eight epilogue warps (TMEM lane
// quarter x half of the group's windows)
// drain TMEM, sum energies and write the images, 8 adjacent image columns per pass (the
// store's pixels run down image columns). A stage is released when both the MMAs and the
// epilogue's energy reads are done. Waits are bounded (DH_FLAG_WAIT_TIMEOUT).
#include "dh_internal.cuh"
#include "tc_sm100.cuh"

namespace dh {
namespace {

using namespace tc;

constexpr int kSpanEpiWarps = 8;
constexpr int kSpanWaiter = 2 + kSpanEpiWarps;  // the warp that watches the MMA warp's mbarriers
// named barriers: 1-4 pair the epilogue warps of a lane quarter; the MMA warp's stages use
// kSpanStageBar + slot (slot < kSpanMaxStages = 4), so 5-8
constexpr int kSpanStageBar = 5;
constexpr int kSpanThreads = 64 + 32 * kSpanEpiWarps + 32;
constexpr int kSpanMaxG = 8;
constexpr int kSpanMaxStages = 4;
constexpr int kNacc = 4;  // partial accumulators per buffer (k-step kk goes to kk % 4)
constexpr size_t kSpanSmemLimit = 232448;
constexpr float kInvScale2 = (float)(1.0 / (kSpanOperandScale * kSpanOperandScale));


// the two 16-bit values of a 32-bit word (lower address first) as floats
template <bool BF16>
__device__ __forceinline__ float2 word_to_f32x2(uint32_t w) {
  if constexpr (BF16) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
  } else {
    __half2 hv;
    memcpy(&hv, &w, 4);
    return __half22float2(hv);
  }
}
// acc + x^2 for each FP16 half of w (x: lower address, y: upper), with the mixed-precision
// FMA (FP16 inputs, FP32 accumulator, one rounding): no separate conversion to FP32
__device__ __forceinline__ float2 sq_acc_f16x2(uint32_t w, float2 acc) {
  asm("{\n\t.reg .f16 lo, hi;\n\t"
      "mov.b32 {lo, hi}, %2;\n\t"
      "fma.rn.f32.f16 %0, lo, lo, %0;\n\t"
      "fma.rn.f32.f16 %1, hi, hi, %1;\n\t}"
      : "+f"(acc.x), "+f"(acc.y)
      : "r"(w));
  return acc;
}
// energies of one 4-frame chunk of this lane's row type for its pixel pair (x: even pixel,
// y: odd pixel) from the chunk's four 32-bit words
template <bool BF16>
__device__ __forceinline__ float2 chunk_sq(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
  if constexpr (BF16) {
    const float2 f0 = word_to_f32x2<BF16>(w0), f1 = word_to_f32x2<BF16>(w1);
    const float2 f2 = word_to_f32x2<BF16>(w2), f3 = word_to_f32x2<BF16>(w3);
    return __fadd2_rn(__ffma2_rn(f0, f0, __fmul2_rn(f1, f1)), __ffma2_rn(f2, f2, __fmul2_rn(f3, f3)));
  } else {  // (w0^2 + w1^2) + (w2^2 + w3^2), the same pairing
    const float2 a = sq_acc_f16x2(w1, sq_acc_f16x2(w0, make_float2(0.f, 0.f)));
    const float2 b = sq_acc_f16x2(w3, sq_acc_f16x2(w2, make_float2(0.f, 0.f)));
    return __fadd2_rn(a, b);
  }
}
// Barrier `id` of the 64 threads of one lane quarter's two epilogue warps, returning whether
// any of them passed true (both warps see the same answer and take the same branch).
__device__ __forceinline__ bool pair_sync_or(int id, bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.or.pred po, %2, 64, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(id)
      : "memory");
  return r != 0;
}

template <int CPW, bool BF16>
__global__ void __launch_bounds__(kSpanThreads, 1)
k_project_span(const __grid_constant__ CUtensorMap tmA, const uint8_t *__restrict__ Bimg, long long group_bytes,
               int img_bytes, int first_slot, int s, int T, int n_windows, int G, int rows, int n_pad,
               int tmem_cols, int nbuf, int stages, int cpg, float *__restrict__ images, int nx, int ny,
               uint32_t *__restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  // aligned by indexing the shared array itself, so that pointers derived from it stay in the
  // shared address space and plain loads and stores compile to shared-memory instructions
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int stage_bytes = rows * 256;  // two 64-pixel boxes of `rows` rows
  uint8_t *stage0 = smem;
  uint8_t *bsm = smem + stages * stage_bytes;
  const int rows_used = 2 * (T + (G - 1) * s);  // span rows (a multiple of 8)
  float *scratch = reinterpret_cast<float *>(bsm + img_bytes);  // [2][rows_used / 8][128]
  uint64_t *full = reinterpret_cast<uint64_t *>(bsm + img_bytes + 2 * (rows_used / 8) * 512);
  uint64_t *empty = full + kSpanMaxStages;
  uint64_t *acc_full = empty + kSpanMaxStages;
  uint64_t *acc_empty = acc_full + 4;
  uint64_t *bfull = acc_empty + 4;
  uint64_t *bempty = bfull + 1;
  uint64_t *mma_done = bempty + 1;
  uint64_t *prog = mma_done + 1;  // [kSpanMaxStages]: a slot's MMAs completed (MMA warp only)
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(prog + kSpanMaxStages);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long npix = (long long)nx * ny;
  const int n_groups = (n_windows + G - 1) / G;
  const long long units = (long long)n_groups * cpg;
  const long long uper = units / gridDim.x, urem = units % gridDim.x;
  const long long u_begin = blockIdx.x * uper + (blockIdx.x < urem ? blockIdx.x : urem);
  const long long u_end = u_begin + uper + (blockIdx.x < urem ? 1 : 0);
  const int gx = nx >> 3;

  if (threadIdx.x == 0) {
    for (int i = 0; i < stages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1 + kSpanEpiWarps);
      mbar_init(&prog[i], 1);
    }
    for (int b = 0; b < nbuf; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 32 * kSpanEpiWarps); }
    mbar_init(bfull, 1);
    mbar_init(bempty, 1);
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_barrier_init();
    prefetch_tmap(&tmA);
  }
  // nbuf (2 or 4) accumulator buffers, each kNacc partial accumulators of n_pad columns
  const int acc_stride = kNacc * n_pad;
  if (warp == 1) { tmem_alloc(tmem_holder, tmem_cols); tmem_relinquish(); }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  auto fail = [&]() { atomicOr(status, DH_FLAG_WAIT_TIMEOUT); *abort_flag = 1; };

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer
      int slot = 0; uint32_t ph = 0, bph = 0;
      int cur = -1;
      long long issued = 0;
      bool b_pending = false, ok = true;
      for (long long u = u_begin; u < u_end && ok && !*abort_flag; ++u) {
        const int grp = (int)(u / cpg), cg = (int)(u % cpg);
        if (grp != cur) {  // the group's banded operand
          if (!mbar_wait(bempty, bph ^ 1)) { fail(); break; }
          mbar_arrive_expect_tx(bfull, (uint32_t)img_bytes);
          bulk_load(bsm, Bimg + grp * group_bytes, (uint32_t)img_bytes, bfull);
          b_pending = true;
          bph ^= 1;
          cur = grp;
        }
        const int row = 2 * (first_slot + grp * G * s);
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
        if (b_pending) mbar_wait(bfull, bph ^ 1);
      }
    }
  } else if (warp == 1) {  // ---------------- MMA issuer: D[128 px x n_pad] = span^T x operand^T
    // The whole warp runs the loop and lane 0 issues; tile k waits on named barrier
    // kSpanStageBar + k % stages, which the waiter passes once the tile has landed, its
    // accumulator buffer is free and (first tile of a group) the group's operand is in place;
    // no shared-memory step inside the loop (a shared-memory access waits for the issued MMAs'
    // operand reads) and no exit of its own.
    const uint32_t idesc = idesc_f16(BF16, true, false, 128, n_pad);
    const int k_steps = rows / 16;
    const int half_bytes = img_bytes / 2;
    int slot = 0, it = 0;
    for (long long u = u_begin; u < u_end; ++u) {
      const int grp = (int)(u / cpg);
      for (int i = 0; i < 8; ++i, ++it) {
        const int buf = it % nbuf;
        named_sync(kSpanStageBar + slot, 64);
        fence_after_sync();
        if (lane == 0) {
          const uint32_t d = tmem + buf * acc_stride;
          // descriptors advance by their start-address field (address >> 4; shared memory is
          // below 256 KiB, so the 14-bit field never carries)
          const uint64_t adesc0 = smem_desc(smem_u32(stage0 + slot * stage_bytes), rows * 128, 1024, kSwizzle128);
          // The tensor cores' accumulator truncates to its own ulp at every step, and the
          // discarded projections are close to the window's whole energy, which the epilogue
          // subtracts them from. So k-step kk goes to partial accumulator kk % 4 (shorter
          // chains of smaller sums; the epilogue adds the partials in FP32), and the small lo
          // products go in first, while the partials are small.
          for (int half = 1; half >= 0; --half) {
            const uint64_t bdesc0 = smem_desc(smem_u32(bsm) + half * half_bytes, 16, 1024, kSwizzle128);
            for (int kk = 0; kk < k_steps; ++kk) {
              const uint64_t adesc = adesc0 + (uint64_t)(kk * 128);  // 2048 bytes per k-step
              const uint64_t bdesc = bdesc0 + (uint64_t)(((kk >> 2) * n_pad * 128 + (kk & 3) * 32) >> 4);
              mma_f16(d + (kk & (kNacc - 1)) * n_pad, adesc, bdesc, idesc, (half == 1 && kk < kNacc) ? 0u : 1u);
            }
          }
          mma_commit(&empty[slot]);
          mma_commit(&prog[slot]);
          mma_commit(&acc_full[buf]);
        }
        __syncwarp();
        if (++slot == stages) slot = 0;
      }
      const bool last_of_group = (u + 1 == u_end) || ((int)((u + 1) / cpg) != grp);
      if (lane == 0 && last_of_group) mma_commit(bempty);
      __syncwarp();
    }
    if (lane == 0) mma_commit(mma_done);  // every MMA completes before the tensor memory is freed
    __syncwarp();
    mbar_wait(mma_done, 0);
  } else if (warp == kSpanWaiter) {  // ---------------- waiter
    // Fewer than `stages` tiles ahead of the MMA warp (a tile's data needs its slot released
    // by the MMAs of the tile `stages` before): one pending arrival per named barrier at most.
    // After a failed wait or an abort it stops waiting for data and arrives once the MMAs of
    // the tile `stages` before have completed (prog, committed by the MMA warp alone: the
    // slot's `empty` also counts the epilogue, which stops on an abort).
    int slot = 0, it = 0, cur = -1, released = 0;
    uint32_t ph = 0, bph = 0;
    bool ok = true;
    for (long long u = u_begin; u < u_end; ++u) {
      const int grp = (int)(u / cpg);
      if (ok && grp != cur) {
        ok = !__any_sync(0xffffffffu, *abort_flag != 0) && __all_sync(0xffffffffu, mbar_wait(bfull, bph));
        bph ^= 1;
        cur = grp;
      }
      for (int i = 0; i < 8; ++i, ++it) {
        const int buf = it % nbuf;
        if (ok) ok = !__any_sync(0xffffffffu, *abort_flag != 0) &&
                     __all_sync(0xffffffffu, mbar_wait(&acc_empty[buf], ((it / nbuf) & 1) ^ 1)) &&
                     __all_sync(0xffffffffu, mbar_wait(&full[slot], ph));
        if (!ok) {
          if (lane == 0 && !*abort_flag) fail();
          // without the data wait, keep at most one pending arrival on this named barrier:
          // wait (bounded) for the MMAs of the stage stages before, which the MMA warp
          // issued after passing the barrier for that stage
          if (released >= stages) (void)__all_sync(0xffffffffu, mbar_wait(&prog[slot], ph ^ 1));
        }
        named_arrive(kSpanStageBar + slot, 64);
        ++released;
        if (++slot == stages) { slot = 0; ph ^= 1; }
      }
    }
  } else {  // ------------------------------ epilogue: lane quarter q, windows 4h..4h+3
    const int e = warp - 2;
    const int q = warp & 3, h = e >> 2;
    const int L = 32 * q + lane;  // pixel of the tile = TMEM lane
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    const bool odd = (L & 1) != 0;
    // Energies in two phases per tile. Phase 1: the two warps of a lane quarter split the
    // span's 4-frame chunks and store each pixel's chunk energy in a scratch buffer (one per
    // tile parity). A lane loads the 32-bit word holding its pixel and its neighbour's (L ^ 1)
    // from the Re rows (even lanes) or the Im rows (odd lanes) and the pair combines them.
    // Phase 2, after the pair's barrier: each warp sums the chunk energies of its windows.
    // Byte offsets within a chunk (4 frames = 8 rows = 1024 bytes) of this lane's word in
    // row 2k + (L & 1), 128-byte swizzle: the 16-byte chunk index XOR row % 8.
    uint32_t off[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = 2 * k + (L & 1);
      off[k] = r * 128 + ((((L & 63) >> 3) ^ r) << 4) + ((L & 6) << 1);
    }
    const int nch = rows_used / 8;          // 4-frame chunks of the span
    const int c_half = (nch + 1) / 2;
    const int c_lo = h == 0 ? 0 : c_half, c_hi = h == 0 ? c_half : nch;
    const int dch = s / 4, mch = T / 4;     // window step and window length in chunks
    const int box_off = (L >> 6) * rows * 128;  // this pixel's 64-pixel box within a stage
    int slot = 0, it = 0;
    uint32_t ph = 0;
    bool stop = false;
    for (long long u = u_begin; u < u_end && !stop; ++u) {
      const int grp = (int)(u / cpg), cg = (int)(u % cpg);
      const int gw = grp * G;
      const int g_here = n_windows - gw < G ? n_windows - gw : G;  // windows of this group
      const int j_n = g_here - 4 * h;                                // of this half
      float out[4][8];
      const bool aborted = __any_sync(0xffffffffu, *abort_flag != 0);
      for (int i = 0; i < 8; ++i, ++it) {
        const int buf = it % nbuf;   // accumulator buffer
        const int sbuf = it & 1;     // scratch buffer (the pair's barrier separates its reuse)
        bool bad = aborted;
        if (!bad)
          bad = !__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (it / nbuf) & 1)) ||
                !__all_sync(0xffffffffu, mbar_wait(&full[slot], ph));
        float v[4 * CPW];
        if (!bad) {
          fence_after_sync();
          if (j_n > 0) {  // the four partial accumulators: loads issued together, one wait
            const uint32_t ta = tmem + lane_addr + buf * acc_stride + 4 * h * CPW;
            if constexpr (CPW == 4) {
              float t[64];
#pragma unroll
              for (int a = 0; a < 4; ++a) tmem_ld16_nowait(ta + a * n_pad, *reinterpret_cast<float(*)[16]>(&t[16 * a]));
              tmem_wait_ld(t);
#pragma unroll
              for (int x = 0; x < 16; ++x) v[x] = (t[x] + t[16 + x]) + (t[32 + x] + t[48 + x]);
            } else {
#pragma unroll
              for (int r = 0; r < 2; ++r) {
                float t[64];
                tmem_ld32_nowait(ta + (2 * r) * n_pad, *reinterpret_cast<float(*)[32]>(&t[0]));
                tmem_ld32_nowait(ta + (2 * r + 1) * n_pad, *reinterpret_cast<float(*)[32]>(&t[32]));
                tmem_wait_ld(t);
#pragma unroll
                for (int x = 0; x < 32; ++x) v[x] = r == 0 ? t[x] + t[32 + x] : v[x] + (t[x] + t[32 + x]);
              }
            }
          }
          fence_before_sync();
          mbar_arrive(&acc_empty[buf]);
          // phase 1: this warp's chunks of the tile
          const uint8_t *a_b = stage0 + slot * stage_bytes + box_off + c_lo * 1024;
          const uint32_t *pk0 = reinterpret_cast<const uint32_t *>(a_b + off[0]);
          const uint32_t *pk1 = reinterpret_cast<const uint32_t *>(a_b + off[1]);
          const uint32_t *pk2 = reinterpret_cast<const uint32_t *>(a_b + off[2]);
          const uint32_t *pk3 = reinterpret_cast<const uint32_t *>(a_b + off[3]);
          float *ws = scratch + (sbuf * nch + c_lo) * 128 + L;
          // the pair's chunk energy: own row type of own pixel + partner's of the same pixel
          auto pair_sum = [&](float2 e) -> float {
            const float keep = odd ? e.y : e.x, send = odd ? e.x : e.y;
            return keep + __shfl_xor_sync(0xffffffffu, send, 1);
          };
          int c = c_lo;
          for (; c + 3 < c_hi; c += 4) {  // 4 chunks (1024 bytes = 256 words each) in flight
            uint32_t w[4][4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              w[k][0] = pk0[256 * k]; w[k][1] = pk1[256 * k]; w[k][2] = pk2[256 * k]; w[k][3] = pk3[256 * k];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) ws[128 * k] = pair_sum(chunk_sq<BF16>(w[k][0], w[k][1], w[k][2], w[k][3]));
            pk0 += 1024; pk1 += 1024; pk2 += 1024; pk3 += 1024; ws += 512;
          }
          for (; c < c_hi; ++c) {
            ws[0] = pair_sum(chunk_sq<BF16>(pk0[0], pk1[0], pk2[0], pk3[0]));
            pk0 += 256; pk1 += 256; pk2 += 256; pk3 += 256; ws += 128;
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[slot]);  // the stage's reads are done
        }
        // the pair's chunk energies are complete; a failure anywhere in the pair stops both
        if (pair_sync_or(1 + q, bad)) { fail(); stop = true; break; }
        // phase 2: the windows of this half
        if (j_n > 0) {
          const float *col = scratch + sbuf * nch * 128 + L;  // chunk c at col[c * 128]
          int a = 4 * h * dch;
          float E;
          {  // the first window's chunks (a multiple of 4 of them): four independent sums
            float e4[4] = {0.f, 0.f, 0.f, 0.f};
            for (int c = a; c < a + mch; c += 4) {
#pragma unroll
              for (int k = 0; k < 4; ++k) e4[k] += col[(c + k) * 128];
            }
            E = (e4[0] + e4[1]) + (e4[2] + e4[3]);
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (j < j_n) {
              if (j > 0) {
                float in = 0.f, outg = 0.f;
                for (int c = 0; c < dch; ++c) {
                  in += col[(a + mch + c) * 128];
                  outg += col[(a + c) * 128];
                }
                E += in - outg;
                a += dch;
              }
              float dsum = 0.f;
#pragma unroll
              for (int c = 0; c < CPW; ++c) dsum = fmaf(v[j * CPW + c], v[j * CPW + c], dsum);
              dsum *= kInvScale2;  // the operand carries V x 2^10
              // shift register: after the 8 tiles, out[j][7 - i] holds tile i
#pragma unroll
              for (int k = 7; k > 0; --k) out[j][k] = out[j][k - 1];
              out[j][0] = fmaxf(E - dsum, 0.f);
            }
          }
        }
        if (++slot == stages) { slot = 0; ph ^= 1; }
      }
      if (stop) break;
      const int kx0 = (cg % gx) * 8, ky = (cg / gx) * 128 + L;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j < j_n) {
          float4 *dst = reinterpret_cast<float4 *>(images + (long long)(gw + 4 * h + j) * npix + (long long)ky * nx + kx0);
          dst[0] = make_float4(out[j][7], out[j][6], out[j][5], out[j][4]);
          dst[1] = make_float4(out[j][3], out[j][2], out[j][1], out[j][0]);
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, tmem_cols);
  }
}

template <int CPW, bool BF16>
dh_status project_span_t(Plan &p, const SpanLayout &sl, int first_slot, int n_windows, float *images, int woff,
                         cudaStream_t s) {
  auto kern = k_project_span<CPW, BF16>;
  static bool attr = false;
  if (!attr) {
    DH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpanSmemLimit));
    attr = true;
  }
  // span tiles: 64 pixels x sl.rows rows x 1 block of the store
  const uint64_t rows_all = 2ull * p.max_frames;
  const uint64_t dims[3] = {64, rows_all, (uint64_t)p.npix / 64};
  const uint64_t strides[2] = {64 * 2, rows_all * 64 * 2};
  const uint32_t box[3] = {64, (uint32_t)sl.rows, 1};
  CUtensorMap tmA;
  dh_status st = encode_3d(&tmA, p.d_H, BF16, dims, strides, box);
  if (st != DH_OK) return st;
  const int stage_bytes = sl.rows * 256;
  const size_t smem = (size_t)sl.stages * stage_bytes + sl.img_bytes + sl.scr_bytes + 1024 + 256;
  const int cpg = (int)(p.npix / 1024);  // 8-tile column groups per window
  const int n_groups = (n_windows + sl.G - 1) / sl.G;
  const long long units = (long long)n_groups * cpg;
  const int grid = (int)(units < p.num_sms ? units : p.num_sms);
  const uint8_t *B = static_cast<const uint8_t *>(p.d_B) + (size_t)woff * p.B_window_bytes;
  ProfScope ps(p, K_PROJECT_SPAN, s);
  kern<<<grid, kSpanThreads, smem, s>>>(tmA, B, (long long)sl.G * (long long)p.B_window_bytes, sl.img_bytes,
                                        first_slot, sl.stride, p.T, n_windows, sl.G, sl.rows, sl.n_pad,
                                        sl.tmem_cols, sl.nbuf, sl.stages, cpg, images, p.nx, p.ny, p.d_status);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

}  // namespace

SpanLayout span_layout(const Plan &p, int slot_stride, int n_windows, int k0, int k1) {
  SpanLayout sl;
  // FP16 storage only: its hi + lo operand carries V to ~22 bits, which keeps the subtraction
  // of the discarded power from the energy accurate (BF16 parts carry ~16 bits)
  if (p.prec != DH_PREC_FP16 || !p.tmaps_ok || p.proj_mode != 0) return sl;
  const int T = p.T, s = slot_stride;
  if (s < 4 || s % 4 != 0 || s >= T || n_windows < 2) return sl;
  if (p.ny < 128 || p.nx % 8 != 0) return sl;
  const int nD = k0 + (T - 1 - k1);
  const int cpw = 2 * nD <= 4 ? 4 : (2 * nD <= 8 ? 8 : 0);
  if (cpw == 0) return sl;
  int G = (128 - T) / s + 1;  // span rows 2 (T + (G - 1) s) <= 256
  if (G > kSpanMaxG) G = kSpanMaxG;
  if (G > n_windows) G = n_windows;
  for (; G >= 2; --G) {
    const int rows = (2 * (T + (G - 1) * s) + 15) / 16 * 16;
    // every epilogue warp reads the columns of 4 windows: cover them even where G is not 4 or 8
    const int n_pad = ((G > 4 ? 8 : 4) * cpw + 15) / 16 * 16;
    // four partial accumulators (more were measured to gain nothing: the remaining error is
    // the FP32 rounding of the energy and of the subtracted power); each needs a k-step
    if (rows < 16 * kNacc) continue;
    const int nacc = kNacc;
    // accumulator buffers: 4 where tensor memory has room (the MMAs run further ahead of the
    // epilogue), else 2
    const int nbuf = 4 * nacc * n_pad <= 512 ? 4 : 2;
    int tmem_cols = 32;
    while (tmem_cols < nbuf * nacc * n_pad) tmem_cols *= 2;
    const int k_pad = (rows + 63) / 64 * 64;
    const int img = 2 * n_pad * k_pad * 2;
    // a group's operand lives in the operand slots of its G windows
    if ((size_t)img > (size_t)G * p.B_window_bytes) continue;
    const int scr = 2 * ((T + (G - 1) * s) / 4) * 512;  // chunk energies, two tile parities
    const size_t fixed = (size_t)img + scr + 1024 + 256;
    if (fixed + (size_t)rows * 256 * 2 > kSpanSmemLimit) continue;
    int stages = (int)((kSpanSmemLimit - fixed) / ((size_t)rows * 256));
    if (stages > kSpanMaxStages) stages = kSpanMaxStages;
    sl.G = G; sl.cpw = cpw; sl.rows = rows; sl.n_pad = n_pad; sl.k_pad = k_pad; sl.stride = s;
    sl.img_bytes = img; sl.stages = stages; sl.nacc = nacc; sl.tmem_cols = tmem_cols; sl.scr_bytes = scr;
    sl.nbuf = nbuf;
    return sl;
  }
  return sl;
}

dh_status launch_project_span(Plan &p, const SpanLayout &sl, int first_slot, int n_windows, float *images, int woff,
                              cudaStream_t s) {
  if (sl.G < 2) return DH_ERR_STATE;
  const bool bf16 = p.prec == DH_PREC_BF16;
  if (sl.cpw == 4) return bf16 ? project_span_t<4, true>(p, sl, first_slot, n_windows, images, woff, s)
                               : project_span_t<4, false>(p, sl, first_slot, n_windows, images, woff, s);
  return bf16 ? project_span_t<8, true>(p, sl, first_slot, n_windows, images, woff, s)
              : project_span_t<8, false>(p, sl, first_slot, n_windows, images, woff, s);
}

}  // namespace dh
