// Eq. 1 with the 32-point DFT stages of each 1024-point transform on the tensor cores.
//
// A 1024-point DFT along one axis, X[x1 + 32 x2] = sum_k a[k] w^(x k) (w = exp(+2 pi i / 1024),
// k = 32 k1 + k2), is two batched 32-point DFTs with a twiddle between them (Cooley-Tukey):
//   stage A, per k2:  b[x1, k2] = sum_k1 W[x1, k1] a[32 k1 + k2]      (W the 32-point DFT)
//   twiddle:          b'[x1, k2] = b[x1, k2] w^(x1 k2)
//   stage B, per x1:  X[x1 + 32 x2] = sum_k2 W[x2, k2] b'[x1, k2].
// Each stage is one real GEMM per tile of 128 vectors (M = 128, K = 64 = the 32 real and 32
// imaginary parts, N = 64): [Re v | Im v] = [Re u | Im u] [[Wr, Wi], [-Wi, Wr]] (W is
// symmetric). tcgen05.mma kind::f16 with FP32 accumulation in tensor memory; the data and W
// are both split into FP16 hi + lo parts and three products (hi hi, hi lo, lo hi) are
// accumulated, which keeps the transform at FP32-level accuracy (~1e-6 relative; a single
// FP16 operand would add an error comparable to the 16-bit storage rounding).
//
// Work is done by warpgroups (4 warps, 128 threads), two per CTA, each on its own item --
// 4 rows (row pass) or 4 columns (column pass) of one frame: 128 vectors, one M-tile -- with
// its own shared-memory operand buffer, 64 tensor-memory columns, MMA barrier and named
// barrier, so the warpgroups of an SM overlap each other's tensor-core waits with arithmetic:
//   converter   the item's 32 values per (row or column, k2) -> K-major operand rows
//               (128-byte rows, 128-byte swizzle), FP16 hi and lo
//   stage A     12 MMAs (4 K-steps x 3 products), one commit
//   epilogue A  tcgen05.ld of the thread's accumulator row, twiddle, split -> the
//               MN-major operand of stage B (K = the 32-point index k2, M = (row, x1))
//   stage B     12 MMAs
//   epilogue B  row pass: y chirp of the row -> the FP32 intermediate; column pass: the
//               16-bit (or FP32) hologram planes.
// The intermediate between the passes is private to this render: per frame, 256 tiles of 4
// columns, tile x1 * 8 + j holding columns x1 + 32 (4 j + c), c = 0..3, as [y][4] FP32
// complex (32 KB, one bulk copy). A row thread then writes its 4 columns of a tile as 32
// contiguous bytes, and the column converter reads 256 contiguous bytes per warp.
// Power-of-two scales keep every FP16 operand below 2^14 for any 16-bit input: the row
// pass's stage B input is scaled by 1/4 (in the twiddle table), the intermediate by 1/32
// (with the y chirp), the column pass's stage B input by 1/4, and the column output by 128.
// Included by render.cu inside its anonymous namespace (uses its store helpers).

namespace tcr {

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
  return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

constexpr int N = 1024;
constexpr int ITEM = 4;                    // rows or columns per item (= warps per warpgroup)
constexpr int WG_THREADS = 128;
constexpr int WGS = 2;                     // warpgroups per CTA
constexpr int THREADS = WG_THREADS * WGS;
constexpr int ITEMS_PER_FRAME = N / ITEM;  // per pass
constexpr long long NPIX = (long long)N * N;
constexpr int OP_BYTES = 128 * 128;        // one M-tile operand (128 x 64 FP16), hi or lo
constexpr int WORK_BYTES = 2 * OP_BYTES;   // per warpgroup: hi | lo; also the column tile
constexpr int TILE_ELEMS = ITEM * N;       // complex values of one column tile (32 KB)
constexpr int W_BYTES = 64 * 128;          // the DFT embedding (64 x 64 FP16), hi or lo
constexpr int TWP_BYTES = 16 * 32 * 16;    // twiddle pairs [a / 2][lane]: (wx_a, wx_a+1, wy_a, wy_a+1)
constexpr int TWN_BYTES = 16 * 32 * 8;     // [a / 2][lane]: (-wy_a, -wy_a+1)
constexpr int CXM_BYTES = N * 16;          // per x: (c.x, c.y, -2^23 c.x, -2^23 c.y)
// dynamic shared memory: work[0] | work[1] | W hi | W lo | twp | twn | cxm (+ 1 KB alignment)
constexpr int OFF_W = WGS * WORK_BYTES;
constexpr int OFF_TWP = OFF_W + 2 * W_BYTES;
constexpr int OFF_TWN = OFF_TWP + TWP_BYTES;
constexpr int OFF_CXM = OFF_TWN + TWN_BYTES;
constexpr int SMEM_BYTES = OFF_CXM + CXM_BYTES + 1024;
constexpr uint32_t TMEM_COLS = 128;        // 64 accumulator columns per warpgroup
constexpr float ROW_B_SCALE = 0.25f;       // stage B input scale (folded into the twiddles)
constexpr float MID_SCALE = 1.0f / 32.0f;  // the intermediate holds Y / 32
constexpr float COL_OUT_SCALE = 128.0f;    // 1 / (MID_SCALE x ROW_B_SCALE)
constexpr uint32_t IDESC_K = tc::idesc_f16(false, false, false, 128, 64);
constexpr uint32_t IDESC_MN = tc::idesc_f16(false, true, false, 128, 64);

// Layout of the device tables (the plan's tensor-core render tables).
constexpr int GLOB_W = 0;                      // W hi then W lo, plain [n][k] FP16 rows
constexpr int GLOB_TWP = 2 * W_BYTES;          // twiddle pairs and their negated sines,
constexpr int GLOB_TWN = GLOB_TWP + TWP_BYTES; // as in shared memory
constexpr int GLOB_BYTES = GLOB_TWN + TWN_BYTES;

// Per-warpgroup state of the tensor-core items.
struct Ctx {
  uint8_t *work;            // this warpgroup's operand buffer, 1024-aligned
  uint8_t *w;               // W hi, then W lo (1024-aligned)
  const float4 *twp;        // [a / 2][lane]
  const float2 *twn;
  const float4 *cxm;
  uint64_t *mma_bar;        // this warpgroup's MMA barrier
  volatile int *stage_ok;   // its leader's outcome of the last MMA wait
  uint32_t mma_phase;
  uint32_t tmem;            // this warpgroup's 64 accumulator columns (lane 0)
  int wg;                   // warpgroup index in the CTA
  bool ok;                  // false once a wait gave up
};

__device__ __forceinline__ void wg_sync(const Ctx &c) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + c.wg), "r"(WG_THREADS) : "memory");
}
// warpgroup barrier that also returns whether v holds on every thread of the warpgroup
__device__ __forceinline__ bool wg_all(const Ctx &c, bool v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(v ? 1 : 0), "r"(1 + c.wg), "r"(WG_THREADS)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ bool wg_leader() { return (threadIdx.x & (WG_THREADS - 1)) == 0; }

// FP16 hi + lo of two FP32 values (a at the lower address): hi = rn(a), lo = rn(a - hi), the
// difference taken by the mixed-precision FMA from the FP16 hi itself (exact: a - hi fits
// FP32). neg1 is FP16 -1.
__device__ __forceinline__ uint32_t split_pair(float a, float b, uint16_t neg1, uint32_t &lo) {
  uint32_t h;
  asm("{\n\t.reg .f16 h0, h1;\n\t.reg .f32 r0, r1;\n\t"
      "cvt.rn.f16x2.f32 %0, %3, %2;\n\t"
      "mov.b32 {h0, h1}, %0;\n\t"
      "fma.rn.f32.f16 r0, h0, %4, %2;\n\t"
      "fma.rn.f32.f16 r1, h1, %4, %3;\n\t"
      "cvt.rn.f16x2.f32 %1, r1, r0;\n\t}"
      : "=r"(h), "=r"(lo)
      : "f"(a), "f"(b), "h"(neg1));
  return h;
}
__device__ __forceinline__ uint16_t f16_neg1() { return __half_as_ushort(__float2half(-1.0f)); }

// Byte offset of 16-byte chunk j of row r of a K-major operand (128-byte rows, 128-byte
// swizzle: chunk j of row r sits at chunk j ^ (r mod 8) of its 1024-byte atom).
__device__ __forceinline__ uint32_t kmaj_chunk(int r, int j) {
  return ((uint32_t)(r >> 3) << 10) + ((uint32_t)(r & 7) << 7) + ((uint32_t)(j ^ (r & 7)) << 4);
}
// Byte offset of 16-byte chunk c (8 M-elements) of K-row k in M-chunk h (64 elements) of an
// MN-major operand: 64 K-rows of 128 bytes per M-chunk, the same swizzle by K-row.
__device__ __forceinline__ uint32_t mnmaj_chunk(int h, int k, int c) {
  return ((uint32_t)h << 13) + ((uint32_t)(k >> 3) << 10) + ((uint32_t)(k & 7) << 7) +
         ((uint32_t)(c ^ (k & 7)) << 4);
}

// Stage A operand row r: K = [Re v[0..31] | Im v[0..31]], hi and lo.
__device__ __forceinline__ void write_kmajor_row(const Ctx &c, int r, const float2 (&v)[32]) {
  uint8_t *hi = c.work, *lo = c.work + OP_BYTES;
  const uint16_t neg1 = f16_neg1();
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = ((j & 3) << 3) + 2 * e;
      h[e] = j < 4 ? split_pair(v[k].x, v[k + 1].x, neg1, l[e]) : split_pair(v[k].y, v[k + 1].y, neg1, l[e]);
    }
    const uint32_t off = kmaj_chunk(r, j);
    *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// One stage of this warpgroup: its operand writes (and tensor-memory reads) are ordered
// before the MMAs, its leader issues 4 K-steps x 3 products, commits and waits for their
// completion (bounded), and a warpgroup barrier hands the result and the outcome on.
__device__ __forceinline__ void run_stage(Ctx &c, bool mn_major) {
  tc::fence_before_sync();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  wg_sync(c);
  if (wg_leader()) {
    tc::fence_after_sync();
    const uint32_t ahi = tc::smem_u32(c.work), alo = ahi + OP_BYTES, b0 = tc::smem_u32(c.w);
    const uint32_t id = mn_major ? IDESC_MN : IDESC_K;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      uint64_t dh, dl;
      if (mn_major) {
        dh = tc::smem_desc(ahi + 2048 * kk, 8192, 1024, tc::kSwizzle128);
        dl = tc::smem_desc(alo + 2048 * kk, 8192, 1024, tc::kSwizzle128);
      } else {
        dh = tc::smem_desc(ahi + 32 * kk, 16, 1024, tc::kSwizzle128);
        dl = tc::smem_desc(alo + 32 * kk, 16, 1024, tc::kSwizzle128);
      }
      const uint64_t wh = tc::smem_desc(b0 + 32 * kk, 16, 1024, tc::kSwizzle128);
      const uint64_t wl = tc::smem_desc(b0 + W_BYTES + 32 * kk, 16, 1024, tc::kSwizzle128);
      tc::mma_f16(c.tmem, dh, wh, id, kk > 0 ? 1u : 0u);
      tc::mma_f16(c.tmem, dh, wl, id, 1u);
      tc::mma_f16(c.tmem, dl, wh, id, 1u);
    }
    tc::mma_commit(c.mma_bar);
    *c.stage_ok = tc::mbar_wait(c.mma_bar, c.mma_phase) ? 1 : 0;
  }
  wg_sync(c);
  c.mma_phase ^= 1;
  tc::fence_after_sync();
  if (!*c.stage_ok) c.ok = false;
}

// This thread's accumulator row (warp q of the warpgroup reads lanes 32 q .. 32 q + 31).
__device__ __forceinline__ void load_acc(const Ctx &c, float (&d)[64]) {
  const int q = (threadIdx.x >> 5) & 3;
  tc::tmem_ld64(c.tmem + ((uint32_t)(32 * q) << 16), d);
}

// Epilogue A: accumulator row 32 q + lane (q = warp in the warpgroup) holds b[a] for the 32
// outputs a of one 32-point DFT (d[a] real, d[32 + a] imaginary); b[a] w^(a lane) / 4 goes to
// the MN-major stage B operand at K-rows lane (Re) and 32 + lane (Im), M = 32 q + a.
__device__ __forceinline__ void epilogue_a(const Ctx &c) {
  const int lane = threadIdx.x & 31, q = (threadIdx.x >> 5) & 3;
  float d[64];
  load_acc(c, d);
  uint8_t *hi = c.work, *lo = c.work + OP_BYTES;
  const int h = q >> 1, c0 = (q & 1) << 2;
  const uint16_t neg1 = f16_neg1();
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int a = 8 * cc + 2 * e, p = a >> 1;
      const float4 w = c.twp[p * 32 + lane];   // (wx_a, wx_a+1, wy_a, wy_a+1)
      const float2 nw = c.twn[p * 32 + lane];  // (-wy_a, -wy_a+1)
      const float2 R = make_float2(d[a], d[a + 1]), I = make_float2(d[32 + a], d[33 + a]);
      const float2 wx = make_float2(w.x, w.y), wy = make_float2(w.z, w.w);
      const float2 re = __ffma2_rn(R, wx, __fmul2_rn(I, nw));
      const float2 im = __ffma2_rn(R, wy, __fmul2_rn(I, wx));
      rh[e] = split_pair(re.x, re.y, neg1, rl[e]);
      ih[e] = split_pair(im.x, im.y, neg1, il[e]);
    }
    const uint32_t o_re = mnmaj_chunk(h, lane, c0 + cc), o_im = mnmaj_chunk(h, 32 + lane, c0 + cc);
    *reinterpret_cast<uint4 *>(hi + o_re) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
    *reinterpret_cast<uint4 *>(lo + o_re) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
    *reinterpret_cast<uint4 *>(hi + o_im) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
    *reinterpret_cast<uint4 *>(lo + o_im) = make_uint4(il[0], il[1], il[2], il[3]);
  }
}

// Loads row (it % 256) * 4 + q (q = warp in the warpgroup) of frame it / 256 into pf: its 128
// 16-byte chunks, chunk lane + 32 k in pf[k] (read once: streaming loads).
__device__ __forceinline__ void row_load(uint4 (&pf)[4], const uint16_t *__restrict__ frames,
                                         long long frame_stride, int it) {
  const int lane = threadIdx.x & 31, q = (threadIdx.x >> 5) & 3;
  const uint4 *src = reinterpret_cast<const uint4 *>(
      frames + (long long)(it / ITEMS_PER_FRAME) * frame_stride + (long long)((it % ITEMS_PER_FRAME) * ITEM + q) * N);
#pragma unroll
  for (int k = 0; k < 4; ++k) pf[k] = __ldcs(src + lane + 32 * k);
}

// Row item: rows y0 .. y0 + 3 of one frame, row y0 + q in `pf` (row_load). Output: the
// frame's intermediate `dst` (Y / 32). `parked()` runs once the rows are in shared memory
// (the caller loads the next rows into pf there); `freed()` runs on every thread of the
// warpgroup once its operand buffer is free (after stage B).
template <typename Parked, typename Freed>
__device__ __forceinline__ void row_item(Ctx &c, const uint4 (&pf)[4], int y0, const float2 *__restrict__ cy,
                                         float2 *__restrict__ dst, Parked parked, Freed freed) {
  const int lane = threadIdx.x & 31, q = (threadIdx.x >> 5) & 3;
  wg_sync(c);  // the previous item is done with the buffer and the accumulators
  uint4 *park = reinterpret_cast<uint4 *>(c.work + q * 2048);
#pragma unroll
  for (int k = 0; k < 4; ++k) park[lane + 32 * k] = pf[k];
  parked();
  __syncwarp();
  const uint16_t *row = reinterpret_cast<const uint16_t *>(c.work + q * 2048);
  float2 v[32];
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) {
    // (2^23 + I) c - 2^23 c = I c with one rounding: the uint16 -> float conversion rides on
    // the chirp's FMA
    const float f = __uint_as_float(0x4b000000u | row[32 * k1 + lane]);
    const float4 t = c.cxm[32 * k1 + lane];
    v[k1] = make_float2(fmaf(f, t.x, t.z), fmaf(f, t.y, t.w));
  }
  wg_sync(c);  // every parked row is read before the operand overwrites them
  write_kmajor_row(c, (q << 5) + lane, v);
  run_stage(c, false);
  epilogue_a(c);
  run_stage(c, true);
  freed();
  // epilogue B: accumulator row 32 q + lane holds X[lane + 32 x2] / 4 of row y = y0 + q;
  // Y / 32 = X cy / 32 goes to tile lane * 8 + x2 / 4, column x2 % 4, row y
  const int y = y0 + q;
  float d[64];
  load_acc(c, d);
  const float2 cyy = cy[y];
  const float sy = MID_SCALE / ROW_B_SCALE;
  const float2 cr = make_float2(cyy.x * sy, cyy.x * sy), ci = make_float2(cyy.y * sy, cyy.y * sy);
  const float2 nci = make_float2(-ci.x, -ci.y);
  float4 *out = reinterpret_cast<float4 *>(dst + (long long)(lane * 8) * TILE_ELEMS + (long long)y * ITEM);
#pragma unroll
  for (int x2 = 0; x2 < 32; x2 += 2) {
    const float2 R = make_float2(d[x2], d[x2 + 1]), I = make_float2(d[32 + x2], d[33 + x2]);
    const float2 re = __ffma2_rn(R, cr, __fmul2_rn(I, nci));
    const float2 im = __ffma2_rn(R, ci, __fmul2_rn(I, cr));
    out[(x2 >> 2) * (TILE_ELEMS / 2) + ((x2 & 2) >> 1)] = make_float4(re.x, im.x, re.y, im.y);
  }
}

// Bulk copy of one 32 KB column tile into this warpgroup's buffer, completing on `bar`
// (its leader issues it; generic accesses of the buffer are ordered before it by the
// fence and the preceding warpgroup barrier).
__device__ __forceinline__ void issue_tile(const Ctx &c, const float2 *src, uint64_t *bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc::mbar_arrive_expect_tx(bar, WORK_BYTES);
  tc::bulk_load(c.work, src, WORK_BYTES / 2, bar);
  tc::bulk_load(c.work + WORK_BYTES / 2, reinterpret_cast<const char *>(src) + WORK_BYTES / 2, WORK_BYTES / 2, bar);
}

// Column item: the 4-column tile `src` (tile x1 * 8 + j of one frame: columns x1 + 32 (4 j + c))
// lands in this warpgroup's buffer on `bar` (already issued). Waits for it (bounded), reads
// it, drops its lines from L2, runs the two stages and writes the hologram planes of `slot`.
// `freed()` runs on every thread once the buffer is free (the caller may issue the next
// tile's copy). Returns false, uniformly over the warpgroup, if a wait gave up.
template <typename OutT, typename Freed>
__device__ __forceinline__ bool col_item(Ctx &c, const float2 *__restrict__ src, uint64_t *bar, uint32_t &phase,
                                         int x1, int j, OutT *__restrict__ H, long long rows_total, int slot,
                                         uint32_t &maxbits, Freed freed) {
  const int lane = threadIdx.x & 31, q = (threadIdx.x >> 5) & 3;
  const int tid = threadIdx.x & (WG_THREADS - 1);
  const bool got = tc::mbar_wait(bar, phase);
  phase ^= 1;
  if (got)
    for (int off = tid * 128; off < WORK_BYTES; off += WG_THREADS * 128)
      l2_discard(reinterpret_cast<const char *>(src) + off);
  // converter: thread (column xc = lane & 3, l2 = 8 q + lane / 4) reads Y[32 l1 + l2][xc]
  // (a warp reads 256 contiguous bytes per l1) for operand row 32 xc + l2
  const int xc = lane & 3, l2 = (q << 3) + (lane >> 2);
  const float2 *tile = reinterpret_cast<const float2 *>(c.work);
  float2 v[32];
#pragma unroll
  for (int l1 = 0; l1 < 32; ++l1) v[l1] = tile[(32 * l1 + l2) * ITEM + xc];
  // the copy's outcome, and every read of the tile before the operand overwrites it
  if (!wg_all(c, got)) {
    c.ok = false;
    return false;
  }
  write_kmajor_row(c, (xc << 5) + l2, v);
  run_stage(c, false);
  epilogue_a(c);
  run_stage(c, true);
  freed();
  // epilogue B: accumulator row 32 q + lane holds H[lane + 32 y2][kx] / 128 for column q of
  // the tile: kx = x1 + 32 (4 j + q)
  const int kx = x1 + 32 * (ITEM * j + q);
  float d[64];
  load_acc(c, d);
  float mx = __uint_as_float(maxbits);
  if constexpr (sizeof(OutT) == 4) {  // FP32 planes: [slot][re|im][p]
    OutT *re = H + (long long)slot * 2 * NPIX + (long long)kx * N;
    OutT *im = re + NPIX;
#pragma unroll
    for (int y2 = 0; y2 < 32; ++y2) {
      const float a = d[y2] * COL_OUT_SCALE, b = d[32 + y2] * COL_OUT_SCALE;
      mx = fmaxf(mx, fmaxf(fabsf(a), fabsf(b)));
      st_stream(re + lane + 32 * y2, a);
      st_stream(im + lane + 32 * y2, b);
    }
  } else {  // 16-bit planes in 64-pixel blocks: [p / 64][row = 2 slot + c][p % 64], p = kx N + y
    const long long bstride = rows_total << 6;
    OutT *base = H + (2ll * slot << 6) + (long long)kx * (N / 64) * bstride + lane;
#pragma unroll
    for (int y2 = 0; y2 < 32; ++y2) {
      const float a = d[y2] * COL_OUT_SCALE, b = d[32 + y2] * COL_OUT_SCALE;
      mx = fmaxf(mx, fmaxf(fabsf(a), fabsf(b)));
      OutT *qp = base + (y2 >> 1) * bstride + ((y2 & 1) << 5);
      st_stream(qp, to_store<OutT>(a));
      st_stream(qp + 64, to_store<OutT>(b));
    }
  }
  maxbits = __float_as_uint(mx);
  return true;
}

// Per-CTA set-up: shared-memory carve-up, tables, the warpgroups' MMA barriers and 128
// tensor-memory columns (warp 0 allocates). Ends with a CTA barrier.
__device__ __forceinline__ void setup(Ctx &c, uint8_t *sm, uint64_t *mma_bars, uint32_t *tmem_holder,
                                      int *stage_ok, const uint8_t *__restrict__ glob,
                                      const float2 *__restrict__ cx) {
  c.wg = threadIdx.x / WG_THREADS;
  c.work = sm + c.wg * WORK_BYTES;
  c.w = sm + OFF_W;
  c.twp = reinterpret_cast<const float4 *>(sm + OFF_TWP);
  c.twn = reinterpret_cast<const float2 *>(sm + OFF_TWN);
  c.cxm = reinterpret_cast<const float4 *>(sm + OFF_CXM);
  c.mma_bar = mma_bars + c.wg;
  c.stage_ok = stage_ok + c.wg;
  c.mma_phase = 0;
  c.ok = true;
  const uint4 *wgl = reinterpret_cast<const uint4 *>(glob + GLOB_W);
  for (int e = threadIdx.x; e < 2 * 64 * 8; e += blockDim.x) {  // 16-byte chunks of W hi, W lo
    const int part = e >> 9, n = (e >> 3) & 63, j = e & 7;
    *reinterpret_cast<uint4 *>(sm + OFF_W + part * W_BYTES + kmaj_chunk(n, j)) = wgl[e];
  }
  const uint4 *tg = reinterpret_cast<const uint4 *>(glob + GLOB_TWP);
  uint4 *ts = reinterpret_cast<uint4 *>(sm + OFF_TWP);
  for (int e = threadIdx.x; e < (TWP_BYTES + TWN_BYTES) / 16; e += blockDim.x) ts[e] = tg[e];
  float4 *cm = reinterpret_cast<float4 *>(sm + OFF_CXM);
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const float2 v = cx[e];
    cm[e] = make_float4(v.x, v.y, -8388608.f * v.x, -8388608.f * v.y);  // exact scaling
  }
  if (threadIdx.x == 0) {
    for (int g = 0; g < WGS; ++g) tc::mbar_init(mma_bars + g, 1);
    tc::fence_barrier_init();
  }
  if ((threadIdx.x >> 5) == 0) {
    tc::tmem_alloc(tmem_holder, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  c.tmem = *tmem_holder + 64 * c.wg;
}

// Per-CTA tear-down: every thread's tensor-memory use is done; warp 0 frees the columns.
__device__ __forceinline__ void teardown(const Ctx &c) {
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if ((threadIdx.x >> 5) == 0) {
    __syncwarp();
    tc::tmem_dealloc(c.tmem, TMEM_COLS);  // warp 0 belongs to warpgroup 0: c.tmem is the base
  }
}

}  // namespace tcr

// ---------------------------------------------------------------- tensor-core render, chunks
// Row pass over a chunk of 1024^2 frames: one warpgroup item = 4 consecutive rows of a frame.
__global__ void __launch_bounds__(tcr::THREADS, 2)
k_render_rows_tc(const uint16_t *__restrict__ frames, long long frame_stride, const uint8_t *__restrict__ tcg,
                 const float2 *__restrict__ cx, const float2 *__restrict__ cy, float2 *__restrict__ mid,
                 int n_items, uint32_t *__restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t mma_bars[tcr::WGS];
  __shared__ uint32_t tmem_holder;
  __shared__ int stage_ok[tcr::WGS];
  tcr::Ctx c;
  tcr::setup(c, tcr::align1024(smem_raw), mma_bars, &tmem_holder, stage_ok, tcg, cx);
  const int stride = (int)gridDim.x * tcr::WGS;
  int item = (int)blockIdx.x * tcr::WGS + c.wg;
  uint4 pf[4];
  if (item < n_items) tcr::row_load(pf, frames, frame_stride, item);
  for (; item < n_items && c.ok; item += stride) {
    const int f = item / tcr::ITEMS_PER_FRAME, y0 = (item % tcr::ITEMS_PER_FRAME) * tcr::ITEM;
    const int nxt = item + stride;
    tcr::row_item(c, pf, y0, cy, mid + (long long)f * tcr::NPIX, [&]() {
      if (nxt < n_items) tcr::row_load(pf, frames, frame_stride, nxt);
    }, []() {});
  }
  if (!c.ok && tcr::wg_leader()) {
    atomicOr(status, DH_FLAG_WAIT_TIMEOUT);
    tc::mbar_wait(c.mma_bar, c.mma_phase ^ 1);  // MMAs of a stage that gave up, before tear-down
  }
  tcr::teardown(c);
}

// Column pass over a chunk: one warpgroup item = one 4-column tile of a frame, written to
// hologram slot slot0 + f. The next tile's copy is issued as soon as the current one's
// operand buffer is free, so it lands during the current item's last epilogue.
template <typename OutT>
__global__ void __launch_bounds__(tcr::THREADS, 2)
k_render_cols_tc(const float2 *__restrict__ mid, const uint8_t *__restrict__ tcg, const float2 *__restrict__ cx,
                 OutT *__restrict__ H, long long rows_total, int slot0, int n_items, uint32_t *__restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t mma_bars[tcr::WGS];
  __shared__ __align__(8) uint64_t tile_bars[tcr::WGS];
  __shared__ uint32_t tmem_holder;
  __shared__ int stage_ok[tcr::WGS];
  tcr::Ctx c;
  tcr::setup(c, tcr::align1024(smem_raw), mma_bars, &tmem_holder, stage_ok, tcg, cx);
  if (threadIdx.x == 0) {
    for (int g = 0; g < tcr::WGS; ++g) tc::mbar_init(tile_bars + g, 1);
    tc::fence_barrier_init();
  }
  __syncthreads();
  uint64_t *bar = tile_bars + c.wg;
  const int stride = (int)gridDim.x * tcr::WGS;
  int item = (int)blockIdx.x * tcr::WGS + c.wg;
  auto src_of = [&](int it) {
    return mid + (long long)(it / tcr::ITEMS_PER_FRAME) * tcr::NPIX +
           (long long)(it % tcr::ITEMS_PER_FRAME) * tcr::TILE_ELEMS;
  };
  uint32_t phase = 0, maxbits = 0;
  // a copy issued for the next item and not yet waited on: it completes the phase `phase`
  bool pending = false;
  if (item < n_items && tcr::wg_leader()) tcr::issue_tile(c, src_of(item), bar);
  for (; item < n_items && c.ok; item += stride) {
    const int nxt = item + stride, tt = item % tcr::ITEMS_PER_FRAME;
    pending = false;
    if (!tcr::col_item<OutT>(c, src_of(item), bar, phase, tt >> 3, tt & 7, H, rows_total,
                             slot0 + item / tcr::ITEMS_PER_FRAME, maxbits, [&]() {
                               if (nxt < n_items) {
                                 if (tcr::wg_leader()) tcr::issue_tile(c, src_of(nxt), bar);
                                 pending = true;
                               }
                             }))
      break;
  }
  if (!c.ok && tcr::wg_leader()) {
    atomicOr(status, DH_FLAG_WAIT_TIMEOUT);
    // before the CTA exits: a copy that did not complete in time (its phase is phase ^ 1
    // after the failed wait), a copy issued for the next item, and MMAs of a stage that gave up
    tc::mbar_wait(bar, pending ? phase : phase ^ 1);
    tc::mbar_wait(c.mma_bar, c.mma_phase ^ 1);
  }
  if (maxbits >= overflow_bits<OutT>()) atomicOr(status, DH_FLAG_STORE_OVERFLOW);
  tcr::teardown(c);
}
