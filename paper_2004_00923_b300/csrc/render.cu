// Eq. 1 on the GPU: Fresnel rendering of 16-bit interferograms into holograms.
//
//   H[t,y,x] = s * sum_{k,l} I[t,l,k] c(k) c(l) exp(+2 pi i (x k / n_x + y l / n_y)),
//   c(k) = exp(-i pi a (k - n/2)^2),  a = pitch^2 / (lambda z),  s = 1/sqrt(n_x n_y).
//
// Two passes over each frame, both on FP32 CUDA cores:
//   rows:    uint16 load -> x chirp (scale folded in) -> n_x-point FFT -> y chirp ->
//            mid, written transposed (mid[f][kx][y]) through a shared staging tile
//   columns: mid (L2-resident chunk of frames, read contiguously) -> n_y-point FFT ->
//            16/32-bit planes of H in column-major pixel order p = kx n_y + ky
// Every transform is done by P threads of one warp (or of one CTA for n >= 2048), with
// coalesced global loads and stores on both passes.
// The FFT is a Stockham auto-sort transform (Govindaraju et al., SC'08 formulation):
// each thread keeps R points in registers, runs an in-register radix-R DIF transform with
// compile-time twiddles, and exchanges through padded shared memory between passes.
// Inter-pass twiddles come from FP64-built tables. Frames are processed in chunks whose
// intermediate fits in L2, so HBM sees only the uint16 input and the hologram output.
#include "dh_internal.cuh"
#include "tc_sm100.cuh"

#include <math.h>
#include <vector>

namespace dh {
namespace {

// cos / sin (2 pi m / 64), m = 0..63 (mathematical constants, rounded to float)
constexpr float kCos64[64] = {
    1.000000000e+00f, 9.951847267e-01f, 9.807852804e-01f, 9.569403357e-01f,
    9.238795325e-01f, 8.819212643e-01f, 8.314696123e-01f, 7.730104534e-01f,
    7.071067812e-01f, 6.343932842e-01f, 5.555702330e-01f, 4.713967368e-01f,
    3.826834324e-01f, 2.902846773e-01f, 1.950903220e-01f, 9.801714033e-02f,
    6.123233996e-17f, -9.801714033e-02f, -1.950903220e-01f, -2.902846773e-01f,
    -3.826834324e-01f, -4.713967368e-01f, -5.555702330e-01f, -6.343932842e-01f,
    -7.071067812e-01f, -7.730104534e-01f, -8.314696123e-01f, -8.819212643e-01f,
    -9.238795325e-01f, -9.569403357e-01f, -9.807852804e-01f, -9.951847267e-01f,
    -1.000000000e+00f, -9.951847267e-01f, -9.807852804e-01f, -9.569403357e-01f,
    -9.238795325e-01f, -8.819212643e-01f, -8.314696123e-01f, -7.730104534e-01f,
    -7.071067812e-01f, -6.343932842e-01f, -5.555702330e-01f, -4.713967368e-01f,
    -3.826834324e-01f, -2.902846773e-01f, -1.950903220e-01f, -9.801714033e-02f,
    -1.836970199e-16f, 9.801714033e-02f, 1.950903220e-01f, 2.902846773e-01f,
    3.826834324e-01f, 4.713967368e-01f, 5.555702330e-01f, 6.343932842e-01f,
    7.071067812e-01f, 7.730104534e-01f, 8.314696123e-01f, 8.819212643e-01f,
    9.238795325e-01f, 9.569403357e-01f, 9.807852804e-01f, 9.951847267e-01f,
};
constexpr float kSin64[64] = {
    0.000000000e+00f, 9.801714033e-02f, 1.950903220e-01f, 2.902846773e-01f,
    3.826834324e-01f, 4.713967368e-01f, 5.555702330e-01f, 6.343932842e-01f,
    7.071067812e-01f, 7.730104534e-01f, 8.314696123e-01f, 8.819212643e-01f,
    9.238795325e-01f, 9.569403357e-01f, 9.807852804e-01f, 9.951847267e-01f,
    1.000000000e+00f, 9.951847267e-01f, 9.807852804e-01f, 9.569403357e-01f,
    9.238795325e-01f, 8.819212643e-01f, 8.314696123e-01f, 7.730104534e-01f,
    7.071067812e-01f, 6.343932842e-01f, 5.555702330e-01f, 4.713967368e-01f,
    3.826834324e-01f, 2.902846773e-01f, 1.950903220e-01f, 9.801714033e-02f,
    1.224646799e-16f, -9.801714033e-02f, -1.950903220e-01f, -2.902846773e-01f,
    -3.826834324e-01f, -4.713967368e-01f, -5.555702330e-01f, -6.343932842e-01f,
    -7.071067812e-01f, -7.730104534e-01f, -8.314696123e-01f, -8.819212643e-01f,
    -9.238795325e-01f, -9.569403357e-01f, -9.807852804e-01f, -9.951847267e-01f,
    -1.000000000e+00f, -9.951847267e-01f, -9.807852804e-01f, -9.569403357e-01f,
    -9.238795325e-01f, -8.819212643e-01f, -8.314696123e-01f, -7.730104534e-01f,
    -7.071067812e-01f, -6.343932842e-01f, -5.555702330e-01f, -4.713967368e-01f,
    -3.826834324e-01f, -2.902846773e-01f, -1.950903220e-01f, -9.801714033e-02f,
};
constexpr float kRsqrt2 = 0.7071067811865475244f;

// Threads of a render CTA (FFTs per CTA = kCtaThreads / P, at most 16; one FFT when it
// needs more threads). 128 threads measured faster at 512^2 and much slower at 2048^2.
constexpr int kCtaThreads = 256;
// log2 of the radix of an FFT length's passes. Measured: radix 32 at 1024 (two passes; radix
// 16, three passes, was 22% slower) and at 2048 (32 x 32 x 2; 21% faster than 16 x 16 x 8).
__host__ __device__ constexpr int log_radix(int logn) {
  return logn == 6 ? 3 : (logn == 5 || logn == 9 || logn == 10 || logn == 11) ? 5 : 4;
}

__host__ __device__ constexpr int bitrev(int k, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r = (r << 1) | ((k >> i) & 1);
  return r;
}

// An FFT spec, the template argument of every length-dependent piece below: log2 of the
// length in the low 4 bits, log2 of the radix above them (0: the length's default radix,
// log_radix). The plan picks the radix per axis (dh_plan_set_option DH_OPT_FFT_RADIX, or the
// autotuner) among the default and the one alternative instantiated per length: radix 16 at
// 512, 1024 and 2048, radix 32 at 4096.
__host__ __device__ constexpr int sp_logn(int sp) { return sp & 15; }
__host__ __device__ constexpr int sp_logr(int sp) { return (sp >> 4) != 0 ? (sp >> 4) : log_radix(sp & 15); }
__host__ __device__ constexpr int alt_logr(int logn) {
  return logn >= 9 && logn <= 11 ? 4 : logn == 12 ? 5 : 0;
}

// Factorisation of one FFT length: L passes of radix R, then (if R2 > 1) one pass of
// radix R2 in which each thread runs B = R / R2 butterflies. P threads per transform.
template <int LOGN>
struct Shape {
  static constexpr int N = 1 << sp_logn(LOGN);
  static constexpr int LOGR = sp_logr(LOGN);
  static constexpr int R = 1 << LOGR;
  static constexpr int P = N / R;
  static constexpr int L = sp_logn(LOGN) / LOGR;
  static constexpr int LOGR2 = sp_logn(LOGN) - L * LOGR;
  static constexpr int R2 = 1 << LOGR2;
  static constexpr int B = R / R2;
  static constexpr int NPASS = L + (R2 > 1 ? 1 : 0);
  static constexpr int PADN = N + (N >> LOGR);  // padded shared-memory length
  static constexpr int RSTRIDE = (PADN + 1) & ~1;  // per-transform region, 16-byte multiple
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Complex sum and difference with the paired FP32 instructions of this architecture (one
// instruction for both components; each component rounds exactly as the scalar FADD does,
// a - b being fma(b, -1, a)).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// x * w_N^I with w_N = exp(+2 pi i / N), N <= 64, I < N/2: compile-time constants.
template <int N, int I>
__device__ __forceinline__ float2 tw_mul(float2 x) {
  constexpr int M = (I * (64 / N)) & 63;
  if constexpr (M == 0) {
    return x;
  } else if constexpr (M == 16) {
    return make_float2(-x.y, x.x);
  } else if constexpr (M == 8) {
    return make_float2((x.x - x.y) * kRsqrt2, (x.x + x.y) * kRsqrt2);
  } else if constexpr (M == 24) {
    return make_float2(-(x.x + x.y) * kRsqrt2, (x.x - x.y) * kRsqrt2);
  } else {
    constexpr float c = kCos64[M], s = kSin64[M];
    // (x.x c - x.y s, x.x s + x.y c): the products x.y (-s, c) rounded, then one paired FMA,
    // the same roundings as fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c)
    return __ffma2_rn(make_float2(x.x, x.x), make_float2(c, s), __fmul2_rn(make_float2(x.y, x.y), make_float2(-s, c)));
  }
}

// Radix-2 decimation in frequency over v[O], v[O+S], ..., v[O+(N-1)S]; the result is
// left in bit-reversed order: v[O + S*bitrev(k)] = X[k].
template <int N, int S, int O, int I, int RR>
__device__ __forceinline__ void dif_level(float2 (&v)[RR]) {
  if constexpr (I < N / 2) {
    const float2 a = v[O + I * S], b = v[O + (I + N / 2) * S];
    v[O + I * S] = cadd(a, b);
    v[O + (I + N / 2) * S] = tw_mul<N, I>(csub(a, b));
    dif_level<N, S, O, I + 1, RR>(v);
  }
}
template <int N, int S, int O, int RR>
__device__ __forceinline__ void dif(float2 (&v)[RR]) {
  if constexpr (N > 1) {
    dif_level<N, S, O, 0, RR>(v);
    dif<N / 2, S, O, RR>(v);
    dif<N / 2, S, O + (N / 2) * S, RR>(v);
  }
}
template <int N, int S, int Q, int RR>
__device__ __forceinline__ void dif_each(float2 (&v)[RR]) {
  if constexpr (Q < S) {
    dif<N, S, Q, RR>(v);
    dif_each<N, S, Q + 1, RR>(v);
  }
}

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// One length-N transform spread over P threads (index j). On entry v[r] = x[j + r P];
// on exit element j + i P of the transform is v[out_reg(i)]. `freed()` runs on every thread
// once it has made its last read of `sm` (for the column tile: of the whole buffer).
template <int LOGN, bool CTA_SYNC>
struct Engine {
  using S = Shape<LOGN>;
  // exchanges of a transform spread over several warps synchronise only those warps (a
  // named barrier per transform), unless the transform is the whole CTA
  static __device__ __forceinline__ void sync() {
    if constexpr (!CTA_SYNC) {
      __syncwarp();
    } else if constexpr (S::P >= kCtaThreads) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / S::P), "r"(S::P) : "memory");
    }
  }
  static __device__ __forceinline__ int pad(int i) { return i + (i >> S::LOGR); }
  static __host__ __device__ constexpr int out_reg(int i) {
    return S::R2 == 1 ? bitrev(i, S::LOGR)
                      : (i % S::B) + S::B * bitrev(i / S::B, S::LOGR2);
  }

  template <typename Freed = NoHook>
  static __device__ __forceinline__ void run(float2 (&v)[S::R], float2 *sm, int j,
                                             const float2 *__restrict__ tw, Freed freed = Freed()) {
    if constexpr (S::NPASS == 1) freed();
    dif<S::R, 1, 0, S::R>(v);  // pass 0 (span 1): no inter-pass twiddles
    if constexpr (S::NPASS > 1) {
      sync();  // earlier readers of sm are done
#pragma unroll
      for (int r = 0; r < S::R; ++r) sm[pad(j * S::R + r)] = v[bitrev(r, S::LOGR)];
      sync();
      int tw_off = 0;
#pragma unroll
      for (int p = 1; p < S::L; ++p) {
        const int Ns = 1 << (p * S::LOGR);
#pragma unroll
        for (int r = 0; r < S::R; ++r) v[r] = sm[pad(j + r * S::P)];
        if (p == S::L - 1 && S::R2 == 1) freed();
        const int m = j & (Ns - 1);
#pragma unroll
        for (int r = 1; r < S::R; ++r) v[r] = cmul(v[r], tw[tw_off + (r - 1) * Ns + m]);
        tw_off += (S::R - 1) * Ns;
        dif<S::R, 1, 0, S::R>(v);
        if (p == S::L - 1 && S::R2 == 1) return;
        sync();
        const int base = (j >> (p * S::LOGR)) * Ns * S::R + m;
#pragma unroll
        for (int r = 0; r < S::R; ++r) sm[pad(base + r * Ns)] = v[bitrev(r, S::LOGR)];
        sync();
      }
      if constexpr (S::R2 > 1) {
        constexpr int NsE = 1 << (S::L * S::LOGR);
#pragma unroll
        for (int i = 0; i < S::R; ++i) v[i] = sm[pad(j + i * S::P)];
        freed();
#pragma unroll
        for (int q = 0; q < S::B; ++q) {
          const int b = j + q * S::P;
#pragma unroll
          for (int r2 = 1; r2 < S::R2; ++r2)
            v[q + S::B * r2] = cmul(v[q + S::B * r2], tw[tw_off + (r2 - 1) * NsE + b]);
        }
        dif_each<S::R2, S::B, 0, S::R>(v);
      }
    }
  }
};

// FFTs per CTA (256 threads, or one FFT when it needs more threads than that).
// FFTs per CTA, and the CTAs per SM the register budget gives each pass.
template <int LOGN>
__host__ __device__ constexpr int fpc() {
  return Shape<LOGN>::P >= kCtaThreads ? 1
                                       : (kCtaThreads / Shape<LOGN>::P < 16 ? kCtaThreads / Shape<LOGN>::P : 16);
}
template <int LOGN>
__host__ __device__ constexpr int cta_threads() { return fpc<LOGN>() * Shape<LOGN>::P; }
// CTAs per SM each pass is compiled for: threads counted in whole warps (a CTA of fewer
// threads still holds a warp's registers), row items with 32 complex values a thread at
// 2 x 256 threads (<= 128 registers), 16 values at 3 x 256, 8 at 4 x 256; column items
// (no uint16 prefetch in flight) one step higher, except 32 values from 2048 up, which
// spill at 3 x 256 (2048: 15.1 ms for 512 frames at 2 x 256 against 17.0 at 3 x 256).
// Measured: the radix-16 lengths (4096, 256) gain 3-8% over 2 x 256, the radix-32 ones
// (512, 1024) keep 2 x 256.
template <int LOGN>
__host__ __device__ constexpr int warp_threads() { return cta_threads<LOGN>() < 32 ? 32 : cta_threads<LOGN>(); }
template <int LOGN>
__host__ __device__ constexpr int rows_per_sm() {
  return warp_threads<LOGN>() <= 256
             ? (Shape<LOGN>::R >= 32 ? 512 : Shape<LOGN>::R >= 16 ? 768 : 1024) / warp_threads<LOGN>() : 1;
}
template <int LOGN>
__host__ __device__ constexpr int cols_per_sm() {
  return warp_threads<LOGN>() <= 256
             ? (Shape<LOGN>::R >= 32 ? (sp_logn(LOGN) >= 11 ? 512 : 768) : 1024) / warp_threads<LOGN>() : 1;
}

template <typename T> __device__ __forceinline__ T to_store(float x);
template <> __device__ __forceinline__ float to_store<float>(float x) { return x; }
template <> __device__ __forceinline__ __half to_store<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
// Hologram planes are written once per render and read back by later kernels: store them
// with the streaming hint so they do not push the intermediate out of L2.
__device__ __forceinline__ void st_stream(float *p, float v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(__half *p, __half v) {
  asm volatile("st.global.cs.b16 [%0], %1;" ::"l"(p), "h"(__half_as_ushort(v)) : "memory");
}
__device__ __forceinline__ void st_stream(__nv_bfloat16 *p, __nv_bfloat16 v) {
  asm volatile("st.global.cs.b16 [%0], %1;" ::"l"(p), "h"(__bfloat16_as_ushort(v)) : "memory");
}
// Drop a 128-byte line of the intermediate from L2 without writing it back (its data is
// dead once the column pass has copied its tile).
__device__ __forceinline__ void l2_discard(const void *p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// Overflow watch of the stored planes: the largest |value| bits a thread wrote, compared once
// with the smallest FP32 magnitude that does not store as a finite value of the storage type
// (FP32: Inf/NaN; FP16: >= 65520, which rounds to Inf; BF16: >= 3.3961775e38). NaN bits
// exceed every threshold.
template <typename T> __host__ __device__ constexpr uint32_t overflow_bits();
template <> __host__ __device__ constexpr uint32_t overflow_bits<float>() { return 0x7f800000u; }
template <> __host__ __device__ constexpr uint32_t overflow_bits<__half>() { return 0x477ff000u; }
template <> __host__ __device__ constexpr uint32_t overflow_bits<__nv_bfloat16>() { return 0x7f7f8000u; }

// The row-pass output `mid` of a frame is stored in tiles of CW = fpc(log2 n_y) columns:
// tile t holds columns [t CW, t CW + CW) for every y, row-major [y][CW], and inside a row of
// the tile the column index is XOR-swizzled by sw(y) = (y >> log2(16/CW)) & (CW - 1). A row
// transform then writes each output as part of a CW-element run of one tile row (64 bytes
// for CW = 8), and the column pass reads a whole tile with one bulk copy and walks its
// columns in shared memory without bank conflicts.
__device__ __forceinline__ int mid_swz(int y, int cw_log) {
  return (y >> (4 - cw_log)) & ((1 << cw_log) - 1);
}
// element offset inside one frame's intermediate (< n_x n_y <= 2^24)
__device__ __forceinline__ int mid_index(int kx, int y, int ny, int cw_log) {
  const int t = kx >> cw_log, c = kx & ((1 << cw_log) - 1);
  return ((t * ny + y) << cw_log) + (c ^ mid_swz(y, cw_log));
}

// ---------------------------------------------------------------- work items
// Row work: FPC consecutive rows y0.. of one frame. `pf` holds their uint16 samples (16-byte
// chunks, thread-strided, loaded by row_prefetch); each transform's input row is parked at
// the head of its own exchange region, then `parked()` runs (the caller issues the next
// prefetch there, so it overlaps this item's transforms); `freed()` runs on each thread after
// its last read of shared memory. Output: the frame's intermediate.
template <int LOGN>
struct RowCfg {
  using S = Shape<LOGN>;
  static constexpr int FPC = fpc<LOGN>();
  static constexpr int NT = FPC * S::P;            // threads
  static constexpr int CHUNKS = FPC * S::N / 8;    // 16-byte chunks of the uint16 rows
  static constexpr int CPT = CHUNKS / NT;          // chunks per thread (= R / 8)
  static constexpr int CPR = S::N / 8;             // chunks per row
};

// PER_WARP (transforms of one warp each, P = 32): warp w loads the chunks of row y0 + w only,
// so it can stage them in its own exchange region without a CTA barrier.
template <int LOGN, bool PER_WARP = false>
__device__ __forceinline__ void row_prefetch(uint4 (&pf)[RowCfg<LOGN>::CPT], const uint16_t *__restrict__ frame,
                                             int y0) {
  using C = RowCfg<LOGN>;
  const uint4 *src = reinterpret_cast<const uint4 *>(frame + (long long)y0 * Shape<LOGN>::N);
  if constexpr (PER_WARP) {
    static_assert(Shape<LOGN>::P == 32 && C::CPR == 32 * C::CPT, "one row a warp");
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < C::CPT; ++k) pf[k] = __ldcs(src + w * C::CPR + lane + 32 * k);  // read once
  } else {
#pragma unroll
    for (int k = 0; k < C::CPT; ++k) pf[k] = __ldcs(src + threadIdx.x + k * C::NT);  // read once
  }
}

template <int LOGN, bool LEAD_SYNC = true, bool PER_WARP = false, typename Parked, typename Freed = NoHook>
__device__ __forceinline__ void row_work(const uint4 (&pf)[RowCfg<LOGN>::CPT], float2 *smem, int y0, int ny,
                                         int cw_log, const float2 *__restrict__ cx,
                                         const float2 *__restrict__ cy, const float2 *__restrict__ tw,
                                         float2 *__restrict__ dst, const uint16_t *__restrict__ mean,
                                         Parked parked, Freed freed = Freed()) {
  using S = Shape<LOGN>;
  using C = RowCfg<LOGN>;
  using E = Engine<LOGN, (S::P > 32)>;
  const int fft = threadIdx.x / S::P, j = threadIdx.x % S::P;
  float2 *sm = smem + fft * S::RSTRIDE;
  const int y = y0 + fft;
  if constexpr (LEAD_SYNC) __syncthreads();  // every transform is done with its region (previous item)
  if constexpr (PER_WARP) {  // this warp's row, into its own region
#pragma unroll
    for (int k = 0; k < C::CPT; ++k) reinterpret_cast<uint4 *>(sm)[(threadIdx.x & 31) + 32 * k] = pf[k];
    parked();
    __syncwarp();
  } else {
#pragma unroll
    for (int k = 0; k < C::CPT; ++k) {
      const int c = threadIdx.x + k * C::NT, row = c / C::CPR, cr = c % C::CPR;
      reinterpret_cast<uint4 *>(smem + row * S::RSTRIDE)[cr] = pf[k];
    }
    parked();
    __syncthreads();
  }
  const uint16_t *row16 = reinterpret_cast<const uint16_t *>(sm);
  float2 v[S::R];
  if (mean == nullptr) {
#pragma unroll
    for (int r = 0; r < S::R; ++r) {
      const int x = j + r * S::P;
      const float a = __uint_as_float(0x4b000000u | row16[x]) - 8388608.f;  // exact: u < 2^23
      const float2 c = cx[x];
      v[r] = make_float2(a * c.x, a * c.y);
    }
  } else {  // the residual I - mean of the frame's window (exact: both integers below 2^16)
    const uint16_t *mrow = mean + (long long)y * S::N;
#pragma unroll
    for (int r = 0; r < S::R; ++r) {
      const int x = j + r * S::P;
      // the difference d (|d| < 2^16) taken in integers, then made a float by placing it in
      // the mantissa of 2^23 + 2^22 (one 3-input add, one float subtraction, exact)
      const int d = (int)row16[x] - (int)__ldg(mrow + x);
      const float a = __int_as_float(0x4b400000 + d) - 12582912.f;
      const float2 c = cx[x];
      v[r] = make_float2(a * c.x, a * c.y);
    }
  }
  E::run(v, sm, j, tw, freed);  // its first exchange store is ordered after the reads above
  const float2 cyy = cy[y];
  if ((S::P & ((1 << cw_log) - 1)) == 0) {
    // kx = j + i P: the tile column and the swizzle are fixed per thread, and successive
    // outputs are P n_y elements apart
    float2 *d = dst + mid_index(j, y, ny, cw_log);
    const int step = S::P * ny;
#pragma unroll
    for (int i = 0; i < S::R; ++i) d[i * step] = cmul(v[E::out_reg(i)], cyy);
  } else {
#pragma unroll
    for (int i = 0; i < S::R; ++i)
      dst[mid_index(j + i * S::P, y, ny, cw_log)] = cmul(v[E::out_reg(i)], cyy);
  }
}

// Bytes of one column tile (FPC columns of the intermediate, contiguous), and the bulk copy
// of one into shared memory that completes on `bar` (one thread issues it).
template <int LOGN>
__host__ __device__ constexpr int tile_bytes() { return fpc<LOGN>() * Shape<LOGN>::N * (int)sizeof(float2); }

template <int LOGN>
__device__ __forceinline__ void issue_tile(const float2 *__restrict__ src, float2 *smem, uint64_t *bar) {
  constexpr int TILE_BYTES = tile_bytes<LOGN>();
  constexpr int CHUNK = TILE_BYTES < 16384 ? TILE_BYTES : 16384;
  tc::mbar_arrive_expect_tx(bar, TILE_BYTES);
  const char *s8 = reinterpret_cast<const char *>(src);
#pragma unroll
  for (int off = 0; off < TILE_BYTES; off += CHUNK)
    tc::bulk_load(reinterpret_cast<char *>(smem) + off, s8 + off, CHUNK, bar);
}

// Column work: one tile of FPC (= CW) columns [kx0, kx0 + FPC) of one frame. The tile
// (contiguous, CW n_y FP32 complex values) arrives by bulk asynchronous copy into shared
// memory (thread 0 issues it; `issued()` then runs on every thread); each transform
// (P threads) reads its column, runs in place in the same buffer, and writes the hologram
// planes of `slot` in column-major pixel order p = kx n_y + ky. `landed()` runs on thread 0
// once every thread has read the tile and dropped its lines from L2; `freed()` runs on each
// thread after its last read of the buffer. Returns false (after a barrier) if the copy did
// not complete within the wait budget; `copy_ok` false on thread 0 skips the copy (a failed
// wait before it); `preissued` (the same on every thread) says the copy is already in flight
// on `bar` (issue_tile).
template <int LOGN, typename OutT, bool TAIL_SYNC = true, typename Issued, typename Landed,
          typename Freed = NoHook>
__device__ __forceinline__ bool col_work(const float2 *__restrict__ src, float2 *smem, uint64_t *bar,
                                         uint32_t &phase, int *abort_flag, bool copy_ok, bool preissued,
                                         int kx0, OutT *__restrict__ H, long long npix, long long rows_total,
                                         int slot, uint32_t &maxbits, const float2 *__restrict__ tw,
                                         Issued issued, Landed landed, Freed freed = Freed()) {
  using S = Shape<LOGN>;
  constexpr int FPC = fpc<LOGN>();
  constexpr int CW_LOG = FPC == 16 ? 4 : FPC == 8 ? 3 : FPC == 4 ? 2 : FPC == 2 ? 1 : 0;
  constexpr int TILE_BYTES = tile_bytes<LOGN>();
  using E = Engine<LOGN, (S::P > 32)>;
  const int fft = threadIdx.x / S::P, j = threadIdx.x % S::P;
  float2 *sm = smem + fft * S::RSTRIDE;
  if (threadIdx.x == 0 && !preissued) {
    if (copy_ok) {
      issue_tile<LOGN>(src, smem, bar);
    } else {
      *abort_flag = 1;
      tc::mbar_arrive(bar);  // completes the phase without data so no thread waits it out
    }
  }
  issued();
  const bool got = tc::mbar_wait(bar, phase);
  if (!got) *abort_flag = 1;
  phase ^= 1;
  // the tile is in shared memory: its lines of the intermediate need no write-back (the
  // next writer of this part of the intermediate overwrites it whole, and may start only
  // after `landed()`, which the barrier below orders after every thread's discards). A
  // thread 0 that skips the copy sets the abort flag before its arrival, so the wait orders
  // that write before this read.
  if (got && !*abort_flag)
    for (int off = threadIdx.x * 128; off < TILE_BYTES; off += blockDim.x * 128)
      l2_discard(reinterpret_cast<const char *>(src) + off);
  float2 v[S::R];
  if constexpr (S::P % 16 == 0) {  // y = j + r P keeps the swizzle of j
    const float2 *col = smem + j * FPC + (fft ^ mid_swz(j, CW_LOG));
#pragma unroll
    for (int r = 0; r < S::R; ++r) v[r] = col[r * S::P * FPC];
  } else {
#pragma unroll
    for (int r = 0; r < S::R; ++r) {
      const int y = j + r * S::P;
      v[r] = smem[y * FPC + (fft ^ mid_swz(y, CW_LOG))];
    }
  }
  __syncthreads();  // the tile is consumed; its buffer becomes the exchange regions
  if (*abort_flag) return false;
  if (threadIdx.x == 0 && copy_ok) landed();
  E::run(v, sm, j, tw, freed);
  const int kx = kx0 + fft;
  // largest |component| stored, for the overflow flag: `maxbits` holds a non-negative float's
  // bits, which order as the values do (the values are finite: finite inputs and tables)
  float mx = __uint_as_float(maxbits);
  if constexpr (sizeof(OutT) == 4) {  // FP32 planes: [slot][re|im][p]
    OutT *re = H + (long long)slot * 2 * npix + (long long)kx * S::N;
    OutT *im = re + npix;
#pragma unroll
    for (int i = 0; i < S::R; ++i) {
      const float2 o = v[E::out_reg(i)];
      mx = fmaxf(mx, fmaxf(fabsf(o.x), fabsf(o.y)));
      st_stream(re + j + i * S::P, o.x);
      st_stream(im + j + i * S::P, o.y);
    }
  } else {  // 16-bit planes in 64-pixel blocks: [p / 64][row = 2 slot + c][p % 64]
    const long long pix0 = (long long)kx * S::N;  // a multiple of 64 when n_y >= 64
    OutT *base = H + (2ll * slot << 6);
    const long long bstride = rows_total << 6;
#pragma unroll
    for (int i = 0; i < S::R; ++i) {
      const float2 o = v[E::out_reg(i)];
      const OutT a = to_store<OutT>(o.x), b = to_store<OutT>(o.y);
      mx = fmaxf(mx, fmaxf(fabsf(o.x), fabsf(o.y)));
      OutT *q;
      if constexpr (S::N >= 64) {
        const int e = j + i * S::P;  // < n_y
        q = base + ((pix0 >> 6) + (e >> 6)) * bstride + (e & 63);
      } else {
        const long long pix = pix0 + j + i * S::P;
        q = base + (pix >> 6) * bstride + (pix & 63);
      }
      st_stream(q, a);
      st_stream(q + 64, b);
    }
  }
  maxbits = __float_as_uint(mx);
  if constexpr (TAIL_SYNC) __syncthreads();  // all transforms are done with the buffer before the next copy
  return true;
}

#include "render_tc.cuh"

// Row pass over a chunk of frames: one item = FPC consecutive rows of one frame.
template <int LOGN, bool MEAN>
__global__ void __launch_bounds__(cta_threads<LOGN>(), rows_per_sm<LOGN>())
k_render_rows(const uint16_t *__restrict__ frames, long long frame_stride, int ny, int cw_log,
              const float2 *__restrict__ cx, const float2 *__restrict__ cy,
              const float2 *__restrict__ tw, float2 *__restrict__ mid, int n_items,
              const uint16_t *__restrict__ mean, int mean_every, int mean_first) {
  using C = RowCfg<LOGN>;
  extern __shared__ float2 smem[];
  const int groups = ny / C::FPC;
  const long long npix = (long long)Shape<LOGN>::N * ny;
  uint4 pf[C::CPT];
  auto frame_of = [&](int item) { return frames + (long long)(item / groups) * frame_stride; };
  if (blockIdx.x < n_items) row_prefetch<LOGN>(pf, frame_of(blockIdx.x), (blockIdx.x % groups) * C::FPC);
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int f = item / groups, y0 = (item % groups) * C::FPC;
    const int nxt = item + (int)gridDim.x;
    row_work<LOGN>(pf, smem, y0, ny, cw_log, cx, cy, tw, mid + (long long)f * npix,
                   MEAN ? mean + (long long)((mean_first + f) / mean_every) * npix : nullptr, [&]() {
      if (nxt < n_items) row_prefetch<LOGN>(pf, frame_of(nxt), (nxt % groups) * C::FPC);
    });
  }
}

// Column pass over a chunk of frames: one item = one tile of FPC columns of one frame,
// written to hologram slot slot0 + f. A bulk copy that does not complete within the wait
// budget raises DH_FLAG_WAIT_TIMEOUT and the CTA stops.
template <int LOGN, typename OutT>
__global__ void __launch_bounds__(cta_threads<LOGN>(), cols_per_sm<LOGN>())
k_render_cols(const float2 *__restrict__ mid, int nx, const float2 *__restrict__ tw,
              OutT *__restrict__ H, long long npix, long long rows_total, int slot0, int n_items,
              uint32_t *__restrict__ status) {
  constexpr int FPC = fpc<LOGN>();
  extern __shared__ float2 smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  const int groups = nx / FPC;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
    abort_flag = 0;
  }
  __syncthreads();
  uint32_t phase = 0;
  uint32_t maxbits = 0;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int f = item / groups, t = item % groups;
    const float2 *src = mid + (long long)f * npix + (long long)t * FPC * Shape<LOGN>::N;
    if (!col_work<LOGN, OutT>(src, smem, &bar, phase, &abort_flag, true, false, t * FPC, H, npix, rows_total,
                              slot0 + f, maxbits, tw, []() {}, []() {}))
      break;
  }
  if (abort_flag && threadIdx.x == 0) {
    atomicOr(status, DH_FLAG_WAIT_TIMEOUT);
    tc::mbar_wait(&bar, phase ^ 1);  // let a late copy land before the CTA exits
  }
  if (maxbits >= overflow_bits<OutT>()) atomicOr(status, DH_FLAG_STORE_OVERFLOW);
}

// ---------------------------------------------------------------- fused, persistent render
// One launch renders every frame of a call (square frames whose row and column items both
// use 256 threads). Work items are taken from a global ticket counter in a fixed order:
// phase k holds the row items of frame k interleaved with the column items of frame k - lag
// (0 < lag < ring), so a frame's rows have had lag phases to finish before its columns run.
// The row-pass output goes to a ring of `ring` frame-sized intermediates, small enough to
// stay in L2, instead of a chunk of frames:
//   - a column item of frame f waits until the row items of frame f are complete;
//   - a row item of frame f waits until the column items of frame f - ring have copied
//     their tiles out of the ring slot it overwrites.
// Every item waits only on items with lower tickets, and a ticket is only ever held by a
// running CTA, so the waits cannot deadlock whatever the residency. Waits are bounded: on
// expiry the CTA raises DH_FLAG_WAIT_TIMEOUT and stops (CTAs waiting on it then time out
// too). Ring writes (generic proxy) are fenced against the column items' bulk copies (async
// proxy) on both sides of the release/acquire pair that publishes them.
constexpr int kMaxRing = 64;  // ring slots the counter array (1 + 2 kMaxRing words) serves

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// shared-memory counter: the release orders this thread's earlier accesses before the add,
// the acquire orders those of the adds read before this one ahead of what follows
__device__ __forceinline__ int atom_add_acq_rel_shared(int *p, int v) {
  int old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;"
               : "=r"(old) : "r"(tc::smem_u32(p)), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ int ld_acquire_cta_shared(const int *p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(tc::smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_cta_shared(int *p, int v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(tc::smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ bool wait_geq(const unsigned *p, unsigned target,
                                         long long budget = tc::kWaitBudget) {
  if (ld_acquire(p) >= target) return true;
  const long long t0 = clock64();
  while (ld_acquire(p) < target) {
    if (clock64() - t0 > budget) return false;
    __nanosleep(128);
  }
  return true;
}

template <int LOGN, typename OutT, bool MEAN>
__global__ void __launch_bounds__(kCtaThreads, rows_per_sm<LOGN>())
k_render_fused(const uint16_t *__restrict__ frames, long long frame_stride, int n_frames, int cw_log,
               const float2 *__restrict__ cx, const float2 *__restrict__ cy, const float2 *__restrict__ tw,
               int tw_len,
               float2 *__restrict__ mid, int ring, int lag, OutT *__restrict__ H, long long rows_total,
               int slot0, unsigned *__restrict__ sync, uint32_t *__restrict__ status, int stall_cycles,
               const uint16_t *__restrict__ mean, int mean_every, int mean_first) {
  using S = Shape<LOGN>;
  using RC = RowCfg<LOGN>;
  constexpr int FPC = fpc<LOGN>();  // rows per row item = columns per column item
  constexpr int N = S::N;
  constexpr int NI = N / FPC;       // row items = column items per frame
  constexpr long long NPIX = (long long)N * N;
  static_assert(RC::NT == kCtaThreads, "fused render needs full-size items on both axes");
  // one transform a warp (n = 1024): a row item's warps stage their rows each on their own,
  // with no CTA barrier inside the item; the last warp to finish records the item's ring slot
  // in `pend_rs`, and thread 0 releases its FPC rows (rows_done counts rows) right after the
  // next item-start barrier, so that the release's wait for the ring writes overlaps the other
  // warps' work. Measured for 2048 frames at 1024^2: one release per warp 9.72 ms, one per
  // item by its last warp 9.47 ms, deferred to the next item 9.38 ms.
  constexpr bool PW = S::P == 32;
  constexpr unsigned ROWS_PER_FRAME = PW ? (unsigned)N : (unsigned)NI;
  extern __shared__ float2 smem[];
  // the CTA lives for the whole launch: its twiddle and chirp tables are copied into shared
  // memory once, after the exchange / tile buffer
  constexpr int XCHG = (FPC * S::RSTRIDE > FPC * S::N ? FPC * S::RSTRIDE : FPC * S::N);
  float2 *s_tw = smem + XCHG, *s_cx = s_tw + tw_len, *s_cy = s_cx + N;
  for (int e = threadIdx.x; e < tw_len; e += blockDim.x) s_tw[e] = tw[e];
  for (int e = threadIdx.x; e < N; e += blockDim.x) { s_cx[e] = cx[e]; s_cy[e] = cy[e]; }
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  __shared__ int tk[2];
  // The next item's tile copy, when the next item is a column item, is issued during the
  // current item by the last warp to make its final read of the buffer (n_freed counts them),
  // so it lands while the current item finishes; `preissued` is the ticket it was issued for.
  __shared__ int n_freed, preissued;
  __shared__ int n_rows_fin;  // warps of the current row item that have written their row
  __shared__ int pend_rs;     // 1 + the ring slot of a finished row item not yet released, or 0
  unsigned *tickets = sync, *rows_done = sync + 1, *cols_done = sync + 1 + ring;
  const int total = (n_frames + lag) * 2 * NI;
  // thread 0 takes tickets two items ahead: the one it takes at an item's start is published
  // at the next item's start, so the atomic's round trip overlaps a whole item. Every ticket a
  // CTA holds is larger than the one it runs and the items only wait on smaller tickets, so
  // the smallest unfinished item can always proceed.
  int pending = 0;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
    abort_flag = 0;
    n_freed = 0;
    n_rows_fin = 0;
    pend_rs = 0;
    preissued = -1;
    tk[0] = (int)atomicAdd(tickets, 1u);
    pending = (int)atomicAdd(tickets, 1u);
    // stall test: a bounded wait on the word after the counters, which nothing sets, runs
    // out in every CTA before any item starts (so no CTA waits on an item left undone)
    if (stall_cycles > 0 && !wait_geq(sync + 1 + 2 * kMaxRing, 1u, stall_cycles)) abort_flag = 1;
  }
  __syncthreads();
  const bool stalled = abort_flag;  // read after the barrier: the same in every thread
  // ticket i: phase k = i / (2 NI); even positions are row items of frame k, odd ones column
  // items of frame k - lag; the item index is the position / 2
  auto is_row = [](int i) { return ((i % (2 * NI)) & 1) == 0; };
  auto frame_of = [&](int i) { return i / (2 * NI) - (is_row(i) ? 0 : lag); };
  auto item_of = [](int i) { return (i % (2 * NI)) >> 1; };
  auto valid = [&](int i) { const int f = frame_of(i); return i < total && f >= 0 && f < n_frames; };
  int cur = tk[0];
  uint4 pf[RC::CPT];
  if (valid(cur) && is_row(cur))
    row_prefetch<LOGN, PW>(pf, frames + (long long)frame_of(cur) * frame_stride, item_of(cur) * FPC);
  uint32_t phase = 0;
  uint32_t maxbits = 0;
  int b = 1;
  bool pre_unwaited = false;  // a copy issued early for `cur` that no one has waited on
  while (!stalled && cur < total) {
    // one barrier per item start: thread 0 publishes the next ticket, takes the one after it
    // and, for a row item, waits for its ring slot; the barrier also ends the previous item's
    // use of shared memory
    if (threadIdx.x == 0) {
      tk[b] = pending;
      pending = (int)atomicAdd(tickets, 1u);
      if (valid(cur) && is_row(cur)) {
        const int f = frame_of(cur);
        // while it waits, thread 0 also releases the previous row item's rows as soon as its
        // last warp has recorded them: with a ring of few frames the awaited column items may
        // need exactly those rows
        const unsigned *slot = cols_done + f % ring;
        const unsigned target = (unsigned)(f / ring) * NI;
        if (ld_acquire(slot) < target) {
          const long long t0 = clock64();
          while (ld_acquire(slot) < target) {
            const int pr = ld_acquire_cta_shared(&pend_rs);
            if (pr) {
              pend_rs = 0;
              red_release_add(rows_done + pr - 1, (unsigned)FPC);
            }
            if (clock64() - t0 > tc::kWaitBudget) { abort_flag = 1; break; }
            __nanosleep(128);
          }
        }
      }
    }
    __syncthreads();
    // the previous item's rows, if it was a row item (its last warp recorded the slot before
    // the barrier, after counting every warp's ring writes)
    if (threadIdx.x == 0 && pend_rs) {
      red_release_add(rows_done + pend_rs - 1, (unsigned)FPC);
      pend_rs = 0;
    }
    const int nxt = tk[b];
    b ^= 1;
    const bool pre = preissued == cur;  // read before any write of this item (see freed)
    pre_unwaited = pre;
    if (abort_flag) break;
    // the next item's uint16 rows are loaded while this item runs (or right away when this
    // ticket names no item)
    auto prefetch_next = [&]() {
      if (valid(nxt) && is_row(nxt))
        row_prefetch<LOGN, PW>(pf, frames + (long long)frame_of(nxt) * frame_stride, item_of(nxt) * FPC);
    };
    // every warp of the CTA calls this once, after its last read of the buffer; the last one
    // issues the next column item's tile copy if that item's rows are done. Each warp has read
    // `preissued` for this item before its call, and the counter's acquire-release orders
    // all those reads, and all the warps' buffer reads, before the copy and the new value.
    const bool early = valid(nxt) && !is_row(nxt);
    auto freed = [&]() {
      if (!early) return;
      __syncwarp();
      if ((threadIdx.x & 31) == 0 && atom_add_acq_rel_shared(&n_freed, 1) == kCtaThreads / 32 - 1) {
        n_freed = 0;  // the next item's adds follow the next item-start barrier
        // one look, no wait: the current item may be a row item of the same frame, whose rows
        // are released only after it ends; if they are not all done the column item issues
        // its own copy
        const int fn = frame_of(nxt), rn = fn % ring;
        if (ld_acquire(rows_done + rn) >= (unsigned)(fn / ring + 1) * ROWS_PER_FRAME) {
          fence_proxy_async_global();  // the rows' ring writes, for the copy
          fence_proxy_async_shared();  // the buffer's reads, before the copy's writes
          issue_tile<LOGN>(mid + (long long)rn * NPIX + (long long)item_of(nxt) * FPC * N, smem, &bar);
          preissued = nxt;
        }
      }
    };
    if (!valid(cur)) {
      prefetch_next();
    } else {
      const int f = frame_of(cur), i = item_of(cur), rs = f % ring;
      float2 *ring_f = mid + (long long)rs * NPIX;
      if (is_row(cur)) {
        row_work<LOGN, false, PW>(pf, smem, i * FPC, N, cw_log, s_cx, s_cy, s_tw, ring_f,
                                  MEAN ? mean + (long long)((mean_first + f) / mean_every) * NPIX : nullptr,
                                  prefetch_next,
                                  freed);
        fence_proxy_async_global();  // this thread's ring writes, for later bulk copies
        if constexpr (PW) {
          __syncwarp();
          // the shared counter's acquire-release orders every warp's ring writes (and proxy
          // fences) before the last warp's record, whose release store thread 0 acquires (in its
          // ring-slot wait) or reads after the next item-start barrier; the next item's
          // increments follow that barrier, after the reset
          if ((threadIdx.x & 31) == 0 && atom_add_acq_rel_shared(&n_rows_fin, 1) == kCtaThreads / 32 - 1) {
            n_rows_fin = 0;
            st_release_cta_shared(&pend_rs, rs + 1);
          }
        } else {
          __syncthreads();
          if (threadIdx.x == 0) red_release_add(rows_done + rs, 1u);  // after the CTA's writes
        }
      } else {
        bool ok = true;
        if (threadIdx.x == 0 && !pre) {
          ok = wait_geq(rows_done + rs, (unsigned)(f / ring + 1) * ROWS_PER_FRAME);
          if (ok) fence_proxy_async_global();
        }
        pre_unwaited = false;
        const float2 *src = ring_f + (long long)i * FPC * N;
        if (!col_work<LOGN, OutT, false>(src, smem, &bar, phase, &abort_flag, ok, pre, i * FPC, H, NPIX,
                                         rows_total, slot0 + f, maxbits, s_tw, prefetch_next,
                                         [&]() { red_release_add(cols_done + rs, 1u); }, freed))
          break;
      }
    }
    cur = nxt;
  }
  __syncthreads();  // the last item's rows, if still unreleased
  if (threadIdx.x == 0 && pend_rs) red_release_add(rows_done + pend_rs - 1, (unsigned)FPC);
  if (abort_flag && threadIdx.x == 0) {
    atomicOr(status, DH_FLAG_WAIT_TIMEOUT);
    // let a late copy land before the CTA exits: the last one waited on, and one issued early
    // for an item the CTA stopped before
    tc::mbar_wait(&bar, phase ^ 1);
    if (pre_unwaited) tc::mbar_wait(&bar, phase);
  }
  if (maxbits >= overflow_bits<OutT>()) atomicOr(status, DH_FLAG_STORE_OVERFLOW);
}

// Inspection: one slot's hologram (column-major pixels p = kx n_y + ky; FP32 as planes,
// 16-bit in 64-pixel blocks) to interleaved FP32 in row-major order.
template <typename T>
__global__ void k_hologram_to_f32(const T *__restrict__ H, int nx, int ny, long long rows_total, int slot,
                                  float *__restrict__ out) {
  const long long npix = (long long)nx * ny;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
       p += (long long)gridDim.x * blockDim.x) {
    float r, i;
    if constexpr (sizeof(T) == 4) {
      const T *re = H + 2ll * slot * npix;
      r = re[p];
      i = re[p + npix];
    } else {
      const T *blk = H + (p >> 6) * (rows_total << 6) + (p & 63);
      const long long row = 2ll * slot;
      if constexpr (std::is_same<T, __half>::value) {
        r = __half2float(blk[row << 6]); i = __half2float(blk[(row + 1) << 6]);
      } else {
        r = __bfloat162float(blk[row << 6]); i = __bfloat162float(blk[(row + 1) << 6]);
      }
    }
    const long long kx = p / ny, ky = p % ny;
    out[2 * (ky * nx + kx)] = r;
    out[2 * (ky * nx + kx) + 1] = i;
  }
}

// ----------------------------------------------------------------- host side
// Every FFT spec with instances: the default radix of each length, and the alternatives.
#define DH_FFT_SPECS(X)                                                                   \
  X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(9 | (4 << 4)) X(10 | (4 << 4)) X(11 | (4 << 4)) \
  X(12 | (5 << 4))

// log2 of the column-tile width of the intermediate (the column pass's FFTs per CTA)
int col_tile_log(int spec) {
  int f = 0;
  switch (spec) {
#define DH_CASE(S) case S: f = fpc<S>(); break;
    DH_FFT_SPECS(DH_CASE)
#undef DH_CASE
  }
  int l = 0;
  while ((1 << l) < f) ++l;
  return l;
}

template <int LOGN>
dh_status launch_rows_t(const uint16_t *frames, long long fstride, int ny, const Plan &p,
                        float2 *mid, int nf, const RenderTarget &to, cudaStream_t s) {
  const int cw_log = col_tile_log(col_spec(p));
  using S = Shape<LOGN>;
  constexpr int FPC = fpc<LOGN>();
  const int threads = FPC * S::P;
  // exchange regions (also the uint16 rows and the staging tile)
  const size_t smem = (size_t)FPC * S::RSTRIDE * sizeof(float2);
  // the mean-subtracting variant (mean-residual storage) is a separate instance, so that the
  // plain one keeps its registers
  auto kern = to.mean ? k_render_rows<LOGN, true> : k_render_rows<LOGN, false>;
  static bool attr_set[2] = {false, false};
  if (!attr_set[to.mean ? 1 : 0]) {
    DH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set[to.mean ? 1 : 0] = true;
  }
  int per_sm = 0;
  DH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  const int items = nf * (ny / FPC);
  int grid = per_sm * p.num_sms;
  if (grid < 1) grid = 1;
  if (grid > items) grid = items;
  ProfScope ps(const_cast<Plan &>(p), K_RENDER_ROWS, s);
  kern<<<grid, threads, smem, s>>>(frames, fstride, ny, cw_log, p.d_cx, p.d_cy, p.d_twx, mid, items, to.mean,
                                    to.mean_every, to.mean_first);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

template <int LOGN, typename OutT>
dh_status launch_cols_t(const Plan &p, const float2 *mid, int nf, int slot0, const RenderTarget &to,
                        cudaStream_t s) {
  using S = Shape<LOGN>;
  constexpr int FPC = fpc<LOGN>();
  const int threads = FPC * S::P;
  // one tile of FPC columns; its buffer is reused in place as the exchange regions
  const size_t tile = (size_t)FPC * S::N * sizeof(float2);
  const size_t xchg = (size_t)FPC * S::RSTRIDE * sizeof(float2);
  const size_t smem = tile > xchg ? tile : xchg;
  auto kern = k_render_cols<LOGN, OutT>;
  static bool attr_set = false;
  if (!attr_set) {
    DH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  int per_sm = 0;
  DH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  const int items = nf * (p.nx / FPC);
  int grid = per_sm * p.num_sms;
  if (grid < 1) grid = 1;
  if (grid > items) grid = items;
  ProfScope ps(const_cast<Plan &>(p), K_RENDER_COLS, s);
  kern<<<grid, threads, smem, s>>>(mid, p.nx, p.d_twy, static_cast<OutT *>(to.H), p.npix, to.rows_total, slot0,
                                    items, p.d_status);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

dh_status launch_rows(const Plan &p, const uint16_t *frames, long long fstride, float2 *mid,
                      int nf, const RenderTarget &to, cudaStream_t s) {
  switch (row_spec(p)) {
#define DH_CASE(S) case S: return launch_rows_t<S>(frames, fstride, p.ny, p, mid, nf, to, s);
    DH_FFT_SPECS(DH_CASE)
#undef DH_CASE
  }
  return DH_ERR_UNSUPPORTED_SIZE;
}

template <typename OutT>
dh_status launch_cols_typed(const Plan &p, const float2 *mid, int nf, int slot0, const RenderTarget &to,
                            cudaStream_t s) {
  switch (col_spec(p)) {
#define DH_CASE(S) case S: return launch_cols_t<S, OutT>(p, mid, nf, slot0, to, s);
    DH_FFT_SPECS(DH_CASE)
#undef DH_CASE
  }
  return DH_ERR_UNSUPPORTED_SIZE;
}

int cta_threads_of(int logn);

// Ring and lag of the persistent schedule, in frames. A column item should find its frame's
// rows done and a row item its ring slot free, so both distances should span about 1.5
// rounds of the grid's CTAs, counted in work items (N / FPC per frame and pass): lag =
// ceil(1.5 grid / items per frame), ring = 2 lag, within the plan's intermediate and the
// 64 slots of the counters. The plan's choices override both. ring 0: not applicable.
int fused_ring(const Plan &p, int grid, int items_per_frame) {
  if (p.render_mode != 0 || p.nx != p.ny || p.lognx < 8 || p.lognx > 12) return 0;
  if (cta_threads_of(row_spec(p)) != kCtaThreads) return 0;
  // untuned plans use it where it measured faster than chunks (512^2, 1024^2); an explicit
  // ring or lag (the autotuner's pick) applies it at any square size from 256^2
  if (p.render_ring == 0 && p.render_lag == 0 && (p.lognx < 9 || p.lognx > 10)) return 0;
  long long r = p.render_ring;
  if (r <= 0) r = 2ll * ((3ll * grid + 2ll * items_per_frame - 1) / (2ll * items_per_frame));
  if (r < 2) r = 2;
  if (r > kMaxRing) r = kMaxRing;
  if (r > p.mid_frames) r = p.mid_frames;
  return r >= 2 ? (int)r : 0;
}
int fused_lag(const Plan &p, int ring) {
  int l = p.render_lag > 0 ? p.render_lag : ring / 2;
  if (l > ring - 1) l = ring - 1;
  return l < 1 ? 1 : l;
}

template <int LOGN, typename OutT>
dh_status launch_fused_t(Plan &p, const uint16_t *frames, long long fstride, int nf, int slot0,
                         const RenderTarget &to, cudaStream_t s) {
  if constexpr (cta_threads<LOGN>() != kCtaThreads) {
    return DH_ERR_UNSUPPORTED_SIZE;  // an item of this length needs more threads
  } else {
  using S = Shape<LOGN>;
  constexpr int FPC = fpc<LOGN>();
  const size_t row_smem = (size_t)FPC * S::RSTRIDE * sizeof(float2);
  const size_t tile = (size_t)FPC * S::N * sizeof(float2);
  const int tw_len = twiddle_len(LOGN);
  // exchange / tile buffer, then the twiddle and the two chirp tables
  const size_t smem = (row_smem > tile ? row_smem : tile) + (size_t)(tw_len + 2 * S::N) * sizeof(float2);
  // (mean-residual storage is 16-bit only: FP32 outputs have no mean-subtracting instance)
  auto kern = k_render_fused<LOGN, OutT, false>;
  if constexpr (sizeof(OutT) == 2) {
    if (to.mean) kern = k_render_fused<LOGN, OutT, true>;
  } else {
    if (to.mean) return DH_ERR_STATE;
  }
  static bool attr_set[2] = {false, false};
  if (!attr_set[to.mean ? 1 : 0]) {
    DH_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set[to.mean ? 1 : 0] = true;
  }
  int per_sm = 0;
  DH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCtaThreads, smem));
  if (per_sm < 1) per_sm = 1;
  const int items = 2 * nf * (S::N / FPC);
  int grid = per_sm * p.num_sms;
  if (grid > items) grid = items;
  const int ring = fused_ring(p, grid, S::N / FPC);
  const int lag = fused_lag(p, ring);
  DH_CUDA_TRY(cudaMemsetAsync(p.d_sync, 0, sizeof(unsigned) * (1 + 2 * ring), s));
  ProfScope ps(p, K_RENDER_FUSED, s);
  kern<<<grid, kCtaThreads, smem, s>>>(frames, fstride, nf, col_tile_log(LOGN), p.d_cx, p.d_cy, p.d_twx, tw_len,
                                      p.d_mid,
                               ring, lag, static_cast<OutT *>(to.H), to.rows_total, slot0, p.d_sync,
                               p.d_status, p.test_stall, to.mean, to.mean_every, to.mean_first);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
  }
}

int cta_threads_of(int spec) {
  switch (spec) {
#define DH_CASE(S) case S: return cta_threads<S>();
    DH_FFT_SPECS(DH_CASE)
#undef DH_CASE
  }
  return 0;
}

template <typename OutT>
dh_status launch_fused_typed(Plan &p, const uint16_t *frames, long long fstride, int nf, int slot0,
                             const RenderTarget &to, cudaStream_t s) {
  switch (row_spec(p)) {  // square frames: the same spec on both axes
    case 8: return launch_fused_t<8, OutT>(p, frames, fstride, nf, slot0, to, s);
    case 9: return launch_fused_t<9, OutT>(p, frames, fstride, nf, slot0, to, s);
    case 10: return launch_fused_t<10, OutT>(p, frames, fstride, nf, slot0, to, s);
    case 11: return launch_fused_t<11, OutT>(p, frames, fstride, nf, slot0, to, s);
    case 12: return launch_fused_t<12, OutT>(p, frames, fstride, nf, slot0, to, s);
    case 9 | (4 << 4): return launch_fused_t<9 | (4 << 4), OutT>(p, frames, fstride, nf, slot0, to, s);
    case 10 | (4 << 4): return launch_fused_t<10 | (4 << 4), OutT>(p, frames, fstride, nf, slot0, to, s);
    case 11 | (4 << 4): return launch_fused_t<11 | (4 << 4), OutT>(p, frames, fstride, nf, slot0, to, s);
    case 12 | (5 << 4): return launch_fused_t<12 | (5 << 4), OutT>(p, frames, fstride, nf, slot0, to, s);
  }
  return DH_ERR_UNSUPPORTED_SIZE;
}

}  // namespace

int render_items_per_frame(const Plan &p) { return p.nx >> col_tile_log(row_spec(p)); }

int fft_spec_for(int logn, int radix) {
  if (radix == 0) return logn;
  int lr = 0;
  while ((1 << lr) < radix) ++lr;
  if (lr == log_radix(logn)) return logn;
  return lr == alt_logr(logn) ? (logn | (lr << 4)) : logn;
}
int row_spec(const Plan &p) { return fft_spec_for(p.lognx, p.fft_radix); }
int col_spec(const Plan &p) { return fft_spec_for(p.logny, p.fft_radix); }
bool fft_radix_available(int logn, int radix) {
  return radix == 0 || fft_spec_for(logn, radix) != logn || (1 << log_radix(logn)) == radix;
}

int twiddle_len(int spec) {
  const int logn = sp_logn(spec), logr = sp_logr(spec), R = 1 << logr, L = logn / logr;
  const int logr2 = logn - L * logr, R2 = 1 << logr2;
  int len = 0;
  for (int p = 1; p < L; ++p) len += (R - 1) * (1 << (p * logr));
  if (R2 > 1) len += (R2 - 1) * (1 << (L * logr));
  return len > 0 ? len : 1;
}

// Inter-pass twiddles w_M^e = exp(+2 pi i e / M), the exponent reduced exactly in integers
// before the angle is formed in FP64.
void build_twiddles(int spec, float2 *out) {
  const int logn = sp_logn(spec), logr = sp_logr(spec), R = 1 << logr, L = logn / logr;
  const int logr2 = logn - L * logr, R2 = 1 << logr2, N = 1 << logn;
  const double two_pi = 6.283185307179586476925286766559;
  auto w = [&](long long e, long long M) {
    const double ang = two_pi * (double)(e % M) / (double)M;
    return make_float2((float)cos(ang), (float)sin(ang));
  };
  int off = 0;
  for (int p = 1; p < L; ++p) {
    const int Ns = 1 << (p * logr);
    for (int r = 1; r < R; ++r)
      for (int m = 0; m < Ns; ++m) out[off + (r - 1) * Ns + m] = w((long long)m * r, (long long)Ns * R);
    off += (R - 1) * Ns;
  }
  if (R2 > 1) {
    const int Ns = 1 << (L * logr);
    for (int r = 1; r < R2; ++r)
      for (int m = 0; m < Ns; ++m) out[off + (r - 1) * Ns + m] = w((long long)m * r, N);
  }
  if (off == 0 && R2 == 1) out[0] = make_float2(1.f, 0.f);
}

namespace {
template <typename OutT>
dh_status launch_tc_chunks_t(Plan &p, const uint16_t *frames, long long fstride, int n_frames, int slot0,
                             cudaStream_t s) {
  auto kr = k_render_rows_tc;
  auto kc = k_render_cols_tc<OutT>;
  static bool attr_set = false;
  if (!attr_set) {
    DH_CUDA_TRY(cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, tcr::SMEM_BYTES));
    DH_CUDA_TRY(cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, tcr::SMEM_BYTES));
    attr_set = true;
  }
  const uint8_t *tcg = static_cast<const uint8_t *>(p.d_tc);
  for (int f0 = 0; f0 < n_frames; f0 += p.mid_frames) {
    const int nf = (n_frames - f0) < p.mid_frames ? (n_frames - f0) : p.mid_frames;
    const int items = nf * tcr::ITEMS_PER_FRAME;  // warpgroup items per pass
    int grid = 2 * p.num_sms;
    if (grid * tcr::WGS > items) grid = (items + tcr::WGS - 1) / tcr::WGS;
    {
      ProfScope ps(p, K_RENDER_ROWS_TC, s);
      kr<<<grid, tcr::THREADS, tcr::SMEM_BYTES, s>>>(frames + (long long)f0 * fstride, fstride, tcg, p.d_cx,
                                                     p.d_cy, p.d_mid, items, p.d_status);
      DH_CUDA_TRY(cudaGetLastError());
    }
    {
      ProfScope ps(p, K_RENDER_COLS_TC, s);
      kc<<<grid, tcr::THREADS, tcr::SMEM_BYTES, s>>>(p.d_mid, tcg, p.d_cx, static_cast<OutT *>(p.d_H),
                                                     2ll * p.max_frames, slot0 + f0, items, p.d_status);
      DH_CUDA_TRY(cudaGetLastError());
    }
  }
  return DH_OK;
}
}  // namespace

bool tc_render_applies(const Plan &p) {
  return p.render_fft == 2 && p.nx == tcr::N && p.ny == tcr::N && p.d_tc != nullptr;
}

// Tables of the tensor-core render (1024-point axes): the real embedding [[Wr, Wi], [-Wi, Wr]]
// of the 32-point DFT W[a][b] = exp(+2 pi i a b / 32) as FP16 hi then lo ([n][k] rows of 64),
// then the twiddles w^(a b) / 4 (w = exp(+2 pi i / 1024)) in pairs of consecutive a per lane b,
// [a / 2][b] (wx_a, wx_a+1, wy_a, wy_a+1), then (-wy_a, -wy_a+1). Angles are reduced exactly
// in integers and formed in FP64.
size_t tc_tables_bytes() { return tcr::GLOB_BYTES; }
void build_tc_tables(void *out) {
  const double two_pi = 6.283185307179586476925286766559;
  char *base = static_cast<char *>(out);
  __half *w = reinterpret_cast<__half *>(base + tcr::GLOB_W);
  for (int n = 0; n < 64; ++n)
    for (int k = 0; k < 64; ++k) {
      const int a = n & 31, b = k & 31;
      const double ang = two_pi * (double)((a * b) % 32) / 32.0;
      const double c = cos(ang), sn = sin(ang);
      const double v = n < 32 ? (k < 32 ? c : -sn) : (k < 32 ? sn : c);
      const __half hi = __float2half_rn((float)v);
      const __half lo = __float2half_rn((float)(v - (double)__half2float(hi)));
      w[n * 64 + k] = hi;
      w[64 * 64 + n * 64 + k] = lo;
    }
  auto tw = [&](int a, int b, bool sine) {
    const double ang = two_pi * (double)((a * b) % tcr::N) / (double)tcr::N;
    return (float)(0.25 * (sine ? sin(ang) : cos(ang)));
  };
  float4 *twp = reinterpret_cast<float4 *>(base + tcr::GLOB_TWP);
  float2 *twn = reinterpret_cast<float2 *>(base + tcr::GLOB_TWN);
  for (int pr = 0; pr < 16; ++pr)
    for (int b = 0; b < 32; ++b) {
      const int a = 2 * pr;
      twp[pr * 32 + b] = make_float4(tw(a, b, false), tw(a + 1, b, false), tw(a, b, true), tw(a + 1, b, true));
      twn[pr * 32 + b] = make_float2(-tw(a, b, true), -tw(a + 1, b, true));
    }
}

dh_status launch_render(Plan &p, const uint16_t *frames, long long frame_stride, int n_frames,
                        int slot0, cudaStream_t s) {
  return launch_render_to(p, frames, frame_stride, n_frames, slot0,
                          RenderTarget{p.d_H, p.prec, 2ll * p.max_frames, nullptr, 1}, s);
}

dh_status launch_render_to(Plan &p, const uint16_t *frames, long long frame_stride, int n_frames,
                           int slot0, const RenderTarget &to, cudaStream_t s) {
  // 1024^2 frames with the tensor-core DFT stages (into the plan's own store, no mean)
  if (tc_render_applies(p) && to.H == p.d_H && to.mean == nullptr) {
    switch (p.prec) {
      case DH_PREC_FP32: return launch_tc_chunks_t<float>(p, frames, frame_stride, n_frames, slot0, s);
      case DH_PREC_FP16: return launch_tc_chunks_t<__half>(p, frames, frame_stride, n_frames, slot0, s);
      case DH_PREC_BF16: return launch_tc_chunks_t<__nv_bfloat16>(p, frames, frame_stride, n_frames, slot0, s);
    }
  }
  // square frames from 256^2: every frame of the call in one persistent launch
  if (fused_ring(p, 1, 1)) {
    switch (to.prec) {
      case DH_PREC_FP32: return launch_fused_typed<float>(p, frames, frame_stride, n_frames, slot0, to, s);
      case DH_PREC_FP16: return launch_fused_typed<__half>(p, frames, frame_stride, n_frames, slot0, to, s);
      case DH_PREC_BF16: return launch_fused_typed<__nv_bfloat16>(p, frames, frame_stride, n_frames, slot0, to, s);
    }
  }
  // Chunks of mid_frames frames: the row pass fills the L2-sized intermediate, the column
  // pass drains it, back to back on the caller's stream. (Running the column pass of one
  // chunk beside the row pass of the next was measured slower: both passes are issue-bound
  // and the doubled intermediate no longer stays in L2.)
  for (int f0 = 0; f0 < n_frames; f0 += p.mid_frames) {
    const int nf = (n_frames - f0) < p.mid_frames ? (n_frames - f0) : p.mid_frames;
    RenderTarget chunk = to;  // the chunk's frames start f0 frames into the call
    chunk.mean_first = to.mean_first + f0;
    dh_status st = launch_rows(p, frames + (long long)f0 * frame_stride, frame_stride, p.d_mid, nf, chunk, s);
    if (st != DH_OK) return st;
    switch (to.prec) {
      case DH_PREC_FP32: st = launch_cols_typed<float>(p, p.d_mid, nf, slot0 + f0, chunk, s); break;
      case DH_PREC_FP16: st = launch_cols_typed<__half>(p, p.d_mid, nf, slot0 + f0, chunk, s); break;
      case DH_PREC_BF16: st = launch_cols_typed<__nv_bfloat16>(p, p.d_mid, nf, slot0 + f0, chunk, s); break;
    }
    if (st != DH_OK) return st;
  }
  return DH_OK;
}

dh_status launch_hologram_to_f32(Plan &p, int slot, float *out, cudaStream_t s) {
  const int grid = p.num_sms * 4;
  const long long rows = 2ll * p.max_frames;
  switch (p.prec) {
    case DH_PREC_FP32:
      k_hologram_to_f32<float><<<grid, 256, 0, s>>>(static_cast<float *>(p.d_H), p.nx, p.ny, rows, slot, out);
      break;
    case DH_PREC_FP16:
      k_hologram_to_f32<__half><<<grid, 256, 0, s>>>(static_cast<__half *>(p.d_H), p.nx, p.ny, rows, slot, out);
      break;
    case DH_PREC_BF16:
      k_hologram_to_f32<__nv_bfloat16>
          <<<grid, 256, 0, s>>>(static_cast<__nv_bfloat16 *>(p.d_H), p.nx, p.ny, rows, slot, out);
      break;
  }
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

}  // namespace dh
