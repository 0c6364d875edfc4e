// Eqs. 8-9: temporal demodulation by the unitary DFT, the paper's Fourier alternative to
// the data-derived basis of Eq. 6. Windows one frame apart use a sliding recurrence (below);
// other strides the projection. W has entries w_{t,k} = exp(-2 pi i t k / n_t) / sqrt(n_t)
// (t, k counted from 0); its columns k0..k1 (the frequency filter I_f) form a fixed
// projection operand, built once per call in the layout the eigensolver writes for Eq. 6,
// and every window is projected onto it by the same kernels, |.|^2 summed in the epilogue:
//   M[p] = sum_{k=k0..k1} |sum_t H[t][p] w_{t,k}|^2.
#include <type_traits>

#include "dh_internal.cuh"

namespace dh {
namespace {

template <typename T16> __device__ __forceinline__ T16 to16(float x);
template <> __device__ __forceinline__ __half to16<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
template <typename T16> __device__ __forceinline__ float from16(T16 x);
template <> __device__ __forceinline__ float from16<__half>(__half x) { return __half2float(x); }
template <> __device__ __forceinline__ float from16<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}

// Real embedding of W's kept columns, rows r = 2t + c of X = [Re H_0; Im H_0; ...]:
//   j < nS (Re of bin k0 + j):        B[j][2t] = Re w_tk, B[j][2t+1] = -Im w_tk
//   nS <= j < 2nS (Im of bin k0+j-nS): B[j][2t] = Im w_tk, B[j][2t+1] =  Re w_tk
// rows 2nS..Npad-1 are zero; 16-bit storage keeps a hi part and the rounding residue lo.
__global__ void k_fourier_operand(int T, int k0, int k1, int Npad, int prec, void *__restrict__ Bop) {
  const int M = 2 * T, nS = k1 - k0 + 1;
  const double scale = 1.0 / sqrt((double)T);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Npad * M; e += gridDim.x * blockDim.x) {
    const int j = e / M, r = e % M, t = r >> 1, c = r & 1;
    double v = 0.0;
    if (j < 2 * nS) {
      const int k = k0 + (j < nS ? j : j - nS);
      double sn, cs;
      sincospi(-2.0 * (double)((t * k) % T) / (double)T, &sn, &cs);  // exact angle reduction
      const double re = cs * scale, im = sn * scale;
      v = j < nS ? (c == 0 ? re : -im) : (c == 0 ? im : re);
    }
    if (prec == DH_PREC_FP32) {
      static_cast<float *>(Bop)[e] = (float)v;
    } else if (prec == DH_PREC_FP16) {
      // one FP16 rounding of W (the lo half is zero): its 2^-11 relative rounding moves the
      // image by a few 1e-5, and the overlapping-window span kernel uses the same operand
      __half *hi = static_cast<__half *>(Bop);
      hi[e] = to16<__half>((float)v);
      hi[(long long)Npad * M + e] = to16<__half>(0.f);
    } else {
      __nv_bfloat16 *hi = static_cast<__nv_bfloat16 *>(Bop);
      const __nv_bfloat16 h = to16<__nv_bfloat16>((float)v);
      hi[e] = h;
      hi[(long long)Npad * M + e] = to16<__nv_bfloat16>((float)(v - (double)from16(h)));
    }
  }
}

// Sliding form for windows one frame apart (the paper's Fourier mode renders a window per
// frame). With X_k(s) = sum_t H_{s+t}[p] w_{t,k} (t < T, w of Eq. 8, scale 1/sqrt(T) included),
//   X_k(s + 1) = e^{+2 pi i k / T} (X_k(s) + (H_{s+T}[p] - H_s[p]) / sqrt(T)),
// so each frame is read twice (entering and leaving) and only the kept bins are updated. Every
// segment of windows starts from the direct sum over its first window, which bounds the
// rounding drift of the recurrence (unit-modulus factors: about one FP32 rounding of |X| per
// step). A CTA covers 8 image columns x 32 rows (one pixel a thread, holograms column-major:
// the 32 rows of a column are 32 consecutive pixels) over one segment; each window's powers
// are transposed through shared memory so image rows are written 32 bytes at a time.
template <typename HT> __device__ __forceinline__ float2 load_h(const HT *H, long long rows_total, long long npix,
                                                                int slot, long long p);
template <> __device__ __forceinline__ float2 load_h<float>(const float *H, long long, long long npix, int slot,
                                                            long long p) {
  const float *re = H + (long long)slot * 2 * npix;
  return make_float2(re[p], re[p + npix]);
}
template <> __device__ __forceinline__ float2 load_h<__half>(const __half *H, long long rows_total, long long,
                                                             int slot, long long p) {
  const __half *b = H + (p >> 6) * (rows_total << 6) + (2ll * slot << 6) + (p & 63);
  return make_float2(__half2float(b[0]), __half2float(b[64]));
}
template <> __device__ __forceinline__ float2 load_h<__nv_bfloat16>(const __nv_bfloat16 *H, long long rows_total,
                                                                    long long, int slot, long long p) {
  const __nv_bfloat16 *b = H + (p >> 6) * (rows_total << 6) + (2ll * slot << 6) + (p & 63);
  return make_float2(__bfloat162float(b[0]), __bfloat162float(b[64]));
}

constexpr int kSlideCols = 8, kSlideRows = 32, kSlideThreads = kSlideCols * kSlideRows;

template <typename HT, int NBM>
__global__ void __launch_bounds__(kSlideThreads)
k_fourier_sliding(const HT *__restrict__ H, long long rows_total, int nx, int ny, int T, int k0, int nb,
                  int first_slot, int n_windows, int seg, float *__restrict__ images) {
  extern __shared__ float2 tab[];  // w[t][j] (T x NBM), then the step factors e[j]; bins >= nb zero
  __shared__ float out[2][kSlideRows][kSlideCols + 1];  // powers of a pass's two windows
  const long long npix = (long long)nx * ny;
  const double rs = 1.0 / sqrt((double)T);
  for (int e = threadIdx.x; e < T * NBM + NBM; e += blockDim.x) {
    double sn = 0.0, cs = 0.0;
    if (e < T * NBM) {
      const int t = e / NBM, j = e % NBM, k = k0 + j;
      if (j < nb) sincospi(-2.0 * (double)((t * k) % T) / (double)T, &sn, &cs);
      tab[e] = make_float2((float)(cs * rs), (float)(sn * rs));
    } else {
      const int j = e - T * NBM, k = k0 + j;
      if (j < nb) sincospi(2.0 * (double)(k % T) / (double)T, &sn, &cs);
      tab[e] = make_float2((float)cs, (float)sn);
    }
  }
  __syncthreads();
  const float2 *w = tab, *step = tab + T * NBM;
  const int tiles_y = ny / kSlideRows;
  const int kx0 = (blockIdx.x / tiles_y) * kSlideCols, ky0 = (blockIdx.x % tiles_y) * kSlideRows;
  const int c = threadIdx.x / kSlideRows, r = threadIdx.x % kSlideRows;
  const long long p = (long long)(kx0 + c) * ny + ky0 + r;
  const int w0 = blockIdx.y * seg, w1 = min(w0 + seg, n_windows);
  const float scale = (float)rs;
  float2 X[NBM];
#pragma unroll
  for (int j = 0; j < NBM; ++j) X[j] = make_float2(0.f, 0.f);
  for (int t = 0; t < T; ++t) {  // direct sum over the segment's first window
    const float2 h = load_h<HT>(H, rows_total, npix, first_slot + w0 + t, p);
#pragma unroll
    for (int j = 0; j < NBM; ++j) {
      const float2 q = w[t * NBM + j];
      X[j].x = fmaf(h.x, q.x, fmaf(-h.y, q.y, X[j].x));
      X[j].y = fmaf(h.x, q.y, fmaf(h.y, q.x, X[j].y));
    }
  }
  // two windows per pass (one barrier for both image writes); the frames of the next pass
  // are loaded while this pass computes
  float2 nin[2], nout[2];
  auto fetch = [&](int s, float2 (&hin)[2], float2 (&hout)[2]) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int sq = s + q;  // window sq > w0 advances from sq - 1
      if (sq > w0 && sq < w1) {
        hin[q] = load_h<HT>(H, rows_total, npix, first_slot + sq - 1 + T, p);
        hout[q] = load_h<HT>(H, rows_total, npix, first_slot + sq - 1, p);
      }
    }
  };
  fetch(w0, nin, nout);
  for (int s = w0; s < w1; s += 2) {
    float2 hin[2] = {nin[0], nin[1]}, hout[2] = {nout[0], nout[1]};
    fetch(s + 2, nin, nout);
    float m[2] = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (s + q >= w1) break;
      if (s + q > w0) {  // advance by one frame
        const float2 d = make_float2((hin[q].x - hout[q].x) * scale, (hin[q].y - hout[q].y) * scale);
#pragma unroll
        for (int j = 0; j < NBM; ++j) {
          const float2 a = make_float2(X[j].x + d.x, X[j].y + d.y), e = step[j];
          X[j] = make_float2(fmaf(a.x, e.x, -a.y * e.y), fmaf(a.x, e.y, a.y * e.x));
        }
      }
#pragma unroll
      for (int j = 0; j < NBM; ++j) m[q] = fmaf(X[j].x, X[j].x, fmaf(X[j].y, X[j].y, m[q]));
    }
    out[0][r][c] = m[0];
    out[1][r][c] = m[1];
    __syncthreads();
    // image rows ky0 + i / 8, columns kx0 .. kx0 + 7: 32 contiguous bytes per row
    const int i = threadIdx.x, ry = i / kSlideCols, cx = i % kSlideCols;
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (s + q < w1) images[(long long)(s + q) * npix + (long long)(ky0 + ry) * nx + kx0 + cx] = out[q][ry][cx];
    __syncthreads();
  }
}

// The same recurrence with two pixels a thread (adjacent rows of one image column, pixels p and
// p + 1): their real parts share one register pair and their imaginary parts another, so every
// operation of the recurrence is a paired FP32 instruction (__fadd2_rn, __fmul2_rn, __ffma2_rn)
// with per-bin constant pairs from shared memory; each pixel keeps the same operations in the
// same order as the one-pixel form, so the powers are bitwise those. A pixel pair's stored
// values come in one 32-bit (16-bit storage) or 64-bit (FP32) load. A CTA covers 8 image
// columns x 64 rows.
template <typename HT> __device__ __forceinline__ void load_h2(const HT *H, long long rows_total, long long npix,
                                                               int slot, long long p, float2 &re, float2 &im);
template <> __device__ __forceinline__ void load_h2<float>(const float *H, long long, long long npix, int slot,
                                                           long long p, float2 &re, float2 &im) {
  const float *b = H + (long long)slot * 2 * npix + p;
  re = *reinterpret_cast<const float2 *>(b);
  im = *reinterpret_cast<const float2 *>(b + npix);
}
template <> __device__ __forceinline__ void load_h2<__half>(const __half *H, long long rows_total, long long,
                                                            int slot, long long p, float2 &re, float2 &im) {
  const __half *b = H + (p >> 6) * (rows_total << 6) + (2ll * slot << 6) + (p & 63);
  re = __half22float2(*reinterpret_cast<const __half2 *>(b));
  im = __half22float2(*reinterpret_cast<const __half2 *>(b + 64));
}
template <> __device__ __forceinline__ void load_h2<__nv_bfloat16>(const __nv_bfloat16 *H, long long rows_total,
                                                                   long long, int slot, long long p, float2 &re,
                                                                   float2 &im) {
  const __nv_bfloat16 *b = H + (p >> 6) * (rows_total << 6) + (2ll * slot << 6) + (p & 63);
  re = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(b));
  im = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(b + 64));
}
constexpr int kSlide2Rows = 64;
constexpr int kSlideDepth = 8;  // window steps prefetched ahead (cp.async ring per thread)
// address of the Re (c = 0) or Im (c = 1) values of pixels p, p + 1 in slot `slot`
template <typename HT> __device__ __forceinline__ const HT *pair_addr(const HT *H, long long rows_total,
                                                                      long long npix, int slot, long long p, int c) {
  if constexpr (sizeof(HT) == 4) return H + ((long long)slot * 2 + c) * npix + p;
  else return H + (p >> 6) * (rows_total << 6) + ((2ll * slot + c) << 6) + (p & 63);
}
template <typename HT> __device__ __forceinline__ float2 pair_val(const void *v) {
  if constexpr (sizeof(HT) == 4) return *reinterpret_cast<const float2 *>(v);
  else if constexpr (std::is_same<HT, __half>::value) return __half22float2(*reinterpret_cast<const __half2 *>(v));
  else return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(v));
}
template <int BYTES>
__device__ __forceinline__ void cp_async_bytes(uint32_t dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
template <typename HT, int NBM>
__global__ void __launch_bounds__(kSlideThreads)
k_fourier_sliding2(const HT *__restrict__ H, long long rows_total, int nx, int ny, int T, int k0, int nb,
                   int first_slot, int n_windows, int seg, float *__restrict__ images) {
  // pair tables: w[t][j] as (Re, Re), (Im, Im), (-Im, -Im); step factors e[j] likewise
  extern __shared__ float2 tab2[];
  __shared__ float out[2][kSlide2Rows][kSlideCols + 1];
  // this thread's prefetch ring (kSlideDepth steps x 4 values of 2 pixels), after the tables
  float2 *ring_sm = tab2 + 3 * (T * NBM + NBM);
  const long long npix = (long long)nx * ny;
  const double rs = 1.0 / sqrt((double)T);
  const int nt = T * NBM + NBM;
  for (int e = threadIdx.x; e < nt; e += blockDim.x) {
    double sn = 0.0, cs = 0.0;
    float re, im;
    if (e < T * NBM) {
      const int t = e / NBM, j = e % NBM, k = k0 + j;
      if (j < nb) sincospi(-2.0 * (double)((t * k) % T) / (double)T, &sn, &cs);
      re = (float)(cs * rs); im = (float)(sn * rs);
    } else {
      const int j = e - T * NBM, k = k0 + j;
      if (j < nb) sincospi(2.0 * (double)(k % T) / (double)T, &sn, &cs);
      re = (float)cs; im = (float)sn;
    }
    tab2[3 * e] = make_float2(re, re);
    tab2[3 * e + 1] = make_float2(im, im);
    tab2[3 * e + 2] = make_float2(-im, -im);
  }
  __syncthreads();
  const float2 *w = tab2, *step = tab2 + 3 * T * NBM;
  const int tiles_y = ny / kSlide2Rows;
  const int kx0 = (blockIdx.x / tiles_y) * kSlideCols, ky0 = (blockIdx.x % tiles_y) * kSlide2Rows;
  const int c = threadIdx.x / 32, r2 = threadIdx.x % 32;  // pixels at rows ky0 + 2 r2, + 1
  const long long p = (long long)(kx0 + c) * ny + ky0 + 2 * r2;
  const int w0 = blockIdx.y * seg, w1 = min(w0 + seg, n_windows);
  const float scale = (float)rs;
  const float2 sc2 = make_float2(scale, scale), m1 = make_float2(-1.f, -1.f);
  float2 XR[NBM], XI[NBM];
#pragma unroll
  for (int j = 0; j < NBM; ++j) XR[j] = XI[j] = make_float2(0.f, 0.f);
  for (int t = 0; t < T; ++t) {  // direct sum over the segment's first window
    float2 hr, hi;
    load_h2<HT>(H, rows_total, npix, first_slot + w0 + t, p, hr, hi);
#pragma unroll
    for (int j = 0; j < NBM; ++j) {
      const float2 qr = w[3 * (t * NBM + j)], qi = w[3 * (t * NBM + j) + 1], qn = w[3 * (t * NBM + j) + 2];
      XR[j] = __ffma2_rn(hr, qr, __ffma2_rn(hi, qn, XR[j]));  // fmaf(h.x, q.x, fmaf(-h.y, q.y, X.x))
      XI[j] = __ffma2_rn(hr, qi, __ffma2_rn(hi, qr, XI[j]));  // fmaf(h.x, q.y, fmaf(h.y, q.x, X.y))
    }
  }
  // The frames entering and leaving at window step sq (window sq advances from sq - 1) are
  // copied kSlideDepth steps ahead into this thread's ring in shared memory (cp.async, one
  // commit group per step, completed in order): slot sq % kSlideDepth holds in Re, in Im,
  // out Re, out Im of the pixel pair. Only the thread reads its slots: no barrier is needed.
  constexpr int EB = sizeof(HT) * 2;  // bytes of a pair's Re or Im values
  const uint32_t ring0 = (uint32_t)__cvta_generic_to_shared(ring_sm);
  auto ring_addr = [&](int slot, int j) -> uint32_t {
    return ring0 + (uint32_t)(((slot * 4 + j) * kSlideThreads + threadIdx.x) * EB);
  };
  auto issue = [&](int sq) {  // always commits a group, empty past the segment
    if (sq > w0 && sq < w1) {
      const int sl = sq % kSlideDepth;
      cp_async_bytes<EB>(ring_addr(sl, 0), pair_addr<HT>(H, rows_total, npix, first_slot + sq - 1 + T, p, 0));
      cp_async_bytes<EB>(ring_addr(sl, 1), pair_addr<HT>(H, rows_total, npix, first_slot + sq - 1 + T, p, 1));
      cp_async_bytes<EB>(ring_addr(sl, 2), pair_addr<HT>(H, rows_total, npix, first_slot + sq - 1, p, 0));
      cp_async_bytes<EB>(ring_addr(sl, 3), pair_addr<HT>(H, rows_total, npix, first_slot + sq - 1, p, 1));
    }
    cp_async_commit();
  };
  for (int k = 0; k < kSlideDepth; ++k) issue(w0 + k);
  for (int s = w0; s < w1; s += 2) {
    float2 m[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (s + q >= w1) break;
      cp_async_wait<kSlideDepth - 1>();  // step s + q's group has landed
      if (s + q > w0) {  // advance by one frame
        const int sl = (s + q) % kSlideDepth;
        const uint8_t *rb = reinterpret_cast<const uint8_t *>(ring_sm);
        const float2 hin_r = pair_val<HT>(rb + (ring_addr(sl, 0) - ring0));
        const float2 hin_i = pair_val<HT>(rb + (ring_addr(sl, 1) - ring0));
        const float2 hout_r = pair_val<HT>(rb + (ring_addr(sl, 2) - ring0));
        const float2 hout_i = pair_val<HT>(rb + (ring_addr(sl, 3) - ring0));
        const float2 dr = __fmul2_rn(__ffma2_rn(hout_r, m1, hin_r), sc2);
        const float2 di = __fmul2_rn(__ffma2_rn(hout_i, m1, hin_i), sc2);
#pragma unroll
        for (int j = 0; j < NBM; ++j) {
          const float2 ar = __fadd2_rn(XR[j], dr), ai = __fadd2_rn(XI[j], di);
          const float2 er = step[3 * j], ei = step[3 * j + 1], en = step[3 * j + 2];
          XR[j] = __ffma2_rn(ar, er, __fmul2_rn(ai, en));  // fmaf(a.x, e.x, -a.y * e.y)
          XI[j] = __ffma2_rn(ar, ei, __fmul2_rn(ai, er));  // fmaf(a.x, e.y, a.y * e.x)
        }
      }
#pragma unroll
      for (int j = 0; j < NBM; ++j) m[q] = __ffma2_rn(XR[j], XR[j], __ffma2_rn(XI[j], XI[j], m[q]));
      issue(s + q + kSlideDepth);  // the slot just read is refilled for a later step
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      out[q][2 * r2][c] = m[q].x;
      out[q][2 * r2 + 1][c] = m[q].y;
    }
    __syncthreads();
    // image rows ky0 .. ky0 + 63, columns kx0 .. kx0 + 7: 32 contiguous bytes per row
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (s + q >= w1) break;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int i = threadIdx.x + hh * kSlideThreads, ry = i / kSlideCols, cx = i % kSlideCols;
        images[(long long)(s + q) * npix + (long long)(ky0 + ry) * nx + kx0 + cx] = out[q][ry][cx];
      }
    }
    __syncthreads();
  }
}

template <typename HT, int NBM>
dh_status launch_sliding_t(Plan &p, int first_slot, int n_windows, int k0, int nb, float *images, cudaStream_t s) {
  const int seg = 128;
  ProfScope ps(p, K_FOURIER_SLIDING, s);
  if (p.ny % kSlide2Rows == 0 && NBM <= 24) {  // two pixels a thread (32 bins would spill)
    const size_t smem = (size_t)3 * (p.T * NBM + NBM) * sizeof(float2) +
                        (size_t)kSlideDepth * 4 * kSlideThreads * 2 * sizeof(HT);
    static bool attr = false;
    if (!attr) {
      DH_CUDA_TRY(cudaFuncSetAttribute(k_fourier_sliding2<HT, NBM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));  // tables (<= 37 KB at T = 64) + ring (<= 64 KB)
      attr = true;
    }
    dim3 grid((unsigned)((p.nx / kSlideCols) * (p.ny / kSlide2Rows)), (unsigned)((n_windows + seg - 1) / seg));
    k_fourier_sliding2<HT, NBM><<<grid, kSlideThreads, smem, s>>>(
        static_cast<const HT *>(p.d_H), 2ll * p.max_frames, p.nx, p.ny, p.T, k0, nb, first_slot, n_windows, seg,
        images);
  } else {
    const size_t smem = (size_t)(p.T * NBM + NBM) * sizeof(float2);
    dim3 grid((unsigned)((p.nx / kSlideCols) * (p.ny / kSlideRows)), (unsigned)((n_windows + seg - 1) / seg));
    k_fourier_sliding<HT, NBM><<<grid, kSlideThreads, smem, s>>>(
        static_cast<const HT *>(p.d_H), 2ll * p.max_frames, p.nx, p.ny, p.T, k0, nb, first_slot, n_windows, seg,
        images);
  }
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

// one instantiation per bin count the bands of T = 16, 32, 64 need most (the paper's 17 at
// T = 32), so no lane computes a bin outside the band; other counts are padded with zero
// bins (rows nb..NBM-1 of the tables are zero)
template <typename HT>
dh_status launch_sliding(Plan &p, int first_slot, int n_windows, int k0, int nb, float *images, cudaStream_t s) {
  switch (nb) {
    case 9: return launch_sliding_t<HT, 9>(p, first_slot, n_windows, k0, nb, images, s);
    case 17: return launch_sliding_t<HT, 17>(p, first_slot, n_windows, k0, nb, images, s);
  }
  if (nb <= 8) return launch_sliding_t<HT, 8>(p, first_slot, n_windows, k0, nb, images, s);
  if (nb <= 16) return launch_sliding_t<HT, 16>(p, first_slot, n_windows, k0, nb, images, s);
  if (nb <= 24) return launch_sliding_t<HT, 24>(p, first_slot, n_windows, k0, nb, images, s);
  return launch_sliding_t<HT, 32>(p, first_slot, n_windows, k0, nb, images, s);
}

}  // namespace

dh_status launch_fourier(Plan &p, int first_slot, int slot_stride, int n_windows, int k0, int k1,
                         float *images, cudaStream_t s) {
  const int nS = k1 - k0 + 1;
  // overlapping windows on the tensor cores: 7 windows per load of their frames
  if (fourier_span_applies(p, slot_stride, n_windows, nS))
    return launch_fourier_span(p, first_slot, slot_stride, n_windows, k0, nS, images, s);
  // a window per frame: the sliding recurrence (each frame read twice instead of T times)
  if (slot_stride == 1 && n_windows >= 8 && nS <= 32 && p.ny % kSlideRows == 0 && p.nx % kSlideCols == 0) {
    switch (p.prec) {
      case DH_PREC_FP32: return launch_sliding<float>(p, first_slot, n_windows, k0, nS, images, s);
      case DH_PREC_FP16: return launch_sliding<__half>(p, first_slot, n_windows, k0, nS, images, s);
      case DH_PREC_BF16: return launch_sliding<__nv_bfloat16>(p, first_slot, n_windows, k0, nS, images, s);
    }
  }
  const int nop = p.prec == DH_PREC_FP32 ? 2 * nS : (2 * nS + 15) / 16 * 16;  // operand rows
  {
    ProfScope ps(p, K_FOURIER_OP, s);
    k_fourier_operand<<<(nop * 2 * p.T + 255) / 256, 256, 0, s>>>(p.T, k0, k1, nop, (int)p.prec, p.d_W);
    DH_CUDA_TRY(cudaGetLastError());
  }
  return p.prec == DH_PREC_FP32
             ? launch_project_simt(p, first_slot, slot_stride, n_windows, nop, images, 0, s, p.d_W)
             : launch_project_tc(p, first_slot, slot_stride, n_windows, nop, images, 0, s, p.d_W);
}

}  // namespace dh
