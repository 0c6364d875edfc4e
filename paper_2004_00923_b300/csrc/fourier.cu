// Eqs. 8-9: temporal demodulation by the unitary DFT, the paper's Fourier alternative to
// the data-derived basis of Eq. 6. Windows one frame apart use a sliding recurrence (below);
// other strides the projection. W has entries w_{t,k} = exp(-2 pi i t k / n_t) / sqrt(n_t)
// (t, k counted from 0); its columns k0..k1 (the frequency filter I_f) form a fixed
// projection operand, built once per call in the layout the eigensolver writes for Eq. 6,
// and every window is projected onto it by the same kernels, |.|^2 summed in the epilogue:
//   M[p] = sum_{k=k0..k1} |sum_t H[t][p] w_{t,k}|^2.
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
      __half *hi = static_cast<__half *>(Bop);
      const __half h = to16<__half>((float)v);
      hi[e] = h;
      hi[(long long)Npad * M + e] = to16<__half>((float)(v - (double)from16(h)));
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

template <typename HT, int NBM>
dh_status launch_sliding_t(Plan &p, int first_slot, int n_windows, int k0, int nb, float *images, cudaStream_t s) {
  const int seg = 128;
  const size_t smem = (size_t)(p.T * NBM + NBM) * sizeof(float2);
  dim3 grid((unsigned)((p.nx / kSlideCols) * (p.ny / kSlideRows)), (unsigned)((n_windows + seg - 1) / seg));
  ProfScope ps(p, K_FOURIER_SLIDING, s);
  k_fourier_sliding<HT, NBM><<<grid, kSlideThreads, smem, s>>>(
      static_cast<const HT *>(p.d_H), 2ll * p.max_frames, p.nx, p.ny, p.T, k0, nb, first_slot, n_windows, seg,
      images);
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
