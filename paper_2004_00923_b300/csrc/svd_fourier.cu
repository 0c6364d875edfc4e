// Eqs. 2-3 then Eqs. 8-9: singular value filtering of each window followed by temporal
// demodulation by the unitary DFT (the paper's earlier pipeline, which it describes as too
// heavy for real time on its hardware). Since U Delta = H V (Eq. 2 with V from Eq. 5), the
// filtered stack is H_f = H V_S V_S^{t*} with V_S the kept eigenvectors k0..k1, and Eq. 8 on
// it keeps bins b0..b1 of H_f W: the image is the power of H Q with the T x n_b matrix
//   Q = V_S V_S^{t*} W_band,   Q[t][j] = sum_{k=k0..k1} V[t][k] sum_u conj(V[u][k]) w_{u,b0+j}.
// One CTA per window forms Q in FP64 from the eigensolver's sorted V and packs it as the
// projection operand (the layout Eq. 6 uses), so the projection kernels do the rest.
#include "dh_internal.cuh"

namespace dh {
namespace {

template <typename T16> __device__ __forceinline__ T16 cvt16(float x);
template <> __device__ __forceinline__ __half cvt16<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt16<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
__device__ __forceinline__ float back(__half x) { return __half2float(x); }
__device__ __forceinline__ float back(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename T16>
__device__ __forceinline__ void put(void *Bop, long long base, long long lo_off, long long i, double v) {
  T16 *b = static_cast<T16 *>(Bop) + base;
  const T16 h = cvt16<T16>((float)v);
  b[i] = h;
  b[lo_off + i] = cvt16<T16>((float)(v - (double)back(h)));
}

template <int T>
__global__ void __launch_bounds__(256)
k_svd_fourier_operand(const double *__restrict__ V, int k0, int k1, int b0, int b1, int Npad, int prec,
                      void *__restrict__ Bop, long long B_stride) {
  constexpr int M = 2 * T;
  extern __shared__ double R[];  // [nS][nb][2]: R[k][j] = sum_u conj(V[u][k]) w_{u,b0+j}
  const int w = blockIdx.x;
  const double *Vw = V + 2ll * w * T * T;
  const int nS = k1 - k0 + 1, nb = b1 - b0 + 1;
  const double scale = 1.0 / sqrt((double)T);
  for (int e = threadIdx.x; e < nS * nb; e += blockDim.x) {
    const int k = k0 + e / nb, b = b0 + e % nb;
    double rr = 0.0, ri = 0.0;
    for (int u = 0; u < T; ++u) {
      double sn, cs;
      sincospi(-2.0 * (double)((u * b) % T) / (double)T, &sn, &cs);
      const double vr = Vw[2 * (u * T + k)], vi = -Vw[2 * (u * T + k) + 1];  // conj(V[u][k])
      rr += vr * cs - vi * sn;
      ri += vr * sn + vi * cs;
    }
    R[2 * e] = rr * scale;
    R[2 * e + 1] = ri * scale;
  }
  __syncthreads();
  // Q[t][j] = sum_k V[t][k] R[k][j], packed: row j < nb holds Re of bin b0 + j, row nb + j Im
  for (int e = threadIdx.x; e < Npad * M; e += blockDim.x) {
    const int j = e / M, r = e % M, t = r >> 1, c = r & 1;
    double v = 0.0;
    if (j < 2 * nb) {
      const int jj = j < nb ? j : j - nb;
      double qr = 0.0, qi = 0.0;
      for (int k = 0; k < nS; ++k) {
        const double vr = Vw[2 * (t * T + k0 + k)], vi = Vw[2 * (t * T + k0 + k) + 1];
        const double rr = R[2 * (k * nb + jj)], ri = R[2 * (k * nb + jj) + 1];
        qr += vr * rr - vi * ri;
        qi += vr * ri + vi * rr;
      }
      v = j < nb ? (c == 0 ? qr : -qi) : (c == 0 ? qi : qr);
    }
    if (prec == DH_PREC_FP32) {
      static_cast<float *>(Bop)[w * B_stride + e] = (float)v;
    } else if (prec == DH_PREC_FP16) {
      put<__half>(Bop, w * B_stride, (long long)Npad * M, e, v);
    } else {
      put<__nv_bfloat16>(Bop, w * B_stride, (long long)Npad * M, e, v);
    }
  }
}

template <int T>
dh_status launch_t(Plan &p, int n_windows, int k0, int k1, int b0, int b1, int Npad, int woff,
                   cudaStream_t s) {
  const size_t smem = (size_t)T * T * 2 * sizeof(double);
  static bool attr = false;
  if (!attr) {
    DH_CUDA_TRY(cudaFuncSetAttribute(k_svd_fourier_operand<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    attr = true;
  }
  const long long B_stride = (long long)(p.B_window_bytes / (p.prec == DH_PREC_FP32 ? 4 : 2));
  void *B = static_cast<char *>(p.d_B) + (size_t)woff * p.B_window_bytes;
  ProfScope ps(p, K_SVD_FOURIER_OP, s);
  k_svd_fourier_operand<T><<<n_windows, 256, smem, s>>>(p.d_V + 2ll * woff * T * T, k0, k1, b0, b1, Npad,
                                                         (int)p.prec, B, B_stride);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

}  // namespace

dh_status launch_svd_fourier_operand(Plan &p, int n_windows, int k0, int k1, int b0, int b1, int Npad,
                                     int woff, cudaStream_t s) {
  switch (p.T) {
    case 16: return launch_t<16>(p, n_windows, k0, k1, b0, b1, Npad, woff, s);
    case 32: return launch_t<32>(p, n_windows, k0, k1, b0, b1, Npad, woff, s);
    case 64: return launch_t<64>(p, n_windows, k0, k1, b0, b1, Npad, woff, s);
  }
  return DH_ERR_UNSUPPORTED_SIZE;
}

}  // namespace dh
