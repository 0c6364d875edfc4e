// Eqs. 8-9: temporal demodulation by the unitary DFT, the paper's Fourier alternative to
// the data-derived basis of Eq. 6. W has entries w_{t,k} = exp(-2 pi i t k / n_t) / sqrt(n_t)
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

}  // namespace

dh_status launch_fourier(Plan &p, int first_slot, int slot_stride, int n_windows, int k0, int k1,
                         float *images, cudaStream_t s) {
  const int nS = k1 - k0 + 1;
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
