// Mean-residual storage of the holograms (DH_OPT_RESIDUAL): for a window of T frames, its
// holograms H_t = F(I_t) (Eq. 1, F linear) are stored as D_t = F(I_t - M), M the window's
// temporal mean frame rounded to integers, and mu = F(M) is kept in FP32. Then
// H = mu 1^T + D exactly, so the projection of Eq. 6 is P = D V + mu (1^T V), and Eq. 7's
// power follows from it. The static part of the speckle -- most of |H| -- is no longer in
// the 16-bit values, whose rounding error shrinks with |D| instead of |H|. The covariance of
// Eq. 4 comes from the frames themselves (C = I^T I, exact), so it does not see the storage.
//
//   k_window_mean  M[w][p] = rint(sum_t I[w T + t][p] / T) as uint16 (exact integer sums)
//   k_mu_coef      per window, for each column j of the projection operand (its layout:
//                  j < nS the real part of component k0 + j, nS <= j < 2 nS its imaginary
//                  part), the coefficients of mu's real and imaginary parts in that column:
//                  s_k = sum_t V_tk; Re P_k gets Re(mu s_k) = mu_r Re s_k - mu_i Im s_k and
//                  Im P_k gets Im(mu s_k) = mu_r Im s_k + mu_i Re s_k.
#include "dh_internal.cuh"

namespace dh {
namespace {

// 8 pixels a thread (16-byte loads of every frame of the window), one grid row per window.
__global__ void __launch_bounds__(256)
k_window_mean(const uint16_t *__restrict__ frames, long long frame_stride, int T, int window_stride,
              long long npix, uint16_t *__restrict__ mean) {
  const int w = blockIdx.y;
  const long long p8 = (blockIdx.x * 256ll + threadIdx.x) * 8;
  if (p8 >= npix) return;
  const uint16_t *f0 = frames + (long long)w * window_stride * frame_stride + p8;
  uint32_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int t = 0; t < T; ++t) {
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(f0 + (long long)t * frame_stride));
    const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc[2 * k] += w4[k] & 0xFFFFu;
      acc[2 * k + 1] += w4[k] >> 16;
    }
  }
  uint32_t out[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t lo = (acc[2 * k] + (uint32_t)T / 2) / (uint32_t)T;
    const uint32_t hi = (acc[2 * k + 1] + (uint32_t)T / 2) / (uint32_t)T;
    out[k] = lo | (hi << 16);
  }
  *reinterpret_cast<uint4 *>(mean + (long long)w * npix + p8) = make_uint4(out[0], out[1], out[2], out[3]);
}

// One CTA per window; V is the window's sorted FP64 eigenvectors [T][T] (re, im interleaved).
__global__ void k_mu_coef(const double *__restrict__ V, int T, int k0, int k1, int Npad,
                          float *__restrict__ coef) {
  const int w = blockIdx.x, j = threadIdx.x;
  if (j >= Npad) return;
  const int nS = k1 - k0 + 1;
  float a = 0.f, b = 0.f;
  if (j < 2 * nS) {
    const int k = k0 + (j < nS ? j : j - nS);
    const double *Vw = V + 2ll * w * T * T;
    double sr = 0.0, si = 0.0;
    for (int t = 0; t < T; ++t) {
      sr += Vw[2 * (t * T + k)];
      si += Vw[2 * (t * T + k) + 1];
    }
    if (j < nS) { a = (float)sr; b = (float)-si; }
    else { a = (float)si; b = (float)sr; }
  }
  // per window: a at [0, 2T), b at [2T, 4T) (Npad <= 2T)
  coef[(long long)w * 4 * T + j] = a;
  coef[(long long)w * 4 * T + 2 * T + j] = b;
}

}  // namespace

dh_status launch_window_mean(Plan &p, const uint16_t *frames, long long frame_stride, int n_windows,
                             int window_stride, cudaStream_t s) {
  const long long blocks = (p.npix / 8 + 255) / 256;
  k_window_mean<<<dim3((unsigned)blocks, (unsigned)n_windows), 256, 0, s>>>(frames, frame_stride, p.T,
                                                                             window_stride, p.npix, p.d_mean);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

dh_status launch_mu_coef(Plan &p, int n_windows, int k0, int k1, int Npad, int woff, cudaStream_t s) {
  k_mu_coef<<<n_windows, 128, 0, s>>>(p.d_V + 2ll * woff * p.T * p.T, p.T, k0, k1, Npad,
                                      p.d_mucoef + 4ll * woff * p.T);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

}  // namespace dh
