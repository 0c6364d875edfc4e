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
//
// The u-column form (used when the operand's padding leaves two columns free): expanding
// |P_k|^2 = |(DV)_k + mu s_k|^2 and summing over the kept components S,
//   M = sum_{k in S} |(DV)_k|^2 + 2 Re(conj(mu) D u) + |mu|^2 sigma,
//   u_t = sum_{k in S} V_tk conj(s_k),   sigma = sum_{k in S} |s_k|^2,
// so D u is one more projection, computed by the same MMAs from two more operand columns
// (the real embedding of u, written here into the last two of the Npad columns, which the
// eigensolver left zero), and the epilogue's cost per pixel stays that of the plain power
// plus three FMAs instead of two FMAs per column.
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

// u-column form: one CTA of 128 threads per window (T <= 64). s_k and sigma in FP64, then
// u_t (thread t) and its two operand columns, split into hi + lo 16-bit parts like the
// eigenvectors' columns: column Npad - 2 gives Re(D u) (rows 2t, 2t + 1: Re u_t, -Im u_t),
// column Npad - 1 gives Im(D u) (Im u_t, Re u_t).
template <typename T16>
__global__ void k_mu_ucol(const double *__restrict__ V, int T, int k0, int k1, int Npad,
                          float *__restrict__ coef, T16 *__restrict__ Bop, long long B_stride) {
  __shared__ double sr[64], si[64];
  const int w = blockIdx.x, tid = threadIdx.x;
  const double *Vw = V + 2ll * w * T * T;
  if (tid < T) {
    double a = 0.0, b = 0.0;
    if (tid >= k0 && tid <= k1)
      for (int t = 0; t < T; ++t) {
        a += Vw[2 * (t * T + tid)];
        b += Vw[2 * (t * T + tid) + 1];
      }
    sr[tid] = a;
    si[tid] = b;
  }
  __syncthreads();
  if (tid == 0) {
    double sig = 0.0;
    for (int k = k0; k <= k1; ++k) sig += sr[k] * sr[k] + si[k] * si[k];
    coef[(long long)w * 4 * T] = (float)sig;
  }
  if (tid < T) {
    double ur = 0.0, ui = 0.0;  // u_t = sum_k V_tk conj(s_k)
    for (int k = k0; k <= k1; ++k) {
      const double vr = Vw[2 * (tid * T + k)], vi = Vw[2 * (tid * T + k) + 1];
      ur += vr * sr[k] + vi * si[k];
      ui += vi * sr[k] - vr * si[k];
    }
    const int M = 2 * T;
    T16 *hi = Bop + (long long)w * B_stride, *lo = hi + (long long)Npad * M;
    const long long j0 = (long long)(Npad - 2) * M, j1 = (long long)(Npad - 1) * M;
    const double vals[4] = {ur, -ui, ui, ur};
    const long long idx[4] = {j0 + 2 * tid, j0 + 2 * tid + 1, j1 + 2 * tid, j1 + 2 * tid + 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T16 h = T16((float)vals[q]);
      hi[idx[q]] = h;
      lo[idx[q]] = T16((float)(vals[q] - (double)(float)h));
    }
  }
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

dh_status launch_mu_coef(Plan &p, int n_windows, int k0, int k1, int Npad, int woff, bool ucol, cudaStream_t s) {
  if (ucol) {
    if (Npad < 2 * (k1 - k0 + 1) + 2 || Npad > 2 * p.T || p.T > 64) return DH_ERR_STATE;
    const long long B_stride = (long long)(p.B_window_bytes / 2);
    char *B = static_cast<char *>(p.d_B) + (size_t)woff * p.B_window_bytes;
    if (p.prec == DH_PREC_BF16)
      k_mu_ucol<__nv_bfloat16><<<n_windows, 128, 0, s>>>(p.d_V + 2ll * woff * p.T * p.T, p.T, k0, k1, Npad,
                                                          p.d_mucoef + 4ll * woff * p.T,
                                                          reinterpret_cast<__nv_bfloat16 *>(B), B_stride);
    else
      k_mu_ucol<__half><<<n_windows, 128, 0, s>>>(p.d_V + 2ll * woff * p.T * p.T, p.T, k0, k1, Npad,
                                                   p.d_mucoef + 4ll * woff * p.T, reinterpret_cast<__half *>(B),
                                                   B_stride);
  } else {
    k_mu_coef<<<n_windows, 128, 0, s>>>(p.d_V + 2ll * woff * p.T * p.T, p.T, k0, k1, Npad,
                                        p.d_mucoef + 4ll * woff * p.T);
  }
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

}  // namespace dh
