// Eqs. 6-7 on FP32 CUDA cores (the plain path): for every pixel p of window w,
//   M[p] = sum_j ( sum_r X[r][p] B[j][r] )^2
// with X the 2T rows [Re H_0; Im H_0; ...] and B the real embedding of the retained
// eigenvectors (rows 0..nS-1 give Re of (H V)_k, rows nS..2nS-1 give Im), i.e.
// M = sum_{k=k0..k1} |(H V)[p][k]|^2. The projected stack H V is never stored.
#include "dh_internal.cuh"

namespace dh {
namespace {

template <int T>
__global__ void __launch_bounds__(256)
k_project_simt(const float *__restrict__ H, long long npix, int first_slot, int slot_stride,
               const float *__restrict__ Bop, long long B_stride, int nrows, int blocks_per_window,
               int nx, int ny, float *__restrict__ images) {
  constexpr int M = 2 * T;
  extern __shared__ float4 bs4[];
  const int w = blockIdx.x / blocks_per_window, b = blockIdx.x % blocks_per_window;
  const float4 *src = reinterpret_cast<const float4 *>(Bop + w * B_stride);
  for (int e = threadIdx.x; e < nrows * M / 4; e += blockDim.x) bs4[e] = src[e];
  __syncthreads();
  const float *X = H + (long long)(first_slot + w * slot_stride) * 2 * npix;
  const long long chunk = npix / blocks_per_window;
  const long long p_end = (b + 1) * chunk;
  float *img = images + (long long)w * npix;
  for (long long p = b * chunk + threadIdx.x; p < p_end; p += blockDim.x) {
    float x[M];
#pragma unroll
    for (int r = 0; r < M; ++r) x[r] = X[(long long)r * npix + p];
    float m = 0.f;
    for (int j = 0; j < nrows; ++j) {
      const float4 *bj = bs4 + j * (M / 4);
      float acc = 0.f;
#pragma unroll
      for (int r4 = 0; r4 < M / 4; ++r4) {
        const float4 v = bj[r4];
        acc = fmaf(x[4 * r4], v.x, acc);
        acc = fmaf(x[4 * r4 + 1], v.y, acc);
        acc = fmaf(x[4 * r4 + 2], v.z, acc);
        acc = fmaf(x[4 * r4 + 3], v.w, acc);
      }
      m = fmaf(acc, acc, m);
    }
    img[(p % ny) * nx + p / ny] = m;  // holograms are column-major: p = kx n_y + ky
  }
}

template <int T>
dh_status launch_t(Plan &p, int first_slot, int slot_stride, int n_windows, int nrows,
                   float *images, int woff, cudaStream_t s, const void *shared_op) {
  // about 4 CTAs per SM in total, at least 256 pixels per CTA
  long long bpw = 1;
  while (bpw * 2 * n_windows <= 8ll * p.num_sms && p.npix / (bpw * 2) >= 256) bpw *= 2;
  const size_t smem = (size_t)nrows * 2 * T * sizeof(float);
  static bool attr = false;
  if (!attr) {
    DH_CUDA_TRY(cudaFuncSetAttribute(k_project_simt<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(4 * T * T * sizeof(float))));
    attr = true;
  }
  const long long B_stride = (long long)(p.B_window_bytes / sizeof(float));
  const float *op = shared_op ? static_cast<const float *>(shared_op)
                              : static_cast<const float *>(p.d_B) + (long long)woff * B_stride;
  ProfScope ps(p, K_PROJECT_SIMT, s);
  k_project_simt<T><<<(int)(n_windows * bpw), 256, smem, s>>>(
      static_cast<const float *>(p.d_H), p.npix, first_slot, slot_stride, op,
      shared_op ? 0 : B_stride, nrows, (int)bpw, p.nx, p.ny, images);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

}  // namespace

dh_status launch_project_simt(Plan &p, int first_slot, int slot_stride, int n_windows, int Npad,
                              float *images, int woff, cudaStream_t s, const void *shared_op) {
  switch (p.T) {
    case 16: return launch_t<16>(p, first_slot, slot_stride, n_windows, Npad, images, woff, s, shared_op);
    case 32: return launch_t<32>(p, first_slot, slot_stride, n_windows, Npad, images, woff, s, shared_op);
    case 64: return launch_t<64>(p, first_slot, slot_stride, n_windows, Npad, images, woff, s, shared_op);
  }
  return DH_ERR_UNSUPPORTED_SIZE;
}

}  // namespace dh
