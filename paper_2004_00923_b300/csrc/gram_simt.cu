// Eq. 4 on FP32 CUDA cores (the plain path): partial real Gram matrices
//   G = X X^T,  X = the 2T rows [Re H_0; Im H_0; Re H_1; Im H_1; ...] over a pixel range.
// Each CTA owns one (window, pixel range) unit and accumulates products in FP32 over
// 256-pixel runs, then in FP64; units are summed in FP64 by the reduction kernel. Chunks of
// 32 pixels are double-buffered in shared memory: the next chunk's copy (cp.async, 8-byte
// pieces) is in flight while the current one is multiplied.
// C[t][u] = (G[2t][2u] + G[2t+1][2u+1]) + i (G[2t][2u+1] - G[2t+1][2u]).
#include "dh_internal.cuh"

namespace dh {
namespace {

template <int T>
__global__ void __launch_bounds__(256)
k_gram_simt(const float *__restrict__ H, long long npix, int first_slot, int slot_stride,
            int units, long long pix_per_unit, double *__restrict__ part) {
  constexpr int M = 2 * T;
  constexpr int TM = M / 16;
  constexpr int KC = 32;
  constexpr int LD = KC + 2;  // row stride: 8-byte aligned pairs, conflict-free columns
  __shared__ __align__(16) float xs[2][M * LD];
  const int w = blockIdx.x / units, u = blockIdx.x % units;
  const float *X = H + (long long)(first_slot + w * slot_stride) * 2 * npix + u * pix_per_unit;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[TM][TM];
  double acc64[TM][TM];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int k = 0; k < TM; ++k) acc[i][k] = 0.f, acc64[i][k] = 0.0;
  // copy of chunk `pc` into buffer `b`: 8-byte pieces, consecutive threads along a row
  auto issue = [&](long long pc, int b) {
    if (pc < pix_per_unit) {
      for (int e = threadIdx.x; e < M * (KC / 2); e += 256) {
        const int r = e / (KC / 2), k = 2 * (e % (KC / 2));
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&xs[b][r * LD + k]);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(X + (long long)r * npix + pc + k)
                     : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  issue(0, 0);
  int chunk = 0;
  for (long long pc = 0; pc < pix_per_unit; pc += KC, ++chunk) {
    const int cb = chunk & 1;
    issue(pc + KC, cb ^ 1);  // the other buffer: its readers passed the barrier below
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // this chunk's copy has landed
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < KC; k += 2) {
      float2 a[TM], b[TM];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        a[i] = *reinterpret_cast<const float2 *>(&xs[cb][(ty + 16 * i) * LD + k]);
        b[i] = *reinterpret_cast<const float2 *>(&xs[cb][(tx + 16 * i) * LD + k]);
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int q = 0; q < TM; ++q) {
          acc[i][q] = fmaf(a[i].x, b[q].x, acc[i][q]);
          acc[i][q] = fmaf(a[i].y, b[q].y, acc[i][q]);
        }
    }
    __syncthreads();
    if ((chunk & 7) == 7) {
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int q = 0; q < TM; ++q) acc64[i][q] += (double)acc[i][q], acc[i][q] = 0.f;
    }
  }
  double *dst = part + (long long)(w * units + u) * M * M;
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int q = 0; q < TM; ++q)
      dst[(ty + 16 * i) * M + tx + 16 * q] = acc64[i][q] + (double)acc[i][q];
}

template <int T>
dh_status launch_t(Plan &p, int first_slot, int slot_stride, int n_windows, int units,
                   cudaStream_t s) {
  const long long ppu = p.npix / units;
  ProfScope ps(p, K_GRAM_SIMT, s);
  k_gram_simt<T><<<n_windows * units, 256, 0, s>>>(static_cast<const float *>(p.d_H), p.npix,
                                                  first_slot, slot_stride, units, ppu, p.d_part);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

}  // namespace

// Partial Gram matrices of one window's rows X (2T rows of npix FP32, row r at
// X + r * npix) into part[u][2T][2T], u < units; npix / units must be a multiple of 32.
dh_status launch_gram_simt_rows(const float *X, long long npix, int T, int units, double *part,
                                cudaStream_t s) {
  const long long ppu = npix / units;
  switch (T) {
    case 16: k_gram_simt<16><<<units, 256, 0, s>>>(X, npix, 0, 0, units, ppu, part); break;
    case 32: k_gram_simt<32><<<units, 256, 0, s>>>(X, npix, 0, 0, units, ppu, part); break;
    case 64: k_gram_simt<64><<<units, 256, 0, s>>>(X, npix, 0, 0, units, ppu, part); break;
    default: return DH_ERR_UNSUPPORTED_SIZE;
  }
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

// Loads the module of every instance launch_gram_simt_rows uses (under lazy module loading a
// kernel's first launch would otherwise load it, which can allocate and synchronise).
dh_status preload_gram_simt_rows() {
  cudaFuncAttributes fa;
  DH_CUDA_TRY(cudaFuncGetAttributes(&fa, k_gram_simt<16>));
  DH_CUDA_TRY(cudaFuncGetAttributes(&fa, k_gram_simt<32>));
  DH_CUDA_TRY(cudaFuncGetAttributes(&fa, k_gram_simt<64>));
  return DH_OK;
}

// Split-K units per window: a function of the frame size only (never of the batch), so a
// window's covariance is bitwise the same alone and inside any batch.
int gram_units(long long npix) {
  long long u = npix / 4096;
  if (u < 1) u = 1;
  if (u > 64) u = 64;
  return (int)u;
}

dh_status launch_gram_simt(Plan &p, int first_slot, int slot_stride, int n_windows,
                           int *parts_per_window, cudaStream_t s) {
  const int units = gram_units(p.npix);
  *parts_per_window = units;
  switch (p.T) {
    case 16: return launch_t<16>(p, first_slot, slot_stride, n_windows, units, s);
    case 32: return launch_t<32>(p, first_slot, slot_stride, n_windows, units, s);
    case 64: return launch_t<64>(p, first_slot, slot_stride, n_windows, units, s);
  }
  return DH_ERR_UNSUPPORTED_SIZE;
}

}  // namespace dh
