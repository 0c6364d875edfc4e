// Display normalisation: the paper divides every displayed image by its own average value,
// which cancels the strong frame-to-frame variations of the power images. The mean of each
// image is reduced in FP64 by one CTA (a fixed order, so repeated calls agree bitwise); a
// second kernel writes the normalised FP32 image and/or 8-bit display codes
//   code = clamp(rint(gain * M / mean), 0, 255)   (mean -> code `gain`),
// the headless stand-in for a display: a caller-owned device buffer (a ring, a file).
#include "dh_internal.cuh"

namespace dh {
namespace {

constexpr int kMeanThreads = 1024;

__global__ void __launch_bounds__(kMeanThreads)
k_image_mean(const float *__restrict__ images, long long npix, double *__restrict__ means) {
  __shared__ double red[kMeanThreads / 32];
  const float4 *img = reinterpret_cast<const float4 *>(images + (long long)blockIdx.x * npix);
  double acc = 0.0;
  for (long long i = threadIdx.x; i < npix / 4; i += kMeanThreads) {
    const float4 v = img[i];
    acc += ((double)v.x + (double)v.y) + ((double)v.z + (double)v.w);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) means[blockIdx.x] = v / (double)npix;
  }
}

__global__ void __launch_bounds__(256)
k_normalize(const float *__restrict__ images, long long npix, const double *__restrict__ means,
            float gain, float *__restrict__ norm, uint8_t *__restrict__ disp) {
  const int w = blockIdx.y;
  const double mean = means[w];
  const float inv = (float)(1.0 / mean), scale = (float)((double)gain / mean);
  const float4 *src = reinterpret_cast<const float4 *>(images + (long long)w * npix);
  for (long long i = blockIdx.x * 256ll + threadIdx.x; i < npix / 4; i += 256ll * gridDim.x) {
    const float4 v = src[i];
    if (norm) reinterpret_cast<float4 *>(norm + (long long)w * npix)[i] =
        make_float4(v.x * inv, v.y * inv, v.z * inv, v.w * inv);
    if (disp) {
      const float c[4] = {v.x * scale, v.y * scale, v.z * scale, v.w * scale};
      uchar4 u;
      u.x = (uint8_t)fminf(fmaxf(rintf(c[0]), 0.f), 255.f);
      u.y = (uint8_t)fminf(fmaxf(rintf(c[1]), 0.f), 255.f);
      u.z = (uint8_t)fminf(fmaxf(rintf(c[2]), 0.f), 255.f);
      u.w = (uint8_t)fminf(fmaxf(rintf(c[3]), 0.f), 255.f);
      reinterpret_cast<uchar4 *>(disp + (long long)w * npix)[i] = u;
    }
  }
}

}  // namespace
}  // namespace dh

using namespace dh;

extern "C" dh_status dh_normalize_images(const float *images_dev, int n_images, int64_t npix,
                                         float *normalized_dev, uint8_t *display_dev,
                                         float display_gain, double *means_dev, void *stream) {
  if (!images_dev || !means_dev || n_images < 1 || npix < 4 || (npix & 3) != 0 || n_images > 65535 ||
      !(display_gain > 0.f))
    return DH_ERR_INVALID_ARG;
  auto misaligned = [](const void *q, uintptr_t a) { return (reinterpret_cast<uintptr_t>(q) & (a - 1)) != 0; };
  if (misaligned(images_dev, 16) || misaligned(normalized_dev, 16) || misaligned(display_dev, 4) ||
      misaligned(means_dev, 8))
    return DH_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_image_mean<<<n_images, kMeanThreads, 0, s>>>(images_dev, npix, means_dev);
  DH_CUDA_TRY(cudaGetLastError());
  if (normalized_dev || display_dev) {
    long long bx = (npix / 4 + 255) / 256;
    if (bx > 64) bx = 64;
    k_normalize<<<dim3((unsigned)bx, (unsigned)n_images), 256, 0, s>>>(images_dev, npix, means_dev, display_gain,
                                                                       normalized_dev, display_dev);
    DH_CUDA_TRY(cudaGetLastError());
  }
  return DH_OK;
}
