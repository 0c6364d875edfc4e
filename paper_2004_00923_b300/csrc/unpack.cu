// 12-bit packed camera frames (the GenICam pixel format Mono12p: pixel i of a frame occupies
// bits [12 i, 12 i + 12) of the frame's bytes read as one little-endian bit string, so two
// pixels fill three bytes) expanded to the uint16 frames the render of Eq. 1 reads. The host
// pipeline of dh_pca_batch_host_packed12 copies the packed bytes (3/4 of the uint16 bytes) and
// expands them on the device.
//
// One thread expands 8 pixels: three 32-bit words (12 bytes, 4-byte aligned when the frame
// stride is) into one 16-byte store. Bound by HBM (1.5 bytes read + 2 written a pixel).
#include "dh_internal.cuh"

namespace dh {
namespace {

__global__ void __launch_bounds__(256)
k_unpack_mono12p(const uint8_t *__restrict__ src, long long src_stride_bytes, long long npix,
                 uint16_t *__restrict__ dst, long long dst_stride_elems) {
  const long long g = blockIdx.x * 256ll + threadIdx.x;  // group of 8 pixels
  if (g * 8 >= npix) return;
  const int f = blockIdx.y;
  const uint32_t *w = reinterpret_cast<const uint32_t *>(src + (long long)f * src_stride_bytes + g * 12);
  const uint32_t w0 = __ldcs(w), w1 = __ldcs(w + 1), w2 = __ldcs(w + 2);
  // bits 0-11, 12-23, 24-35, 36-47, 48-59, 60-71, 72-83, 84-95 of w2:w1:w0
  const uint32_t p0 = w0 & 0xFFFu, p1 = (w0 >> 12) & 0xFFFu;
  const uint32_t p2 = (w0 >> 24) | ((w1 & 0xFu) << 8), p3 = (w1 >> 4) & 0xFFFu;
  const uint32_t p4 = (w1 >> 16) & 0xFFFu, p5 = (w1 >> 28) | ((w2 & 0xFFu) << 4);
  const uint32_t p6 = (w2 >> 8) & 0xFFFu, p7 = w2 >> 20;
  *reinterpret_cast<uint4 *>(dst + (long long)f * dst_stride_elems + g * 8) =
      make_uint4(p0 | (p1 << 16), p2 | (p3 << 16), p4 | (p5 << 16), p6 | (p7 << 16));
}

}  // namespace

dh_status launch_unpack_mono12p(const uint8_t *src, long long src_stride_bytes, long long npix, int n_frames,
                                uint16_t *dst, long long dst_stride_elems, cudaStream_t s) {
  if (n_frames < 1) return DH_OK;
  const long long blocks = (npix / 8 + 255) / 256;
  k_unpack_mono12p<<<dim3((unsigned)blocks, (unsigned)n_frames), 256, 0, s>>>(src, src_stride_bytes, npix, dst,
                                                                                dst_stride_elems);
  DH_CUDA_TRY(cudaGetLastError());
  return DH_OK;
}

}  // namespace dh

using namespace dh;

extern "C" dh_status dh_unpack_mono12p(const uint8_t *src_dev, int64_t src_stride_bytes, int64_t npix,
                                       int n_frames, uint16_t *dst_dev, int64_t dst_stride_elems, void *stream) {
  if (!src_dev || !dst_dev || n_frames < 0 || npix < 8 || (npix & 7) != 0 || n_frames > 65535) return DH_ERR_INVALID_ARG;
  if (src_stride_bytes < npix / 2 * 3 || (src_stride_bytes & 3) != 0 || dst_stride_elems < npix ||
      (dst_stride_elems & 7) != 0)
    return DH_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(src_dev) & 3) != 0 || (reinterpret_cast<uintptr_t>(dst_dev) & 15) != 0)
    return DH_ERR_INVALID_ARG;
  return launch_unpack_mono12p(src_dev, src_stride_bytes, npix, n_frames, dst_dev, dst_stride_elems,
                               static_cast<cudaStream_t>(stream));
}
