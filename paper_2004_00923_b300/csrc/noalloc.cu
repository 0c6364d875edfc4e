// dh_covariance_noalloc: the covariance C = H^{t*} H of one window computed without
// allocating any device memory.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree (or any allocating
// routine) once they are running -- for example a frame-grabber callback or a real-time
// acquisition thread, where an allocation can synchronise the device and stall the camera
// stream, or host code whose device memory is owned by another framework's allocator. They
// pass their holograms and an output buffer; the split-K scratch lives in the file-scope
// device array below, which every GPU that loads this library holds until the process
// exits.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current), caches it per device, and loads the
// modules of every kernel the entry point launches, for all T (under lazy module loading a
// kernel's first launch would load it, and loading a module can allocate and synchronise).
// So the first call on a device may allocate: make one call per device before real-time use
// and before any stream capture; from the second call on nothing is allocated or loaded.
// All calls on a device share the one array, so calls whose kernels overlap on the GPU race
// (serialise them, e.g. on one stream). Every partial matrix is fully overwritten before it
// is read. The status word after the partials (the reduction's non-finite flag) is cleared
// at the start of every call and is not reported: a non-finite covariance shows up as
// NaN/Inf entries of C_dev itself.
#include "dh_internal.cuh"

#include <mutex>

namespace dh {
namespace {

// Scratch for the per-unit partial Gram matrices: 2 MiB, i.e. 16 partial 128x128 FP64
// matrices (T = 64) or 64 partial 64x64 ones (T = 32), plus a status word.
constexpr size_t kScratchBytes = 2u << 20;
constexpr int kMaxUnits = 64;
static __device__ __align__(256) unsigned char g_cov_scratch[kScratchBytes + 256];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

dh_status scratch_for_current_device(void **out) {
  int dev = -1;
  DH_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return DH_ERR_UNSUPPORTED_SIZE;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    DH_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_cov_scratch));
    dh_status st = preload_gram_simt_rows();
    if (st == DH_OK) st = preload_reduce_cov_window();
    if (st != DH_OK) return st;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return DH_OK;
}

}  // namespace
}  // namespace dh

using namespace dh;

extern "C" dh_status dh_covariance_noalloc(const float *planes_dev, int64_t npix, int T, double *C_dev,
                                           void *stream) {
  if (!planes_dev || !C_dev || npix < 32 || (npix % 32) != 0) return DH_ERR_INVALID_ARG;
  // the planes are copied in 8-byte pieces and C is written as doubles
  if ((reinterpret_cast<uintptr_t>(planes_dev) & 7u) != 0 || (reinterpret_cast<uintptr_t>(C_dev) & 7u) != 0)
    return DH_ERR_INVALID_ARG;
  if (!(T == 16 || T == 32 || T == 64)) return DH_ERR_UNSUPPORTED_SIZE;
  if (npix > (1ll << 28)) return DH_ERR_UNSUPPORTED_SIZE;
  const size_t part_bytes = (size_t)(2 * T) * (2 * T) * sizeof(double);
  // units: a power of two that divides npix / 32, at least 4096 pixels each when possible,
  // and no more partial matrices than the scratch array holds
  int units = 1;
  while (units * 2 <= kMaxUnits && (size_t)(units * 2) * part_bytes <= kScratchBytes &&
         npix % (32ll * units * 2) == 0 && npix / (units * 2) >= 4096)
    units *= 2;
  void *scratch = nullptr;
  dh_status st = scratch_for_current_device(&scratch);
  if (st != DH_OK) return st;
  double *part = static_cast<double *>(scratch);
  uint32_t *status = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(scratch) + kScratchBytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DH_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
  if ((st = launch_gram_simt_rows(planes_dev, npix, T, units, part, s)) != DH_OK) return st;
  return launch_reduce_cov_window(part, units, T, C_dev, status, s);
}
