// Arithmetic-rate measurement for the rooflines: the FP32 and FP64 FMA throughput this GPU
// sustains at its current clocks. The render of Eq. 1 is bound by FP32 instruction issue and
// the eigensolver's refinement by the FP64 pipe, so their fractions divide by these measured
// rates rather than by nominal unit counts.
//
// Each thread runs kChains independent FMA chains (enough to cover the pipe latency) for
// `iters` rounds; a chain's final value is stored (to a one-element buffer) only if it equals
// a value it can never reach, which keeps the work live without memory traffic. FLOPs = 2 per
// FMA lane.
#include "dh_internal.cuh"

namespace dh {
namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <typename T>
__device__ __forceinline__ T fma_op(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_op<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double fma_op<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float2 fma_op<float2>(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <typename T>
__device__ __forceinline__ T splat(float v);
template <> __device__ __forceinline__ float splat<float>(float v) { return v; }
template <> __device__ __forceinline__ double splat<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ float2 splat<float2>(float v) { return make_float2(v, v + 0.5f); }

template <typename T>
__device__ __forceinline__ bool is_sentinel(T v);
template <> __device__ __forceinline__ bool is_sentinel<float>(float v) { return v == -1.2345e30f; }
template <> __device__ __forceinline__ bool is_sentinel<double>(double v) { return v == -1.2345e300; }
template <> __device__ __forceinline__ bool is_sentinel<float2>(float2 v) { return v.x == -1.2345e30f; }

// x <- x * m + a keeps |x| bounded (m < 1), so no value overflows or goes subnormal.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_rate(int iters, T *__restrict__ sink) {
  T x[kChains];
  const float seed = 1.0f + 1e-3f * (float)(threadIdx.x & 31);
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = splat<T>(seed + (float)c);
  const T m = splat<T>(0.999f), a = splat<T>(0.001f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma_op<T>(x[c], m, a);
  }
#pragma unroll
  for (int c = 0; c < kChains; ++c)
    if (is_sentinel<T>(x[c])) *sink = x[c];
}

template <typename T>
dh_status time_rate(int iters, int blocks, int lanes, float *ms, double *flops, cudaStream_t s) {
  cudaEvent_t a = nullptr, b = nullptr;
  T *sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(T));
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) {
    k_fma_rate<T><<<blocks, kThreads, 0, s>>>(iters, sink);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) {
    k_fma_rate<T><<<blocks, kThreads, 0, s>>>(iters, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return fail_cuda(e);
  // FMAs per thread: iters x 8 x kChains, each on `lanes` values
  *flops = 2.0 * lanes * (double)iters * 8.0 * kChains * (double)blocks * kThreads;
  return DH_OK;
}

}  // namespace
}  // namespace dh

using namespace dh;

extern "C" dh_status dh_measure_fma_rate(int kind, int iters, int blocks_per_sm, float *ms, double *flops,
                                         void *stream) {
  if (!ms || !flops || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 64) return DH_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  DH_CUDA_TRY(cudaGetDevice(&dev));
  DH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * blocks_per_sm;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (kind) {
    case 0: return time_rate<float>(iters, blocks, 1, ms, flops, s);
    case 1: return time_rate<float2>(iters, blocks, 2, ms, flops, s);
    case 2: return time_rate<double>(iters, blocks, 1, ms, flops, s);
  }
  return DH_ERR_INVALID_ARG;
}
