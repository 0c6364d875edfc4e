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
#include "tc_sm100.cuh"

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


// ---------------------------------------------------------------- tensor-core issue rate
// tcgen05.mma kind::f16 (M = 128, N = 128, K = 16, FP32 accumulation) issued in stages of four
// from one thread of one CTA per SM, with a tcgen05.commit per stage, in three forms:
//   0: back to back (the tensor cores' rate for this shape);
//   1: the issuing warp waits on an mbarrier (already complete) before each stage, as a
//      pipeline's MMA warp waits for its stage's data;
//   2: a second warp does that wait and releases the issuing warp through a named barrier.
// The operands are constant FP16 tiles in shared memory (128-byte swizzle, K-major).
constexpr int kMmaStageSlots = 4;
constexpr int kMmaSmem = kMmaStageSlots * 16384 + 1024;

template <int FORM>
__global__ void __launch_bounds__(128, 1) k_mma_issue(int stages, long long *__restrict__ cycles) {
  using namespace tc;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t ready[kMmaStageSlots], released[kMmaStageSlots], done;
  __shared__ uint32_t holder;
  for (int i = threadIdx.x; i < kMmaStageSlots * 16384 / 4; i += blockDim.x)
    reinterpret_cast<uint32_t *>(smem)[i] = 0x3C003C00u;  // FP16 1.0
  if (threadIdx.x == 0) {
    for (int j = 0; j < kMmaStageSlots; ++j) { mbar_init(&ready[j], 1); mbar_init(&released[j], 1); }
    mbar_init(&done, 1);
    fence_barrier_init();
    for (int j = 0; j < kMmaStageSlots; ++j) mbar_arrive(&ready[j]);  // phase 0 of each completes
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x < 32) { tmem_alloc(&holder, 128); tmem_relinquish(); }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = holder;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t idesc = idesc_f16(false, false, false, 128, 128);
  if (warp == 0) {
    const long long t0 = clock64();
    bool ok = true;
    for (int st = 0; st < stages; ++st) {
      const int slot = st % kMmaStageSlots;
      if (FORM == 1) ok = ok && __all_sync(0xffffffffu, mbar_wait(&ready[slot], 0));
      if (FORM == 2) named_sync(1 + slot, 64);
      fence_after_sync();
      if (lane == 0) {
        const uint32_t base = smem_u32(smem + slot * 16384);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint64_t desc = smem_desc(base + 32 * k, 16, 1024, kSwizzle128);
          mma_f16(tmem, desc, desc, idesc, (st > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(&released[slot]);
      }
      __syncwarp();
    }
    if (lane == 0) mma_commit(&done);
    __syncwarp();
    ok = __all_sync(0xffffffffu, mbar_wait(&done, 0)) && ok;
    if (lane == 0) cycles[blockIdx.x] = ok ? clock64() - t0 : -1;
  } else if (FORM == 2 && warp == 1) {  // the waiter: lock-step with the issuing warp
    for (int st = 0; st < stages; ++st) {
      const int slot = st % kMmaStageSlots;
      __all_sync(0xffffffffu, mbar_wait(&ready[slot], 0));
      named_sync(1 + slot, 64);
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

template <int FORM>
dh_status time_mma_issue(int stages, float *ms, double *cycles_per_mma, double *flops, cudaStream_t s) {
  int dev = 0, sms = 0;
  DH_CUDA_TRY(cudaGetDevice(&dev));
  DH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // more shared memory than half an SM holds: one CTA per SM, so each has its own tensor cores
  const int smem = 120 * 1024;
  static_assert(kMmaSmem <= 120 * 1024, "operand tiles fit");
  DH_CUDA_TRY(cudaFuncSetAttribute(k_mma_issue<FORM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  long long *d_cyc = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaMalloc(&d_cyc, sizeof(long long) * sms);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) {
    k_mma_issue<FORM><<<sms, 128, smem, s>>>(stages, d_cyc);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) {
    k_mma_issue<FORM><<<sms, 128, smem, s>>>(stages, d_cyc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  long long mx = 0;
  if (e == cudaSuccess) {
    long long *h = new long long[sms];
    e = cudaMemcpy(h, d_cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
    for (int i = 0; e == cudaSuccess && i < sms; ++i) mx = h[i] < 0 ? -1 : (mx < 0 ? mx : (h[i] > mx ? h[i] : mx));
    delete[] h;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (d_cyc) cudaFree(d_cyc);
  if (e != cudaSuccess) return fail_cuda(e);
  if (mx < 0) return DH_ERR_TIMEOUT;
  *cycles_per_mma = (double)mx / (4.0 * stages);
  *flops = 2.0 * 128 * 128 * 16 * 4.0 * stages * sms;
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

extern "C" dh_status dh_measure_mma_issue(int form, int stages, float *ms, double *cycles_per_mma, double *flops,
                                          void *stream) {
  if (!ms || !cycles_per_mma || !flops || stages < 1 || stages > (1 << 24)) return DH_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (form) {
    case 0: return time_mma_issue<0>(stages, ms, cycles_per_mma, flops, s);
    case 1: return time_mma_issue<1>(stages, ms, cycles_per_mma, flops, s);
    case 2: return time_mma_issue<2>(stages, ms, cycles_per_mma, flops, s);
  }
  return DH_ERR_INVALID_ARG;
}
