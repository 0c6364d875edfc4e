// Tracing: optional per-kernel device timing. When enabled on a plan, every kernel the
// plan launches is bracketed by a pair of CUDA events recorded on the launch stream;
// dh_profile_read() synchronises and returns launches and total milliseconds per kernel.
// Every launch is also inside an NVTX range named for its stage (always on: without a tool
// attached an NVTX call returns at once), so that profilers can attribute kernels to stages
// (e.g. ncu --nvtx --nvtx-include "render_fused/").
#include "dh_internal.cuh"

#include <nvtx3/nvToolsExt.h>

#include <vector>

struct dh_plan;

namespace dh {

namespace {
struct ProfState {
  struct Rec { int kid; cudaEvent_t a, b; };
  std::vector<Rec> recs;      // recorded since the last read
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
const char *kNames[K_COUNT] = {"render_rows", "render_cols", "gram_simt", "gram_tc",
                               "reduce_cov", "jacobi", "project_simt", "project_tc",
                               "fourier_operand", "svd_fourier_operand", "render_fused", "gram_raw",
                               "reduce_raw", "fourier_sliding", "band_gram", "band_reduce",
                               "band_cov", "project_span", "fourier_span", "render_rows_tc",
                               "render_cols_tc", "render_fused_tc"};
}  // namespace

const char *kernel_name(int kid) { return kid >= 0 && kid < K_COUNT ? kNames[kid] : "?"; }

ProfScope::ProfScope(Plan &plan, int k, cudaStream_t st) : p(plan), kid(k), s(st), slot(-1) {
  nvtxRangePushA(kernel_name(k));
  if (!p.prof) return;
  // launches being captured into a CUDA graph are not timed (the events would become graph
  // nodes, not timestamps of a run)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  ProfState *ps = static_cast<ProfState *>(p.prof);
  ProfState::Rec r{kid, ps->get(), ps->get()};
  cudaEventRecord(r.a, s);
  ps->recs.push_back(r);
  slot = (int)ps->recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (p.prof && slot >= 0) {
    ProfState *ps = static_cast<ProfState *>(p.prof);
    cudaEventRecord(ps->recs[slot].b, s);
  }
  nvtxRangePop();
}

void profile_free(Plan &p) {
  if (!p.prof) return;
  ProfState *ps = static_cast<ProfState *>(p.prof);
  for (auto &r : ps->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : ps->pool) cudaEventDestroy(e);
  delete ps;
  p.prof = nullptr;
}

dh_status profile_enable(Plan &p, int on) {
  if (on && !p.prof) p.prof = new ProfState();
  if (!on) profile_free(p);
  return DH_OK;
}

int profile_read(Plan &p, int n, const char **names, int *launches, double *total_ms) {
  for (int k = 0; k < n && k < K_COUNT; ++k) {
    if (names) names[k] = kNames[k];
    if (launches) launches[k] = 0;
    if (total_ms) total_ms[k] = 0.0;
  }
  if (!p.prof) return K_COUNT;
  ProfState *ps = static_cast<ProfState *>(p.prof);
  for (auto &r : ps->recs) {
    float ms = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms, r.a, r.b);
    if (r.kid < n) {
      if (launches) launches[r.kid] += 1;
      if (total_ms) total_ms[r.kid] += ms;
    }
    ps->pool.push_back(r.a);
    ps->pool.push_back(r.b);
  }
  ps->recs.clear();
  return K_COUNT;
}

}  // namespace dh
