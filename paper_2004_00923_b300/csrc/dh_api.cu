// The C ABI of libdh (declared in include/dh.h): plan lifetime, argument checks, device
// buffers and the order of the stages. Every step of the computation runs in the
// library's own CUDA kernels; this file only validates, allocates and launches.
#include "dh_internal.cuh"

#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <algorithm>
#include <vector>

struct dh_plan {
  dh::Plan p;
  std::atomic<int> busy{0};
  std::atomic<int> refs{1};   // the caller's handle + one per live view of this plan
  std::atomic<int> views{0};  // live views sharing this plan's hologram store
  dh_plan *base = nullptr;    // for a view: the plan whose store it reads
};

struct dh_graph {
  cudaGraphExec_t exec = nullptr;
};

namespace dh {

static thread_local std::string g_last_error = "no error";

const char *set_cuda_error(cudaError_t e) {
  g_last_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
  return g_last_error.c_str();
}

dh_status fail_cuda(cudaError_t e) {
  set_cuda_error(e);
  (void)cudaGetLastError();  // clear a non-sticky error
  return e == cudaErrorMemoryAllocation ? DH_ERR_OOM : DH_ERR_CUDA;
}


namespace {

bool pow2_in_range(int n) { return n >= kMinDim && n <= kMaxDim && (n & (n - 1)) == 0; }

template <typename Ptr>
dh_status dalloc(Plan &p, Ptr **ptr, size_t bytes) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) return fail_cuda(e);
  *ptr = static_cast<Ptr *>(q);
  p.bytes += bytes;
  return DH_OK;
}

template <typename Ptr>
void dfree(Ptr *&ptr) {
  if (ptr) cudaFree((void *)ptr);
  ptr = nullptr;
}

// Per-window buffers: covariance partials, C, lambda, V and the projection operand.
void free_windows(Plan &p) {
  dfree(p.d_part); dfree(p.d_C); dfree(p.d_lam); dfree(p.d_V); dfree(p.d_B); dfree(p.d_W);
  dfree(p.d_mean); dfree(p.d_mu); dfree(p.d_mucoef);
  p.tmaps_ok = false;
  p.bytes -= p.window_bytes;
  p.window_bytes = 0;
}

void free_store(Plan &p) {
  free_windows(p);
  if (p.is_view) {
    p.d_H = nullptr;  // owned by the base plan
  } else {
    dfree(p.d_H);
    dfree(p.d_mid);
  }
}

bool tc_render_sizes(const Plan &p) { return p.nx == 1024 && p.ny == 1024; }

size_t table_bytes(const Plan &p) {
  return sizeof(float2) * (p.nx + p.ny + twiddle_len(p.lognx) + twiddle_len(p.logny)) + 16 +
         (tc_render_sizes(p) ? tc_tables_bytes() : 0);
}

// Device bytes of every buffer a plan allocates, from its sizes, reservation and precision.
struct StoreSizes {
  size_t tables, H, mid, part, C, lam, V, B, W, resid;
  int mid_frames, parts_total;
  size_t B_window;
  size_t windows() const { return part + C + lam + V + B + W + resid; }
  size_t total() const { return tables + H + mid + windows(); }
};

StoreSizes store_sizes(const Plan &p) {
  StoreSizes z{};
  const int M = 2 * p.T;
  const size_t hb = p.prec == DH_PREC_FP32 ? 4 : 2;
  z.tables = table_bytes(p);
  z.H = (size_t)p.max_frames * 2 * p.npix * hb;
  // row-pass intermediate: a chunk of frames sized to stay in L2 (~96 MiB of the 126 MB),
  // never more frames than the plan has slots
  long long mf = (96ll << 20) / (p.npix * (long long)sizeof(float2));
  if (mf > 64) mf = 64;
  if (mf > p.max_frames) mf = p.max_frames;
  if (mf < 1) mf = 1;
  z.mid_frames = (int)mf;
  z.mid = (size_t)mf * p.npix * sizeof(float2);
  z.parts_total = p.max_windows * parts_per_window(p);
  z.part = (size_t)z.parts_total * M * M * sizeof(double);
  z.C = (size_t)p.max_windows * p.T * p.T * 2 * sizeof(double);
  z.lam = (size_t)p.max_windows * p.T * sizeof(double);
  z.V = z.C;
  // operand of Eq. 6 per window: FP32 [2T][2T], or 16-bit hi and lo [2][2T][2T]
  const size_t bw = p.prec == DH_PREC_FP32 ? (size_t)M * M * 4 : (size_t)2 * M * M * 2;
  z.B_window = (bw + 1023) / 1024 * 1024;
  // + room for the last group's operand of the grouped projection (at most 64 KiB)
  z.B = z.B_window * p.max_windows + (p.prec == DH_PREC_FP32 ? 0 : (64u << 10));
  // one operand shared by every window (Eq. 8); 16-bit plans also hold there the banded group
  // operand of the tensor-core sliding DFT (at most 2 x 240 x 256 16-bit values)
  z.W = z.B_window;
  if (p.prec != DH_PREC_FP32 && z.W < (256u << 10)) z.W = 256u << 10;
  // mean-residual storage: mean frames (uint16), mu (FP32 complex), mu coefficients
  z.resid = p.residual ? (size_t)p.max_windows * ((size_t)p.npix * (2 + 8) + 16ull * p.T) : 0;
  return z;
}

// (Re)allocate the per-window buffers for max_windows windows of length T over the store.
dh_status alloc_windows(Plan &p) {
  free_windows(p);
  const StoreSizes z = store_sizes(p);
  dh_status st;
  p.parts_total = z.parts_total;
  p.B_window_bytes = z.B_window;
  if ((st = dalloc(p, &p.d_part, z.part)) != DH_OK) return st;
  if ((st = dalloc(p, &p.d_C, z.C)) != DH_OK) return st;
  if ((st = dalloc(p, &p.d_lam, z.lam)) != DH_OK) return st;
  if ((st = dalloc(p, &p.d_V, z.V)) != DH_OK) return st;
  if ((st = dalloc(p, &p.d_B, z.B)) != DH_OK) return st;
  if ((st = dalloc(p, &p.d_W, z.W)) != DH_OK) return st;
  if (p.residual) {
    if ((st = dalloc(p, &p.d_mean, (size_t)p.max_windows * p.npix * 2)) != DH_OK) return st;
    if ((st = dalloc(p, &p.d_mu, (size_t)p.max_windows * p.npix * 8)) != DH_OK) return st;
    if ((st = dalloc(p, &p.d_mucoef, (size_t)p.max_windows * 16 * p.T)) != DH_OK) return st;
  }
  p.W_bytes = z.W;
  p.window_bytes = z.windows();
  DH_CUDA_TRY(cudaMemset(p.d_B, 0, z.B));
  if (p.prec != DH_PREC_FP32) {
    if ((st = make_tensor_maps(p)) != DH_OK) return st;
  }
  return DH_OK;
}

// (Re)allocate everything whose size depends on the reservation or the precision. A view
// takes the store of `base` instead of allocating one.
dh_status alloc_store(Plan &p, const Plan *base = nullptr) {
  free_store(p);
  p.band_frames = 0;  // a new store has no band yet
  const StoreSizes z = store_sizes(p);
  // the host-buffer pipeline's buffers (kept across reservations) stay counted
  const size_t pipe = 2 * p.pipe.stage_elems * sizeof(uint16_t) + 2 * p.pipe.pstage_bytes +
                      p.pipe.img_elems * sizeof(float) + p.pipe.eig_elems * sizeof(double);
  p.bytes = (p.is_view ? 0 : z.tables) + pipe;
  p.H_elem_bytes = p.prec == DH_PREC_FP32 ? 4 : 2;
  dh_status st;
  if (p.is_view) {
    p.d_H = base->d_H;
  } else {
    if ((st = dalloc(p, &p.d_H, z.H)) != DH_OK) return st;
    p.mid_frames = z.mid_frames;
    if ((st = dalloc(p, &p.d_mid, z.mid)) != DH_OK) return st;
  }
  return alloc_windows(p);
}

// The CUDA-core FFT radix of the plan (0 = each length's default, 16 or 32 where that radix is
// instantiated for an axis length): the inter-pass twiddle tables follow it. Synchronous.
dh_status set_fft_radix(Plan &p, int radix) {
  if (radix != 0 && radix != 16 && radix != 32) return DH_ERR_INVALID_ARG;
  if (p.is_view) return DH_ERR_STATE;
  if (!fft_radix_available(p.lognx, radix) && !fft_radix_available(p.logny, radix))
    return DH_ERR_UNSUPPORTED_SIZE;
  const int old_rx = row_spec(p), old_cy = col_spec(p);
  const int keep = p.fft_radix;
  p.fft_radix = radix;
  const int rx = row_spec(p), cy = col_spec(p);
  if (rx == old_rx && cy == old_cy) return DH_OK;
  std::vector<float2> twx(twiddle_len(rx)), twy(twiddle_len(cy));
  build_twiddles(rx, twx.data());
  build_twiddles(cy, twy.data());
  cudaError_t e = cudaDeviceSynchronize();  // no render in flight reads the old tables
  if (e != cudaSuccess) { p.fft_radix = keep; return fail_cuda(e); }
  dfree(p.d_twx); dfree(p.d_twy);
  p.bytes -= sizeof(float2) * (twiddle_len(old_rx) + twiddle_len(old_cy));
  dh_status st = dalloc(p, &p.d_twx, twx.size() * sizeof(float2));
  if (st == DH_OK) st = dalloc(p, &p.d_twy, twy.size() * sizeof(float2));
  if (st != DH_OK) return st;
  e = cudaMemcpy(p.d_twx, twx.data(), twx.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p.d_twy, twy.data(), twy.size() * sizeof(float2), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? DH_OK : fail_cuda(e);
}

// Mean-residual storage for dh_pca_batch's windows (16-bit storage): the mean frame, mu and
// coefficient buffers are allocated with the per-window buffers (synchronous).
dh_status set_residual(Plan &p, int on) {
  if (on != 0 && on != 1) return DH_ERR_INVALID_ARG;
  if (on && p.prec == DH_PREC_FP32) return DH_ERR_STATE;
  if (on == p.residual) return DH_OK;
  DH_CUDA_TRY(cudaDeviceSynchronize());
  p.residual = on;
  return alloc_windows(p);
}

// Split-K units per window of the tensor-core covariance (0 = the default for the frame size):
// a power of two dividing n / 256, so that every window length's pixel chunks tile a unit.
// The per-window partial buffers are reallocated (synchronous).
dh_status set_gram_units(Plan &p, int units) {
  if (units < 0 || units > 1024 || (units & (units - 1)) != 0) return DH_ERR_INVALID_ARG;
  if (p.prec == DH_PREC_FP32) return DH_ERR_STATE;  // the tensor-core covariance only
  if (units > 0 && p.npix % (256ll * units) != 0) return DH_ERR_UNSUPPORTED_SIZE;
  if (units == p.gram_units) return DH_OK;
  DH_CUDA_TRY(cudaDeviceSynchronize());
  p.gram_units = units;
  return alloc_windows(p);
}

std::vector<float2> chirp_table(int n, double a) {
  // c(k) = exp(-i pi a (k - n/2)^2) / sqrt(n); the phase a d^2 is reduced mod 2 in FP64
  std::vector<float2> c(n);
  const double inv = 1.0 / std::sqrt((double)n);
  const double pi = 3.141592653589793238462643383279502884;
  for (int k = 0; k < n; ++k) {
    const double d = (double)(k - n / 2);
    const double ph = std::fmod(a * (d * d), 2.0);
    c[k] = make_float2((float)(std::cos(pi * ph) * inv), (float)(-std::sin(pi * ph) * inv));
  }
  return c;
}

// Windows [first_slot + w * slot_stride, + T), w < n_windows, optionally rendering the frames
// they need first. The windows can be processed in groups: each group's covariance runs on
// the caller's stream, its eigensolver on the plan's aux stream, and the projections follow
// on the caller's stream once each group's eigenvectors are ready; the call ends with the
// caller's stream joined to everything it launched. Two groups are used only with every
// frame rendered first: an eigensolver beside the persistent render, which fills every SM,
// was measured slower (both slowed down on the shared SMs).
// With b0 >= 0 the operand of Eq. 6 is replaced, per window, by the SVD-filter + DFT operand
// of Eqs. 2-3 and 8-9 (components k0..k1 kept, bins b0..b1). With `raw` (uint16 frames,
// window w's first frame at raw + w * slot_stride * raw_stride) and the plan's raw-domain
// option, the covariance is formed from those frames (C = I^T I) instead of the holograms.
dh_status pca_impl(Plan &p, const uint16_t *frames, long long frame_stride, int first_slot,
                   int slot_stride, int n_windows, int k0, int k1, float *images, double *eig_user,
                   cudaStream_t s, int b0 = -1, int b1 = -1, const uint16_t *raw = nullptr,
                   long long raw_stride = 0) {
  // mean-residual storage: disjoint windows with their frames at hand, Eqs. 4-7 only
  if (p.residual && (!frames || !raw || slot_stride != p.T || b0 >= 0 || p.cov_mode == 2 || p.prec == DH_PREC_FP32))
    return DH_ERR_STATE;
  const int nS = b0 >= 0 ? b1 - b0 + 1 : k1 - k0 + 1;  // projected columns
  int nop = p.prec == DH_PREC_FP32 ? 2 * nS : (2 * nS + 15) / 16 * 16;  // operand rows
  // residual storage: the u-column form where two more operand columns fit (residual.cu)
  p.resid_ucol = 0;
  if (p.residual && b0 < 0 && (2 * nS + 2 + 15) / 16 * 16 <= 2 * p.T) {
    nop = (2 * nS + 2 + 15) / 16 * 16;
    p.resid_ucol = 1;
  }
  // overlapping windows: grouped projection (one group layout for the whole call)
  const SpanLayout span = b0 < 0 ? span_layout(p, slot_stride, n_windows, k0, k1) : SpanLayout{};
  // Two groups where the eigensolver (one CTA per window) can run beside the other group's
  // tensor-core covariance and projection: those launches then leave one SM per eigensolver
  // CTA (their own CTAs, by registers or shared memory, cannot share an SM with it), and
  // every frame is rendered first, since the persistent render fills all SMs.
  const bool two = p.group_mode == 0 && b0 < 0 && span.G == 0 && (p.cov_mode == 0 || p.cov_mode == 1) &&
                   p.prec != DH_PREC_FP32 && n_windows >= 32 && n_windows <= p.num_sms;
  const int G = two ? 2 : 1;
  struct Budget {  // the SM budget applies to one launch at a time
    Plan &p;
    ~Budget() { p.sm_budget = 0; }
  } budget{p};
  int w0s[Plan::kMaxGroups], nws[Plan::kMaxGroups];
  for (int g = 0, w0 = 0; g < G; ++g) {
    nws[g] = n_windows / G + (g < n_windows % G ? 1 : 0);
    w0s[g] = w0;
    w0 += nws[g];
  }
  int rendered = 0;  // frames (slots relative to first_slot) already rendered
  dh_status st;
  if (p.residual) {  // the windows' mean frames M, and mu = F(M) in FP32
    if ((st = launch_window_mean(p, frames, frame_stride, n_windows, slot_stride, s)) != DH_OK) return st;
    if ((st = launch_render_to(p, p.d_mean, p.npix, n_windows, 0,
                               RenderTarget{p.d_mu, DH_PREC_FP32, 0, nullptr, 1}, s)) != DH_OK)
      return st;
  }
  for (int g = 0; g < G; ++g) {
    const int w0 = w0s[g], nw = nws[g];
    if (frames) {
      const int need = (G > 1 ? n_windows - 1 : w0 + nw - 1) * slot_stride + p.T;
      if (need > rendered) {
        const RenderTarget to{p.d_H, p.prec, 2ll * p.max_frames, p.residual ? p.d_mean : nullptr, p.T,
                              rendered};
        st = launch_render_to(p, frames + (long long)rendered * frame_stride, frame_stride, need - rendered,
                              first_slot + rendered, to, s);
        if (st != DH_OK) return st;
        rendered = need;
      }
    }
    const int fs = first_slot + w0 * slot_stride;
    int parts = 0;
    if (raw && (p.cov_mode == 1 || p.residual)) {
      p.sm_budget = g > 0 ? p.num_sms - nws[g - 1] : 0;  // beside the previous group's eigensolver
      st = launch_gram_raw(p, raw, raw_stride, (n_windows - 1) * slot_stride + p.T, w0 * slot_stride, slot_stride,
                           nw, &parts, s);
      p.sm_budget = 0;
      if (st != DH_OK) return st;
      if ((st = launch_reduce_raw(p, nw, parts, w0, s)) != DH_OK) return st;
    } else if (p.cov_mode == 2) {
      const Plan *o = p.band_owner;
      if (!o || o->band_frames == 0 || fs < o->band_first ||
          (long long)fs + (long long)(nw - 1) * slot_stride + p.T > (long long)o->band_first + o->band_frames)
        return DH_ERR_STATE;  // the windows are not inside the store's current band
      if ((st = launch_band_cov(p, *o, fs, slot_stride, nw, w0, s)) != DH_OK) return st;
    } else {
      p.sm_budget = g > 0 ? p.num_sms - nws[g - 1] : 0;  // beside the previous group's eigensolver
      st = p.prec == DH_PREC_FP32 ? launch_gram_simt(p, fs, slot_stride, nw, &parts, s)
                                  : launch_gram_tc(p, fs, slot_stride, nw, &parts, s);
      p.sm_budget = 0;
      if (st != DH_OK) return st;
      if ((st = launch_reduce(p, nw, parts, w0, s)) != DH_OK) return st;
    }
    DH_CUDA_TRY(cudaEventRecord(p.ev_grp[g], s));
    DH_CUDA_TRY(cudaStreamWaitEvent(p.aux, p.ev_grp[g], 0));
    st = launch_jacobi(p, nw, k0, k1, nop, eig_user ? eig_user + (long long)w0 * p.T : nullptr, w0, p.aux,
                       span.G > 0 ? &span : nullptr);
    if (st != DH_OK) return st;
    if (b0 >= 0 && (st = launch_svd_fourier_operand(p, nw, k0, k1, b0, b1, nop, w0, p.aux)) != DH_OK)
      return st;
    if (p.residual && (st = launch_mu_coef(p, nw, k0, k1, nop, w0, p.resid_ucol != 0, p.aux)) != DH_OK) return st;
    DH_CUDA_TRY(cudaEventRecord(p.ev_jac[g], p.aux));
  }
  for (int g = 0; g < G; ++g) {
    DH_CUDA_TRY(cudaStreamWaitEvent(s, p.ev_jac[g], 0));
    const int fs = first_slot + w0s[g] * slot_stride;
    float *img = images + (long long)w0s[g] * p.npix;
    // beside the next group's eigensolver. At T = 32 an eigensolver CTA (50.7 KB of shared
    // memory) fits beside one projection CTA (99.6 KB, two per SM otherwise), so whichever
    // launch comes first, 2 x SMs - (eigensolver CTAs) projection CTAs stay resident: a
    // budget of SMs - CTAs / 2 (measured: 1.75 -> 1.64 ms for the two projections of a
    // 64-window step). Elsewhere each eigensolver CTA keeps a whole SM.
    p.sm_budget = g + 1 < G ? p.num_sms - (p.T == 32 ? nws[g + 1] / 2 : nws[g + 1]) : 0;
    if (span.G > 0)
      st = launch_project_span(p, span, fs, nws[g], img, w0s[g], s);
    else
      st = p.prec == DH_PREC_FP32 ? launch_project_simt(p, fs, slot_stride, nws[g], nop, img, w0s[g], s)
                                  : launch_project_tc(p, fs, slot_stride, nws[g], nop, img, w0s[g], s);
    p.sm_budget = 0;
    if (st != DH_OK) return st;
  }
  return DH_OK;
}

}  // namespace

void note_stream(Plan &p, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    p.touched_all = true;  // a graph's launch stream is not known here
    return;
  }
  for (int i = 0; i < p.n_touched; ++i)
    if (p.touched[i] == s) return;
  if (p.n_touched < Plan::kMaxTouched) p.touched[p.n_touched++] = s;
  else p.touched_all = true;
}

namespace {

struct Busy {
  std::atomic<int> &b;
  bool ok;
  explicit Busy(std::atomic<int> &x) : b(x) { int z = 0; ok = b.compare_exchange_strong(z, 1); }
  ~Busy() { if (ok) b.store(0); }
};

// Branch streams of the batch executor, one set per device: a batch forks branches from the
// caller's stream and joins them back before returning.
struct Executor {
  static constexpr int kBranches = 8;
  static constexpr int kMaxItems = 64;
  std::mutex mu;
  cudaStream_t st[kBranches] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kBranches] = {};
  cudaEvent_t ev[2 * kMaxItems] = {};  // after each item's render part and windows part
  bool ready = false;

  cudaError_t init() {
    if (ready) return cudaSuccess;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int b = 0; b < kBranches && e == cudaSuccess; ++b) {
      e = cudaStreamCreateWithFlags(&st[b], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming);
    }
    for (int k = 0; k < 2 * kMaxItems && e == cudaSuccess; ++k)
      e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    ready = e == cudaSuccess;
    return e;
  }
};

Executor &executor(int device) {
  static std::mutex mu;
  static std::map<int, Executor *> per_device;
  std::lock_guard<std::mutex> lk(mu);
  Executor *&x = per_device[device];
  if (!x) x = new Executor();  // lives for the process: streams outlast every plan
  return *x;
}

}  // namespace

Plan &plan_of(dh_plan *h) { return h->p; }

// Entry points of the serving runtime (server.cu) into one plan, under the plan's guard.
dh_status plan_pca(dh_plan *h, int first_slot, int slot_stride, int n_windows, int k0, int k1,
                   float *images, double *eigvals, cudaStream_t s) {
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  note_stream(h->p, s);
  return pca_impl(h->p, nullptr, 0, first_slot, slot_stride, n_windows, k0, k1, images, eigvals, s);
}

dh_status plan_render(dh_plan *h, const uint16_t *frames, long long stride, int n, int slot0,
                      cudaStream_t s) {
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  note_stream(h->p, s);
  return launch_render(h->p, frames, stride, n, slot0, s);
}

}  // namespace dh

using namespace dh;

extern "C" {

const char *dh_version(void) { return "libdh 0.1 (sm_103a)"; }

const char *dh_last_error(void) { return g_last_error.c_str(); }

const char *dh_status_string(dh_status s) {
  switch (s) {
    case DH_OK: return "ok";
    case DH_ERR_INVALID_ARG: return "invalid argument";
    case DH_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case DH_ERR_OOM: return "out of device memory";
    case DH_ERR_CUDA: return "CUDA error";
    case DH_ERR_TIMEOUT: return "device-side wait timed out";
    case DH_ERR_FRAME_GAP: return "frame sequence gap";
    case DH_ERR_STATE: return "plan busy or in the wrong state";
  }
  return "unknown status";
}

dh_status dh_plan_create(dh_plan_t *out, int nx, int ny, double lambda_m, double z_m,
                         double pitch_m, int T) {
  if (!out) return DH_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(std::isfinite(lambda_m) && lambda_m > 0) || !(std::isfinite(z_m) && z_m > 0) ||
      !(std::isfinite(pitch_m) && pitch_m > 0))
    return DH_ERR_INVALID_ARG;
  if (!pow2_in_range(nx) || !pow2_in_range(ny) || !(T == 16 || T == 32 || T == 64))
    return DH_ERR_UNSUPPORTED_SIZE;
  dh_plan *h = new (std::nothrow) dh_plan();
  if (!h) return DH_ERR_OOM;
  Plan &p = h->p;
  p.nx = nx; p.ny = ny; p.T = T;
  p.lognx = ilog2(nx); p.logny = ilog2(ny);
  p.npix = (long long)nx * ny;
  p.lambda = lambda_m; p.z = z_m; p.pitch = pitch_m;
  p.a = pitch_m * pitch_m / (lambda_m * z_m);
  p.max_frames = T;
  p.max_windows = 1;
  p.band_owner = &p;
  cudaError_t e = cudaGetDevice(&p.device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, p.device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p.aux, cudaStreamNonBlocking);
  for (int k = 0; k < Plan::kMaxGroups && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&p.ev_grp[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.ev_jac[k], cudaEventDisableTiming);
  }
  dh_status st = e == cudaSuccess ? DH_OK : fail_cuda(e);
  if (st == DH_OK) {
    std::vector<float2> cx = chirp_table(nx, p.a), cy = chirp_table(ny, p.a);
    std::vector<float2> twx(twiddle_len(p.lognx)), twy(twiddle_len(p.logny));
    build_twiddles(p.lognx, twx.data());
    build_twiddles(p.logny, twy.data());
    if ((st = dalloc(p, &p.d_cx, cx.size() * sizeof(float2))) == DH_OK &&
        (st = dalloc(p, &p.d_cy, cy.size() * sizeof(float2))) == DH_OK &&
        (st = dalloc(p, &p.d_twx, twx.size() * sizeof(float2))) == DH_OK &&
        (st = dalloc(p, &p.d_twy, twy.size() * sizeof(float2))) == DH_OK &&
        (st = dalloc(p, &p.d_status, sizeof(uint32_t))) == DH_OK &&
        (st = dalloc(p, &p.d_sync, sizeof(unsigned) * (2 + 2 * 64))) == DH_OK) {
      cudaError_t c = cudaMemcpy(p.d_cx, cx.data(), cx.size() * sizeof(float2), cudaMemcpyHostToDevice);
      if (c == cudaSuccess) c = cudaMemcpy(p.d_cy, cy.data(), cy.size() * sizeof(float2), cudaMemcpyHostToDevice);
      if (c == cudaSuccess) c = cudaMemcpy(p.d_twx, twx.data(), twx.size() * sizeof(float2), cudaMemcpyHostToDevice);
      if (c == cudaSuccess) c = cudaMemcpy(p.d_twy, twy.data(), twy.size() * sizeof(float2), cudaMemcpyHostToDevice);
      if (c == cudaSuccess) c = cudaMemset(p.d_status, 0, sizeof(uint32_t));
      if (c == cudaSuccess) c = cudaMemset(p.d_sync, 0, sizeof(unsigned) * (2 + 2 * 64));
      if (c == cudaSuccess && tc_render_sizes(p)) {
        std::vector<char> tct(tc_tables_bytes());
        build_tc_tables(tct.data());
        st = dalloc(p, &p.d_tc, tct.size());
        if (st == DH_OK) c = cudaMemcpy(p.d_tc, tct.data(), tct.size(), cudaMemcpyHostToDevice);
      }
      if (st == DH_OK) st = c == cudaSuccess ? alloc_store(p) : fail_cuda(c);
    }
  }
  if (st != DH_OK) {
    dh_destroy(h);
    return st;
  }
  *out = h;
  return DH_OK;
}

namespace {
// Frees a plan once neither the caller's handle nor a view refers to it any more.
void release(dh_plan_t h) {
  if (!h || h->refs.fetch_sub(1) != 1) return;
  Plan &p = h->p;
  cudaDeviceSynchronize();
  free_store(p);
  profile_free(p);
  for (int k = 0; k < Plan::kMaxGroups; ++k) {
    if (p.ev_grp[k]) cudaEventDestroy(p.ev_grp[k]);
    if (p.ev_jac[k]) cudaEventDestroy(p.ev_jac[k]);
  }
  if (p.aux) cudaStreamDestroy(p.aux);
  Plan::HostPipe &q = p.pipe;
  if (q.up) cudaStreamDestroy(q.up);
  if (q.down) cudaStreamDestroy(q.down);
  for (cudaEvent_t ev : {q.start, q.done, q.finished, q.copied[0], q.copied[1], q.freed[0], q.freed[1]})
    if (ev) cudaEventDestroy(ev);
  dfree(q.stage[0]); dfree(q.stage[1]); dfree(q.pstage[0]); dfree(q.pstage[1]); dfree(q.img); dfree(q.eig);
  dfree(p.d_band); dfree(p.d_band_part);
  dfree(p.d_cx); dfree(p.d_cy); dfree(p.d_twx); dfree(p.d_twy); dfree(p.d_status); dfree(p.d_sync);
  dfree(p.d_tc);
  dh_plan *base = h->base;
  delete h;
  if (base) {
    base->views.fetch_sub(1);
    release(base);
  }
}
}  // namespace

void dh_destroy(dh_plan_t h) { release(h); }

dh_status dh_plan_create_view(dh_plan_t *out, dh_plan_t base_h, int T) {
  if (!out) return DH_ERR_INVALID_ARG;
  *out = nullptr;
  if (!base_h) return DH_ERR_INVALID_ARG;
  if (!(T == 16 || T == 32 || T == 64)) return DH_ERR_UNSUPPORTED_SIZE;
  while (base_h->base) base_h = base_h->base;  // a view of a view reads the same store
  const Plan &b = base_h->p;
  if (T > b.max_frames) return DH_ERR_INVALID_ARG;
  dh_plan *h = new (std::nothrow) dh_plan();
  if (!h) return DH_ERR_OOM;
  Plan &p = h->p;
  p.is_view = true;
  p.nx = b.nx; p.ny = b.ny; p.T = T; p.lognx = b.lognx; p.logny = b.logny; p.npix = b.npix;
  p.lambda = b.lambda; p.z = b.z; p.pitch = b.pitch; p.a = b.a;
  p.prec = b.prec;
  p.device = b.device; p.num_sms = b.num_sms;
  p.max_frames = b.max_frames;
  p.max_windows = 1;
  base_h->refs.fetch_add(1);
  base_h->views.fetch_add(1);
  h->base = base_h;
  p.band_owner = &base_h->p;
  cudaError_t e = cudaStreamCreateWithFlags(&p.aux, cudaStreamNonBlocking);
  for (int k = 0; k < Plan::kMaxGroups && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&p.ev_grp[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.ev_jac[k], cudaEventDisableTiming);
  }
  dh_status st = e == cudaSuccess ? dalloc(p, &p.d_status, sizeof(uint32_t)) : fail_cuda(e);
  if (st == DH_OK) {
    cudaError_t c = cudaMemset(p.d_status, 0, sizeof(uint32_t));
    st = c == cudaSuccess ? alloc_store(p, &b) : fail_cuda(c);
  }
  if (st != DH_OK) {
    release(h);
    return st;
  }
  *out = h;
  return DH_OK;
}

dh_status dh_plan_set_precision(dh_plan_t h, dh_precision prec) {
  if (!h) return DH_ERR_INVALID_ARG;
  if (prec != DH_PREC_FP32 && prec != DH_PREC_FP16 && prec != DH_PREC_BF16) return DH_ERR_INVALID_ARG;
  // a view follows its base's storage; a base cannot change it under live views
  if (h->base || h->views.load() > 0) return DH_ERR_STATE;
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  DH_CUDA_TRY(cudaDeviceSynchronize());
  h->p.prec = prec;
  if (prec == DH_PREC_FP32) h->p.cov_mode = 0;
  return alloc_store(h->p);
}

dh_status dh_plan_reserve(dh_plan_t h, int max_frames, int max_windows) {
  if (!h || max_frames < h->p.T || max_windows < 1) return DH_ERR_INVALID_ARG;
  if (h->base) {
    // a view reserves windows only; its slots are the base's
    if (max_frames > h->base->p.max_frames) return DH_ERR_INVALID_ARG;
  } else if (h->views.load() > 0 && max_frames != h->p.max_frames) {
    return DH_ERR_STATE;
  }
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  DH_CUDA_TRY(cudaDeviceSynchronize());
  h->p.max_windows = max_windows;
  // a view's slots are its base's, and a base with live views keeps its store in place
  // (the views hold its address): only the per-window buffers change
  if (h->base || h->views.load() > 0) return alloc_windows(h->p);
  h->p.max_frames = max_frames;
  return alloc_store(h->p);
}

size_t dh_plan_device_bytes(dh_plan_t h) { return h ? h->p.bytes : 0; }

dh_status dh_plan_get_option(dh_plan_t h, int option, int *value) {
  if (!h || !value) return DH_ERR_INVALID_ARG;
  switch (option) {
    case DH_OPT_RENDER_SCHEDULE: *value = h->p.render_mode; return DH_OK;
    case DH_OPT_RENDER_RING: *value = h->p.render_ring; return DH_OK;
    case DH_OPT_RENDER_LAG: *value = h->p.render_lag; return DH_OK;
    case DH_OPT_COVARIANCE: *value = h->p.cov_mode; return DH_OK;
    case DH_OPT_PROJECTION: *value = h->p.proj_mode; return DH_OK;
    case DH_OPT_WINDOW_GROUPS: *value = h->p.group_mode; return DH_OK;
    case DH_OPT_TEST_STALL: *value = h->p.test_stall; return DH_OK;
    case DH_OPT_RENDER_FFT: *value = h->p.render_fft; return DH_OK;
    case DH_OPT_FFT_RADIX: *value = h->p.fft_radix; return DH_OK;
    case DH_OPT_GRAM_UNITS: *value = h->p.gram_units; return DH_OK;
    case DH_OPT_RESIDUAL: *value = h->p.residual; return DH_OK;
  }
  return DH_ERR_INVALID_ARG;
}

// The autotuner. Render time does not depend on the pixel values (no data-dependent control
// flow), nor does the covariance's, so every candidate is timed on zero frames (best of
// three after a warm-up) and the fastest kept:
//   1. the DFT arithmetic of Eq. 1: the CUDA-core FFT at each length's default radix, at the
//      alternative radix where one is instantiated, and the tensor-core DFT stages (1024^2);
//   2. for the CUDA-core FFT, the schedule: chunks, and the persistent ring at the automatic
//      lag, half of it and twice it (ring twice the lag), and the automatic ring with one
//      frame more lag;
//   3. for 16-bit storage, the covariance's split-K units: the default for the frame size,
//      half and twice it (timed on up to 32 windows of the store).
// Schedules give bitwise the same holograms; the radix, the DFT arithmetic and the split-K
// units change only the rounding.
dh_status dh_plan_autotune(dh_plan_t h, int n_frames, void *stream) {
  if (!h || n_frames < 1) return DH_ERR_INVALID_ARG;
  Plan &p = h->p;
  if (p.is_view) return DH_ERR_STATE;
  if (n_frames > p.max_frames) n_frames = p.max_frames;
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint16_t *zeros = nullptr;
  DH_CUDA_TRY(cudaMalloc(&zeros, (size_t)n_frames * p.npix * sizeof(uint16_t)));
  const int saved[6] = {p.render_mode, p.render_ring, p.render_lag, p.render_fft, p.fft_radix, p.gram_units};
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaMemsetAsync(zeros, 0, (size_t)n_frames * p.npix * sizeof(uint16_t), s);
  dh_status st = e == cudaSuccess ? DH_OK : fail_cuda(e);
  // best of three timed runs of f() after a warm-up, in ms (1e30 on failure)
  auto time_of = [&](auto f) -> float {
    if (st != DH_OK || (st = f()) != DH_OK) return 1e30f;
    float tmin = 1e30f;
    for (int rep = 0; rep < 3 && st == DH_OK; ++rep) {
      e = cudaEventRecord(a, s);
      if (e == cudaSuccess) st = f();
      if (st == DH_OK && e == cudaSuccess) e = cudaEventRecord(b, s);
      if (st == DH_OK && e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (st == DH_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e != cudaSuccess && st == DH_OK) st = fail_cuda(e);
      if (st == DH_OK && ms < tmin) tmin = ms;
    }
    return st == DH_OK ? tmin : 1e30f;
  };
  auto render = [&]() { return launch_render(p, zeros, p.npix, n_frames, 0, s); };

  // 1. DFT arithmetic, each with the default schedule
  struct Fft { int fft, radix; };
  std::vector<Fft> ffts = {{1, 0}};
  for (int rx : {16, 32}) {
    const bool alt = (fft_spec_for(p.lognx, rx) != p.lognx) || (fft_spec_for(p.logny, rx) != p.logny);
    if (alt) ffts.push_back({1, rx});
  }
  if (p.d_tc) ffts.push_back({2, 0});
  p.render_mode = 0; p.render_ring = 0; p.render_lag = 0;
  float best = 1e30f;
  Fft fpick = {1, 0};
  for (const Fft &f : ffts) {
    if (st != DH_OK) break;
    p.render_fft = f.fft;
    if ((st = set_fft_radix(p, f.radix)) != DH_OK) break;
    const float ms = time_of(render);
    if (ms < best) { best = ms; fpick = f; }
  }
  if (st == DH_OK) {
    p.render_fft = fpick.fft;
    st = set_fft_radix(p, fpick.radix);
  }

  // 2. schedules of the CUDA-core FFT
  struct Cand { int mode, ring, lag; };
  Cand pick = {0, 0, 0};
  if (st == DH_OK && p.render_fft != 2) {
    std::vector<Cand> cands = {{1, 0, 0}};
    // automatic lag of this plan (grid of 2 CTAs per SM, the persistent kernel's residency)
    const int items = render_items_per_frame(p);
    const long long grid = 2ll * p.num_sms;
    const int lag = (int)((3 * grid + 2ll * items - 1) / (2ll * items));
    for (int l : {lag, lag / 2, 2 * lag})
      if (l >= 1 && 2 * l <= 64 && 2 * l <= p.mid_frames) cands.push_back({0, 2 * l, l});
    // one frame more lag in the same ring (a larger ring spills the intermediate from L2)
    if (lag >= 2 && 2 * lag <= 64 && 2 * lag <= p.mid_frames) cands.push_back({0, 2 * lag, lag + 1});
    if (p.mid_frames >= 3 && lag == 1) cands.push_back({0, 3, 1});
    best = 1e30f;
    for (const Cand &c : cands) {
      p.render_mode = c.mode; p.render_ring = c.ring; p.render_lag = c.lag;
      const float ms = time_of(render);
      if (ms < best) { best = ms; pick = c; }
    }
  }
  p.render_mode = pick.mode; p.render_ring = pick.ring; p.render_lag = pick.lag;

  // 3. split-K units of the tensor-core covariance (16-bit storage)
  const int n_win = std::min(std::min(p.max_windows, p.max_frames / p.T), 32);
  if (st == DH_OK && p.prec != DH_PREC_FP32 && n_win >= 1) {
    const int u0 = gram_tc_default_units(p.npix);
    int upick = 0;
    best = 1e30f;
    for (int u : {u0, u0 / 2, 2 * u0, u0 / 4}) {
      if (u < 1 || p.npix % (256ll * u) != 0) continue;
      if ((st = set_gram_units(p, u == u0 ? 0 : u)) != DH_OK) break;
      int parts = 0;
      const float ms = time_of([&]() { return launch_gram_tc(p, 0, p.T, n_win, &parts, s); });
      if (ms < best) { best = ms; upick = u == u0 ? 0 : u; }
    }
    if (st == DH_OK) st = set_gram_units(p, upick);
  }
  if (st != DH_OK) {
    p.render_mode = saved[0]; p.render_ring = saved[1]; p.render_lag = saved[2]; p.render_fft = saved[3];
    set_fft_radix(p, saved[4]);
    set_gram_units(p, saved[5]);
  }
  cudaStreamSynchronize(s);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(zeros);
  return st;
}

dh_status dh_plan_set_option(dh_plan_t h, int option, int value) {
  if (!h) return DH_ERR_INVALID_ARG;
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  switch (option) {
    case DH_OPT_RENDER_SCHEDULE:
      if (value != 0 && value != 1) return DH_ERR_INVALID_ARG;
      h->p.render_mode = value;
      return DH_OK;
    case DH_OPT_RENDER_RING:
      if (value < 0 || value > 64 || value == 1) return DH_ERR_INVALID_ARG;
      h->p.render_ring = value;
      return DH_OK;
    case DH_OPT_RENDER_LAG:
      if (value < 0 || value > 63) return DH_ERR_INVALID_ARG;
      h->p.render_lag = value;
      return DH_OK;
    case DH_OPT_COVARIANCE:
      if (value < 0 || value > 2) return DH_ERR_INVALID_ARG;
      if (value != 0 && h->p.prec == DH_PREC_FP32) return DH_ERR_STATE;  // tensor-core paths only
      h->p.cov_mode = value;
      return DH_OK;
    case DH_OPT_PROJECTION:
      if (value != 0 && value != 1) return DH_ERR_INVALID_ARG;
      h->p.proj_mode = value;
      return DH_OK;
    case DH_OPT_WINDOW_GROUPS:
      if (value != 0 && value != 1) return DH_ERR_INVALID_ARG;
      h->p.group_mode = value;
      return DH_OK;
    case DH_OPT_TEST_STALL:
      if (value < 0 || value > 100000000) return DH_ERR_INVALID_ARG;
      h->p.test_stall = value;
      return DH_OK;
    case DH_OPT_RENDER_FFT:
      if (value < 0 || value > 2) return DH_ERR_INVALID_ARG;
      if (value == 2 && !h->p.d_tc) return DH_ERR_UNSUPPORTED_SIZE;
      h->p.render_fft = value;
      return DH_OK;
    case DH_OPT_FFT_RADIX:
      return set_fft_radix(h->p, value);
    case DH_OPT_GRAM_UNITS:
      return set_gram_units(h->p, value);
    case DH_OPT_RESIDUAL:
      return set_residual(h->p, value);
  }
  return DH_ERR_INVALID_ARG;
}

size_t dh_plan_footprint(int nx, int ny, int T, dh_precision prec, int max_frames, int max_windows) {
  if (!pow2_in_range(nx) || !pow2_in_range(ny) || !(T == 16 || T == 32 || T == 64) ||
      max_frames < T || max_windows < 1 ||
      (prec != DH_PREC_FP32 && prec != DH_PREC_FP16 && prec != DH_PREC_BF16))
    return 0;
  Plan p;
  p.nx = nx; p.ny = ny; p.T = T;
  p.lognx = ilog2(nx); p.logny = ilog2(ny);
  p.npix = (long long)nx * ny;
  p.prec = prec;
  p.max_frames = max_frames;
  p.max_windows = max_windows;
  return store_sizes(p).total();
}

dh_status dh_render_frames(dh_plan_t h, const uint16_t *frames_dev, int64_t frame_stride_elems,
                           int n_frames, int first_slot, void *stream) {
  if (!h || !frames_dev || n_frames < 1 || first_slot < 0) return DH_ERR_INVALID_ARG;
  Plan &p = h->p;
  if (frame_stride_elems < p.npix || (long long)first_slot + n_frames > p.max_frames)
    return DH_ERR_INVALID_ARG;
  if (p.is_view) return DH_ERR_STATE;  // views render nothing: render through the base plan
  // frames are read with 16-byte vector loads
  if ((reinterpret_cast<uintptr_t>(frames_dev) & 15u) != 0 || (frame_stride_elems & 7) != 0)
    return DH_ERR_INVALID_ARG;
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  note_stream(p, static_cast<cudaStream_t>(stream));
  return launch_render(p, frames_dev, frame_stride_elems, n_frames, first_slot,
                       static_cast<cudaStream_t>(stream));
}

dh_status dh_pca_windows(dh_plan_t h, int first_slot, int slot_stride, int n_windows, int k0,
                         int k1, float *images_dev, double *eigvals_dev, void *stream) {
  if (!h || !images_dev || n_windows < 1 || first_slot < 0 || slot_stride < 1) return DH_ERR_INVALID_ARG;
  Plan &p = h->p;
  if (k0 < 0 || k1 < k0 || k1 >= p.T) return DH_ERR_INVALID_ARG;
  if (n_windows > p.max_windows) return DH_ERR_INVALID_ARG;
  if ((long long)first_slot + (long long)(n_windows - 1) * slot_stride + p.T > p.max_frames)
    return DH_ERR_INVALID_ARG;
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  note_stream(p, static_cast<cudaStream_t>(stream));
  return pca_impl(p, nullptr, 0, first_slot, slot_stride, n_windows, k0, k1, images_dev, eigvals_dev,
                  static_cast<cudaStream_t>(stream));
}

dh_status dh_svd_fourier_windows(dh_plan_t h, int first_slot, int slot_stride, int n_windows, int k0,
                                int k1, int b0, int b1, float *images_dev, double *eigvals_dev,
                                void *stream) {
  if (!h || !images_dev || n_windows < 1 || first_slot < 0 || slot_stride < 1) return DH_ERR_INVALID_ARG;
  Plan &p = h->p;
  if (k0 < 0 || k1 < k0 || k1 >= p.T || b0 < 0 || b1 < b0 || b1 >= p.T) return DH_ERR_INVALID_ARG;
  if (n_windows > p.max_windows) return DH_ERR_INVALID_ARG;
  if ((long long)first_slot + (long long)(n_windows - 1) * slot_stride + p.T > p.max_frames)
    return DH_ERR_INVALID_ARG;
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  note_stream(p, static_cast<cudaStream_t>(stream));
  return pca_impl(p, nullptr, 0, first_slot, slot_stride, n_windows, k0, k1, images_dev, eigvals_dev,
                  static_cast<cudaStream_t>(stream), b0, b1);
}

dh_status dh_fourier_windows(dh_plan_t h, int first_slot, int slot_stride, int n_windows, int k0,
                            int k1, float *images_dev, void *stream) {
  if (!h || !images_dev || n_windows < 1 || first_slot < 0 || slot_stride < 1) return DH_ERR_INVALID_ARG;
  Plan &p = h->p;
  if (k0 < 0 || k1 < k0 || k1 >= p.T) return DH_ERR_INVALID_ARG;
  if ((long long)first_slot + (long long)(n_windows - 1) * slot_stride + p.T > p.max_frames)
    return DH_ERR_INVALID_ARG;
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  note_stream(p, static_cast<cudaStream_t>(stream));
  return launch_fourier(p, first_slot, slot_stride, n_windows, k0, k1, images_dev,
                        static_cast<cudaStream_t>(stream));
}

dh_status dh_band_gram(dh_plan_t h, int first_slot, int n_frames, void *stream) {
  if (!h || first_slot < 0 || n_frames < 1) return DH_ERR_INVALID_ARG;
  dh_plan *root = h;
  while (root->base) root = root->base;
  Plan &p = root->p;
  if (p.prec == DH_PREC_FP32) return DH_ERR_STATE;
  if ((long long)first_slot + n_frames > p.max_frames) return DH_ERR_INVALID_ARG;
  Busy g(root->busy);
  if (!g.ok) return DH_ERR_STATE;
  const int blocks = (n_frames + 63) / 64;
  if (blocks > p.band_cap) {  // first use (or a longer band): allocate
    DH_CUDA_TRY(cudaDeviceSynchronize());
    dfree(p.d_band); dfree(p.d_band_part);
    const size_t cell = 2ull * 128 * 128 * sizeof(double);
    p.bytes -= (size_t)p.band_cap * cell * (1 + band_units(p.npix));
    p.band_cap = 0;
    dh_status st;
    if ((st = dalloc(p, &p.d_band, (size_t)blocks * cell)) != DH_OK) return st;
    if ((st = dalloc(p, &p.d_band_part, (size_t)blocks * band_units(p.npix) * cell)) != DH_OK) return st;
    p.band_cap = blocks;
  }
  note_stream(p, static_cast<cudaStream_t>(stream));
  dh_status st = launch_band_gram(p, first_slot, n_frames, static_cast<cudaStream_t>(stream));
  if (st != DH_OK) return st;
  p.band_first = first_slot;
  p.band_frames = n_frames;
  return DH_OK;
}

dh_status dh_render_stack(dh_plan_t h, const uint16_t *frames_dev, int64_t frame_stride_elems,
                          void *stream) {
  if (!h) return DH_ERR_INVALID_ARG;
  return dh_render_frames(h, frames_dev, frame_stride_elems, h->p.T, 0, stream);
}

dh_status dh_pca_window(dh_plan_t h, int k0, int k1, float *image_dev, double *eigvals_host,
                        void *stream) {
  if (!h) return DH_ERR_INVALID_ARG;
  dh_status st = dh_pca_windows(h, 0, h->p.T, 1, k0, k1, image_dev, nullptr, stream);
  if (st != DH_OK || !eigvals_host) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DH_CUDA_TRY(cudaMemcpyAsync(eigvals_host, h->p.d_lam, sizeof(double) * h->p.T,
                              cudaMemcpyDeviceToHost, s));
  DH_CUDA_TRY(cudaStreamSynchronize(s));
  return DH_OK;
}

dh_status dh_pca_batch(dh_plan_t h, const uint16_t *frames_dev, int64_t frame_stride_elems,
                       int n_windows, int window_stride_frames, int k0, int k1, float *images_dev,
                       double *eigvals_dev, void *stream) {
  if (!h || !frames_dev || !images_dev || n_windows < 1 || window_stride_frames < 1) return DH_ERR_INVALID_ARG;
  Plan &p = h->p;
  if (k0 < 0 || k1 < k0 || k1 >= p.T) return DH_ERR_INVALID_ARG;
  const long long nf = (long long)(n_windows - 1) * window_stride_frames + p.T;
  if (nf > p.max_frames || n_windows > p.max_windows) return DH_ERR_INVALID_ARG;
  if (frame_stride_elems < p.npix || (frame_stride_elems & 7) != 0 ||
      (reinterpret_cast<uintptr_t>(frames_dev) & 15u) != 0)
    return DH_ERR_INVALID_ARG;
  if (p.is_view) return DH_ERR_STATE;
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  note_stream(p, static_cast<cudaStream_t>(stream));
  return pca_impl(p, frames_dev, frame_stride_elems, 0, window_stride_frames, n_windows, k0, k1,
                  images_dev, eigvals_dev, static_cast<cudaStream_t>(stream), -1, -1, frames_dev,
                  frame_stride_elems);
}

// The host pipeline of dh_pca_batch_host and dh_pca_batch_host_packed12. `frames_host` holds
// uint16 frames `host_stride` elements apart, or (packed) Mono12p frames `host_stride` bytes
// apart, which are copied as bytes and expanded on the device into the uint16 staging buffer.
static dh_status host_batch(dh_plan_t h, const void *frames_host, int64_t host_stride, bool packed,
                            int n_windows, int window_stride_frames, int k0, int k1, float *images_host,
                            double *eigvals_host, void *stream) {
  if (!h || !frames_host || !images_host || n_windows < 1 || window_stride_frames < 1) return DH_ERR_INVALID_ARG;
  Plan &p = h->p;
  if (p.is_view) return DH_ERR_STATE;
  if (k0 < 0 || k1 < k0 || k1 >= p.T) return DH_ERR_INVALID_ARG;
  const int ws = window_stride_frames, T = p.T;
  const long long nf_all = (long long)(n_windows - 1) * ws + T;
  if (nf_all > p.max_frames || n_windows > p.max_windows) return DH_ERR_INVALID_ARG;
  if (packed ? (host_stride < p.npix / 2 * 3 || (host_stride & 3) != 0)
             : (host_stride < p.npix || (host_stride & 7) != 0))
    return DH_ERR_INVALID_ARG;
  // the uint16 frames the render reads: the caller's stride, or dense after expansion
  const int64_t frame_stride_elems = packed ? p.npix : host_stride;
  const size_t host_frame_bytes = packed ? (size_t)host_stride : (size_t)host_stride * sizeof(uint16_t);
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  // groups of windows whose new frames fit a 256-frame staging buffer (one window per group
  // when windows are further apart than T: only its own frames are copied)
  const int cap = T > 256 ? T : 256;
  const int G = ws > T ? 1 : (cap - T) / ws + 1;
  Plan::HostPipe &q = p.pipe;
  const size_t stage_elems = (size_t)cap * frame_stride_elems;
  const size_t img_elems = (size_t)p.max_windows * p.npix, eig_elems = (size_t)p.max_windows * T;
  if (!q.up) {
    DH_CUDA_TRY(cudaStreamCreateWithFlags(&q.up, cudaStreamNonBlocking));
    DH_CUDA_TRY(cudaStreamCreateWithFlags(&q.down, cudaStreamNonBlocking));
    for (cudaEvent_t *ev : {&q.start, &q.done, &q.finished, &q.copied[0], &q.copied[1], &q.freed[0], &q.freed[1]})
      DH_CUDA_TRY(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
  }
  if (q.stage_elems < stage_elems) {
    DH_CUDA_TRY(cudaDeviceSynchronize());
    dfree(q.stage[0]); dfree(q.stage[1]);
    p.bytes -= 2 * q.stage_elems * sizeof(uint16_t);
    q.stage_elems = 0;
    dh_status st;
    if ((st = dalloc(p, &q.stage[0], stage_elems * sizeof(uint16_t))) != DH_OK) return st;
    if ((st = dalloc(p, &q.stage[1], stage_elems * sizeof(uint16_t))) != DH_OK) return st;
    q.stage_elems = stage_elems;
  }
  const size_t pstage_bytes = packed ? (size_t)cap * host_frame_bytes : 0;
  if (q.pstage_bytes < pstage_bytes) {  // the packed bytes' own staging buffers
    DH_CUDA_TRY(cudaDeviceSynchronize());
    dfree(q.pstage[0]); dfree(q.pstage[1]);
    p.bytes -= 2 * q.pstage_bytes;
    q.pstage_bytes = 0;
    dh_status st;
    if ((st = dalloc(p, &q.pstage[0], pstage_bytes)) != DH_OK) return st;
    if ((st = dalloc(p, &q.pstage[1], pstage_bytes)) != DH_OK) return st;
    q.pstage_bytes = pstage_bytes;
  }
  if (q.img_elems < img_elems || q.eig_elems < eig_elems) {
    DH_CUDA_TRY(cudaDeviceSynchronize());
    dfree(q.img); dfree(q.eig);
    p.bytes -= q.img_elems * sizeof(float) + q.eig_elems * sizeof(double);
    q.img_elems = q.eig_elems = 0;
    dh_status st;
    if ((st = dalloc(p, &q.img, img_elems * sizeof(float))) != DH_OK) return st;
    if ((st = dalloc(p, &q.eig, eig_elems * sizeof(double))) != DH_OK) return st;
    q.img_elems = img_elems; q.eig_elems = eig_elems;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  note_stream(p, s);
  DH_CUDA_TRY(cudaEventRecord(q.start, s));  // copies follow earlier work on the caller's stream
  DH_CUDA_TRY(cudaStreamWaitEvent(q.up, q.start, 0));
  DH_CUDA_TRY(cudaStreamWaitEvent(q.down, q.start, 0));
  long long rendered = 0;  // frames 0 .. rendered-1 are in their slots (ws <= T)
  for (int w0 = 0, grp = 0; w0 < n_windows; ++grp) {
    // full groups, then the last ones halve (G/2, G/4, ..., 1, 1): less work follows the last
    // copy, whose end the call cannot finish before (each window's result does not depend on
    // the grouping)
    const int left = n_windows - w0;
    const int nw = left > G ? G : left > 1 ? (left + 1) / 2 : left;
    long long f0, nf;
    if (ws > T) {
      f0 = (long long)w0 * ws;
      nf = T;
    } else {
      f0 = rendered;
      nf = (long long)(w0 + nw - 1) * ws + T - rendered;
      rendered += nf;
    }
    const int b = grp & 1;
    if (grp >= 2) DH_CUDA_TRY(cudaStreamWaitEvent(q.up, q.freed[b], 0));  // group grp-2 rendered
    const char *src = static_cast<const char *>(frames_host) + (size_t)f0 * host_frame_bytes;
    DH_CUDA_TRY(cudaMemcpyAsync(packed ? static_cast<void *>(q.pstage[b]) : static_cast<void *>(q.stage[b]), src,
                                (size_t)nf * host_frame_bytes, cudaMemcpyHostToDevice, q.up));
    DH_CUDA_TRY(cudaEventRecord(q.copied[b], q.up));
    DH_CUDA_TRY(cudaStreamWaitEvent(s, q.copied[b], 0));
    dh_status st;
    if (packed && (st = launch_unpack_mono12p(q.pstage[b], host_stride, p.npix, (int)nf, q.stage[b],
                                              frame_stride_elems, s)) != DH_OK)
      return st;
    st = launch_render(p, q.stage[b], frame_stride_elems, (int)nf, (int)f0, s);
    if (st != DH_OK) return st;
    // the raw-domain covariance reads the staged frames: only when the group's windows lie
    // wholly in them (windows T or more frames apart)
    st = pca_impl(p, nullptr, 0, w0 * ws, ws, nw, k0, k1, q.img + (size_t)w0 * p.npix,
                  eigvals_host ? q.eig + (size_t)w0 * T : nullptr, s, -1, -1,
                  ws >= T ? q.stage[b] : nullptr, frame_stride_elems);
    if (st != DH_OK) return st;
    DH_CUDA_TRY(cudaEventRecord(q.freed[b], s));
    DH_CUDA_TRY(cudaEventRecord(q.done, s));
    DH_CUDA_TRY(cudaStreamWaitEvent(q.down, q.done, 0));
    DH_CUDA_TRY(cudaMemcpyAsync(images_host + (size_t)w0 * p.npix, q.img + (size_t)w0 * p.npix,
                                (size_t)nw * p.npix * sizeof(float), cudaMemcpyDeviceToHost, q.down));
    if (eigvals_host)
      DH_CUDA_TRY(cudaMemcpyAsync(eigvals_host + (size_t)w0 * T, q.eig + (size_t)w0 * T,
                                  (size_t)nw * T * sizeof(double), cudaMemcpyDeviceToHost, q.down));
    w0 += nw;
  }
  DH_CUDA_TRY(cudaEventRecord(q.finished, q.down));
  DH_CUDA_TRY(cudaStreamWaitEvent(s, q.finished, 0));  // the caller's stream ends with the results
  return DH_OK;
}

dh_status dh_pca_batch_host(dh_plan_t h, const uint16_t *frames_host, int64_t frame_stride_elems,
                            int n_windows, int window_stride_frames, int k0, int k1, float *images_host,
                            double *eigvals_host, void *stream) {
  return host_batch(h, frames_host, frame_stride_elems, false, n_windows, window_stride_frames, k0, k1,
                    images_host, eigvals_host, stream);
}

dh_status dh_pca_batch_host_packed12(dh_plan_t h, const uint8_t *frames_host, int64_t frame_stride_bytes,
                                     int n_windows, int window_stride_frames, int k0, int k1, float *images_host,
                                     double *eigvals_host, void *stream) {
  return host_batch(h, frames_host, frame_stride_bytes, true, n_windows, window_stride_frames, k0, k1,
                    images_host, eigvals_host, stream);
}

dh_status dh_debug_hologram(dh_plan_t h, int slot, float *out_dev, void *stream) {
  if (!h || !out_dev || slot < 0 || slot >= h->p.max_frames) return DH_ERR_INVALID_ARG;
  return launch_hologram_to_f32(h->p, slot, out_dev, static_cast<cudaStream_t>(stream));
}

dh_status dh_debug_covariance(dh_plan_t h, int w, double *out_dev, void *stream) {
  if (!h || !out_dev || w < 0 || w >= h->p.max_windows) return DH_ERR_INVALID_ARG;
  const size_t n = (size_t)h->p.T * h->p.T * 2;
  DH_CUDA_TRY(cudaMemcpyAsync(out_dev, h->p.d_C + n * w, n * sizeof(double), cudaMemcpyDeviceToDevice,
                              static_cast<cudaStream_t>(stream)));
  return DH_OK;
}

dh_status dh_debug_eigvecs(dh_plan_t h, int w, double *out_dev, void *stream) {
  if (!h || !out_dev || w < 0 || w >= h->p.max_windows) return DH_ERR_INVALID_ARG;
  const size_t n = (size_t)h->p.T * h->p.T * 2;
  DH_CUDA_TRY(cudaMemcpyAsync(out_dev, h->p.d_V + n * w, n * sizeof(double), cudaMemcpyDeviceToDevice,
                              static_cast<cudaStream_t>(stream)));
  return DH_OK;
}

dh_status dh_profile_enable(dh_plan_t h, int on) {
  if (!h) return DH_ERR_INVALID_ARG;
  Busy g(h->busy);
  if (!g.ok) return DH_ERR_STATE;
  return profile_enable(h->p, on);
}

int dh_profile_read(dh_plan_t h, int n, const char **names, int *launches, double *total_ms) {
  if (!h) return 0;
  return profile_read(h->p, n, names, launches, total_ms);
}

dh_status dh_plan_status(dh_plan_t h, uint32_t *flags) {
  if (!h || !flags) return DH_ERR_INVALID_ARG;
  Plan &p = h->p;
  // wait for the plan's own work only: the streams its calls launched on, its second stream
  // and its host-copy streams; the whole device only if it lost track (see note_stream)
  if (p.touched_all) {
    DH_CUDA_TRY(cudaDeviceSynchronize());
  } else {
    for (int i = 0; i < p.n_touched; ++i) DH_CUDA_TRY(cudaStreamSynchronize(p.touched[i]));
    for (cudaStream_t q : {p.pipe.up, p.pipe.down})
      if (q) DH_CUDA_TRY(cudaStreamSynchronize(q));
  }
  // read and clear the word on the plan's own non-blocking stream (no implicit
  // synchronisation with the legacy default stream)
  DH_CUDA_TRY(cudaStreamSynchronize(p.aux));
  uint32_t v = 0;
  DH_CUDA_TRY(cudaMemcpyAsync(&v, p.d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, p.aux));
  DH_CUDA_TRY(cudaMemsetAsync(p.d_status, 0, sizeof(uint32_t), p.aux));
  DH_CUDA_TRY(cudaStreamSynchronize(p.aux));
  p.n_touched = 0;
  p.touched_all = false;
  *flags = v;
  return (v & DH_FLAG_WAIT_TIMEOUT) ? DH_ERR_TIMEOUT : DH_OK;
}

// ---------------------------------------------------------------- CUDA graphs
dh_status dh_graph_begin(void *stream) {
  if (!stream) return DH_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
  DH_CUDA_TRY(cudaStreamBeginCapture(static_cast<cudaStream_t>(stream), cudaStreamCaptureModeThreadLocal));
  return DH_OK;
}

dh_status dh_graph_end(void *stream, dh_graph_t *out) {
  if (!stream || !out) return DH_ERR_INVALID_ARG;
  *out = nullptr;
  cudaGraph_t graph = nullptr;
  DH_CUDA_TRY(cudaStreamEndCapture(static_cast<cudaStream_t>(stream), &graph));
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail_cuda(e);
  dh_graph *g = new (std::nothrow) dh_graph();
  if (!g) {
    cudaGraphExecDestroy(exec);
    return DH_ERR_OOM;
  }
  g->exec = exec;
  *out = g;
  return DH_OK;
}

dh_status dh_graph_launch(dh_graph_t g, void *stream) {
  if (!g || !g->exec) return DH_ERR_INVALID_ARG;
  DH_CUDA_TRY(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
  return DH_OK;
}

void dh_graph_destroy(dh_graph_t g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
}

// ---------------------------------------------------------------- batches
dh_status dh_batch_run(const dh_batch_item *items, int n_items, void *stream) {
  if (!items || n_items < 1 || n_items > Executor::kMaxItems) return DH_ERR_INVALID_ARG;
  // validate everything before launching anything
  std::vector<dh_plan *> plans, roots(n_items);
  for (int i = 0; i < n_items; ++i) {
    const dh_batch_item &it = items[i];
    if (!it.plan) return DH_ERR_INVALID_ARG;
    dh_plan *root = it.plan;
    while (root->base) root = root->base;
    roots[i] = root;
    const Plan &p = it.plan->p;
    if (it.frames_dev) {
      if (it.n_frames < 1 || it.render_slot < 0 || it.frame_stride_elems < p.npix ||
          (it.frame_stride_elems & 7) != 0 || (reinterpret_cast<uintptr_t>(it.frames_dev) & 15u) != 0 ||
          (long long)it.render_slot + it.n_frames > root->p.max_frames)
        return DH_ERR_INVALID_ARG;
    }
    if (it.n_windows < 0 || (it.n_windows == 0 && !it.frames_dev)) return DH_ERR_INVALID_ARG;
    if (it.n_windows > 0) {
      if (!it.images_dev || it.first_slot < 0 || it.slot_stride < 1 || it.n_windows > p.max_windows ||
          it.k0 < 0 || it.k1 < it.k0 || it.k1 >= p.T ||
          (long long)it.first_slot + (long long)(it.n_windows - 1) * it.slot_stride + p.T > p.max_frames)
        return DH_ERR_INVALID_ARG;
    }
    for (dh_plan *q : {it.plan, root}) {
      bool seen = false;
      for (dh_plan *y : plans) seen |= y == q;
      if (!seen) plans.push_back(q);
    }
  }
  // every plan involved is held for the duration of the enqueue
  std::vector<std::unique_ptr<Busy>> held;
  for (dh_plan *q : plans) {
    held.emplace_back(new Busy(q->busy));
    if (!held.back()->ok) return DH_ERR_STATE;
  }
  int device = 0;
  DH_CUDA_TRY(cudaGetDevice(&device));
  Executor &x = executor(device);
  std::lock_guard<std::mutex> lk(x.mu);
  DH_CUDA_TRY(x.init());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the branches join back into the caller's stream: waiting on it covers them
  for (dh_plan *q : plans) note_stream(q->p, s);
  // Branches: one per store for its renders, one per plan for its windows, in order of first
  // appearance (wrapping onto shared streams beyond kBranches, which only adds ordering).
  // The windows of different plans over one store (views) run concurrently once the store's
  // earlier renders are done; a later render of a store waits for its earlier readers.
  std::vector<const void *> keys;
  auto branch_of = [&](const void *key) {
    int k = 0;
    while (k < (int)keys.size() && keys[k] != key) ++k;
    if (k == (int)keys.size()) keys.push_back(key);
    return k % Executor::kBranches;
  };
  DH_CUDA_TRY(cudaEventRecord(x.fork, s));
  bool forked[Executor::kBranches] = {};
  auto stream_of = [&](int b) -> cudaStream_t {
    if (!forked[b]) {
      forked[b] = true;
      if (cudaStreamWaitEvent(x.st[b], x.fork, 0) != cudaSuccess) return nullptr;
    }
    return x.st[b];
  };
  dh_status st = DH_OK;
  for (int i = 0; i < n_items && st == DH_OK; ++i) {
    const dh_batch_item &it = items[i];
    dh_plan *root = roots[i];
    int store_render = -1;  // latest earlier render part of this store
    for (int j = i - 1; j >= 0 && store_render < 0; --j)
      if (roots[j] == root && items[j].frames_dev) store_render = 2 * j;
    if (it.frames_dev) {
      cudaStream_t bs = stream_of(branch_of(root));
      if (!bs) { st = fail_cuda(cudaGetLastError()); break; }
      // readers of this store since its last render finish first
      for (int j = i - 1; j >= 0; --j) {
        if (roots[j] != root) continue;
        if (items[j].n_windows > 0) {
          cudaError_t e = cudaStreamWaitEvent(bs, x.ev[2 * j + 1], 0);
          if (e != cudaSuccess) { st = fail_cuda(e); break; }
        }
        if (items[j].frames_dev) break;  // readers before that render waited for it already
      }
      if (st != DH_OK) break;
      st = launch_render(root->p, it.frames_dev, it.frame_stride_elems, it.n_frames, it.render_slot, bs);
      if (st == DH_OK) {
        cudaError_t e = cudaEventRecord(x.ev[2 * i], bs);
        if (e != cudaSuccess) st = fail_cuda(e);
      }
      store_render = 2 * i;
    }
    if (st == DH_OK && it.n_windows > 0) {
      cudaStream_t bs = stream_of(branch_of(it.plan));
      if (!bs) { st = fail_cuda(cudaGetLastError()); break; }
      if (store_render >= 0) {
        cudaError_t e = cudaStreamWaitEvent(bs, x.ev[store_render], 0);
        if (e != cudaSuccess) { st = fail_cuda(e); break; }
      }
      st = pca_impl(it.plan->p, nullptr, 0, it.first_slot, it.slot_stride, it.n_windows, it.k0, it.k1,
                    it.images_dev, it.eigvals_dev, bs);
      if (st == DH_OK) {
        cudaError_t e = cudaEventRecord(x.ev[2 * i + 1], bs);
        if (e != cudaSuccess) st = fail_cuda(e);
      }
    }
  }
  // join every forked branch, also after an error, so the caller's stream never runs ahead
  for (int b = 0; b < Executor::kBranches; ++b) {
    if (!forked[b]) continue;
    cudaError_t e = cudaEventRecord(x.join[b], x.st[b]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, x.join[b], 0);
    if (e != cudaSuccess && st == DH_OK) st = fail_cuda(e);
  }
  return st;
}

}  // extern "C"
