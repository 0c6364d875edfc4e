// The serving runtime (dh_server_*, include/dh.h): several synthetic or real camera streams,
// each with a device-resident plan, frame ring and output ring, admitted against an HBM
// budget. A push copies a stream's new frames to the device, renders them (Eq. 1) and, for
// every 32/64-frame window the push completes, runs Eqs. 4-7 and copies the image and the
// eigenvalues to pinned host memory; a host callback stamps the completion time. Every
// camera stream has its own CUDA stream, so windows of different streams overlap on the
// device as they become ready (continuous batching, no global queue).
#include "dh_internal.cuh"

#include <chrono>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <new>
#include <vector>

// launch pipeline of one plan's windows, defined with the plan ABI
struct dh_plan;
namespace dh {
dh_status plan_pca(dh_plan *h, int first_slot, int slot_stride, int n_windows, int k0, int k1,
                   float *images, double *eigvals, cudaStream_t s);
dh_status plan_render(dh_plan *h, const uint16_t *frames, long long stride, int n, int slot0,
                      cudaStream_t s);
}  // namespace dh

namespace {

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Done {
  int stream_id;
  int64_t window;
  int slot;
  double t_ready, t_done;
};

struct Pending {  // one in-flight window, handed to the completion callback
  dh_server *srv;
  int stream_id;
  int64_t window;
  int slot;
  double t_ready;
};

}  // namespace

struct CamStream {
  int id = 0;
  dh_plan_t plan = nullptr;
  int nx = 0, ny = 0, T = 0, k0 = 0, k1 = 0, ring = 0;
  long long npix = 0;
  cudaStream_t cs = nullptr;
  uint16_t *d_frames = nullptr;  // [2T][npix] device frame ring
  float *d_images = nullptr;     // [ring][npix]
  double *d_eig = nullptr;       // [ring][T]
  float *h_images = nullptr;     // pinned [ring][npix]
  double *h_eig = nullptr;       // pinned [ring][T]
  std::vector<int> slot_used;    // 1 from launch until dh_server_release
  int64_t next_frame = 0;
  size_t bytes = 0;              // device bytes charged to the budget
};

struct dh_server {
  size_t budget = 0, used = 0;
  int device = 0;
  std::string tune_path;  // autotune cache applied to admitted streams' plans (empty: none)
  bool tune_autotune = false;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  std::mutex mu;        // streams, budget
  std::mutex done_mu;   // completion queue (also taken by the driver's callback thread)
  std::map<int, CamStream *> streams;
  std::deque<Done> done;
  int next_id = 0;
};

namespace {

void CUDART_CB on_window_done(void *arg) {
  // runs on the CUDA driver's callback thread once the window's copies to the host ended;
  // no CUDA calls are allowed here
  Pending *p = static_cast<Pending *>(arg);
  dh_server *srv = p->srv;
  const double t = now_s(srv->t0);
  {
    std::lock_guard<std::mutex> lk(srv->done_mu);
    srv->done.push_back(Done{p->stream_id, p->window, p->slot, p->t_ready, t});
  }
  delete p;  // the record belonged to this callback alone
}

size_t stream_device_bytes(int nx, int ny, int T, dh_precision prec, int ring) {
  const size_t npix = (size_t)nx * ny;
  const size_t plan = dh_plan_footprint(nx, ny, T, prec, 2 * T, 1);
  if (!plan) return 0;
  return plan + (size_t)2 * T * npix * sizeof(uint16_t) + (size_t)ring * npix * sizeof(float) +
         (size_t)ring * T * sizeof(double);
}

void free_stream(CamStream *c) {
  if (c->cs) cudaStreamSynchronize(c->cs);  // every completion callback of the stream has run
  if (c->cs) cudaStreamDestroy(c->cs);
  if (c->d_frames) cudaFree(c->d_frames);
  if (c->d_images) cudaFree(c->d_images);
  if (c->d_eig) cudaFree(c->d_eig);
  if (c->h_images) cudaFreeHost(c->h_images);
  if (c->h_eig) cudaFreeHost(c->h_eig);
  dh_destroy(c->plan);
  delete c;
}

}  // namespace

using namespace dh;

extern "C" {

dh_status dh_server_create(dh_server_t *out, size_t hbm_budget_bytes) {
  if (!out || hbm_budget_bytes == 0) return DH_ERR_INVALID_ARG;
  *out = nullptr;
  dh_server *s = new (std::nothrow) dh_server();
  if (!s) return DH_ERR_OOM;
  s->budget = hbm_budget_bytes;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) {
    delete s;
    return fail_cuda(e);
  }
  *out = s;
  return DH_OK;
}

size_t dh_server_stream_bytes(int nx, int ny, int T, dh_precision prec, int ring_windows) {
  if (ring_windows < 1) return 0;
  return stream_device_bytes(nx, ny, T, prec, ring_windows);
}

dh_status dh_server_add_stream(dh_server_t s, int nx, int ny, double lambda_m, double z_m,
                               double pitch_m, int T, dh_precision prec, int k0, int k1,
                               int ring_windows, int *stream_id) {
  if (!s || !stream_id || ring_windows < 1 || k0 < 0 || k1 < k0 || k1 >= T) return DH_ERR_INVALID_ARG;
  *stream_id = -1;
  const size_t need = stream_device_bytes(nx, ny, T, prec, ring_windows);
  if (!need) return DH_ERR_UNSUPPORTED_SIZE;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->used + need > s->budget) return DH_ERR_OOM;  // admission denied: nothing allocated
  CamStream *c = new (std::nothrow) CamStream();
  if (!c) return DH_ERR_OOM;
  c->nx = nx; c->ny = ny; c->T = T; c->k0 = k0; c->k1 = k1; c->ring = ring_windows;
  c->npix = (long long)nx * ny;
  dh_status st = dh_plan_create(&c->plan, nx, ny, lambda_m, z_m, pitch_m, T);
  if (st == DH_OK && prec != DH_PREC_FP32) st = dh_plan_set_precision(c->plan, prec);
  if (st == DH_OK) st = dh_plan_reserve(c->plan, 2 * T, 1);
  cudaError_t e = cudaSuccess;
  if (st == DH_OK) e = cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) st = fail_cuda(e);
  if (st == DH_OK && !s->tune_path.empty()) {  // the autotune cache: apply, or tune and save
    int found = 0;
    st = dh_plan_tune_load(c->plan, s->tune_path.c_str(), &found);
    if (st == DH_OK && !found && s->tune_autotune) {
      st = dh_plan_autotune(c->plan, 2 * T, c->cs);
      if (st == DH_OK) st = dh_plan_tune_save(c->plan, s->tune_path.c_str());
    }
  }
  if (st == DH_OK) {
    if (e == cudaSuccess) e = cudaMalloc(&c->d_frames, (size_t)2 * T * c->npix * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_images, (size_t)ring_windows * c->npix * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_eig, (size_t)ring_windows * T * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_images, (size_t)ring_windows * c->npix * sizeof(float));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_eig, (size_t)ring_windows * T * sizeof(double));
    if (e != cudaSuccess) st = fail_cuda(e);
  }
  if (st != DH_OK) {
    free_stream(c);
    return st;
  }
  c->slot_used.assign(ring_windows, 0);
  c->bytes = dh_plan_device_bytes(c->plan) + (size_t)2 * T * c->npix * sizeof(uint16_t) +
             (size_t)ring_windows * c->npix * sizeof(float) + (size_t)ring_windows * T * sizeof(double);
  c->id = s->next_id++;
  s->used += c->bytes;
  s->streams[c->id] = c;
  *stream_id = c->id;
  return DH_OK;
}

dh_status dh_server_set_tune_cache(dh_server_t s, const char *path, int autotune) {
  if (!s || (autotune != 0 && autotune != 1)) return DH_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->tune_path = path ? path : "";
  s->tune_autotune = path && autotune == 1;
  return DH_OK;
}

dh_status dh_server_stream_option(dh_server_t s, int stream_id, int option, int *value) {
  if (!s || !value) return DH_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->streams.find(stream_id);
  if (it == s->streams.end()) return DH_ERR_INVALID_ARG;
  return dh_plan_get_option(it->second->plan, option, value);
}

dh_status dh_server_remove_stream(dh_server_t s, int stream_id) {
  if (!s) return DH_ERR_INVALID_ARG;
  CamStream *c = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->streams.find(stream_id);
    if (it == s->streams.end()) return DH_ERR_INVALID_ARG;
    c = it->second;
    s->streams.erase(it);
    s->used -= c->bytes;
  }
  cudaStreamSynchronize(c->cs);  // every callback of the stream has run
  {
    std::lock_guard<std::mutex> lk(s->done_mu);
    std::deque<Done> keep;
    for (const Done &d : s->done)
      if (d.stream_id != stream_id) keep.push_back(d);
    s->done.swap(keep);
  }
  free_stream(c);
  return DH_OK;
}

size_t dh_server_used_bytes(dh_server_t s) {
  if (!s) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  return s->used;
}

dh_status dh_server_push(dh_server_t s, int stream_id, const uint16_t *frames_host,
                         int64_t frame_index, int n_frames) {
  if (!s || !frames_host || n_frames < 1) return DH_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->streams.find(stream_id);
  if (it == s->streams.end()) return DH_ERR_INVALID_ARG;
  CamStream *c = it->second;
  const int T = c->T, ring2 = 2 * T;
  if (n_frames > T) return DH_ERR_INVALID_ARG;
  if (frame_index != c->next_frame) return DH_ERR_FRAME_GAP;
  // windows this push completes, and an output slot for each (backpressure when the caller
  // has not released enough earlier results)
  const int64_t last = frame_index + n_frames - 1;
  std::vector<int64_t> wins;
  for (int64_t w = frame_index / T; (w + 1) * T - 1 <= last; ++w)
    if ((w + 1) * T - 1 >= frame_index) wins.push_back(w);
  for (int64_t w : wins)
    if (c->slot_used[(int)(w % c->ring)]) return DH_ERR_STATE;
  const double t_push = now_s(s->t0);
  // frames -> device ring (one copy per contiguous run) -> holograms in slot f mod 2T
  int done_n = 0;
  while (done_n < n_frames) {
    const int64_t f = frame_index + done_n;
    const int slot = (int)(f % ring2);
    const int run = std::min(n_frames - done_n, ring2 - slot);
    DH_CUDA_TRY(cudaMemcpyAsync(c->d_frames + (size_t)slot * c->npix, frames_host + (size_t)done_n * c->npix,
                                (size_t)run * c->npix * sizeof(uint16_t), cudaMemcpyHostToDevice, c->cs));
    dh_status st = plan_render(c->plan, c->d_frames + (size_t)slot * c->npix, c->npix, run, slot, c->cs);
    if (st != DH_OK) return st;
    done_n += run;
  }
  c->next_frame = last + 1;
  for (int64_t w : wins) {
    const int slot = (int)(w % c->ring);
    float *img = c->d_images + (size_t)slot * c->npix;
    double *eig = c->d_eig + (size_t)slot * T;
    dh_status st = plan_pca(c->plan, (int)((w * T) % ring2), T, 1, c->k0, c->k1, img, eig, c->cs);
    if (st != DH_OK) return st;
    DH_CUDA_TRY(cudaMemcpyAsync(c->h_images + (size_t)slot * c->npix, img, (size_t)c->npix * sizeof(float),
                                cudaMemcpyDeviceToHost, c->cs));
    DH_CUDA_TRY(cudaMemcpyAsync(c->h_eig + (size_t)slot * T, eig, (size_t)T * sizeof(double),
                                cudaMemcpyDeviceToHost, c->cs));
    Pending *p = new (std::nothrow) Pending{s, c->id, w, slot, t_push};
    if (!p) return DH_ERR_OOM;
    c->slot_used[slot] = 1;
    cudaError_t e = cudaLaunchHostFunc(c->cs, on_window_done, p);
    if (e != cudaSuccess) {
      delete p;
      return fail_cuda(e);
    }
  }
  return DH_OK;
}

int dh_server_poll(dh_server_t s, dh_window_result *out, int max_results) {
  if (!s || !out || max_results < 1) return 0;
  std::vector<Done> got;
  {
    std::lock_guard<std::mutex> lk(s->done_mu);
    while (!s->done.empty() && (int)got.size() < max_results) {
      got.push_back(s->done.front());
      s->done.pop_front();
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  int n = 0;
  for (const Done &d : got) {
    auto it = s->streams.find(d.stream_id);
    if (it == s->streams.end()) continue;
    CamStream *c = it->second;
    dh_window_result &r = out[n++];
    r.stream_id = d.stream_id;
    r.window = d.window;
    r.image_host = c->h_images + (size_t)d.slot * c->npix;
    r.eigvals_host = c->h_eig + (size_t)d.slot * c->T;
    r.t_ready_s = d.t_ready;
    r.t_done_s = d.t_done;
  }
  return n;
}

dh_status dh_server_release(dh_server_t s, int stream_id, int64_t window) {
  if (!s || window < 0) return DH_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->streams.find(stream_id);
  if (it == s->streams.end()) return DH_ERR_INVALID_ARG;
  CamStream *c = it->second;
  c->slot_used[(int)(window % c->ring)] = 0;
  return DH_OK;
}

double dh_server_clock(dh_server_t s) { return s ? now_s(s->t0) : 0.0; }

dh_status dh_server_drain(dh_server_t s) {
  if (!s) return DH_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto &kv : s->streams) DH_CUDA_TRY(cudaStreamSynchronize(kv.second->cs));
  return DH_OK;
}

void dh_server_destroy(dh_server_t s) {
  if (!s) return;
  std::vector<CamStream *> all;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &kv : s->streams) all.push_back(kv.second);
    s->streams.clear();
  }
  for (CamStream *c : all) free_stream(c);
  delete s;
}

}  // extern "C"
