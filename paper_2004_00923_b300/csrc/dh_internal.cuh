// Internal declarations shared by the translation units of libdh.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dh.h"

namespace dh {

constexpr int kMaxDim = 4096;
constexpr int kMinDim = 16;

// One device-resident plan (see dh.h). Host-side bookkeeping plus device buffers.
struct Plan {
  int nx = 0, ny = 0, T = 0, lognx = 0, logny = 0;
  long long npix = 0;
  double lambda = 0, z = 0, pitch = 0, a = 0;
  dh_precision prec = DH_PREC_FP32;
  int device = 0;
  int num_sms = 148;

  // a view computes windows of its own length T over another plan's hologram store; it
  // holds no store, intermediate or tables of its own and renders nothing
  bool is_view = false;
  int max_frames = 0;   // hologram slots
  int max_windows = 0;  // windows per dh_pca_windows call

  // tables
  float2 *d_cx = nullptr, *d_cy = nullptr;   // chirp * 1/sqrt(n) per axis
  float2 *d_twx = nullptr, *d_twy = nullptr; // Stockham twiddles per axis
  void *d_tc = nullptr;                      // tensor-core render tables (1024^2 frames)
  // arithmetic of Eq. 1's DFTs: 0 = automatic, 1 = CUDA cores, 2 = tensor cores (1024^2)
  int render_fft = 0;
  // radix of the CUDA-core FFT passes: 0 = each length's default, else 16 or 32 where that
  // radix is instantiated for an axis length (the other axes keep their default)
  int fft_radix = 0;
  // split-K units per window of the tensor-core covariance: 0 = the default for the frame
  // size, else a power of two dividing n / 256 (DH_OPT_GRAM_UNITS, the autotuner)
  int gram_units = 0;
  // mean-residual storage (DH_OPT_RESIDUAL, 16-bit storage): windows of dh_pca_batch store
  // D = F(I - M) with M the window's rounded mean frame, mu = F(M) in FP32
  int residual = 0;
  uint16_t *d_mean = nullptr;  // [max_windows][npix] uint16
  float *d_mu = nullptr;       // [max_windows][re | im][npix] FP32
  float *d_mucoef = nullptr;   // [max_windows][a (2T) | b (2T)] FP32, or [sigma, ...]
  // per call: the residual projection takes mu's cross term from two operand columns (the
  // u-column form, see residual.cu) instead of per-column coefficients
  int resid_ucol = 0;
  // render intermediate (row-pass output): a chunk of frames sized to stay in L2
  float2 *d_mid = nullptr;
  int mid_frames = 0;
  // render schedule: 0 = one persistent launch over a ring of intermediates where it
  // applies (square frames from 256^2), else chunks; 1 = always chunks of two launches
  int render_mode = 0;
  int render_ring = 0, render_lag = 0;  // persistent schedule: ring frames, lag (0 = automatic)
  // covariance source: 0 holograms (Eq. 4 as written), 1 the uint16 frames (C = I^T I) where
  // the call has them, 2 the banded Gram of the store (dh_band_gram)
  int cov_mode = 0;
  // projection of Eqs. 6-7: 0 = automatic (overlapping windows share their tile loads and use
  // the complement of the discarded components where that applies), 1 = per window always
  int proj_mode = 0;
  // window groups of one call: 0 = automatic (two where the eigensolver can overlap the
  // covariance and projection of the other group), 1 = one group
  int group_mode = 0;
  // SMs the next tensor-core covariance or projection launch may fill (0 = all): the rest
  // are left to an eigensolver running beside it
  int sm_budget = 0;
  unsigned *d_sync = nullptr;  // ticket and ring counters of the persistent render, then one
                               // word nothing ever sets (the stall test's wait target)
  // test only (DH_OPT_TEST_STALL): cycles the persistent render's CTAs wait on that word
  // before their first item; the wait always runs out (0 = off)
  int test_stall = 0;
  // streams the plan's calls launched work on since the last status read (dh_plan_status
  // synchronises only these); touched_all: more streams than the list holds, or work
  // captured into a graph (whose launch stream the plan does not see)
  static constexpr int kMaxTouched = 8;
  cudaStream_t touched[kMaxTouched] = {};
  int n_touched = 0;
  bool touched_all = false;
  // second stream: the eigensolver of one group of windows overlaps the next group's work
  cudaStream_t aux = nullptr;
  static constexpr int kMaxGroups = 4;
  cudaEvent_t ev_grp[kMaxGroups] = {}, ev_jac[kMaxGroups] = {};
  // hologram store: [max_frames][2][npix] of the storage type
  void *d_H = nullptr;
  size_t H_elem_bytes = 4;
  // covariance partials: [max_windows][parts_per_window][2T][2T] FP64
  double *d_part = nullptr;
  int parts_total = 0;  // partial Gram matrices the buffer holds (all windows)
  double *d_C = nullptr;    // [max_windows][T][T][2]
  double *d_lam = nullptr;  // [max_windows][T]
  double *d_V = nullptr;    // [max_windows][T][T][2]
  void *d_B = nullptr;      // projection operand per window
  size_t B_window_bytes = 0;
  void *d_W = nullptr;      // projection operand shared by all windows (Eq. 8's DFT columns)
  size_t W_bytes = 0;
  uint32_t *d_status = nullptr;

  // tensor maps for the tensor-core kernels (16-bit storage only)
  CUtensorMap tmap_H;
  CUtensorMap tmap_B;
  CUtensorMap tmap_band;  // 64 pixels x 128 rows (64 frames) boxes, for the banded Gram
  bool tmaps_ok = false;
  // banded Gram of the store (held by the plan that owns the store; views read the owner's)
  const Plan *band_owner = nullptr;
  double *d_band = nullptr, *d_band_part = nullptr;
  int band_cap = 0;                     // 64-frame blocks the buffers hold
  int band_first = 0, band_frames = 0;  // slots the current band covers

  // host-buffer pipeline (dh_pca_batch_host), created on first use: copy streams, two
  // staging buffers of frames, device images / eigenvalues of the batch
  struct HostPipe {
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t start = nullptr, done = nullptr, finished = nullptr;
    cudaEvent_t copied[2] = {}, freed[2] = {};
    uint16_t *stage[2] = {};
    size_t stage_elems = 0;
    uint8_t *pstage[2] = {};  // packed 12-bit frames as copied (dh_pca_batch_host_packed12)
    size_t pstage_bytes = 0;
    float *img = nullptr;
    double *eig = nullptr;
    size_t img_elems = 0, eig_elems = 0;
  } pipe;
  size_t bytes = 0;         // device bytes the plan itself allocated
  size_t window_bytes = 0;  // the part of `bytes` in per-window buffers
  int busy = 0;
  void *prof = nullptr;  // per-kernel event timing state (profile.cu), null when disabled
};

// ---------------------------------------------------------------- tracing
enum KernelId {
  K_RENDER_ROWS = 0, K_RENDER_COLS, K_GRAM_SIMT, K_GRAM_TC, K_REDUCE_COV, K_JACOBI,
  K_PROJECT_SIMT, K_PROJECT_TC, K_FOURIER_OP, K_SVD_FOURIER_OP, K_RENDER_FUSED, K_GRAM_RAW,
  K_REDUCE_RAW, K_FOURIER_SLIDING, K_BAND_GRAM, K_BAND_REDUCE, K_BAND_COV, K_PROJECT_SPAN, K_FOURIER_SPAN,
  K_RENDER_ROWS_TC, K_RENDER_COLS_TC, K_RENDER_FUSED_TC, K_COUNT
};
const char *kernel_name(int kid);
dh_status profile_enable(Plan &p, int on);
int profile_read(Plan &p, int n, const char **names, int *launches, double *total_ms);
void profile_free(Plan &p);
// Brackets one kernel launch with CUDA events on its stream when the plan's profiler is on.
struct ProfScope {
  Plan &p;
  int kid;
  cudaStream_t s;
  int slot;
  ProfScope(Plan &plan, int k, cudaStream_t st);
  ~ProfScope();
};

// ---------------------------------------------------------------- host helpers
const char *set_cuda_error(cudaError_t e);
// Record that plan work was launched on stream s (for dh_plan_status).
void note_stream(Plan &p, cudaStream_t s);
dh_status fail_cuda(cudaError_t e);

#define DH_CUDA_TRY(expr)                         \
  do {                                            \
    cudaError_t e__ = (expr);                     \
    if (e__ != cudaSuccess) return fail_cuda(e__); \
  } while (0)

// ---------------------------------------------------------------- stage launchers
// Eq. 1: render n_frames frames into hologram slots [slot0, slot0 + n_frames).
dh_status launch_render(Plan &p, const uint16_t *frames, long long frame_stride, int n_frames,
                        int slot0, cudaStream_t s);
// Where a render writes: H of storage type `prec` (16-bit: [p / 64][rows_total][64] blocks;
// FP32: planes [slot][re|im][npix]), and optionally, per frame, the window mean frame it
// subtracts first: frame f of the call uses mean + ((mean_first + f) / mean_every) * npix
// (uint16).
struct RenderTarget {
  void *H;
  dh_precision prec;
  long long rows_total;
  const uint16_t *mean;
  int mean_every;
  int mean_first = 0;
};
dh_status launch_render_to(Plan &p, const uint16_t *frames, long long frame_stride, int n_frames,
                           int slot0, const RenderTarget &to, cudaStream_t s);
// FFT specs of the render: log2 length in the low 4 bits, log2 radix above (0 = default);
// the plan's radix choice (0 = default, or 16 / 32 where that radix is instantiated for the
// length) per axis, and whether a radix is available for a length
int fft_spec_for(int logn, int radix);
int row_spec(const Plan &p);
int col_spec(const Plan &p);
bool fft_radix_available(int logn, int radix);
void build_twiddles(int spec, float2 *host_out);  // host, FP64 -> FP32
// work items per frame and pass of the render (square frames): N / FFTs per CTA
int render_items_per_frame(const Plan &p);
int twiddle_len(int spec);
// tensor-core render of 1024^2 frames: whether the plan uses it, and its tables
bool tc_render_applies(const Plan &p);
size_t tc_tables_bytes();
void build_tc_tables(void *host_out);

// Partial Gram matrices per window (split-K over pixels), fixed per frame size.
int gram_units(long long npix);
int gram_tc_parts(const Plan &p);
int gram_tc_default_units(long long npix);
int gram_raw_parts(const Plan &p);
// partial Gram matrices a window may need (hologram or raw-domain covariance)
inline int parts_per_window(const Plan &p) {
  const int h = p.prec == DH_PREC_FP32 ? gram_units(p.npix) : gram_tc_parts(p);
  const int r = gram_raw_parts(p);
  return h > r ? h : r;
}
// Eq. 4, FP32 CUDA cores: partial real Gram matrices of X = [Re H_t ; Im H_t] rows.
dh_status launch_gram_simt(Plan &p, int first_slot, int slot_stride, int n_windows,
                           int *parts_per_window, cudaStream_t s);
// Eq. 4, tensor cores (16-bit storage).
dh_status launch_gram_tc(Plan &p, int first_slot, int slot_stride, int n_windows,
                         int *parts_per_window, cudaStream_t s);
// Eq. 4 from the uint16 frames (C = I^T I, exact): partial Gram matrices of the hi / lo byte
// rows of windows [first_frame + w * window_stride, + T) of `frames` (n_frames frames,
// frame_stride elements apart), then their FP64 reduction into C.
dh_status launch_gram_raw(Plan &p, const uint16_t *frames, long long frame_stride, int n_frames,
                          int first_frame, int window_stride, int n_windows, int *parts_per_window,
                          cudaStream_t s);
dh_status launch_reduce_raw(Plan &p, int n_windows, int parts_per_window, int woff, cudaStream_t s);
// Banded Gram of slots [first_slot, first_slot + n_frames) into p.d_band (16-bit storage), and
// the covariance of windows [woff, woff + n_windows) of plan p assembled from owner's band.
int band_units(long long npix);
dh_status launch_band_gram(Plan &p, int first_slot, int n_frames, cudaStream_t s);
dh_status launch_band_cov(Plan &p, const Plan &owner, int first_slot, int slot_stride, int n_windows, int woff,
                          cudaStream_t s);
// Eq. 4 final FP64 reduction, then Eq. 5 + ordering + operand build for Eq. 6, for windows
// [woff, woff + n_windows) of the plan's per-window buffers.
dh_status launch_reduce(Plan &p, int n_windows, int parts_per_window, int woff, cudaStream_t s);
// Layout of the grouped projection of overlapping windows (csrc/project_span.cu): G windows
// of slot stride `stride` per group, each group's banded operand (hi + lo 16-bit images of
// n_pad x k_pad, 128-byte swizzled, `img_bytes` in all) stored in the operand slots of its
// windows; G = 0 when the per-window projection is used.
// 3-D tiled tensor map over 16-bit data (128-byte swizzle, zero fill out of bounds).
dh_status encode_3d(CUtensorMap *map, void *base, bool bf16, const uint64_t dims[3],
                    const uint64_t strides_bytes[2], const uint32_t box[3]);
// Scale of the grouped projection's operand entries (a power of two; see k_span_operand).
constexpr double kSpanOperandScale = 1024.0;
struct SpanLayout {
  int G = 0, cpw = 0, rows = 0, n_pad = 0, k_pad = 0, stride = 0, img_bytes = 0, stages = 0;
  int nacc = 0, tmem_cols = 0;  // partial accumulators per buffer; TMEM columns allocated
  int scr_bytes = 0;            // shared scratch of per-pixel chunk energies
  int nbuf = 0;                 // TMEM accumulator buffers (2 or 4)
};
SpanLayout span_layout(const Plan &p, int slot_stride, int n_windows, int k0, int k1);
dh_status launch_project_span(Plan &p, const SpanLayout &sl, int first_slot, int n_windows, float *images,
                              int woff, cudaStream_t s);
// With span (G > 0) the eigensolver writes the discarded components' banded group operand
// instead of the per-window operand of Eq. 6.
dh_status launch_jacobi(Plan &p, int n_windows, int k0, int k1, int Npad, double *eig_user, int woff,
                        cudaStream_t s, const SpanLayout *span = nullptr);
// Eqs. 6-7 (and 8-9).
// images points at window woff's image; woff selects the windows' operands, unless
// shared_op is given: then every window projects onto that one operand (one window's
// layout, as d_W holds it).
dh_status launch_project_simt(Plan &p, int first_slot, int slot_stride, int n_windows, int Npad,
                              float *images, int woff, cudaStream_t s, const void *shared_op = nullptr);
dh_status launch_project_tc(Plan &p, int first_slot, int slot_stride, int n_windows, int Npad,
                            float *images, int woff, cudaStream_t s, const void *shared_op = nullptr);
// Eqs. 8-9 for overlapping windows on the tensor cores, 7 windows per span load (FP16 storage,
// 17 kept bins, slot stride < T, n_y >= 128): whether it applies, and the launch (operand
// built into d_W first).
bool fourier_span_applies(const Plan &p, int slot_stride, int n_windows, int nS);
dh_status launch_fourier_span(Plan &p, int first_slot, int slot_stride, int n_windows, int k0, int nS,
                              float *images, cudaStream_t s);
// Eqs. 2-3 then 8-9: per window, the operand Q = V_S V_S^{t*} W_band from the sorted
// eigenvectors of windows [woff, woff + n_windows), replacing the Eq. 6 operand.
dh_status launch_svd_fourier_operand(Plan &p, int n_windows, int k0, int k1, int b0, int b1, int Npad,
                                     int woff, cudaStream_t s);
// Eqs. 8-9: power of the DFT bins k0..k1 of every window.
dh_status launch_fourier(Plan &p, int first_slot, int slot_stride, int n_windows, int k0, int k1,
                         float *images, cudaStream_t s);
dh_status make_tensor_maps(Plan &p);

// single-window helpers used by the allocation-free covariance entry point
dh_status launch_gram_simt_rows(const float *X, long long npix, int T, int units, double *part,
                                cudaStream_t s);
dh_status launch_reduce_cov_window(const double *part, int parts, int T, double *C, uint32_t *status,
                                   cudaStream_t s);
// load the modules of the kernels the two helpers above launch, for every T
dh_status preload_gram_simt_rows();
dh_status preload_reduce_cov_window();

// mean-residual storage: the windows' rounded mean frames into p.d_mean, and after the
// eigensolver the projection's mu coefficients into p.d_mucoef (ucol: sigma there, and u's
// two columns into the last two of the Npad operand columns)
dh_status launch_unpack_mono12p(const uint8_t *src, long long src_stride_bytes, long long npix, int n_frames,
                                uint16_t *dst, long long dst_stride_elems, cudaStream_t s);  // unpack.cu
dh_status launch_window_mean(Plan &p, const uint16_t *frames, long long frame_stride, int n_windows,
                             int window_stride, cudaStream_t s);
dh_status launch_mu_coef(Plan &p, int n_windows, int k0, int k1, int Npad, int woff, bool ucol, cudaStream_t s);

// conversions for inspection
dh_status launch_hologram_to_f32(Plan &p, int slot, float *out, cudaStream_t s);

inline int ilog2(long long v) {
  int l = 0;
  while ((1ll << l) < v) ++l;
  return l;
}

}  // namespace dh
