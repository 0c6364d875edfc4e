/*
 * dh.h -- C ABI of libdh: real-time digital holography of the retina by principal
 * component analysis (Puyo et al., arXiv 2004.00923) on one NVIDIA B300 (sm_103a).
 *
 * The library computes, for windows of n_t consecutive 16-bit interferograms
 * I(x, y, t) of n_x x n_y pixels:
 *   1. Fresnel holograms H(x, y, t) of every frame (Eq. 1, one 2-D FFT per frame),
 *   2. the covariance C = H^{t*} H of each window (Eq. 4),
 *   3. its eigendecomposition C = V Lambda V^{t*} (Eq. 5),
 *   4. the power image M(x, y) = sum_{k=k0..k1} |(H V)(x, y, k)|^2 (Eqs. 6-7).
 *
 * Conventions shared by every entry point:
 *  - Discrete form of Eq. 1 used here: with a = pitch^2 / (lambda z) and centred input
 *    coordinates, H[t,y,x] = s sum_{k,l} I[t,l,k] c(k) c(l) exp(+2 pi i (xk/n_x + yl/n_y)),
 *    c(k) = exp(-i pi a (k - n/2)^2), s = 1/sqrt(n_x n_y). The output chirp and the
 *    constant prefactor of Eq. 1 have unit modulus per pixel; they cancel in C and in
 *    |H V|^2 and are not applied. Output pixels are in natural FFT order.
 *  - Eigenvalues are ordered DEcreasing and components are numbered from 0; (k0, k1)
 *    is the inclusive retained range in that order (the paper orders increasingly
 *    from 1: its index j is component k = n_t - j here).
 *  - Device pointers are CUDA device addresses owned by the caller; the library never
 *    frees them. Host pointers are plain host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Every call is asynchronous on that stream unless its comment says otherwise.
 *  - Errors are returned as dh_status; nothing is thrown across the ABI. After
 *    DH_ERR_CUDA, dh_last_error() gives the CUDA error text.
 *  - A plan is not re-entrant: calls on one plan from two host threads at once return
 *    DH_ERR_STATE.
 */
#ifndef DH_H_
#define DH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dh_plan *dh_plan_t;   /* opaque, library-owned */
typedef struct dh_graph *dh_graph_t; /* opaque, library-owned */

typedef enum {
  DH_OK = 0,
  DH_ERR_INVALID_ARG = 1,
  DH_ERR_UNSUPPORTED_SIZE = 2,
  DH_ERR_OOM = 3,
  DH_ERR_CUDA = 4,
  DH_ERR_TIMEOUT = 5,
  DH_ERR_FRAME_GAP = 6,
  DH_ERR_STATE = 7
} dh_status;

/* Storage type of the holograms H (paper: single-precision cuComplex, "plain" here).
 * DH_PREC_FP32: H stored FP32; covariance and projection on FP32 CUDA cores.
 * DH_PREC_FP16 / DH_PREC_BF16: H stored as 16-bit real/imaginary planes; covariance and
 * projection run on the tensor cores (tcgen05, FP32 accumulation), with the eigenvector
 * operand split into hi + lo 16-bit parts. */
typedef enum { DH_PREC_FP32 = 0, DH_PREC_FP16 = 1, DH_PREC_BF16 = 2 } dh_precision;

/* Device status bits returned by dh_plan_status(). */
#define DH_FLAG_STORE_OVERFLOW 0x1u  /* a hologram value was not finite after 16-bit storage */
#define DH_FLAG_NONFINITE_C 0x2u     /* the covariance held a NaN/Inf */
#define DH_FLAG_EIG_NOT_CONVERGED 0x4u
#define DH_FLAG_WAIT_TIMEOUT 0x8u    /* a bounded device-side wait gave up (kernel skipped work) */

/* Create a plan for n_x x n_y frames (powers of two in [16, 4096]) and windows of
 * T frames (T in {16, 32, 64}); lambda_m, z_m, pitch_m > 0 are the wavelength, the
 * sensor-to-object distance and the pixel pitch of Eq. 1, in metres. Builds the chirp
 * and twiddle tables in FP64 on the host and allocates the device buffers for one
 * window of FP32 holograms on the current CUDA device. Synchronous.
 * Errors: DH_ERR_INVALID_ARG (NULL out, non-positive/non-finite optics),
 * DH_ERR_UNSUPPORTED_SIZE (n_x, n_y or T), DH_ERR_OOM, DH_ERR_CUDA. */
dh_status dh_plan_create(dh_plan_t *out, int nx, int ny, double lambda_m, double z_m,
                         double pitch_m, int T);

/* Release every device buffer of the plan. NULL-safe. Synchronises the device. A plan
 * whose store live views still read keeps that store until its last view is destroyed. */
void dh_destroy(dh_plan_t plan);

/* A view: a plan for windows of T' frames (T' in {16, 32, 64}, T' <= the base's slots)
 * over the hologram store of `base`, so that windows of several lengths share one
 * rendering of each frame (Eq. 1 is per frame; Eqs. 4-7 are per window). The view has
 * its own covariance, eigenvector and projection buffers (one window until
 * dh_plan_reserve(view, ., max_windows)), the base's frame size, optics and storage
 * type, and renders nothing: dh_render_frames / dh_render_stack / dh_pca_batch on a
 * view return DH_ERR_STATE. While views live, dh_plan_set_precision on the base and a
 * dh_plan_reserve that changes its slot count return DH_ERR_STATE. Work on the base and
 * on its views touches the same store: order it (one stream, or events) as for one plan.
 * A view of a view reads the same store. The paper renders each frame once and runs one
 * window length; views extend that to several lengths at once. Synchronous.
 * Errors: DH_ERR_INVALID_ARG (NULL out or base, T' above the base's slots),
 * DH_ERR_UNSUPPORTED_SIZE (T'), DH_ERR_OOM, DH_ERR_CUDA. */
dh_status dh_plan_create_view(dh_plan_t *out, dh_plan_t base, int T);

/* Select the hologram storage type (default DH_PREC_FP32). Reallocates the hologram
 * store; previously rendered holograms are discarded. Synchronous. */
dh_status dh_plan_set_precision(dh_plan_t plan, dh_precision prec);

/* Reserve device storage for up to max_frames rendered frames (hologram "slots") and
 * up to max_windows windows per dh_pca_windows call. Default: T slots, 1 window.
 * Synchronous; previously rendered holograms are discarded when the store grows. */
dh_status dh_plan_reserve(dh_plan_t plan, int max_frames, int max_windows);

/* Plan options (dh_plan_set_option).
 * DH_OPT_RENDER_SCHEDULE: how Eq. 1 is scheduled. 0 (default): for square frames from
 *   256 x 256, every frame of a render call in one persistent launch that interleaves the
 *   row and column FFT passes of consecutive frames over a small L2-resident ring of
 *   intermediates (a frame's column work starts as soon as its rows are done; other sizes
 *   use chunks). 1: chunks of frames, each a row-pass launch then a column-pass launch.
 *   Both give bitwise the same holograms. */
#define DH_OPT_RENDER_SCHEDULE 0
/* DH_OPT_RENDER_RING: frames of intermediate in the persistent schedule's ring, 2..64
 *   (capped by the plan's intermediate), 0 = automatic (twice the lag).
 * DH_OPT_RENDER_LAG: frames between a frame's row pass and its column pass in that
 *   schedule, 1..63 (capped at ring - 1), 0 = automatic (half the ring; the automatic ring
 *   makes it about 1.5 rounds of the grid's CTAs in work items). */
#define DH_OPT_RENDER_RING 1
#define DH_OPT_RENDER_LAG 2
/* DH_OPT_COVARIANCE: 0 (default): C = H^{t*} H from the holograms, as Eq. 4 is written.
 *   1: wherever the call has the uint16 frames at hand (dh_pca_batch; dh_pca_batch_host when
 *   windows are T or more frames apart), C = I^T I from the frames themselves -- equal in
 *   exact arithmetic because the Fresnel transform of Eq. 1 is unitary per frame -- computed
 *   exactly on the tensor cores (each value split into two bytes, integer accumulation):
 *   half the bytes read and no storage rounding in C (exact while sum I^2 < 2^53). 16-bit
 *   hologram storage only (DH_ERR_STATE for FP32 plans). Holograms are still rendered for
 *   the projection of Eqs. 6-7. */
/*   2: C from the banded Gram of the store computed by dh_band_gram (below): windows of any
 *   length and stride inside the band take their C from it without reading the holograms
 *   again (DH_ERR_STATE for windows outside the band). 16-bit storage only. */
#define DH_OPT_COVARIANCE 3
/* DH_OPT_PROJECTION: 0 (default): overlapping windows (slot stride s < T, s a multiple of
 *   4; FP16 storage, n_y >= 128, n_x a multiple of 8) with at most 4 discarded components
 *   (k0 + T - 1 - k1 <= 4) are projected in groups of up to 8: each pixel tile of a group's
 *   span of frames is read once for all its windows, and each window's power is taken as
 *   its energy sum_t |H_t|^2 minus its discarded components' power (equal to Eq. 7 because
 *   V is unitary). Other calls project per window. 1: per window always (Eq. 7 over the
 *   kept components). */
#define DH_OPT_PROJECTION 4
/* DH_OPT_WINDOW_GROUPS: 0 (default): a call whose covariance comes from the tensor cores
 *   (16-bit storage; DH_OPT_COVARIANCE 0, or 1 with the frames at hand) and whose windows are
 *   projected one by one, with 32 to (SMs) windows, runs in two groups of windows: the
 *   eigensolver of one group (one CTA per window) runs beside the covariance of the next
 *   group, and the eigensolver of that group beside the projection of the first, each pair
 *   on disjoint SMs (the covariance and projection launches leave one SM per eigensolver
 *   CTA). 1: one group always. Both give bitwise the same results. */
#define DH_OPT_WINDOW_GROUPS 5
/* DH_OPT_TEST_STALL (test only, for the failure path): value > 0 makes every CTA of the
 *   persistent render (DH_OPT_RENDER_SCHEDULE 0) first wait `value` SM cycles (at most 1e8)
 *   on a device word that nothing sets; the bounded wait runs out, the CTA raises
 *   DH_FLAG_WAIT_TIMEOUT and skips its work (no CTA is left waiting on another), and the next
 *   dh_plan_status returns DH_ERR_TIMEOUT. The holograms of that call are not written. It
 *   does the same to the waiter warp of the 16-bit tensor-core covariance (DH_OPT_COVARIANCE
 *   0): its first wait, on a barrier that completes only at the end of the launch, runs out,
 *   and the launch takes its abort path (the covariances of that call are not formed).
 *   0 (default): off. */
#define DH_OPT_TEST_STALL 6
/* DH_OPT_RENDER_FFT: the arithmetic of Eq. 1's DFTs. 0 (default): automatic. 1: the
 *   CUDA-core FFT (FP32 Stockham passes). 2: for 1024 x 1024 frames, each 1024-point DFT as two
 *   batched 32-point DFTs on the tensor cores (FP16 hi + lo operands, three products, FP32
 *   accumulation; ~1e-7 relative, like the FP32 FFT) with the twiddles, chirps and stores on
 *   the CUDA cores; DH_ERR_UNSUPPORTED_SIZE for other sizes. */
#define DH_OPT_RENDER_FFT 7
/* DH_OPT_FFT_RADIX: the radix of the CUDA-core FFT passes of Eq. 1. 0 (default): each
 *   length's own (32 at 32, 512, 1024 and 2048; 8 at 64; 16 otherwise); 16 or 32: that radix
 *   on every axis whose length has it instantiated (16 at 512, 1024, 2048; 32 at 4096; each
 *   length's default), the other axes keep their default; DH_ERR_UNSUPPORTED_SIZE if no axis
 *   has it. Results differ from the default only in rounding. Synchronous. Views: DH_ERR_STATE.
 * DH_OPT_GRAM_UNITS: split-K units per window of the tensor-core covariance of Eq. 4 (16-bit
 *   storage; DH_ERR_STATE for FP32 plans): 0 (default) = the frame size's own, else a power of
 *   two dividing n_x n_y / 256 (DH_ERR_UNSUPPORTED_SIZE otherwise). A window's covariance stays
 *   bitwise the same alone and in any batch for a given setting; settings differ only in the
 *   order of the FP64 partial sums. Reallocates the per-window buffers (synchronous). */
#define DH_OPT_FFT_RADIX 8
#define DH_OPT_GRAM_UNITS 9
/* DH_OPT_RESIDUAL: mean-residual storage (16-bit storage only; DH_ERR_STATE for FP32 plans).
 *   1: dh_pca_batch with windows exactly T frames apart stores each window's holograms as
 *   D_t = F(I_t - M) (Eq. 1 of the residual, F linear), M the window's temporal mean frame
 *   rounded to integers, keeps mu = F(M) in FP32, projects P = D V + mu (1^T V) (equal to H V
 *   since H = mu 1^T + D), and takes C = I^T I from the frames (exact). The 16-bit rounding
 *   then scales with |D| rather than |H|, whose static part is removed; the tensor-core DFT
 *   render is not used. Other calls on the plan return DH_ERR_STATE while it is on.
 *   Allocates per window 2 n_x n_y bytes of mean frames, 8 n_x n_y of mu (synchronous).
 *   0 (default): off. */
#define DH_OPT_RESIDUAL 10
dh_status dh_plan_set_option(dh_plan_t plan, int option, int value);
dh_status dh_plan_get_option(dh_plan_t plan, int option, int *value);

/* Autotuner: times every candidate on zero frames (render and covariance time do not depend
 * on the values; best of three after a warm-up) and keeps the fastest in the plan's options:
 *   1. the DFT arithmetic of Eq. 1 (DH_OPT_RENDER_FFT 1 at the default and at the alternative
 *      DH_OPT_FFT_RADIX, and 2 for 1024 x 1024 frames), each with the default schedule;
 *   2. for the CUDA-core FFT, the schedule (DH_OPT_RENDER_SCHEDULE, _RING, _LAG): chunks; the
 *      persistent ring at the automatic lag, half and twice it; the automatic ring with one
 *      frame more lag;
 *   3. 16-bit storage: the covariance's split-K units (DH_OPT_GRAM_UNITS: the default, half,
 *      twice and a quarter of it), on up to 32 windows of the store.
 * Schedules give bitwise the same holograms; radix, DFT arithmetic and split-K units change
 * only the rounding. Renders n_frames (capped at the plan's slots) frames; discards rendered
 * holograms; allocates and frees a temporary frame buffer; synchronises `stream` and the
 * device. Call it after dh_plan_reserve, before any graph capture. */
dh_status dh_plan_autotune(dh_plan_t plan, int n_frames, void *stream);

/* The autotuner's persistent cache: a JSON file {"version": 1, "entries": {key: {option: value,
 * ...}}} whose key is the plan's frame size, T, precision, device name and SM count, and whose
 * values are the options the autotuner sets (render_schedule, render_ring, render_lag,
 * render_fft, fft_radix, gram_units).
 * dh_plan_tune_load: applies the plan's entry if the file has one (*found = 1), else changes
 *   nothing (*found = 0; also when the file does not exist). DH_ERR_INVALID_ARG for a file that
 *   is not such JSON, or an entry with a value the options reject (nothing applied).
 * dh_plan_tune_save: writes the plan's current options as its entry, keeping every other
 *   entry (written to path.tmp, then renamed over path). DH_ERR_INVALID_ARG if an existing
 *   file cannot be parsed (it is left as it is) or written.
 * Host-side file I/O only; the options they set behave as dh_plan_set_option. */
dh_status dh_plan_tune_load(dh_plan_t plan, const char *path, int *found);
dh_status dh_plan_tune_save(dh_plan_t plan, const char *path);

/* Bytes of device memory the plan holds now (all buffers). */
size_t dh_plan_device_bytes(dh_plan_t plan);

/* Bytes of device memory a plan of these sizes holds after dh_plan_set_precision(prec) and
 * dh_plan_reserve(max_frames, max_windows), computed without creating it (admission
 * control budgets with it). 0 for arguments dh_plan_create / dh_plan_reserve reject. */
size_t dh_plan_footprint(int nx, int ny, int T, dh_precision prec, int max_frames,
                         int max_windows);

/* Eq. 1 for n_frames frames: frame i (uint16, row-major n_y x n_x, caller-owned device
 * memory at frames_dev + i * frame_stride_elems) is rendered into hologram slot
 * first_slot + i. Requires frame_stride_elems >= n_x n_y and a multiple of 8,
 * frames_dev 16-byte aligned (frames are read with 16-byte loads), and the slots within
 * the reservation; otherwise DH_ERR_INVALID_ARG. Asynchronous. */
dh_status dh_render_frames(dh_plan_t plan, const uint16_t *frames_dev,
                           int64_t frame_stride_elems, int n_frames, int first_slot,
                           void *stream);

/* Eqs. 4-7 for n_windows windows; window w covers slots
 * [first_slot + w * slot_stride, ... + T). Writes image w (FP32, n_y x n_x row-major) to
 * images_dev + w * n_x n_y, and, if eigvals_dev is not NULL, the T eigenvalues of window
 * w (FP64, decreasing) to eigvals_dev + w * T. 0 <= k0 <= k1 < T. Overlapping windows
 * (slot_stride < T) share the rendered holograms. Asynchronous. */
dh_status dh_pca_windows(dh_plan_t plan, int first_slot, int slot_stride, int n_windows,
                         int k0, int k1, float *images_dev, double *eigvals_dev,
                         void *stream);

/* Banded covariance of a hologram store (16-bit storage): the real Gram of the rows Re H_f,
 * Im H_f for every pair of frames fewer than 64 apart among slots [first_slot, first_slot +
 * n_frames), computed once on the tensor cores (64-frame blocks b; the products X_b X_b^T and
 * X_b X_{b+1}^T, so each frame is read three times). Every
 * window of T <= 64 frames inside those slots -- any start, any stride, any plan over the
 * store (a view, or the plan itself) with DH_OPT_COVARIANCE = 2 -- then takes its Eq. 4
 * covariance from the band instead of reading its T frames again: for overlapping windows
 * (sliding windows of several lengths) this replaces re-reading each frame once per window
 * containing it. Call it on any plan of the store after rendering; it replaces the store's
 * previous band (stream-ordered: windows enqueued before it on other streams must have
 * finished). The first call (and a longer band) allocates the band buffers synchronously,
 * so make it once before a graph capture; asynchronous otherwise. DH_ERR_STATE for FP32
 * storage, DH_ERR_INVALID_ARG for slots outside the reservation. The paper computes C per
 * window; this computes the whole sequence's band at once. */
dh_status dh_band_gram(dh_plan_t plan, int first_slot, int n_frames, void *stream);

/* Eqs. 8-9, the paper's Fourier alternative to Eqs. 4-7: temporal demodulation of each
 * window by the unitary DFT W, w_{t,k} = exp(-2 pi i t k / T) / sqrt(T) (t, k counted from
 * 0), keeping the frequency bins k0..k1 (0 <= k0 <= k1 < T; the paper's filter indices
 * n_1..n_2 count from 1, so its n_1 = 8, n_2 = 24 at T = 32 are bins 7..23), and summing
 * their power: image w (FP32, n_y x n_x row-major, at images_dev + w * n_x n_y) is
 * M[p] = sum_{k=k0..k1} |sum_t H_t[p] w_{t,k}|^2 for window w = slots
 * [first_slot + w * slot_stride, + T). No covariance or eigendecomposition is computed;
 * windows of any number and stride (stride 1 = a new window per frame) share the rendered
 * holograms. Runs on the tensor cores for 16-bit storage (the DFT operand rounded once to
 * FP16 with FP16 holograms, which adds a few 1e-5 to the image's relative error; split into
 * hi + lo BF16 parts with BF16 holograms), on FP32 CUDA cores for FP32 storage. Overlapping windows (stride < T)
 * are computed together where possible: 7 at a time from one load of their frames on the
 * tensor cores (FP16 storage, 17 bins as the paper's 7..23 at T = 32, n_y >= 128), else one
 * frame read twice per window by a sliding DFT recurrence (stride 1). Asynchronous. */
dh_status dh_fourier_windows(dh_plan_t plan, int first_slot, int slot_stride, int n_windows,
                             int k0, int k1, float *images_dev, void *stream);

/* Eqs. 2-3 then Eqs. 8-9, the paper's earlier pipeline: singular value filtering of each
 * window, keeping components k0..k1 of the decreasing order (H_f = U Delta I_f V^{t*} =
 * H V I_f V^{t*}, V from Eqs. 4-5), then temporal demodulation of H_f by the unitary DFT,
 * keeping bins b0..b1 (counted from 0), and the power sum of Eq. 9. Image w and, if
 * eigvals_dev is not NULL, window w's T eigenvalues are written as by dh_pca_windows.
 * 0 <= k0 <= k1 < T, 0 <= b0 <= b1 < T. Asynchronous. */
dh_status dh_svd_fourier_windows(dh_plan_t plan, int first_slot, int slot_stride, int n_windows,
                                 int k0, int k1, int b0, int b1, float *images_dev,
                                 double *eigvals_dev, void *stream);

/* The single-window calls of the paper's statement of the problem: render T frames
 * (frames_dev + t * frame_stride_elems, t < T) into slots [0, T). Asynchronous. */
dh_status dh_render_stack(dh_plan_t plan, const uint16_t *frames_dev,
                          int64_t frame_stride_elems, void *stream);

/* PCA of the window held in slots [0, T): image to image_dev (n_y x n_x FP32). If
 * eigvals_host is not NULL the call synchronises `stream` and copies the T eigenvalues
 * (FP64, decreasing) to it. */
dh_status dh_pca_window(dh_plan_t plan, int k0, int k1, float *image_dev,
                        double *eigvals_host, void *stream);

/* Render then demodulate n_windows windows whose first frames are
 * window_stride_frames apart: frames are rendered once into slots
 * [0, (n_windows - 1) * window_stride_frames + T) and window w uses slots
 * [w * window_stride_frames, + T). Asynchronous. */
dh_status dh_pca_batch(dh_plan_t plan, const uint16_t *frames_dev,
                       int64_t frame_stride_elems, int n_windows,
                       int window_stride_frames, int k0, int k1, float *images_dev,
                       double *eigvals_dev, void *stream);

/* Display normalisation of n_images FP32 images of npix pixels each (back to back at
 * images_dev, e.g. the output of dh_pca_windows): the paper divides every displayed image by
 * its own average value. Writes each image's mean (FP64, fixed-order reduction) to
 * means_dev[i]; if normalized_dev is not NULL, image / mean (FP32, may equal images_dev); if
 * display_dev is not NULL, 8-bit display codes clamp(rint(gain * M / mean), 0, 255) (FP32
 * product; the mean maps to code `display_gain`), n_images x npix bytes: the headless
 * output of a display path (no graphics stack is used). Requires npix a multiple of 4,
 * 16-byte aligned images and normalized buffers, display_gain > 0. Asynchronous. */
dh_status dh_normalize_images(const float *images_dev, int n_images, int64_t npix,
                              float *normalized_dev, uint8_t *display_dev, float display_gain,
                              double *means_dev, void *stream);

/* dh_pca_batch from HOST memory, overlapping the transfers with the computation: frames
 * (uint16, frame i at frames_host + i * frame_stride_elems) are copied to the device in
 * groups of windows (up to 256 frames a group; the last groups halve down to one window, so
 * little work follows the last copy) on a copy stream, into two alternating
 * staging buffers, while the caller's stream renders and demodulates the previous group; the
 * images (n_windows x n_x n_y FP32) and, if eigvals_host is not NULL, the eigenvalues
 * (n_windows x T FP64) of each group are copied back on a second copy stream as soon as the
 * group is done. Use pinned host memory for the copies to overlap (pageable memory works,
 * with synchronous copies). The host buffers must stay valid until `stream` has passed this
 * call; `stream` is ordered after every copy. The staging buffers and the device images are
 * allocated on first use (synchronously) and kept by the plan. Asynchronous otherwise.
 * The paper's pipeline streams camera frames through a host buffer in the same way. */
dh_status dh_pca_batch_host(dh_plan_t plan, const uint16_t *frames_host, int64_t frame_stride_elems,
                            int n_windows, int window_stride_frames, int k0, int k1,
                            float *images_host, double *eigvals_host, void *stream);

/* dh_pca_batch_host for 12-bit camera frames in the packed pixel format Mono12p (GenICam
 * PFNC): pixel i of a frame occupies bits [12 i, 12 i + 12) of the frame's bytes read as one
 * little-endian bit string (two pixels in three bytes; pixel i = frame row-major index y n_x +
 * x). Frame i starts at frames_host + i * frame_stride_bytes (at least n_x n_y 3/2 bytes, a
 * multiple of 4). The packed bytes are copied (3/4 of the uint16 bytes) and expanded to uint16
 * on the device; everything else, including the results, is as dh_pca_batch_host with those
 * uint16 frames. The paper's camera delivers 12-bit frames; the format is a deployment choice
 * with no counterpart in the paper. */
dh_status dh_pca_batch_host_packed12(dh_plan_t plan, const uint8_t *frames_host, int64_t frame_stride_bytes,
                                     int n_windows, int window_stride_frames, int k0, int k1,
                                     float *images_host, double *eigvals_host, void *stream);

/* Expand n_frames (<= 65535) Mono12p frames of npix pixels (a multiple of 8) from device
 * memory (frame f at src_dev + f * src_stride_bytes: >= npix 3/2, a multiple of 4; src_dev
 * 4-byte aligned) to uint16 (frame f at dst_dev + f * dst_stride_elems: >= npix, a multiple
 * of 8; dst_dev 16-byte aligned). Asynchronous on `stream`. The device half of
 * dh_pca_batch_host_packed12, exported for tests and for callers that stage frames
 * themselves. */
dh_status dh_unpack_mono12p(const uint8_t *src_dev, int64_t src_stride_bytes, int64_t npix, int n_frames,
                            uint16_t *dst_dev, int64_t dst_stride_elems, void *stream);

/* Inspection (tests): copy hologram slot `slot` as interleaved FP32 (re, im) pairs,
 * n_x n_y of them, to out_dev. Asynchronous. */
dh_status dh_debug_hologram(dh_plan_t plan, int slot, float *out_dev, void *stream);

/* Inspection (tests): after dh_pca_windows, copy window w's covariance C (Eq. 4) as
 * T x T interleaved FP64 (re, im), row-major, to out_dev. Asynchronous. */
dh_status dh_debug_covariance(dh_plan_t plan, int w, double *out_dev, void *stream);

/* Inspection (tests): after dh_pca_windows, copy window w's eigenvectors V (Eq. 5,
 * columns in decreasing-eigenvalue order) as T x T interleaved FP64 (re, im), V[t][k]
 * row-major, to out_dev. Asynchronous. */
dh_status dh_debug_eigvecs(dh_plan_t plan, int w, double *out_dev, void *stream);

/* Wait for the plan's own work -- the streams its calls launched work on since the last
 * read, its second stream and its host-copy streams (the whole device only if the plan's
 * work was captured into a graph, or ran on more than 8 streams) -- then return the plan's
 * accumulated DH_FLAG_* bits in *flags and clear them. Returns DH_ERR_TIMEOUT when the bits
 * include DH_FLAG_WAIT_TIMEOUT (a bounded device-side wait gave up and its kernel skipped
 * work: that work's results are invalid; the context stays usable), else DH_OK. Not
 * concurrently with other calls on the same plan. */
dh_status dh_plan_status(dh_plan_t plan, uint32_t *flags);

/* Tracing: with on != 0, every kernel the plan launches from now on is bracketed by two
 * CUDA events on its stream (a few microseconds of overhead per launch); on == 0 stops
 * and discards the records. The paper has no tracing facility; this one exists to
 * attribute device time to the stages of Eqs. 1, 4, 5, 6-7. */
dh_status dh_profile_enable(dh_plan_t plan, int on);

/* Synchronise on the recorded events and report, for each of the library's kernels
 * (index k < n), its name (static string), the number of launches and the summed device
 * milliseconds since the last read; the records are then cleared. Any output array may be
 * NULL. Returns the number of kernel kinds the library has (write at most n entries). */
int dh_profile_read(dh_plan_t plan, int n, const char **names, int *launches, double *total_ms);

/* Arithmetic-rate measurement for rooflines (the paper has no counterpart; it serves the
 * measurement of the FP32-bound render of Eq. 1 and the FP64-bound eigensolver of Eq. 5):
 * launches blocks_per_sm (1..64) x SMs CTAs of 256 threads, each thread running 8
 * independent FMA chains for iters x 8 rounds, once to warm up and once timed with CUDA
 * events on `stream` (synchronised). kind 0: scalar FP32 FMA; 1: paired FP32 FMA (two lanes
 * per instruction); 2: FP64 FMA. *ms receives the timed launch's duration and *flops its
 * floating-point operations (2 per FMA lane). */
dh_status dh_measure_fma_rate(int kind, int iters, int blocks_per_sm, float *ms, double *flops,
                              void *stream);

/* Tensor-core issue-rate measurement (the paper has no counterpart; it serves the design and
 * the rooflines of the tensor-core kernels of Eqs. 4 and 6): one CTA per SM issues `stages`
 * (1..2^24) stages of four tcgen05.mma kind::f16 (M = 128, N = 128, K = 16, FP16 operands in
 * shared memory, FP32 accumulation in tensor memory) from one thread, with a commit per stage,
 * once to warm up and once timed with CUDA events on `stream` (synchronised). form 0: back to
 * back; 1: the issuing warp waits on a (completed) mbarrier before each stage; 2: another warp
 * does that wait and releases the issuing warp through a named barrier. *ms receives the timed
 * launch's duration, *cycles_per_mma the slowest CTA's SM cycles per MMA and *flops the
 * launch's floating-point operations. DH_ERR_TIMEOUT if a wait gave up. */
dh_status dh_measure_mma_issue(int form, int stages, float *ms, double *cycles_per_mma, double *flops,
                               void *stream);

/* The covariance of one window, C = H^{t*} H (the FP32 plain path's covariance), without
 * any device allocation, for callers that cannot call cudaMalloc while running (for example
 * a frame-grabber callback in a real-time acquisition loop, where an allocation can
 * synchronise the device, or code whose device memory belongs to another allocator). The
 * paper has no counterpart: it is a deployment variant of the covariance stage.
 *   planes_dev: caller-owned device FP32 array [2T][npix]: row 2t = Re H_t, row 2t+1 = Im H_t
 *               (pixels in any fixed order); npix a positive multiple of 32, <= 2^28;
 *               8-byte aligned (else DH_ERR_INVALID_ARG).
 *   T:          16, 32 or 64 (else DH_ERR_UNSUPPORTED_SIZE).
 *   C_dev:      caller-owned device FP64 output, T x T interleaved (re, im), row-major;
 *               8-byte aligned (else DH_ERR_INVALID_ARG). A non-finite covariance shows up
 *               as NaN/Inf entries here; no flag is reported.
 * Products are FP32 with FP64 accumulation (as the plain path). The split-K scratch is a
 * fixed 2 MiB device array inside the library (16 partial matrices at T = 64, 64 at
 * T <= 32), held by every GPU that loads the library until exit. The first call on a device
 * looks up that array's address and loads the library's kernels for this entry point (which
 * can allocate): make one call per device before real-time use and before any stream
 * capture. All calls share the array, so calls that overlap on the GPU race. Asynchronous
 * on `stream`. */
dh_status dh_covariance_noalloc(const float *planes_dev, int64_t npix, int T, double *C_dev,
                                void *stream);

/* One item of a batch (dh_batch_run). */
typedef struct {
  dh_plan_t plan;                 /* a plan or a view */
  const uint16_t *frames_dev;     /* NULL, or frames to render first (Eq. 1), through the
                                     store's base plan, as dh_render_frames: */
  int64_t frame_stride_elems;     /*   frame i at frames_dev + i * frame_stride_elems */
  int n_frames;                   /*   into slots [render_slot, render_slot + n_frames) */
  int render_slot;
  int first_slot;                 /* then Eqs. 4-7 for n_windows windows, as dh_pca_windows */
  int slot_stride;                /* (n_windows = 0: render only) */
  int n_windows;
  int k0, k1;
  float *images_dev;
  double *eigvals_dev;            /* may be NULL */
} dh_batch_item;

/* Run a batch of up to 64 items over any mix of frame sizes, window lengths and plans, on
 * branch streams forked from `stream` and joined back into it before the call returns (the
 * batch is ordered after earlier work on `stream`; later work waits for all of it; the batch
 * can be captured into one graph with dh_graph_begin). Ordering: the renders of one hologram
 * store run in the given order; the windows of one plan run in the given order; the windows
 * of different plans run concurrently, each after the earlier renders of its store (so the
 * views of one store, and different stores, overlap on the device); a render waits for the
 * earlier windows that read its store. Up to 8 branch streams (more branches share them,
 * which only adds ordering). Every item is validated before anything is launched
 * (DH_ERR_INVALID_ARG); a plan in use by another call gives DH_ERR_STATE. The paper runs
 * one frame size and one window length; this batches several. Asynchronous. */
dh_status dh_batch_run(const dh_batch_item *items, int n_items, void *stream);

/* ---------------------------------------------------------------- serving
 * A server runs several camera streams at once. Each stream has its own plan (frame size,
 * optics, window length T, storage type, retained range), a device frame ring and hologram
 * slots for two windows, an output ring of ring_windows images on the device and in pinned
 * host memory, and its own CUDA stream: windows of different streams run concurrently on
 * the device as soon as each is complete. Streams are admitted against an HBM budget. The
 * paper processes one camera; the server is this library's multi-stream runtime around
 * the same stages (Eqs. 1, 4-7). */
typedef struct dh_server *dh_server_t;

typedef struct {
  int stream_id;
  int64_t window;              /* window w of the stream covers its frames [w T, w T + T) */
  const float *image_host;     /* n_x n_y FP32 image (Eq. 7) in the server's pinned ring */
  const double *eigvals_host;  /* T eigenvalues, decreasing */
  double t_ready_s;            /* server clock when the push completing the window began */
  double t_done_s;             /* server clock when image and eigenvalues were in host memory */
} dh_window_result;

/* A server on the current device with `hbm_budget_bytes` of device memory to admit streams
 * into. Synchronous. */
dh_status dh_server_create(dh_server_t *out, size_t hbm_budget_bytes);

/* Device bytes one stream of these parameters is charged (plan with 2T slots and one
 * window, frame ring of 2T frames, ring_windows images and eigenvalue sets); 0 for
 * unsupported sizes. */
size_t dh_server_stream_bytes(int nx, int ny, int T, dh_precision prec, int ring_windows);

/* Admit a stream: DH_ERR_OOM (nothing allocated) when its bytes exceed what is left of the
 * budget; otherwise allocates it and writes its id. Arguments as dh_plan_create, plus the
 * storage type, the retained range 0 <= k0 <= k1 < T and ring_windows >= 1. Synchronous
 * (allocations may briefly stall the device). */
dh_status dh_server_add_stream(dh_server_t server, int nx, int ny, double lambda_m, double z_m,
                               double pitch_m, int T, dh_precision prec, int k0, int k1,
                               int ring_windows, int *stream_id);

/* Wait for the stream's work, drop its unpolled results, free it and return its bytes to
 * the budget. */
dh_status dh_server_remove_stream(dh_server_t server, int stream_id);

/* Restart from the autotuner's cache (see dh_plan_tune_load): every stream admitted after
 * this call gets its plan's options from the JSON file at `path` when the file has an entry
 * for the stream's frame size, T, storage type and device. With autotune = 1 a stream
 * without an entry is autotuned once at admission (dh_plan_autotune on its 2T slots:
 * synchronous, some milliseconds of device time) and its picks are saved to the file, so
 * that a restarted server rebuilds the same plans without measuring. path = NULL turns it
 * off. The path is copied. An unreadable file makes later admissions fail with
 * DH_ERR_INVALID_ARG (nothing allocated). The paper's pipeline has no counterpart. */
dh_status dh_server_set_tune_cache(dh_server_t server, const char *path, int autotune);

/* One option (DH_OPT_*) of an admitted stream's plan, as dh_plan_get_option. */
dh_status dh_server_stream_option(dh_server_t server, int stream_id, int option, int *value);

/* Device bytes charged to admitted streams. */
size_t dh_server_used_bytes(dh_server_t server);

/* Hand n_frames (1..T) consecutive frames of a stream, starting at frame_index, to the
 * server: host uint16 frames, n_y x n_x row-major, back to back. They are copied to the
 * device (asynchronously when the memory is pinned: keep it unchanged until the window
 * holding the last of them has been polled), rendered, and every window they complete is
 * launched. Returns without waiting for the device.
 * Errors: DH_ERR_FRAME_GAP when frame_index is not the stream's next frame (nothing is
 * done; push the missing frames or remove the stream); DH_ERR_STATE when a completed window
 * needs an output slot whose previous result has not been released (nothing is done:
 * poll, release and push again); DH_ERR_INVALID_ARG. */
dh_status dh_server_push(dh_server_t server, int stream_id, const uint16_t *frames_host,
                         int64_t frame_index, int n_frames);

/* Up to max_results finished windows of any stream, in completion order; non-blocking.
 * Returns how many were written. A result's host buffers stay valid until it is released. */
int dh_server_poll(dh_server_t server, dh_window_result *out, int max_results);

/* Give a result's output slot back to its stream. */
dh_status dh_server_release(dh_server_t server, int stream_id, int64_t window);

/* Seconds since the server was created, the clock of t_ready_s and t_done_s. */
double dh_server_clock(dh_server_t server);

/* Wait until every pushed window of every stream has finished. */
dh_status dh_server_drain(dh_server_t server);

/* Free every stream and the server. NULL-safe. */
void dh_server_destroy(dh_server_t server);

/* CUDA graphs of library calls. dh_graph_begin starts capturing `stream` (a created
 * stream, not NULL: the legacy default stream cannot be captured; capture mode
 * thread-local). Every library call made on that stream until dh_graph_end is recorded,
 * not run, including the work the library forks onto a plan's internal stream and joins
 * back. dh_graph_end ends the capture and instantiates it into *out; dh_graph_launch runs
 * it on a stream (asynchronous), any number of times, against the same buffers and
 * arguments as captured. Calls that synchronise (dh_pca_window with eigvals_host,
 * dh_plan_status, create/reserve/destroy) must not be made during a capture (they fail
 * with DH_ERR_CUDA and invalidate it). Per-kernel tracing skips captured launches. The
 * paper launches library calls one by one; graphs remove the host launch cost of the
 * many short launches of small frames. */
dh_status dh_graph_begin(void *stream);
dh_status dh_graph_end(void *stream, dh_graph_t *out);
dh_status dh_graph_launch(dh_graph_t graph, void *stream);
void dh_graph_destroy(dh_graph_t graph); /* NULL-safe */

/* Text of a status code, and of the last CUDA error recorded by the library. */
const char *dh_status_string(dh_status s);
const char *dh_last_error(void);

/* Library version string. */
const char *dh_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DH_H_ */
