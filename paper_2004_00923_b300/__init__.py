"""Real-time digital holography of the retina by PCA on one B300 (sm_103a).

Python binding of libdh (include/dh.h): every method marshals tensors and the current
CUDA stream into one C-ABI call; all computation runs in the library's CUDA kernels.

    plan = Plan(1024, 1024, 785e-9, 0.35, 20e-6, T=32, precision="fp16",
                max_frames=2048, max_windows=64)
    images, lam = plan.pca_batch(frames, n_windows=64, window_stride=32, k0=2, k1=31)

Paper: Puyo et al., "Real-time digital holography of the retina by principal component
analysis", arXiv 2004.00923 (Eqs. 1, 4, 5, 6, 7).
"""

from __future__ import annotations

import contextlib
import ctypes
import os

import torch

from . import _lib
from ._lib import DHError, PREC  # noqa: F401

__all__ = ["Plan", "Graph", "Server", "capture", "run_batch", "normalize_images", "save_pgm",
           "DHError", "PREC", "version"]


def version() -> str:
    return _lib.load().dh_version().decode()


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: torch.Tensor) -> int:
    return int(t.data_ptr())


class Plan:
    """A device-resident plan: chirp/twiddle tables, hologram store and workspaces."""

    def __init__(self, nx: int, ny: int, lambda_m: float, z_m: float, pitch_m: float, T: int,
                 precision: str = "fp32", max_frames: int | None = None, max_windows: int = 1):
        self._lib = _lib.load()
        self.nx, self.ny, self.T = int(nx), int(ny), int(T)
        self.precision = precision
        h = ctypes.c_void_p()
        _lib.check("dh_plan_create", self._lib.dh_plan_create(
            ctypes.byref(h), self.nx, self.ny, float(lambda_m), float(z_m), float(pitch_m), self.T))
        self._h = h
        if precision != "fp32":
            _lib.check("dh_plan_set_precision", self._lib.dh_plan_set_precision(h, PREC[precision]))
        self.max_frames = max(int(max_frames or T), self.T)
        self.max_windows = int(max_windows)
        if self.max_frames != self.T or self.max_windows != 1:
            _lib.check("dh_plan_reserve",
                       self._lib.dh_plan_reserve(h, self.max_frames, self.max_windows))

    def view(self, T: int, max_windows: int = 1) -> "Plan":
        """A plan for windows of T frames over this plan's hologram store
        (dh_plan_create_view): windows of several lengths share one rendering."""
        v = Plan.__new__(Plan)
        v._lib = self._lib
        v.nx, v.ny, v.T = self.nx, self.ny, int(T)
        v.precision = self.precision
        h = ctypes.c_void_p()
        _lib.check("dh_plan_create_view",
                   self._lib.dh_plan_create_view(ctypes.byref(h), self._h, v.T))
        v._h = h
        v.max_frames = self.max_frames
        v.max_windows = int(max_windows)
        if v.max_windows != 1:
            _lib.check("dh_plan_reserve",
                       self._lib.dh_plan_reserve(h, v.max_frames, v.max_windows))
        return v

    # -- lifetime -------------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.dh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_render_schedule(self, persistent: bool, ring: int = 0, lag: int = 0) -> None:
        """DH_OPT_RENDER_SCHEDULE / _RING / _LAG: one persistent launch over an L2 ring (True,
        the default where it applies; ring and lag 0 = automatic) or chunks of row/column
        launches (False)."""
        for opt, val in ((0, 0 if persistent else 1), (1, int(ring)), (2, int(lag))):
            _lib.check("dh_plan_set_option", self._lib.dh_plan_set_option(self._h, opt, val))

    def set_render_fft(self, kind: str = "auto") -> None:
        """DH_OPT_RENDER_FFT: "auto" (0), "cuda" (1: CUDA-core FFT) or "tensor" (2: 32-point
        DFT stages on the tensor cores, 1024 x 1024 frames)."""
        _lib.check("dh_plan_set_option", self._lib.dh_plan_set_option(
            self._h, 7, {"auto": 0, "cuda": 1, "tensor": 2}[kind]))

    def set_covariance_source(self, source) -> None:
        """DH_OPT_COVARIANCE: "holograms" (Eq. 4 as written, the default; also False), "raw"
        (exact C = I^T I from the uint16 frames where the call has them; also True) or "band"
        (the store's banded Gram, see band_gram)."""
        mode = {False: 0, True: 1, "holograms": 0, "raw": 1, "band": 2}[source]
        _lib.check("dh_plan_set_option", self._lib.dh_plan_set_option(self._h, 3, mode))

    def set_projection(self, grouped: bool = True) -> None:
        """DH_OPT_PROJECTION: grouped (the default: overlapping windows share their tile loads
        and take the power as energy minus the discarded components' power, where that
        applies) or per window (False: Eq. 7 over the kept components, always)."""
        _lib.check("dh_plan_set_option", self._lib.dh_plan_set_option(self._h, 4, 0 if grouped else 1))

    def set_window_groups(self, automatic: bool = True) -> None:
        """DH_OPT_WINDOW_GROUPS: automatic (the default: two groups of windows, each one's
        eigensolver beside the other's covariance or projection, where that applies) or one
        group (False). Both give bitwise the same results."""
        _lib.check("dh_plan_set_option", self._lib.dh_plan_set_option(self._h, 5, 0 if automatic else 1))

    def band_gram(self, first_slot: int, n_frames: int, stream=None) -> None:
        """dh_band_gram: the banded covariance of slots [first_slot, first_slot + n_frames)."""
        _lib.check("dh_band_gram", self._lib.dh_band_gram(self._h, int(first_slot), int(n_frames),
                                                           _stream_ptr(stream)))

    def render_schedule(self) -> dict:
        """The plan's render and covariance options: persistent (bool), ring and lag (0 =
        automatic), fft ("auto" / "cuda" / "tensor"), radix (0 = each length's default) and
        gram_units (0 = the frame size's default)."""
        v = ctypes.c_int(0)
        out = {}
        for opt, key in ((0, "persistent"), (1, "ring"), (2, "lag"), (7, "fft"), (8, "radix"),
                         (9, "gram_units")):
            _lib.check("dh_plan_get_option", self._lib.dh_plan_get_option(self._h, opt, ctypes.byref(v)))
            if opt == 0:
                out[key] = v.value == 0
            elif opt == 7:
                out[key] = {0: "auto", 1: "cuda", 2: "tensor"}[v.value]
            else:
                out[key] = v.value
        return out

    def set_fft_radix(self, radix: int = 0) -> None:
        """DH_OPT_FFT_RADIX: 0 (each length's default), 16 or 32 where instantiated."""
        _lib.check("dh_plan_set_option", self._lib.dh_plan_set_option(self._h, 8, int(radix)))

    def set_residual(self, on: bool = True) -> None:
        """DH_OPT_RESIDUAL: mean-residual storage for pca_batch's windows (16-bit storage)."""
        _lib.check("dh_plan_set_option", self._lib.dh_plan_set_option(self._h, 10, 1 if on else 0))

    def set_gram_units(self, units: int = 0) -> None:
        """DH_OPT_GRAM_UNITS: split-K units per window of the tensor-core covariance (0 =
        the frame size's default)."""
        _lib.check("dh_plan_set_option", self._lib.dh_plan_set_option(self._h, 9, int(units)))

    def autotune(self, n_frames: int = 256, stream=None, cache: str | None = None) -> dict:
        """dh_plan_autotune: time the candidate DFT arithmetic, radix, render schedule and
        covariance split-K units on zero frames and keep the fastest. With `cache`, the plan's
        entry in that JSON file is applied instead when present (dh_plan_tune_load), and the
        picks are saved there after a measurement (dh_plan_tune_save). The returned options
        carry "from_cache"."""
        found = ctypes.c_int(0)
        if cache is not None:
            _lib.check("dh_plan_tune_load", self._lib.dh_plan_tune_load(
                self._h, os.fsencode(cache), ctypes.byref(found)))
        if not found.value:
            _lib.check("dh_plan_autotune", self._lib.dh_plan_autotune(self._h, int(n_frames),
                                                                       _stream_ptr(stream)))
            if cache is not None:
                _lib.check("dh_plan_tune_save", self._lib.dh_plan_tune_save(self._h, os.fsencode(cache)))
        out = self.render_schedule()
        out["from_cache"] = bool(found.value)
        return out

    @property
    def device_bytes(self) -> int:
        return int(self._lib.dh_plan_device_bytes(self._h))

    # -- checks ---------------------------------------------------------------
    def _frames(self, frames: torch.Tensor) -> torch.Tensor:
        if frames.dtype != torch.uint16 or not frames.is_cuda:
            raise TypeError("frames must be a CUDA uint16 tensor [F, ny, nx]")
        if frames.dim() != 3 or frames.shape[1:] != (self.ny, self.nx) or not frames.is_contiguous():
            raise ValueError(f"frames must be contiguous [F, {self.ny}, {self.nx}]")
        return frames

    # -- the C ABI ------------------------------------------------------------
    def render_frames(self, frames: torch.Tensor, first_slot: int = 0, stream=None) -> None:
        """Eq. 1 for every frame of `frames` into slots first_slot, first_slot+1, ..."""
        f = self._frames(frames)
        _lib.check("dh_render_frames", self._lib.dh_render_frames(
            self._h, _ptr(f), self.nx * self.ny, f.shape[0], int(first_slot), _stream_ptr(stream)))

    def pca_windows(self, first_slot: int, slot_stride: int, n_windows: int, k0: int, k1: int,
                    images: torch.Tensor | None = None, eigvals: torch.Tensor | None = None,
                    want_eigvals: bool = True, stream=None):
        """Eqs. 4-7 for windows [first_slot + w*slot_stride, +T). Returns (images, eigvals)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        if images is None:
            images = torch.empty((n_windows, self.ny, self.nx), dtype=torch.float32, device=dev)
        if eigvals is None and want_eigvals:
            eigvals = torch.empty((n_windows, self.T), dtype=torch.float64, device=dev)
        _lib.check("dh_pca_windows", self._lib.dh_pca_windows(
            self._h, int(first_slot), int(slot_stride), int(n_windows), int(k0), int(k1),
            _ptr(images), _ptr(eigvals) if eigvals is not None else None, _stream_ptr(stream)))
        return images, eigvals

    def fourier_windows(self, first_slot: int, slot_stride: int, n_windows: int, k0: int,
                        k1: int, images: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Eqs. 8-9 for windows [first_slot + w*slot_stride, +T): power of the unitary DFT's
        bins k0..k1 (counted from 0). Returns the images [n_windows, ny, nx]."""
        if images is None:
            images = torch.empty((n_windows, self.ny, self.nx), dtype=torch.float32,
                                 device=torch.device("cuda", torch.cuda.current_device()))
        _lib.check("dh_fourier_windows", self._lib.dh_fourier_windows(
            self._h, int(first_slot), int(slot_stride), int(n_windows), int(k0), int(k1),
            _ptr(images), _stream_ptr(stream)))
        return images

    def svd_fourier_windows(self, first_slot: int, slot_stride: int, n_windows: int, k0: int,
                            k1: int, b0: int, b1: int, images: torch.Tensor | None = None,
                            eigvals: torch.Tensor | None = None, want_eigvals: bool = True,
                            stream=None):
        """Eqs. 2-3 then 8-9: SVD filter keeping components k0..k1 (decreasing order), DFT
        bins b0..b1. Returns (images, eigvals)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        if images is None:
            images = torch.empty((n_windows, self.ny, self.nx), dtype=torch.float32, device=dev)
        if eigvals is None and want_eigvals:
            eigvals = torch.empty((n_windows, self.T), dtype=torch.float64, device=dev)
        _lib.check("dh_svd_fourier_windows", self._lib.dh_svd_fourier_windows(
            self._h, int(first_slot), int(slot_stride), int(n_windows), int(k0), int(k1),
            int(b0), int(b1), _ptr(images), _ptr(eigvals) if eigvals is not None else None,
            _stream_ptr(stream)))
        return images, eigvals

    def render_stack(self, frames: torch.Tensor, stream=None) -> None:
        f = self._frames(frames)
        if f.shape[0] < self.T:
            raise ValueError("render_stack needs T frames")
        _lib.check("dh_render_stack", self._lib.dh_render_stack(
            self._h, _ptr(f), self.nx * self.ny, _stream_ptr(stream)))

    def pca_window(self, k0: int, k1: int, image: torch.Tensor | None = None, stream=None):
        """Eqs. 4-7 on slots [0, T); returns (image, eigenvalues as a host float64 tensor)."""
        if image is None:
            image = torch.empty((self.ny, self.nx), dtype=torch.float32,
                                device=torch.device("cuda", torch.cuda.current_device()))
        lam = torch.empty(self.T, dtype=torch.float64)
        _lib.check("dh_pca_window", self._lib.dh_pca_window(
            self._h, int(k0), int(k1), _ptr(image), _ptr(lam), _stream_ptr(stream)))
        return image, lam

    def pca_batch(self, frames: torch.Tensor, n_windows: int, window_stride: int, k0: int, k1: int,
                  images: torch.Tensor | None = None, eigvals: torch.Tensor | None = None,
                  want_eigvals: bool = True, stream=None):
        f = self._frames(frames)
        dev = f.device
        if images is None:
            images = torch.empty((n_windows, self.ny, self.nx), dtype=torch.float32, device=dev)
        if eigvals is None and want_eigvals:
            eigvals = torch.empty((n_windows, self.T), dtype=torch.float64, device=dev)
        _lib.check("dh_pca_batch", self._lib.dh_pca_batch(
            self._h, _ptr(f), self.nx * self.ny, int(n_windows), int(window_stride), int(k0),
            int(k1), _ptr(images), _ptr(eigvals) if eigvals is not None else None,
            _stream_ptr(stream)))
        return images, eigvals

    def pca_batch_host(self, frames_host: torch.Tensor, n_windows: int, window_stride: int,
                       k0: int, k1: int, images_host: torch.Tensor | None = None,
                       eigvals_host: torch.Tensor | None = None, want_eigvals: bool = True,
                       stream=None, sync: bool = True):
        """dh_pca_batch_host: frames in host memory (pinned to overlap the copies), images and
        eigenvalues back in host memory; with sync=True the stream is synchronised."""
        f = frames_host
        if f.dtype != torch.uint16 or f.is_cuda or f.dim() != 3 or f.shape[1:] != (self.ny, self.nx) \
                or not f.is_contiguous():
            raise TypeError(f"frames must be a contiguous host uint16 tensor [F, {self.ny}, {self.nx}]")
        pin = f.is_pinned()
        if images_host is None:
            images_host = torch.empty((n_windows, self.ny, self.nx), dtype=torch.float32, pin_memory=pin)
        if eigvals_host is None and want_eigvals:
            eigvals_host = torch.empty((n_windows, self.T), dtype=torch.float64, pin_memory=pin)
        _lib.check("dh_pca_batch_host", self._lib.dh_pca_batch_host(
            self._h, _ptr(f), self.nx * self.ny, int(n_windows), int(window_stride), int(k0),
            int(k1), _ptr(images_host), _ptr(eigvals_host) if eigvals_host is not None else None,
            _stream_ptr(stream)))
        if sync:
            (stream or torch.cuda.current_stream()).synchronize()
        return images_host, eigvals_host

    def pca_batch_host_packed12(self, frames_packed: torch.Tensor, n_windows: int, window_stride: int,
                                k0: int, k1: int, images_host: torch.Tensor | None = None,
                                eigvals_host: torch.Tensor | None = None, want_eigvals: bool = True,
                                stream=None, sync: bool = True):
        """dh_pca_batch_host_packed12: as pca_batch_host, for Mono12p frames in host memory
        (a contiguous uint8 tensor [F, n_x n_y 3/2], e.g. from pack_mono12p)."""
        f = frames_packed
        nbytes = self.nx * self.ny // 2 * 3
        if f.dtype != torch.uint8 or f.is_cuda or f.dim() != 2 or f.shape[1] != nbytes or not f.is_contiguous():
            raise TypeError(f"frames must be a contiguous host uint8 tensor [F, {nbytes}]")
        pin = f.is_pinned()
        if images_host is None:
            images_host = torch.empty((n_windows, self.ny, self.nx), dtype=torch.float32, pin_memory=pin)
        if eigvals_host is None and want_eigvals:
            eigvals_host = torch.empty((n_windows, self.T), dtype=torch.float64, pin_memory=pin)
        _lib.check("dh_pca_batch_host_packed12", self._lib.dh_pca_batch_host_packed12(
            self._h, _ptr(f), nbytes, int(n_windows), int(window_stride), int(k0), int(k1),
            _ptr(images_host), _ptr(eigvals_host) if eigvals_host is not None else None,
            _stream_ptr(stream)))
        if sync:
            (stream or torch.cuda.current_stream()).synchronize()
        return images_host, eigvals_host

    # -- inspection -----------------------------------------------------------
    def debug_hologram(self, slot: int, stream=None) -> torch.Tensor:
        out = torch.empty((self.ny, self.nx, 2), dtype=torch.float32, device="cuda")
        _lib.check("dh_debug_hologram", self._lib.dh_debug_hologram(
            self._h, int(slot), _ptr(out), _stream_ptr(stream)))
        return torch.view_as_complex(out)

    def debug_covariance(self, w: int = 0, stream=None) -> torch.Tensor:
        out = torch.empty((self.T, self.T, 2), dtype=torch.float64, device="cuda")
        _lib.check("dh_debug_covariance", self._lib.dh_debug_covariance(
            self._h, int(w), _ptr(out), _stream_ptr(stream)))
        return torch.view_as_complex(out)

    def debug_eigvecs(self, w: int = 0, stream=None) -> torch.Tensor:
        out = torch.empty((self.T, self.T, 2), dtype=torch.float64, device="cuda")
        _lib.check("dh_debug_eigvecs", self._lib.dh_debug_eigvecs(
            self._h, int(w), _ptr(out), _stream_ptr(stream)))
        return torch.view_as_complex(out)

    def profile(self, on: bool = True) -> None:
        """Enable/disable per-kernel CUDA-event timing inside the library."""
        _lib.check("dh_profile_enable", self._lib.dh_profile_enable(self._h, 1 if on else 0))

    def profile_read(self) -> dict:
        """{kernel name: (launches, total device ms)} since the last read (synchronises)."""
        n = 64  # more than the library's kernel kinds (the call returns how many it has)
        names = (ctypes.c_char_p * n)()
        launches = (ctypes.c_int * n)()
        ms = (ctypes.c_double * n)()
        k = self._lib.dh_profile_read(self._h, n, names, launches, ms)
        return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(k, n))}

    def status(self) -> int:
        """The plan's DH_FLAG_* bits since the last read (then cleared), after waiting for the
        plan's own work. A timed-out device wait (DH_ERR_TIMEOUT from the C ABI) shows as
        DH_FLAG_WAIT_TIMEOUT (0x8) in the returned bits."""
        flags = ctypes.c_uint32(0)
        rc = self._lib.dh_plan_status(self._h, ctypes.byref(flags))
        if rc != 5:  # DH_ERR_TIMEOUT: reported through the flags
            _lib.check("dh_plan_status", rc)
        return int(flags.value)

    def set_test_stall(self, cycles: int) -> None:
        """DH_OPT_TEST_STALL (test only): the persistent render's CTAs first wait `cycles`
        SM cycles on a device word nothing sets, give up, and skip their work; the 16-bit
        tensor-core covariance's waiter warp does the same and the launch takes its abort path;
        the next status read reports DH_ERR_TIMEOUT. 0 turns it off."""
        _lib.check("dh_plan_set_option", self._lib.dh_plan_set_option(self._h, 6, int(cycles)))


def pack_mono12p(frames) -> torch.Tensor:
    """Host-side packing of 12-bit frames (values < 4096, uint16 [F, ny, nx] as a numpy array or
    a CPU tensor) into Mono12p: pixel i of a frame occupies bits [12 i, 12 i + 12) of the frame's
    bytes read as one little-endian bit string, so pixels 2j and 2j + 1 fill bytes 3j .. 3j + 2.
    Returns a contiguous uint8 tensor [F, ny nx 3/2]. Raises ValueError on values >= 4096."""
    import numpy as np
    a = frames.numpy() if isinstance(frames, torch.Tensor) else np.asarray(frames)
    if a.dtype != np.uint16 or a.ndim != 3 or (a.shape[1] * a.shape[2]) % 2:
        raise TypeError("frames must be uint16 [F, ny, nx] with an even pixel count")
    if a.size and int(a.max()) >= 4096:
        raise ValueError("Mono12p holds 12-bit values (< 4096)")
    v = a.reshape(a.shape[0], -1, 2).astype(np.uint32)
    lo, hi = v[..., 0], v[..., 1]
    out = np.empty((a.shape[0], v.shape[1], 3), dtype=np.uint8)
    out[..., 0] = lo & 0xFF
    out[..., 1] = (lo >> 8) | ((hi & 0xF) << 4)
    out[..., 2] = hi >> 4
    return torch.from_numpy(out.reshape(a.shape[0], -1))


def unpack_mono12p(packed: torch.Tensor, ny: int, nx: int, stream=None) -> torch.Tensor:
    """dh_unpack_mono12p: Mono12p frames on the device (uint8 [F, ny nx 3/2]) to uint16
    [F, ny, nx] on the device."""
    lib = _lib.load()
    if packed.dtype != torch.uint8 or not packed.is_cuda or packed.dim() != 2 or not packed.is_contiguous():
        raise TypeError("packed must be a contiguous CUDA uint8 tensor [F, ny nx 3/2]")
    npix = ny * nx
    out = torch.empty((packed.shape[0], ny, nx), dtype=torch.uint16, device=packed.device)
    _lib.check("dh_unpack_mono12p", lib.dh_unpack_mono12p(_ptr(packed), int(packed.shape[1]), npix,
                                                         int(packed.shape[0]), _ptr(out), npix,
                                                         _stream_ptr(stream)))
    return out


def measure_fma_rate(kind: str = "fp32", iters: int = 4096, blocks_per_sm: int = 4,
                     stream=None) -> dict:
    """dh_measure_fma_rate: the FMA throughput this GPU sustains now. kind: "fp32" (scalar
    FMA), "fp32x2" (paired FMA) or "fp64". Returns {"ms", "flops", "tflops"}."""
    lib = _lib.load()
    k = {"fp32": 0, "fp32x2": 1, "fp64": 2}[kind]
    ms, fl = ctypes.c_float(0), ctypes.c_double(0)
    _lib.check("dh_measure_fma_rate", lib.dh_measure_fma_rate(k, int(iters), int(blocks_per_sm),
                                                              ctypes.byref(ms), ctypes.byref(fl),
                                                              _stream_ptr(stream)))
    return {"ms": float(ms.value), "flops": float(fl.value),
            "tflops": float(fl.value) / (float(ms.value) * 1e-3) / 1e12}


def measure_mma_issue(form: str = "back-to-back", stages: int = 4096, stream=None) -> dict:
    """dh_measure_mma_issue: tcgen05.mma (M = N = 128, K = 16) issue rate, one CTA per SM.
    form: "back-to-back" (0), "mbarrier-wait" (1: the issuing warp waits on an mbarrier each
    stage) or "waiter-warp" (2: another warp waits and releases it by a named barrier).
    Returns {"ms", "cycles_per_mma", "tflops"}."""
    lib = _lib.load()
    f = {"back-to-back": 0, "mbarrier-wait": 1, "waiter-warp": 2}[form]
    ms, cyc, fl = ctypes.c_float(0), ctypes.c_double(0), ctypes.c_double(0)
    _lib.check("dh_measure_mma_issue", lib.dh_measure_mma_issue(f, int(stages), ctypes.byref(ms),
                                                                ctypes.byref(cyc), ctypes.byref(fl),
                                                                _stream_ptr(stream)))
    return {"ms": float(ms.value), "cycles_per_mma": float(cyc.value),
            "tflops": float(fl.value) / (float(ms.value) * 1e-3) / 1e12}


def normalize_images(images: torch.Tensor, normalized: bool = True, display: bool = False,
                     gain: float = 128.0, in_place: bool = False, stream=None):
    """dh_normalize_images on CUDA FP32 images [n, ny, nx]: returns (normalized or None,
    display uint8 or None, means float64 [n])."""
    if images.dtype != torch.float32 or not images.is_cuda or not images.is_contiguous():
        raise TypeError("images must be a contiguous CUDA float32 tensor [n, ny, nx]")
    imgs = images if images.dim() == 3 else images.unsqueeze(0)
    n, npix = imgs.shape[0], imgs.shape[1] * imgs.shape[2]
    means = torch.empty(n, dtype=torch.float64, device=imgs.device)
    norm = (imgs if in_place else torch.empty_like(imgs)) if normalized else None
    disp = torch.empty(imgs.shape, dtype=torch.uint8, device=imgs.device) if display else None
    _lib.check("dh_normalize_images", _lib.load().dh_normalize_images(
        _ptr(imgs), n, npix, _ptr(norm) if norm is not None else None,
        _ptr(disp) if disp is not None else None, float(gain), _ptr(means), _stream_ptr(stream)))
    return norm, disp, means


def save_pgm(path: str, image_u8) -> None:
    """Write an 8-bit image [ny, nx] (host or device tensor) as a binary PGM file."""
    a = image_u8.detach().cpu().numpy() if isinstance(image_u8, torch.Tensor) else image_u8
    ny, nx = a.shape
    with open(path, "wb") as f:
        f.write(f"P5\n{nx} {ny}\n255\n".encode())
        f.write(a.astype("uint8").tobytes())


def run_batch(items, stream=None) -> None:
    """dh_batch_run: `items` is a list of dicts with keys plan (a Plan or view), and
    optionally frames (CUDA uint16 [F, ny, nx] rendered first into slots render_slot...),
    render_slot, first_slot, slot_stride, n_windows, k0, k1, images, eigvals."""
    lib = _lib.load()
    arr = (_lib.BatchItem * len(items))()
    for a, it in zip(arr, items):
        plan = it["plan"]
        a.plan = plan._h.value
        f = it.get("frames")
        if f is not None:
            f = plan._frames(f)
            a.frames_dev, a.frame_stride_elems, a.n_frames = _ptr(f), plan.nx * plan.ny, f.shape[0]
            a.render_slot = int(it.get("render_slot", 0))
        a.n_windows = int(it.get("n_windows", 0))
        if a.n_windows:
            a.first_slot, a.slot_stride = int(it.get("first_slot", 0)), int(it["slot_stride"])
            a.k0, a.k1 = int(it["k0"]), int(it["k1"])
            a.images_dev = _ptr(it["images"])
            ev = it.get("eigvals")
            a.eigvals_dev = _ptr(ev) if ev is not None else None
    _lib.check("dh_batch_run", lib.dh_batch_run(arr, len(items), _stream_ptr(stream)))


class Graph:
    """An instantiated CUDA graph of library calls (dh_graph_*)."""

    def __init__(self):
        self._lib = _lib.load()
        self._h = None

    def launch(self, stream=None) -> None:
        _lib.check("dh_graph_launch", self._lib.dh_graph_launch(self._h, _stream_ptr(stream)))

    def close(self) -> None:
        if self._h is not None and self._h.value:
            self._lib.dh_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@contextlib.contextmanager
def capture(stream: torch.cuda.Stream):
    """Record the library calls made on `stream` (a created stream, made current inside the
    block) into a Graph instead of running them. Pass preallocated output tensors to calls
    made inside the block: nothing may allocate device memory during a capture."""
    lib = _lib.load()
    g = Graph()
    ptr = int(stream.cuda_stream)
    with torch.cuda.stream(stream):
        _lib.check("dh_graph_begin", lib.dh_graph_begin(ptr))
        ok = False
        try:
            yield g
            ok = True
        finally:
            h = ctypes.c_void_p()
            code = lib.dh_graph_end(ptr, ctypes.byref(h))
            g._h = h
            if ok:
                _lib.check("dh_graph_end", code)


class Server:
    """The serving runtime (dh_server_*): camera streams admitted against an HBM budget,
    frames pushed from host memory, finished windows polled with their latency."""

    def __init__(self, hbm_budget_bytes: int):
        self._lib = _lib.load()
        h = ctypes.c_void_p()
        _lib.check("dh_server_create", self._lib.dh_server_create(ctypes.byref(h),
                                                                  int(hbm_budget_bytes)))
        self._h = h
        self.streams = {}  # id -> (nx, ny, T)

    @staticmethod
    def stream_bytes(nx, ny, T, precision="fp16", ring_windows=4) -> int:
        return int(_lib.load().dh_server_stream_bytes(nx, ny, T, PREC[precision], ring_windows))

    def add_stream(self, nx, ny, lambda_m, z_m, pitch_m, T, precision="fp16", k0=2, k1=None,
                   ring_windows=4) -> int:
        """Admit a stream; raises DHError (code 3, DH_ERR_OOM) when the budget is exhausted."""
        sid = ctypes.c_int(-1)
        k1 = T - 1 if k1 is None else k1
        _lib.check("dh_server_add_stream", self._lib.dh_server_add_stream(
            self._h, int(nx), int(ny), float(lambda_m), float(z_m), float(pitch_m), int(T),
            PREC[precision], int(k0), int(k1), int(ring_windows), ctypes.byref(sid)))
        self.streams[sid.value] = (int(nx), int(ny), int(T))
        return sid.value

    def remove_stream(self, sid: int) -> None:
        _lib.check("dh_server_remove_stream", self._lib.dh_server_remove_stream(self._h, sid))
        self.streams.pop(sid, None)

    def set_tune_cache(self, path: str | None, autotune: bool = False) -> None:
        """dh_server_set_tune_cache: streams admitted from now on take their plan options from
        the autotune cache at `path` (and, with autotune, are tuned once and saved when it has
        no entry for them); None turns it off."""
        _lib.check("dh_server_set_tune_cache", self._lib.dh_server_set_tune_cache(
            self._h, os.fsencode(path) if path is not None else None, 1 if autotune else 0))

    def stream_option(self, sid: int, option: int) -> int:
        """dh_server_stream_option: one DH_OPT_* option of a stream's plan."""
        v = ctypes.c_int(0)
        _lib.check("dh_server_stream_option", self._lib.dh_server_stream_option(
            self._h, int(sid), int(option), ctypes.byref(v)))
        return v.value

    @property
    def used_bytes(self) -> int:
        return int(self._lib.dh_server_used_bytes(self._h))

    def push(self, sid: int, frames_host: torch.Tensor, frame_index: int) -> None:
        """Frames [n, ny, nx] uint16 in host memory (pinned for asynchronous copies)."""
        if frames_host.dtype != torch.uint16 or frames_host.is_cuda or not frames_host.is_contiguous():
            raise TypeError("frames must be a contiguous host uint16 tensor")
        _lib.check("dh_server_push", self._lib.dh_server_push(
            self._h, int(sid), _ptr(frames_host), int(frame_index), int(frames_host.shape[0])))

    def poll(self, max_results: int = 64, copy: bool = True):
        """Finished windows: list of dicts (stream, window, image, eigvals, t_ready, t_done).
        With copy=True the image and eigenvalues are copied out and the slot released."""
        arr = (_lib.WindowResult * max_results)()
        n = self._lib.dh_server_poll(self._h, arr, max_results)
        out = []
        for r in arr[:n]:
            nx, ny, T = self.streams[r.stream_id]
            d = {"stream": r.stream_id, "window": int(r.window), "t_ready": r.t_ready_s,
                 "t_done": r.t_done_s}
            if copy:
                img = (ctypes.c_float * (nx * ny)).from_address(r.image_host)
                lam = (ctypes.c_double * T).from_address(r.eigvals_host)
                d["image"] = torch.frombuffer(img, dtype=torch.float32).reshape(ny, nx).clone()
                d["eigvals"] = torch.frombuffer(lam, dtype=torch.float64).clone()
                self.release(r.stream_id, r.window)
            out.append(d)
        return out

    def release(self, sid: int, window: int) -> None:
        _lib.check("dh_server_release", self._lib.dh_server_release(self._h, int(sid), int(window)))

    def clock(self) -> float:
        return float(self._lib.dh_server_clock(self._h))

    def drain(self) -> None:
        _lib.check("dh_server_drain", self._lib.dh_server_drain(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.dh_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
