"""TEST INFRASTRUCTURE: the FP64 CPU oracle for the retinal-holography PCA path.

Only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg may
import this package. The library path never calls it, and it shares no code with the
CUDA library (its C source is `dh_oracle.c` in this folder).

Each wrapper names the equation of Puyo et al. (arXiv 2004.00923) it computes:
  render           Eq. 1 (Fresnel transform, one FFT per frame)
  covariance       Eq. 4 (C = H^{t*} H)
  eig              Eq. 5 (C = V Lambda V^{t*}), decreasing order
  project_power    Eqs. 6-7 (H_breve = H V I_f, M = sum |H_breve|^2)
  pca_window       Eqs. 1, 4, 5, 6, 7 in the paper's order
  fourier_power    Eqs. 8-9 (H_tilde = H W I_f with the unitary DFT W, M = sum |H_tilde|^2)
  fourier_window   Eqs. 1, 8, 9 in the paper's order
  svd_fourier_window  Eqs. 1, 4, 5, then the SVD filter of Eqs. 2-3 and Eqs. 8-9
  normalize / display_u8  display normalisation of an image by its mean (text after Eq. 9)
  fft1d / fft2d    the DFT used inside Eq. 1 (exposed for pins)

Parity status: every function above is pinned by `tests/test_oracle_pins.py`
(direct DFT, closed forms, LAPACK, invariants); nothing is "parity unpinned".
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dh_oracle.c")
_LIB = os.path.join(_HERE, "libdh_oracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, no fast-math, OpenMP) into oracle/libdh_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u16p = ctypes.POINTER(ctypes.c_uint16)
        lib.dho_fft1d.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int]
        lib.dho_fft2d.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int]
        lib.dho_chirp.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
        lib.dho_chirp.restype = None
        lib.dho_render.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u16p,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]
        lib.dho_covariance.argtypes = [ctypes.c_longlong, ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.dho_eig.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp, ctypes.c_double,
                                ctypes.c_int]
        lib.dho_project_power.argtypes = [ctypes.c_longlong, ctypes.c_int, _dp, _dp, _dp, _dp,
                                          ctypes.c_int, ctypes.c_int, _dp]
        lib.dho_pca_window.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u16p,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.dho_fourier_power.argtypes = [ctypes.c_longlong, ctypes.c_int, _dp, _dp, ctypes.c_int,
                                          ctypes.c_int, _dp]
        lib.dho_fourier_window.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u16p,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_int, _dp]
        lib.dho_svd_fourier_window.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u16p,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, _dp, _dp]
        lib.dho_num_threads.argtypes = []
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(_load().dho_num_threads())


def fft1d(x: np.ndarray, sign: int = +1) -> np.ndarray:
    """Unnormalised DFT, X[m] = sum_k x[k] exp(sign 2 pi i m k / n) (inside Eq. 1)."""
    re, im = _c(np.real(x), np.float64).copy(), _c(np.imag(x), np.float64).copy()
    if _load().dho_fft1d(len(re), _ptr(re), _ptr(im), int(sign)) != 0:
        raise ValueError("fft1d: length must be a power of two")
    return re + 1j * im


def fft2d(x: np.ndarray, sign: int = +1) -> np.ndarray:
    """Unnormalised 2-D DFT of an (ny, nx) array, rows then columns."""
    ny, nx = x.shape
    re, im = _c(np.real(x), np.float64).copy(), _c(np.imag(x), np.float64).copy()
    if _load().dho_fft2d(nx, ny, _ptr(re), _ptr(im), int(sign)) != 0:
        raise ValueError("fft2d: sizes must be powers of two")
    return re + 1j * im


def chirp(n: int, a: float) -> np.ndarray:
    """c(k) = exp(-i pi a (k - n/2)^2) (input chirp of Eq. 1)."""
    re, im = np.empty(n), np.empty(n)
    _load().dho_chirp(n, float(a), _ptr(re), _ptr(im))
    return re + 1j * im


def render(frames: np.ndarray, lambda_m: float, z_m: float, pitch_m: float) -> np.ndarray:
    """Eq. 1: uint16 frames [T, ny, nx] -> complex128 holograms [T, ny, nx]."""
    f = _c(frames, np.uint16)
    T, ny, nx = f.shape
    hr, hi = np.empty(f.shape), np.empty(f.shape)
    rc = _load().dho_render(nx, ny, T, f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)),
                            lambda_m, z_m, pitch_m, _ptr(hr), _ptr(hi))
    if rc != 0:
        raise ValueError(f"render failed ({rc})")
    return hr + 1j * hi


def covariance(H: np.ndarray) -> np.ndarray:
    """Eq. 4: C = H^{t*} H for holograms H[T, ...] (frame-major), as complex128 [T, T]."""
    T = H.shape[0]
    Hm = H.reshape(T, -1)
    hr, hi = _c(Hm.real, np.float64), _c(Hm.imag, np.float64)
    cr, ci = np.empty((T, T)), np.empty((T, T))
    rc = _load().dho_covariance(Hm.shape[1], T, _ptr(hr), _ptr(hi), _ptr(cr), _ptr(ci))
    if rc != 0:
        raise ValueError(f"covariance failed ({rc})")
    return cr + 1j * ci


def eig(C: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Eq. 5: Hermitian eigendecomposition by cyclic complex Jacobi.
    Returns (lam[T] decreasing, V[T, T] with eigenvectors as columns, sweeps)."""
    T = C.shape[0]
    cr, ci = _c(C.real, np.float64), _c(C.imag, np.float64)
    lam, vr, vi = np.empty(T), np.empty((T, T)), np.empty((T, T))
    rc = _load().dho_eig(T, _ptr(cr), _ptr(ci), _ptr(lam), _ptr(vr), _ptr(vi), tol, max_sweeps)
    if rc < 0:
        raise RuntimeError(f"Jacobi did not converge ({rc})")
    return lam, vr + 1j * vi, rc


def project_power(H: np.ndarray, V: np.ndarray, k0: int, k1: int) -> np.ndarray:
    """Eqs. 6-7: M[p] = sum_{k=k0..k1} |sum_t H[t, p] V[t, k]|^2, shaped like one frame."""
    T = H.shape[0]
    Hm = H.reshape(T, -1)
    hr, hi = _c(Hm.real, np.float64), _c(Hm.imag, np.float64)
    vr, vi = _c(V.real, np.float64), _c(V.imag, np.float64)
    M = np.empty(Hm.shape[1])
    rc = _load().dho_project_power(Hm.shape[1], T, _ptr(hr), _ptr(hi), _ptr(vr), _ptr(vi),
                                   int(k0), int(k1), _ptr(M))
    if rc != 0:
        raise ValueError(f"project_power failed ({rc})")
    return M.reshape(H.shape[1:])


def pca_window(frames: np.ndarray, lambda_m: float, z_m: float, pitch_m: float,
               k0: int, k1: int):
    """The whole window in the paper's order (Eqs. 1, 4, 5, 6, 7).
    Returns (M [ny, nx] float64, lam [T] decreasing, C [T, T] complex128, sweeps)."""
    f = _c(frames, np.uint16)
    T, ny, nx = f.shape
    M, lam = np.empty((ny, nx)), np.empty(T)
    cr, ci = np.empty((T, T)), np.empty((T, T))
    rc = _load().dho_pca_window(nx, ny, T, f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)),
                                lambda_m, z_m, pitch_m, int(k0), int(k1), _ptr(M), _ptr(lam),
                                _ptr(cr), _ptr(ci))
    if rc < 0:
        raise RuntimeError(f"pca_window failed ({rc})")
    return M, lam, cr + 1j * ci, rc


def fourier_power(H: np.ndarray, k0: int, k1: int) -> np.ndarray:
    """Eqs. 8-9: M[p] = sum_{k=k0..k1} |sum_t H[t, p] w_{t,k}|^2 with the unitary DFT
    w_{t,k} = exp(-2 pi i t k / T) / sqrt(T), bins counted from 0 (the paper's n = k + 1)."""
    T = H.shape[0]
    Hm = H.reshape(T, -1)
    hr, hi = _c(Hm.real, np.float64), _c(Hm.imag, np.float64)
    M = np.empty(Hm.shape[1])
    rc = _load().dho_fourier_power(Hm.shape[1], T, _ptr(hr), _ptr(hi), int(k0), int(k1), _ptr(M))
    if rc != 0:
        raise ValueError(f"fourier_power failed ({rc})")
    return M.reshape(H.shape[1:])


def fourier_window(frames: np.ndarray, lambda_m: float, z_m: float, pitch_m: float,
                   k0: int, k1: int) -> np.ndarray:
    """The Fourier-demodulated window (Eq. 1, then Eqs. 8-9): the image M [ny, nx]."""
    f = _c(frames, np.uint16)
    T, ny, nx = f.shape
    M = np.empty((ny, nx))
    rc = _load().dho_fourier_window(nx, ny, T, f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)),
                                    lambda_m, z_m, pitch_m, int(k0), int(k1), _ptr(M))
    if rc != 0:
        raise RuntimeError(f"fourier_window failed ({rc})")
    return M


def svd_fourier_window(frames: np.ndarray, lambda_m: float, z_m: float, pitch_m: float,
                       k0: int, k1: int, b0: int, b1: int):
    """The SVD-filtered, Fourier-demodulated window (Eq. 1; Eqs. 4-5 for V; H_f = H V I_f
    V^{t*} of Eqs. 2-3 keeping components k0..k1 in decreasing order; Eqs. 8-9 over bins
    b0..b1). Returns (M [ny, nx], lam [T] decreasing)."""
    f = _c(frames, np.uint16)
    T, ny, nx = f.shape
    M, lam = np.empty((ny, nx)), np.empty(T)
    rc = _load().dho_svd_fourier_window(nx, ny, T, f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)),
                                        lambda_m, z_m, pitch_m, int(k0), int(k1), int(b0),
                                        int(b1), _ptr(M), _ptr(lam))
    if rc < 0:
        raise RuntimeError(f"svd_fourier_window failed ({rc})")
    return M, lam


def normalize(M: np.ndarray):
    """An image divided by its own mean (the paper normalises every displayed image by its
    average value). Returns (M / mean, mean) in FP64."""
    M = np.asarray(M, dtype=np.float64)
    mean = float(M.mean())
    return M / mean, mean


def display_value(M: np.ndarray, gain: float = 128.0) -> np.ndarray:
    """The display value gain * M / mean(M) of every pixel, in FP64, with the image's own FP64
    mean (the paper normalises each displayed image by its average value)."""
    N, _ = normalize(M)
    return np.float64(gain) * N


def display_u8(M: np.ndarray, gain: float = 128.0) -> np.ndarray:
    """8-bit display codes of an image: clamp(rint(gain * M / mean(M)), 0, 255), decided in
    FP64 from the image's own FP64 mean; the mean maps to code `gain`."""
    return np.clip(np.rint(display_value(M, gain)), 0, 255).astype(np.uint8)
