"""Helpers shared by the GPU parity test files: the optics of the small workloads, the
stated tolerances and the window check against the FP64 oracle.

Tolerances: image relative L2 <= 1e-4 for the plain FP32 path, <= 1e-3 for the 16-bit fast
form; eigenvalues within 1e-5 * lambda_max (norm-wise: |d lambda_k| <= ||dC||_2).
"""

import numpy as np
import torch

import oracle

LAM, Z, PITCH = 785e-9, 0.35, 20e-6
TOL_IMG = {"fp32": 1e-4, "fp16": 1e-3}
TOL_LAM = 1e-5


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def to_gpu(frames_np):
    return torch.from_numpy(np.ascontiguousarray(frames_np)).cuda()


# Relative covariance error each storage achieves (||dC|| / ||C||, measured against the
# oracle). The image of a retained range [k0, k1] is unique only where the eigenvalue gaps at
# the range boundary are non-zero, and moves by about ||dC|| / gap (Davis-Kahan); only the
# named extreme ranges (a single smallest or largest component) sit on gaps small enough for
# that to exceed the stated tolerance, and only they use check_window_extreme_range.
EPS_C = {"fp32": 1e-8, "fp16": 1e-5}


def boundary_gap(lam, k0, k1):
    gaps = []
    if k0 > 0:
        gaps.append(lam[k0 - 1] - lam[k0])
    if k1 < len(lam) - 1:
        gaps.append(lam[k1] - lam[k1 + 1])
    return min(gaps) / lam[0] if gaps else 1.0


# 16-bit storage rounds every hologram value with unit roundoff u; the resulting covariance
# noise is ~u/sqrt(n) relative per entry and moves eigenvalues by up to ~4 u/sqrt(n) of
# lambda_max. At the workload sizes (n >= 256^2) that is below the stated 1e-5; tiny frames
# used for edge cases get the storage bound instead.
U16 = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


def lam_tol(prec, npix):
    return TOL_LAM if prec == "fp32" else max(TOL_LAM, 4 * U16[prec] / np.sqrt(npix))


# The covariance diagnostic (not one of the stated tolerances, which bound the image and the
# eigenvalues): 5e-6 for FP32 storage; for 16-bit storage 2e-4, or the storage bound
# 16 u / sqrt(n) on frames of a few hundred pixels (measured 6-10 u / sqrt(n) at 256-1024).
def c_tol(prec, npix):
    return 5e-6 if prec == "fp32" else max(2e-4, 16 * U16[prec] / np.sqrt(npix))


def _errors(img, lam, C, frames_np, k0, k1, z):
    M, lam_ref, C_ref, _ = oracle.pca_window(frames_np, LAM, z, PITCH, k0, k1)
    e_img = rel(img, M)
    e_lam = float(np.max(np.abs(lam - lam_ref)) / lam_ref[0])
    e_C = rel(C, C_ref)
    return e_img, e_lam, e_C, boundary_gap(lam_ref, k0, k1)


def check_window(img, lam, C, frames_np, k0, k1, prec, z=Z, label=""):
    """One window against the oracle at the stated tolerances: image <= 1e-4 (FP32) or
    <= 1e-3 (16-bit storage), eigenvalues <= 1e-5 lambda_max (the storage bound for frames
    below 256^2); covariance diagnostic c_tol. Prints the measured errors."""
    e_img, e_lam, e_C, gap = _errors(img, lam, C, frames_np, k0, k1, z)
    print(f"window {label} [{k0},{k1}] {prec}: image {e_img:.2e} (<= {TOL_IMG[prec]:.0e}), "
          f"eigenvalues {e_lam:.2e}, C {e_C:.2e}, boundary gap {gap:.2e}")
    assert e_lam <= lam_tol(prec, frames_np[0].size), e_lam
    assert e_img <= TOL_IMG[prec], (e_img, gap)
    assert e_C <= c_tol(prec, frames_np[0].size), e_C
    return e_img, e_lam, e_C


# the only ranges whose boundary gap may sit below the covariance accuracy of the storage: a
# single component at either end of the spectrum
EXTREME_RANGES = {(0, 0), (31, 31)}


def check_window_extreme_range(img, lam, C, frames_np, k0, k1, prec, z=Z):
    """A named extreme range (EXTREME_RANGES): the image tolerance is max(stated,
    eps_C / gap), with the boundary gap printed and asserted to be the reason."""
    assert (k0, k1) in EXTREME_RANGES, (k0, k1)
    e_img, e_lam, e_C, gap = _errors(img, lam, C, frames_np, k0, k1, z)
    tol_img = max(TOL_IMG[prec], EPS_C[prec] / gap)
    print(f"extreme range [{k0},{k1}] {prec}: image {e_img:.2e} (<= {tol_img:.2e}), "
          f"boundary gap {gap:.2e}, eigenvalues {e_lam:.2e}")
    assert e_lam <= lam_tol(prec, frames_np[0].size), e_lam
    assert e_img <= tol_img, (e_img, gap)
    assert e_C <= c_tol(prec, frames_np[0].size), e_C
    return e_img, e_lam, e_C
