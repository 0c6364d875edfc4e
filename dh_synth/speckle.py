"""Synthetic inline interferograms shaped like the paper's retinal footage.

The paper records 16-bit 1024x1024 interferograms at 500 frames/s (Sec. "experimental
setup", camera paragraph) of I = |E|^2 + |E_LO|^2 + H + H* (the interferogram model
stated after Eq. 1). The footage itself is not public, so frames are drawn from a
seeded model with the same shape and the same kinds of contributions:

  I(x, y, t) = clip(Poisson(kappa * |R + S(x, y, t)|^2), 0, 4095)

with a unit plane reference R = 1 and an object field S that is the sum of
  * a static complex-Gaussian speckle field S_s (E|S_s|^2 = p_static),
  * a dynamic speckle field S_d0 * exp(i theta(x, y, t)) whose phase performs a
    per-pixel random walk with N(0, sigma_doppler^2) steps (E|S_d0|^2 = p_dynamic),
  * a spatially uniform field g(t) = a_drift * exp(i phi(t)), phi ~ U(0, 2 pi) i.i.d.
    per frame (the "global random phase drift").

The numbers below (p_static = 0.3, p_dynamic = 0.05, a_drift = 0.3, kappa = 1500,
12-bit clipping) are this library's reading: the workload description gives the
three contributions, the Doppler step spread and the 12-bit scale, not the powers.

All draws come from one torch.Generator seeded by the caller, so a (seed, device)
pair always yields the same frames. CPU and CUDA generators produce different
streams; a test that compares two implementations must draw once and hand the
same frames to both.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch


@dataclass(frozen=True)
class SpeckleParams:
    nx: int
    ny: int
    sigma_doppler: float = 0.3  # rad per frame, std of the dynamic-speckle phase step
    p_static: float = 0.3
    p_dynamic: float = 0.05
    a_drift: float = 0.3
    kappa: float = 1500.0
    max_count: int = 4095  # 12-bit camera scale


class SpeckleStream:
    """A continuous, gap-free frame sequence (the paper buffers the camera stream
    so that no frame is dropped; windows are cut from this sequence)."""

    def __init__(self, params: SpeckleParams, seed: int, device="cpu"):
        self.p = params
        self.device = torch.device(device)
        self.gen = torch.Generator(device=self.device)
        self.gen.manual_seed(int(seed))
        shape = (params.ny, params.nx)
        f32 = torch.float32
        s = math.sqrt(params.p_static / 2.0)
        d = math.sqrt(params.p_dynamic / 2.0)
        self.s_static = torch.complex(
            torch.randn(shape, generator=self.gen, device=self.device, dtype=f32) * s,
            torch.randn(shape, generator=self.gen, device=self.device, dtype=f32) * s,
        )
        self.s_dyn0 = torch.complex(
            torch.randn(shape, generator=self.gen, device=self.device, dtype=f32) * d,
            torch.randn(shape, generator=self.gen, device=self.device, dtype=f32) * d,
        )
        self.theta = torch.zeros(shape, device=self.device, dtype=f32)
        self.frames_drawn = 0

    def next(self, nframes: int) -> torch.Tensor:
        """Draw the next `nframes` frames as a uint16 tensor [nframes, ny, nx]."""
        p = self.p
        out = torch.empty((nframes, p.ny, p.nx), dtype=torch.uint16, device=self.device)
        for i in range(nframes):
            step = torch.randn(self.theta.shape, generator=self.gen, device=self.device,
                               dtype=torch.float32) * p.sigma_doppler
            self.theta = self.theta + step
            phi = float(torch.rand((), generator=self.gen, device=self.device)) * 2.0 * math.pi
            g = complex(p.a_drift * math.cos(phi), p.a_drift * math.sin(phi))
            field = 1.0 + self.s_static + self.s_dyn0 * torch.polar(
                torch.ones_like(self.theta), self.theta) + g
            rate = p.kappa * (field.real * field.real + field.imag * field.imag)
            counts = torch.poisson(rate, generator=self.gen)
            counts = counts.clamp_(0, p.max_count)
            out[i] = counts.to(torch.int32).to(torch.uint16)
        self.frames_drawn += nframes
        return out


def speckle_window(nx: int, ny: int, T: int, seed: int, device="cpu",
                   sigma_doppler: float = 0.3) -> torch.Tensor:
    """One independent T-frame window (uint16 [T, ny, nx]) drawn from its own seed."""
    return SpeckleStream(SpeckleParams(nx, ny, sigma_doppler=sigma_doppler), seed,
                         device).next(T)


def hadamard_rows(T: int) -> np.ndarray:
    """Sylvester Hadamard matrix of order T (T a power of two), entries +-1, as int64.
    Rows are mutually orthogonal: H H^T = T I."""
    if T < 1 or T & (T - 1):
        raise ValueError("T must be a power of two")
    h = np.ones((1, 1), dtype=np.int64)
    while h.shape[0] < T:
        h = np.block([[h, h], [h, -h]])
    return h


def known_rank_frames(nx: int, ny: int, T: int, c0: int, comps, support_seed: int = 0):
    """Frames whose temporal covariance has a closed-form spectrum.

    `comps` is a list of (hadamard_row_index >= 1, n_pixels, amplitude). Component r
    owns two disjoint random pixel sets S_r+ and S_r- of n_pixels each; the frame
    sequence is c0 + amplitude * h_r(t) on S_r+ and c0 - amplitude * h_r(t) on S_r-,
    with h_r a row of the Sylvester Hadamard matrix. All other pixels are 0.

    Because the Fresnel transform of the method is unitary per frame, the hologram
    covariance equals the Gram matrix of the raw sequences, in which the +/- pairs
    cancel the cross terms:
        C = 2 c0^2 N 1 1^T + sum_r 2 n_r a_r^2 h_r h_r^T,   N = sum_r n_r,
    so its eigenvalues are 2 c0^2 N T, 2 n_r a_r^2 T (one per component) and zeros.
    Returns (frames uint16 [T, ny, nx] numpy, sorted-decreasing eigenvalues float64 [T]).
    """
    h = hadamard_rows(T)
    rng = np.random.default_rng(support_seed)
    n = nx * ny
    total = 2 * sum(cnt for _, cnt, _ in comps)
    if total > n:
        raise ValueError("supports do not fit in the frame")
    perm = rng.permutation(n)
    frames = np.zeros((T, n), dtype=np.int64)
    off = 0
    lam = [2.0 * c0 * c0 * (total // 2) * T]
    for hidx, cnt, amp in comps:
        if not 1 <= hidx < T:
            raise ValueError("Hadamard row must be 1..T-1 (row 0 is the constant row)")
        for sgn in (+1, -1):
            seq = c0 + sgn * amp * h[hidx]
            if seq.min() < 0 or seq.max() > 65535:
                raise ValueError("sequence outside uint16")
            frames[:, perm[off:off + cnt]] = seq[:, None]
            off += cnt
        lam.append(2.0 * cnt * amp * amp * T)
    lam = np.array(sorted(lam + [0.0] * (T - len(lam)), reverse=True))
    return frames.reshape(T, ny, nx).astype(np.uint16), lam
