"""The tensor-core render of 1024 x 1024 frames (DH_OPT_RENDER_FFT = 2): each 1024-point DFT of
Eq. 1 as two batched 32-point DFTs on the tensor cores (FP16 hi + lo operands, three
products, FP32 accumulation), against the FP64 oracle and against the CUDA-core FFT."""

import numpy as np
import pytest
import torch

import oracle
from dh_synth import SpeckleParams, SpeckleStream
from parity_helpers import LAM, PITCH, Z, check_window, rel, to_gpu

pytestmark = pytest.mark.gpu
N = 1024


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


def _holograms(dh, frames, prec, fft, schedule=None):
    F = frames.shape[0]
    with dh.Plan(N, N, LAM, Z, PITCH, T=16, precision=prec, max_frames=max(F, 16)) as plan:
        plan.set_render_fft(fft)
        if schedule is not None:
            plan.set_render_schedule(schedule == "persistent")
        plan.render_frames(to_gpu(frames))
        out = np.stack([plan.debug_hologram(t).cpu().numpy() for t in range(F)])
        assert plan.status() == 0
    return out.astype(np.complex128)


@pytest.mark.parametrize("kind", ["speckle", "full_range"])
def test_tc_render_fp32_matches_oracle(dh, kind):
    if kind == "speckle":
        frames = SpeckleStream(SpeckleParams(N, N), seed=5).next(3).numpy()
    else:  # every 16-bit value: the operand scales must keep FP16 in range
        frames = np.random.default_rng(6).integers(0, 65536, size=(2, N, N), dtype=np.uint16)
    H = oracle.render(frames, LAM, Z, PITCH)
    G = _holograms(dh, frames, "fp32", "tensor")
    for t in range(frames.shape[0]):
        e = rel(G[t], H[t])
        print(f"{kind} frame {t}: tensor-core render against the oracle {e:.2e}")
        assert e <= 3e-6, (t, e)


def test_tc_render_equals_cuda_core_fft_closely(dh):
    frames = SpeckleStream(SpeckleParams(N, N), seed=7).next(2).numpy()
    a = _holograms(dh, frames, "fp32", "tensor")
    b = _holograms(dh, frames, "fp32", "cuda")
    for t in range(2):
        assert rel(a[t], b[t]) <= 3e-6, rel(a[t], b[t])


def test_tc_render_16bit_storage_rounding(dh):
    """FP16 planes: every value within one FP16 rounding (2^-11 relative) of the oracle's,
    plus the render's own ~1e-7 of the frame's scale."""
    frames = SpeckleStream(SpeckleParams(N, N), seed=8).next(2).numpy()
    H = oracle.render(frames, LAM, Z, PITCH)
    G = _holograms(dh, frames, "fp16", "tensor")
    for t in range(2):
        scale = np.abs(H[t]).max()
        bound = 2.0 ** -11 * np.maximum(np.abs(H[t].real), np.abs(H[t].imag)) + 1e-6 * scale + 6e-8
        assert np.all(np.abs(G[t].real - H[t].real) <= bound)
        assert np.all(np.abs(G[t].imag - H[t].imag) <= bound)


def test_tc_render_pca_window_matches_oracle(dh):
    T = 32
    frames = SpeckleStream(SpeckleParams(N, N), seed=9).next(T).numpy()
    with dh.Plan(N, N, LAM, Z, PITCH, T=T, precision="fp16") as plan:
        plan.set_render_fft("tensor")
        plan.render_stack(to_gpu(frames))
        img, lam = plan.pca_window(2, T - 1)
        C = plan.debug_covariance(0).cpu().numpy()
        assert plan.status() == 0
    check_window(img.double().cpu().numpy(), lam.numpy(), C, frames, 2, T - 1, "fp16", label="tc render")
