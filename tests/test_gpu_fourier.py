"""Fourier temporal demodulation (Eqs. 8-9) on the GPU against the FP64 oracle.

Every window's image is the power of the unitary DFT's bins k0..k1 (counted from 0; the
paper's n_1 = 8, n_2 = 24 at n_t = 32 are bins 7..23). Tolerances as for Eqs. 6-7: image
relative L2 <= 1e-4 (FP32 holograms) and <= 1e-3 (16-bit holograms).
"""

import numpy as np
import pytest
import torch

import oracle
from dh_synth import SpeckleParams, SpeckleStream
from parity_helpers import LAM, PITCH, TOL_IMG, Z, rel, to_gpu

pytestmark = pytest.mark.gpu

BANDS = {16: (3, 11), 32: (7, 23), 64: (15, 47)}


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


@pytest.mark.parametrize("T", [16, 32, 64])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_fourier_windows_match_oracle(dh, T, prec):
    k0, k1 = BANDS[T]
    frames = SpeckleStream(SpeckleParams(128, 256), seed=50 + T).next(2 * T).numpy()
    with dh.Plan(128, 256, LAM, Z, PITCH, T=T, precision=prec, max_frames=2 * T) as plan:
        plan.render_frames(to_gpu(frames))
        img = plan.fourier_windows(0, T, 2, k0, k1).cpu().numpy()
        assert plan.status() == 0
    for w in range(2):
        M = oracle.fourier_window(frames[w * T:(w + 1) * T], LAM, Z, PITCH, k0, k1)
        assert rel(img[w], M) <= TOL_IMG[prec], (w, rel(img[w], M))


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_fourier_stride1_sliding_windows(dh, prec):
    """A new window per frame (the paper's Fourier mode runs at the frame rate)."""
    T, n = 32, 9
    frames = SpeckleStream(SpeckleParams(128, 128), seed=60).next(T + n - 1).numpy()
    with dh.Plan(128, 128, LAM, Z, PITCH, T=T, precision=prec, max_frames=T + n - 1) as plan:
        plan.render_frames(to_gpu(frames))
        img = plan.fourier_windows(0, 1, n, 7, 23).cpu().numpy()
    for w in range(n):
        M = oracle.fourier_window(frames[w:w + T], LAM, Z, PITCH, 7, 23)
        assert rel(img[w], M) <= TOL_IMG[prec], (w, rel(img[w], M))


def test_fourier_full_band_is_parseval(dh):
    """All bins kept: the unitary W preserves each pixel's temporal energy."""
    T = 32
    frames = SpeckleStream(SpeckleParams(64, 64), seed=61).next(T).numpy()
    with dh.Plan(64, 64, LAM, Z, PITCH, T=T) as plan:
        plan.render_frames(to_gpu(frames))
        img = plan.fourier_windows(0, T, 1, 0, T - 1)[0].double().cpu().numpy()
        energy = sum((plan.debug_hologram(t).abs() ** 2).double().cpu().numpy() for t in range(T))
    assert rel(img, energy) <= 1e-6


def test_fourier_rejects_bad_bins(dh):
    with dh.Plan(64, 64, LAM, Z, PITCH, T=16) as plan:
        with pytest.raises(dh.DHError) as e:
            plan.fourier_windows(0, 16, 1, 5, 16)
        assert e.value.code == 1
        with pytest.raises(dh.DHError):
            plan.fourier_windows(0, 1, 2, 0, 3)  # window 1 runs past the slots


@pytest.mark.parametrize("T", [16, 32, 64])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_svd_fourier_windows_match_oracle(dh, T, prec):
    """Eqs. 2-3 then 8-9: SVD filter keeping components 2..T-1, then DFT bins. The filter is
    the projector onto the kept eigenvectors; the stated image tolerance applies."""
    from parity_helpers import lam_tol
    b0, b1 = BANDS[T]
    frames = SpeckleStream(SpeckleParams(128, 128), seed=70 + T).next(2 * T).numpy()
    with dh.Plan(128, 128, LAM, Z, PITCH, T=T, precision=prec, max_frames=2 * T,
                 max_windows=2) as plan:
        plan.render_frames(to_gpu(frames))
        img, lam = plan.svd_fourier_windows(0, T, 2, 2, T - 1, b0, b1)
        img, lam = img.cpu().numpy(), lam.cpu().numpy()
        assert plan.status() == 0
    for w in range(2):
        M, lam_ref = oracle.svd_fourier_window(frames[w * T:(w + 1) * T], LAM, Z, PITCH, 2, T - 1,
                                               b0, b1)
        print(f"T={T} {prec} window {w}: image {rel(img[w], M):.2e}")
        assert rel(img[w], M) <= TOL_IMG[prec], (w, rel(img[w], M))
        assert np.max(np.abs(lam[w] - lam_ref)) / lam_ref[0] <= lam_tol(prec, 128 * 128)


@pytest.mark.parametrize("T,b0,b1", [(32, 7, 23), (16, 3, 11), (64, 20, 40)])
def test_fourier_sliding_recurrence_long_run(dh, T, b0, b1):
    """300 windows a frame apart (several restart segments of the sliding recurrence): each
    sampled window equals the direct projection onto W (a one-window call) to FP32 rounding,
    and matches the oracle."""
    n = 300
    frames = SpeckleStream(SpeckleParams(64, 64), seed=80 + T).next(n + T - 1).numpy()
    with dh.Plan(64, 64, LAM, Z, PITCH, T=T, max_frames=n + T - 1) as plan:
        plan.render_frames(to_gpu(frames))
        slide = plan.fourier_windows(0, 1, n, b0, b1).cpu().numpy()
        for w in (0, 1, 127, 128, 129, 255, 256, 299):
            direct = plan.fourier_windows(w, 1, 1, b0, b1)[0].cpu().numpy()
            assert rel(slide[w], direct) <= 1e-5, (w, rel(slide[w], direct))
    for w in (0, 150, 299):
        M = oracle.fourier_window(frames[w:w + T], LAM, Z, PITCH, b0, b1)
        assert rel(slide[w], M) <= TOL_IMG["fp32"], (w, rel(slide[w], M))


@pytest.mark.parametrize("stride,n", [(1, 16), (2, 9), (5, 3)])
def test_fourier_span_equals_single_window_projection(dh, stride, n):
    """Overlapping windows on the tensor-core span path (7 windows per load of their frames,
    FP16, 17 bins): equal to one-window calls (the per-window projection onto W) to FP32
    rounding, over full and ragged groups, and to the oracle."""
    T, b0, b1 = 32, 7, 23
    F = (n - 1) * stride + T
    frames = SpeckleStream(SpeckleParams(256, 128), seed=90 + stride).next(F).numpy()
    with dh.Plan(256, 128, LAM, Z, PITCH, T=T, precision="fp16", max_frames=F) as plan:
        plan.render_frames(to_gpu(frames))
        plan.profile(True)
        span = plan.fourier_windows(0, stride, n, b0, b1).cpu().numpy()
        prof = plan.profile_read()
        plan.profile(False)
        assert prof["fourier_span"][0] == 1, prof
        for w in range(n):
            one = plan.fourier_windows(w * stride, 1, 1, b0, b1)[0].cpu().numpy()
            assert rel(span[w], one) <= 1e-5, (w, rel(span[w], one))
        assert plan.status() == 0
    for w in (0, n - 1):
        M = oracle.fourier_window(frames[w * stride:w * stride + T], LAM, Z, PITCH, b0, b1)
        assert rel(span[w], M) <= TOL_IMG["fp16"], (w, rel(span[w], M))
