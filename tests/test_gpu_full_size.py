"""Parity at the full workload sizes, in the launch configurations the benchmark times.

Headline: 2048 frames of 1024^2 as 64 disjoint 32-frame windows, FP16 storage, the render
schedule the autotuner picks, one dh_pca_batch call. Sliding: 2048 frames of 1024^2, 16/32/64-
frame windows at stride 8 (757 windows) over one store, the banded covariance and the grouped
projection, one batch of three views. The oracle computes a whole window (all 2^20 pixels) in
about a second, so a sample of windows is checked against it element by element (first,
middle and last of each set); every window is checked through a property that holds at any
size: the unitary Fresnel transform preserves each frame's energy, so the eigenvalues of a
window sum to trace C = sum_t ||H_t||^2 = sum_t ||I_t||^2, an exact integer from the frames.
"""

import numpy as np
import pytest
import torch

from dh_synth import SpeckleParams, SpeckleStream
from parity_helpers import LAM, PITCH, Z, check_window

pytestmark = pytest.mark.gpu

N, F = 1024, 2048


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


@pytest.fixture(scope="module")
def frames():
    f = SpeckleStream(SpeckleParams(N, N), seed=2024, device=torch.device("cuda")).next(F)
    # per-frame energies sum_p I^2, exact in int64 (4095^2 * 2^20 < 2^63)
    energy = (f.to(torch.int64) ** 2).sum(dim=(1, 2)).cpu().numpy()
    return f, energy


def window_energy(energy, f0, T):
    return float(energy[f0:f0 + T].sum())


def test_headline_configuration(dh, frames):
    f, energy = frames
    T, nwin = 32, F // 32
    with dh.Plan(N, N, LAM, Z, PITCH, T=T, precision="fp16", max_frames=F, max_windows=nwin) as plan:
        plan.autotune(256)
        img, lam = plan.pca_batch(f, nwin, T, 2, T - 1)
        torch.cuda.synchronize()
        assert plan.status() == 0
        lam = lam.cpu().numpy()
        # every window: sum of eigenvalues = the window's energy (FP16 storage and FP32
        # accumulation of 2^25 products leave ~1e-6)
        for w in range(nwin):
            e = window_energy(energy, w * T, T)
            assert abs(lam[w].sum() - e) <= 5e-6 * e, w
        # sampled windows against the oracle, element by element
        for w in (0, nwin // 2, nwin - 1):
            fr = f[w * T:(w + 1) * T].cpu().numpy()
            C = plan.debug_covariance(w).cpu().numpy()
            check_window(img[w].cpu().numpy().astype(np.float64), lam[w], C, fr, 2, T - 1, "fp16")


def test_sliding_configuration(dh, frames):
    f, energy = frames
    s = 8
    n = {L: (F - L) // s + 1 for L in (16, 32, 64)}
    base = dh.Plan(N, N, LAM, Z, PITCH, T=16, precision="fp16", max_frames=F, max_windows=n[16])
    plans = {16: base, 32: base.view(32, n[32]), 64: base.view(64, n[64])}
    images = {L: torch.empty((n[L], N, N), dtype=torch.float32, device="cuda") for L in n}
    eig = {L: torch.empty((n[L], L), dtype=torch.float64, device="cuda") for L in n}
    try:
        for p in plans.values():
            p.set_covariance_source("band")
        base.render_frames(f)
        base.band_gram(0, F)
        dh.run_batch([{"plan": plans[L], "n_windows": n[L], "first_slot": 0, "slot_stride": s,
                       "k0": 2, "k1": L - 1, "images": images[L], "eigvals": eig[L]}
                      for L in (64, 32, 16)])
        torch.cuda.synchronize()
        for p in plans.values():
            assert p.status() == 0
        for L in n:
            lam = eig[L].cpu().numpy()
            for w in range(n[L]):
                e = window_energy(energy, w * s, L)
                assert abs(lam[w].sum() - e) <= 5e-6 * e, (L, w)
            for w in (0, n[L] // 2, n[L] - 1):
                fr = f[w * s:w * s + L].cpu().numpy()
                C = plans[L].debug_covariance(w).cpu().numpy()
                check_window(images[L][w].cpu().numpy().astype(np.float64), lam[w], C, fr, 2,
                             L - 1, "fp16")
    finally:
        for L in (32, 64):
            plans[L].close()
        base.close()


def test_largest_frames(dh):
    """The largest frame size the library takes, 4096^2 (16 MiB pixels a frame): two 16-frame
    windows, FP16 storage, with the plan's default schedule; window 0 element by element
    against the oracle, both through the energy trace."""
    n, T, nwin = 4096, 16, 2
    f = SpeckleStream(SpeckleParams(n, n), seed=4096, device=torch.device("cuda")).next(T * nwin)
    energy = (f.to(torch.int64) ** 2).sum(dim=(1, 2)).cpu().numpy()
    with dh.Plan(n, n, LAM, Z, PITCH, T=T, precision="fp16", max_frames=T * nwin, max_windows=nwin) as plan:
        img, lam = plan.pca_batch(f, nwin, T, 2, T - 1)
        torch.cuda.synchronize()
        assert plan.status() == 0
        lam = lam.cpu().numpy()
        for w in range(nwin):
            e = window_energy(energy, w * T, T)
            assert abs(lam[w].sum() - e) <= 5e-6 * e, w
        C = plan.debug_covariance(0).cpu().numpy()
        check_window(img[0].cpu().numpy().astype(np.float64), lam[0], C, f[:T].cpu().numpy(), 2, T - 1,
                     "fp16", label="4096^2")
