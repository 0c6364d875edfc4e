"""Degenerate and boundary windows through the C ABI: all-zero frames (C = 0: no rotation,
no division by ||C||), identical frames (C of rank one, T - 1 equal zero eigenvalues), per
window and through the grouped projection of overlapping windows; an empty batch; more
windows than SMs (one group, several CTA rounds of the eigensolver).

For identical frames h_t = h, C = T h^H h 1 1^T: lambda_0 = T ||h||^2, the other eigenvalues
are 0, V_0 = 1 / sqrt(T), and every other eigenvector is orthogonal to 1, so H V_k = h (1^T
V_k) = 0: the power of components 1..T-1 vanishes and components 0..T-1 give T |h|^2 per pixel
(Eq. 7 with V unitary). The same identities hold for the stored 16-bit holograms, which are
identical too.
"""

import numpy as np
import pytest
import torch

import oracle
from dh_synth import speckle_window
from parity_helpers import LAM, PITCH, TOL_IMG, Z, rel, to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


@pytest.mark.parametrize("T", [16, 32, 64])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_all_zero_windows(dh, T, prec):
    """Zero frames: zero eigenvalues and images, no NaN, no flag."""
    n = 3
    frames = np.zeros((n * T, 64, 128), dtype=np.uint16)
    with dh.Plan(128, 64, LAM, Z, PITCH, T=T, precision=prec, max_frames=n * T, max_windows=n) as plan:
        img, lam = plan.pca_batch(to_gpu(frames), n, T, 0, T - 1)
        torch.cuda.synchronize()
        assert plan.status() == 0
        img, lam = img.cpu().numpy(), lam.cpu().numpy()
    assert np.all(img == 0.0) and np.all(lam == 0.0)


@pytest.mark.parametrize("T", [16, 32, 64])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_identical_frames(dh, T, prec):
    """Rank-one C: one eigenvalue T ||h||^2 (the oracle's), T - 1 zeros to 1e-6 of it (the
    covariance's own rounding, ~1e-7 of ||C||, bounds them by Weyl); the discarded-first image
    (components 1..T-1) has no power; the full range gives T |h|^2."""
    one = speckle_window(128, 64, 1, seed=T).numpy()
    frames = np.repeat(one, T, axis=0)
    with dh.Plan(128, 64, LAM, Z, PITCH, T=T, precision=prec, max_frames=T, max_windows=1) as plan:
        plan.render_stack(to_gpu(frames))
        full, lam = plan.pca_window(0, T - 1)
        rest, _ = plan.pca_window(1, T - 1)
        assert plan.status() == 0
        full, rest, lam = full.double().cpu().numpy(), rest.double().cpu().numpy(), lam.numpy()
        hs = plan.debug_hologram(0).cpu().numpy().astype(np.complex128)
    M, lam_ref, _, _ = oracle.pca_window(frames, LAM, Z, PITCH, 0, T - 1)
    if prec == "fp32":
        assert abs(lam[0] - lam_ref[0]) <= 1e-5 * lam_ref[0]
    else:
        # the frames' 16-bit storage rounding is the same in every frame, so it does not
        # average out over the window as it does for distinct frames: pin lambda_0 to the
        # stored hologram instead, T ||h_stored||^2 in FP64
        lam0 = T * float(np.sum(np.abs(hs) ** 2))
        assert abs(lam[0] - lam0) <= 1e-6 * lam0
        assert abs(lam[0] - lam_ref[0]) <= 1e-4 * lam_ref[0]
    assert np.all(np.abs(lam[1:]) <= 1e-6 * lam[0])
    assert rel(full, M) <= TOL_IMG[prec]
    assert np.max(rest) <= 1e-6 * np.mean(full)


def test_identical_frames_grouped_projection(dh):
    """Overlapping windows over constant frames (the grouped projection, which takes the power
    as the window's energy minus its discarded components'): with k0 = 1 the single discarded
    component holds all of the energy, and the images vanish to the rounding of it (energy and
    discarded power are each accurate to ~1e-6; speckle energies reach ~10x their mean)."""
    T, s, n = 32, 8, 9
    F = (n - 1) * s + T
    one = speckle_window(128, 128, 1, seed=7).numpy()
    frames = np.repeat(one, F, axis=0)
    with dh.Plan(128, 128, LAM, Z, PITCH, T=T, precision="fp16", max_frames=F, max_windows=n) as plan:
        img, lam = plan.pca_batch(to_gpu(frames), n, s, 1, T - 1)
        full, _ = plan.pca_batch(to_gpu(frames), n, s, 0, T - 1)
        torch.cuda.synchronize()
        assert plan.status() == 0
        img, full = img.double().cpu().numpy(), full.double().cpu().numpy()
    for w in range(n):
        assert np.max(img[w]) <= 1e-4 * np.mean(full[w]), w


def test_empty_batch_is_an_argument_error(dh):
    """A batch of no windows is rejected before anything launches."""
    frames = to_gpu(speckle_window(64, 64, 16, seed=3).numpy())
    with dh.Plan(64, 64, LAM, Z, PITCH, T=16, precision="fp16") as plan:
        with pytest.raises(dh.DHError) as e:
            plan.pca_batch(frames, 0, 16, 2, 15)
        assert e.value.code == 1
        assert plan.status() == 0


def test_more_windows_than_sms(dh):
    """160 windows (more than the SMs: one group, the eigensolver in several CTA rounds),
    first, middle and last against the oracle."""
    T, n = 16, 160
    frames = np.concatenate([speckle_window(128, 64, T, seed=500 + w).numpy() for w in range(n)])
    with dh.Plan(128, 64, LAM, Z, PITCH, T=T, precision="fp16", max_frames=n * T, max_windows=n) as plan:
        img, lam = plan.pca_batch(to_gpu(frames), n, T, 2, T - 1)
        torch.cuda.synchronize()
        assert plan.status() == 0
        img, lam = img.cpu().numpy(), lam.cpu().numpy()
    for w in (0, n // 2, n - 1):
        M, lam_ref, _, _ = oracle.pca_window(frames[w * T:(w + 1) * T], LAM, Z, PITCH, 2, T - 1)
        assert rel(img[w], M) <= TOL_IMG["fp16"], w
        assert np.max(np.abs(lam[w] - lam_ref)) <= 1e-5 * lam_ref[0], w


@pytest.mark.parametrize("persistent", [True, False])
def test_store_overflow_flag(dh, persistent):
    """16-bit storage beyond its range: a uniform frame at the largest 16-bit value has
    hologram components near 2.3e5 at 256^2 (the oracle's FP64 render), beyond FP16's 65504,
    so the render (persistent or chunked) raises DH_FLAG_STORE_OVERFLOW (0x1); the same frames
    stored in BF16 or FP32 do not, and speckle frames (components near 1.1e4) do not. Only the
    render runs: no window stage reads the non-finite planes."""
    T = 16
    hot = to_gpu(np.full((T, 256, 256), 65535, dtype=np.uint16))
    cool = to_gpu(speckle_window(256, 256, T, seed=0).numpy())
    for prec, frames, want in (("fp16", hot, 1), ("bf16", hot, 0), ("fp32", hot, 0), ("fp16", cool, 0)):
        with dh.Plan(256, 256, LAM, Z, PITCH, T=T, precision=prec) as plan:
            plan.set_render_schedule(persistent)
            plan.render_frames(frames)
            assert plan.status() == want, (prec, want)
            assert plan.status() == 0  # the bits are cleared by the read


def test_nonfinite_covariance_is_flagged(dh):
    """Holograms beyond FP16's range (as in test_store_overflow_flag) make C non-finite. The
    window's call raises DH_FLAG_NONFINITE_C (0x2) and DH_FLAG_EIG_NOT_CONVERGED (0x4) beside
    the overflow bit: every stage runs to its bounded end (the eigensolver's sweeps stop at
    their limit, and its ordering puts NaN eigenvalues last, so the ranks stay a
    permutation). The plan then gives a correct window again."""
    T = 16
    hot = np.full((T, 256, 256), 65535, dtype=np.uint16)
    cool = speckle_window(256, 256, T, seed=3).numpy()
    with dh.Plan(256, 256, LAM, Z, PITCH, T=T, precision="fp16") as plan:
        plan.render_stack(to_gpu(hot))
        plan.pca_window(2, T - 1)
        flags = plan.status()
        assert flags & 0x7 == 0x7, flags
        plan.render_stack(to_gpu(cool))
        img, lam = plan.pca_window(2, T - 1)
        assert plan.status() == 0
    M, lam_ref, _, _ = oracle.pca_window(cool, LAM, Z, PITCH, 2, T - 1)
    assert rel(img.double().cpu().numpy(), M) <= TOL_IMG["fp16"]
    assert np.max(np.abs(lam.numpy() - lam_ref)) <= 1e-5 * lam_ref[0]
