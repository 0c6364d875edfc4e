"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (stated in the workload definition):
  image relative L2 <= 1e-4 for the plain FP32 path, <= 1e-3 for the 16-bit fast form;
  eigenvalues within 1e-5 * lambda_max (norm-wise reading: |d lambda_k| <= ||dC||_2);
FP32 holograms are compared at 3e-6 relative L2 (a few FP32 ulps times log2 N stages),
covariances at 5e-6 relative Frobenius (plain) and 2e-4 (16-bit storage).
"""

import ctypes

import numpy as np
import pytest
import torch

import oracle
from dh_synth import SpeckleParams, SpeckleStream, known_rank_frames, speckle_window
from parity_helpers import (EXTREME_RANGES, LAM, PITCH, TOL_IMG, TOL_LAM, Z, check_window,
                            check_window_extreme_range, lam_tol, rel, to_gpu)

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


# ------------------------------------------------------------------------ Eq. 1
RENDER_SIZES = [(16, 16), (32, 64), (64, 32), (128, 256), (256, 128), (512, 1024),
                (1024, 512), (2048, 16), (16, 2048), (4096, 64), (64, 4096), (1024, 1024)]


@pytest.mark.parametrize("nx,ny", RENDER_SIZES)
def test_render_fp32_matches_oracle(dh, nx, ny):
    f = speckle_window(nx, ny, 2, seed=nx * 7 + ny).numpy()
    with dh.Plan(nx, ny, LAM, Z, PITCH, T=16) as plan:
        plan.render_frames(to_gpu(f), first_slot=3)
        got = [plan.debug_hologram(3 + t).cpu().numpy() for t in range(2)]
        assert plan.status() == 0
    ref = oracle.render(f, LAM, Z, PITCH)
    for t in range(2):
        assert rel(got[t], ref[t]) < 3e-6, (nx, ny, t, rel(got[t], ref[t]))


@pytest.mark.parametrize("prec,tol", [("fp16", 6e-4), ("bf16", 5e-3)])
def test_render_16bit_storage_rounding(dh, prec, tol):
    nx = ny = 256
    f = speckle_window(nx, ny, 2, seed=5).numpy()
    with dh.Plan(nx, ny, LAM, Z, PITCH, T=16, precision=prec) as plan:
        plan.render_frames(to_gpu(f))
        got = plan.debug_hologram(1).cpu().numpy()
        assert plan.status() == 0
    ref = oracle.render(f, LAM, Z, PITCH)[1]
    assert rel(got, ref) < tol


def test_render_point_source_closed_form(dh):
    """Eq. 1 for a delta: |H| = s A at every pixel (FP32 rounding only)."""
    nx = ny = 512
    f = np.zeros((1, ny, nx), dtype=np.uint16)
    f[0, 100, 400] = 4000
    with dh.Plan(nx, ny, LAM, Z, PITCH, T=16) as plan:
        plan.render_frames(to_gpu(f))
        h = plan.debug_hologram(0).cpu().numpy()
    assert np.allclose(np.abs(h), 4000 / nx, rtol=2e-6)


# ------------------------------------------------------------------- whole window
def gpu_windows(dh, frames_np, T, prec, k0, k1, n_windows, stride):
    """prec "fp16-residual": FP16 storage with mean-residual storage (DH_OPT_RESIDUAL)."""
    ny, nx = frames_np.shape[1:]
    residual = prec.endswith("-residual")
    with dh.Plan(nx, ny, LAM, Z, PITCH, T=T, precision=prec.split("-")[0], max_frames=frames_np.shape[0],
                 max_windows=n_windows) as plan:
        if residual:
            plan.set_residual(True)
        images, lam = plan.pca_batch(to_gpu(frames_np), n_windows, stride, k0, k1)
        C = [plan.debug_covariance(w).cpu().numpy() for w in range(n_windows)]
        flags = plan.status()
    return images.cpu().numpy(), lam.cpu().numpy(), C, flags


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_config0_plain_small(dh, prec):
    """8 windows of 32 frames at 256x256, seeds 0..7, k0=2..31 (the small workload).
    The stated tolerances apply as is (no gap allowance)."""
    T, n = 32, 8
    frames = np.concatenate([speckle_window(256, 256, T, seed=w).numpy() for w in range(n)])
    img, lam, C, flags = gpu_windows(dh, frames, T, prec, 2, T - 1, n, T)
    assert flags == 0
    for w in range(n):
        M, lam_ref, _, _ = oracle.pca_window(frames[w * T:(w + 1) * T], LAM, Z, PITCH, 2, T - 1)
        assert rel(img[w], M) <= TOL_IMG[prec]
        assert np.max(np.abs(lam[w] - lam_ref)) <= TOL_LAM * lam_ref[0]


@pytest.mark.parametrize("T", [16, 32, 64])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_window_lengths(dh, T, prec):
    f = speckle_window(128, 64, T, seed=T + 1).numpy()
    img, lam, C, flags = gpu_windows(dh, f, T, prec, 2, T - 1, 1, T)
    assert flags == 0
    check_window(img[0], lam[0], C[0], f, 2, T - 1, prec)


@pytest.mark.parametrize("nx,ny,T", [(16, 16, 16), (32, 16, 16), (16, 32, 32), (64, 16, 32)])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_smallest_frames(dh, nx, ny, T, prec):
    """The smallest frames the library takes (16 pixels a side) through the whole path,
    against the oracle at the stated tolerances (eigenvalues at the storage bound below
    256^2 pixels)."""
    f = speckle_window(nx, ny, T, seed=nx * 7 + ny + T).numpy()
    img, lam, C, flags = gpu_windows(dh, f, T, prec, 2, T - 1, 1, T)
    assert flags == 0
    check_window(img[0], lam[0], C[0], f, 2, T - 1, prec, label=f"{nx}x{ny}")


# FP16 storage of H alone rounds every value by up to 2^-12 relative; the projected image of
# a range then carries ~u sqrt(E / (T M_kept)) relative error, E the energy and M_kept the
# kept power. For the paper's own range (k0 = 12: the 20 weakest components, E / M_kept ~ 500
# on this generator) that is 1.06-1.13e-3 in exact arithmetic with FP16-rounded H (emulated
# from the oracle at 64^2 .. 512^2), above the 1e-3 of the fast form whatever the kernels do.
STORAGE_FLOOR = {("fp16", 12, 31): "FP16 storage alone gives 1.1e-3 at k0 = 12 (E / M_kept ~ 500)"}


# Mean-residual storage ("fp16-residual") removes the window's static part from the 16-bit
# values and meets the stated tolerance there too.
@pytest.mark.parametrize("k0,k1", [(0, 31), (0, 0), (31, 31), (5, 17), (12, 31)])
@pytest.mark.parametrize("prec", ["fp32", "fp16", "fp16-residual"])
def test_retained_ranges(dh, k0, k1, prec, request):
    if (prec, k0, k1) in STORAGE_FLOOR:
        request.applymarker(pytest.mark.xfail(strict=True, reason=STORAGE_FLOOR[(prec, k0, k1)]))
    f = speckle_window(64, 64, 32, seed=77).numpy()
    img, lam, C, _ = gpu_windows(dh, f, 32, prec, k0, k1, 1, 32)
    tol_prec = "fp16" if prec == "fp16-residual" else prec
    if (k0, k1) in EXTREME_RANGES:
        check_window_extreme_range(img[0], lam[0], C[0], f, k0, k1, tol_prec)
    else:
        check_window(img[0], lam[0], C[0], f, k0, k1, tol_prec)


def test_full_range_is_parseval(dh):
    """k0=0, k1=T-1: the image is sum_t |H_t|^2 = sum_t I_t^2 per pixel of the holograms."""
    f = speckle_window(128, 128, 16, seed=3).numpy()
    img, _, _, _ = gpu_windows(dh, f, 16, "fp32", 0, 15, 1, 16)
    H = oracle.render(f, LAM, Z, PITCH)
    assert rel(img[0], np.sum(np.abs(H) ** 2, axis=0)) < 1e-5


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_known_rank_eigenvalues(dh, prec):
    comps = [(1, 300, 300), (5, 200, 700), (30, 100, 1500), (17, 400, 90)]
    f, lam_exact = known_rank_frames(128, 128, 32, 2000, comps, support_seed=1)
    _, lam, _, _ = gpu_windows(dh, f, 32, prec, 2, 31, 1, 32)
    assert np.max(np.abs(lam[0] - lam_exact)) <= lam_tol(prec, f[0].size) * lam_exact[0]


def test_covariance_is_integer_gram(dh):
    """Unitary Fresnel rendering preserves inner products: C = I^T I (exact int64)."""
    f = speckle_window(256, 256, 32, seed=12).numpy()
    _, _, C, _ = gpu_windows(dh, f, 32, "fp32", 2, 31, 1, 32)
    I = f.reshape(32, -1).astype(np.int64)
    G = (I @ I.T).astype(np.float64)
    assert rel(C[0].real, G) < 5e-6
    assert np.max(np.abs(C[0].imag)) < 5e-6 * np.max(G)


# ------------------------------------------------------------ determinism
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_repeated_calls_are_bitwise_equal(dh, prec):
    """The same batch twice on one plan: bitwise the same images and eigenvalues, whatever
    the run-time order of the persistent render's tickets, the split-K covariance units and
    the two window groups sharing SMs (40 windows); the Fourier span path likewise."""
    T, n = 32, 40
    frames = to_gpu(np.concatenate([speckle_window(128, 128, T, seed=900 + w).numpy() for w in range(n)]))
    with dh.Plan(128, 128, LAM, Z, PITCH, T=T, precision=prec, max_frames=n * T, max_windows=n) as plan:
        runs = []
        for _ in range(2):
            img, lam = plan.pca_batch(frames, n, T, 2, T - 1)
            runs.append((img.cpu(), lam.cpu()))
        assert plan.status() == 0
        assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])
        fourier = [plan.fourier_windows(0, 1, 64, 7, 23).cpu() for _ in range(2)]
        assert torch.equal(fourier[0], fourier[1])


# ------------------------------------------------------------ batching semantics
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_window_alone_equals_in_batch(dh, prec):
    """A window's image is bitwise the same computed alone and inside a batch."""
    T = 32
    frames = np.concatenate([speckle_window(128, 128, T, seed=40 + w).numpy() for w in range(5)])
    img_b, lam_b, _, _ = gpu_windows(dh, frames, T, prec, 2, 31, 5, T)
    for w in (0, 3):
        img_1, lam_1, _, _ = gpu_windows(dh, frames[w * T:(w + 1) * T], T, prec, 2, 31, 1, T)
        assert np.array_equal(img_1[0], img_b[w])
        assert np.array_equal(lam_1[0], lam_b[w])


@pytest.mark.parametrize("T,n,ws", [(32, 40, 32), (16, 33, 16), (64, 32, 64), (32, 48, 40)])
def test_two_window_groups_equal_one(dh, T, n, ws):
    """The two-group schedule (each group's eigensolver beside the other group's covariance
    or projection, on SM budgets) gives bitwise the one-group results, with the frames
    rendered inside the call, for an odd split, every window length, and gaps between
    windows; the two-group batch matches the oracle on its first and last window."""
    F = (n - 1) * ws + T
    frames = SpeckleStream(SpeckleParams(128, 128), seed=T + n).next(F)
    out = []
    for automatic in (False, True):
        with dh.Plan(128, 128, LAM, Z, PITCH, T=T, precision="fp16", max_frames=F, max_windows=n) as plan:
            plan.set_window_groups(automatic)
            img, lam = plan.pca_batch(to_gpu(frames.numpy()), n, ws, 2, T - 1)
            torch.cuda.synchronize()
            assert plan.status() == 0
            out.append((img.cpu().numpy(), lam.cpu().numpy()))
            if automatic:
                for w in (0, n - 1):
                    C = plan.debug_covariance(w).cpu().numpy()
                    check_window(out[-1][0][w].astype(np.float64), out[-1][1][w], C,
                                 frames[w * ws:w * ws + T].numpy(), 2, T - 1, "fp16")
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_two_window_groups_equal_one_raw_covariance(dh):
    """The two-group schedule with the covariance taken from the uint16 frames (C = I^T I)
    gives bitwise the one-group results, and matches the oracle on its first and last window."""
    T, n = 32, 36
    F = n * T
    frames = SpeckleStream(SpeckleParams(128, 128), seed=77).next(F)
    out = []
    for automatic in (False, True):
        with dh.Plan(128, 128, LAM, Z, PITCH, T=T, precision="fp16", max_frames=F, max_windows=n) as plan:
            plan.set_covariance_source("raw")
            plan.set_window_groups(automatic)
            img, lam = plan.pca_batch(to_gpu(frames.numpy()), n, T, 2, T - 1)
            torch.cuda.synchronize()
            assert plan.status() == 0
            out.append((img.cpu().numpy(), lam.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    for w in (0, n - 1):
        M, lam_ref, _, _ = oracle.pca_window(frames[w * T:(w + 1) * T].numpy(), LAM, Z, PITCH, 2, T - 1)
        assert rel(out[1][0][w], M) <= TOL_IMG["fp16"]
        assert np.max(np.abs(out[1][1][w] - lam_ref)) <= TOL_LAM * lam_ref[0]


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_overlapping_sliding_windows(dh, prec):
    """Windows at stride 8 < T share rendered holograms; each matches the oracle."""
    T, stride, n = 16, 8, 4
    frames = SpeckleStream(SpeckleParams(128, 64), seed=9).next((n - 1) * stride + T).numpy()
    img, lam, C, _ = gpu_windows(dh, frames, T, prec, 2, T - 1, n, stride)
    for w in range(n):
        check_window(img[w], lam[w], C[w], frames[w * stride:w * stride + T], 2, T - 1, prec)


def test_deterministic(dh):
    f = speckle_window(256, 256, 32, seed=8).numpy()
    a = gpu_windows(dh, f, 32, "fp16", 2, 31, 1, 32)
    b = gpu_windows(dh, f, 32, "fp16", 2, 31, 1, 32)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_invalid_calls_return_errors(dh):
    with dh.Plan(64, 64, LAM, Z, PITCH, T=16) as plan:
        f = to_gpu(speckle_window(64, 64, 16, seed=1).numpy())
        plan.render_stack(f)
        with pytest.raises(dh.DHError) as e:
            plan.pca_windows(0, 16, 1, 3, 16)  # k1 >= T
        assert e.value.code == 1
        with pytest.raises(dh.DHError):
            plan.pca_windows(0, 16, 2, 0, 15)  # more windows than reserved
        with pytest.raises(dh.DHError):
            plan.render_frames(f, first_slot=8)  # slots beyond the reservation
        lib = plan._lib
        for opt, bad in ((0, 2), (1, 1), (1, 65), (2, 64), (3, 3), (4, 2), (5, 2), (5, -1), (6, -1),
                         (6, 100000001), (7, 3), (8, 64), (9, 3), (10, 2), (11, 0)):
            assert lib.dh_plan_set_option(plan._h, opt, bad) == 1, (opt, bad)  # DH_ERR_INVALID_ARG
        v = ctypes.c_int(-1)
        assert lib.dh_plan_get_option(plan._h, 5, ctypes.byref(v)) == 0 and v.value == 0
        plan.set_window_groups(False)
        assert lib.dh_plan_get_option(plan._h, 5, ctypes.byref(v)) == 0 and v.value == 1
        img, lam = plan.pca_window(2, 15)
        assert np.all(np.diff(lam.numpy()) <= 0)


# ------------------------------------------------- tensor-core kernels, storage excluded
@pytest.mark.parametrize("T", [16, 32, 64])
@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_kernels_exact_on_stored_values(dh, T, prec):
    """Separate kernel error from storage rounding: recompute Eq. 4 and Eqs. 6-7 in FP64
    from the 16-bit holograms the GPU stored and the eigenvectors it found. The covariance
    then differs only by FP32 accumulation, the image by the hi+lo split of V."""
    nx, ny, n = 256, 128, 3
    frames = np.concatenate([speckle_window(nx, ny, T, seed=90 + w).numpy() for w in range(n)])
    with dh.Plan(nx, ny, LAM, Z, PITCH, T=T, precision=prec, max_frames=n * T,
                 max_windows=n) as plan:
        images, _ = plan.pca_batch(to_gpu(frames), n, T, 2, T - 1)
        for w in range(n):
            Hs = np.stack([plan.debug_hologram(w * T + t).cpu().numpy() for t in range(T)])
            Hs = Hs.astype(np.complex128).reshape(T, -1)
            C_gpu = plan.debug_covariance(w).cpu().numpy()
            V = plan.debug_eigvecs(w).cpu().numpy()
            C_exact = Hs.conj() @ Hs.T
            assert rel(C_gpu, C_exact) < 1e-6
            P = Hs.T @ V[:, 2:T]
            M_exact = np.sum(np.abs(P) ** 2, axis=1).reshape(ny, nx)
            # V's hi+lo split keeps ~22 (fp16) / ~16 (bf16) significant bits
            assert rel(images[w].cpu().numpy(), M_exact) < (1e-5 if prec == "fp16" else 6e-5)
        assert plan.status() == 0


# ------------------------------------------------------------- eigensolver precision
@pytest.mark.parametrize("T", [16, 32, 64])
def test_eigensolver_reaches_fp64_accuracy(dh, T):
    """Eq. 5 on the GPU's own covariance: the residual and orthonormality of the returned
    eigenpairs are at FP64 level (the FP32 sweeps only supply the starting basis)."""
    f = speckle_window(128, 128, T, seed=300 + T).numpy()
    with dh.Plan(128, 128, LAM, Z, PITCH, T=T, precision="fp32") as plan:
        _, lam = plan.pca_batch(to_gpu(f), 1, T, 2, T - 1)
        C = plan.debug_covariance(0).cpu().numpy()
        V = plan.debug_eigvecs(0).cpu().numpy()
        assert plan.status() == 0
    lam = lam[0].cpu().numpy()
    Ch = 0.5 * (C + C.conj().T)
    nC = np.linalg.norm(Ch, 2)
    assert np.all(np.diff(lam) <= 0)
    assert np.linalg.norm(Ch @ V - V * lam[None, :]) <= 1e-12 * nC * T
    assert np.linalg.norm(V.conj().T @ V - np.eye(T)) <= 1e-12 * T
    ref = np.linalg.eigvalsh(Ch)[::-1]
    assert np.max(np.abs(lam - ref)) <= 1e-12 * nC


# ------------------------------------------------------- persistent render schedule
@pytest.mark.parametrize("n,F", [(256, 9), (512, 7), (1024, 13), (2048, 5), (4096, 3)])
@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_persistent_render_equals_chunked(dh, n, F, prec):
    """The persistent ring schedule (one launch, rows and columns of consecutive frames
    interleaved) and the chunked two-launch schedule compute the same transforms: the
    holograms must be bitwise equal, at every square size it serves, with more frames
    than the ring holds."""
    frames = to_gpu(SpeckleStream(SpeckleParams(n, n), seed=n + F).next(F).numpy())
    out = []
    # chunks; the persistent ring with an explicit ring and lag (so it runs at every size);
    # and the automatic choice
    for sched in ((False, 0, 0), (True, 3, 1), (True, 0, 0)):
        with dh.Plan(n, n, LAM, Z, PITCH, T=16, precision=prec, max_frames=max(F + 2, 16)) as plan:
            plan.set_render_schedule(*sched)
            plan.render_frames(frames, first_slot=2)
            out.append([plan.debug_hologram(2 + t).cpu() for t in range(F)])
            assert plan.status() == 0
    for holo in out[1:]:
        for a, b in zip(out[0], holo):
            assert torch.equal(a, b)


def test_persistent_render_smallest_ring(dh):
    """The smallest ring (2 frame intermediates, lag 1) at 256^2, where the grid's items in
    flight span many more frames than the ring holds: a CTA's ring-slot wait can then need the
    rows of the row item it finished last, whose release it has deferred, so the wait itself
    must publish them. The holograms equal the chunked schedule's bitwise and no wait times
    out."""
    n, F = 256, 40
    frames = to_gpu(SpeckleStream(SpeckleParams(n, n), seed=4242).next(F).numpy())
    out = []
    for sched in ((False, 0, 0), (True, 2, 1)):
        with dh.Plan(n, n, LAM, Z, PITCH, T=16, precision="fp16", max_frames=F) as plan:
            plan.set_render_schedule(*sched)
            plan.render_frames(frames)
            out.append([plan.debug_hologram(t).cpu() for t in range(0, F, 3)])
            assert plan.status() == 0
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a, b)


def test_autotune_picks_are_plan_options(dh):
    """The autotuner's picks are plan options: a plan given the same options explicitly renders
    bitwise the same holograms; picks that change the arithmetic (radix, tensor cores) change
    only the rounding (within 1e-3 of the 16-bit holograms before tuning)."""
    frames = to_gpu(SpeckleStream(SpeckleParams(512, 512), seed=77).next(6).numpy())
    with dh.Plan(512, 512, LAM, Z, PITCH, T=16, precision="fp16", max_frames=16) as plan:
        plan.render_frames(frames)
        before = [plan.debug_hologram(t).cpu() for t in range(6)]
        pick = plan.autotune(16)
        assert {"persistent", "ring", "lag", "fft", "radix", "gram_units"} <= set(pick)
        plan.render_frames(frames)
        after = [plan.debug_hologram(t).cpu() for t in range(6)]
    with dh.Plan(512, 512, LAM, Z, PITCH, T=16, precision="fp16", max_frames=16) as again:
        again.set_render_schedule(pick["persistent"], pick["ring"], pick["lag"])
        again.set_render_fft(pick["fft"])
        again.set_fft_radix(pick["radix"])
        again.set_gram_units(pick["gram_units"])
        again.render_frames(frames)
        explicit = [again.debug_hologram(t).cpu() for t in range(6)]
    for a, b, c in zip(before, after, explicit):
        assert torch.equal(b, c)
        assert rel(b.numpy(), a.numpy()) <= 1e-3


# ------------------------------------------------------- host buffers, overlapped copies
@pytest.mark.parametrize("T,ws,n", [(16, 16, 40), (16, 8, 50), (16, 40, 7), (32, 32, 9)])
@pytest.mark.parametrize("pinned", [True, False])
def test_batch_from_host_buffers_equals_device_batch(dh, T, ws, n, pinned):
    """dh_pca_batch_host (groups of windows copied in while earlier groups compute) gives
    bitwise the device-buffer batch's images and eigenvalues, for windows apart by T, by
    less (overlapping) and by more (gaps), from pinned and from pageable memory."""
    F = (n - 1) * ws + T
    frames = SpeckleStream(SpeckleParams(128, 64), seed=T + ws + n).next(F)
    host = frames.pin_memory() if pinned else frames.clone()
    with dh.Plan(128, 64, LAM, Z, PITCH, T=T, precision="fp16", max_frames=F, max_windows=n) as plan:
        img_d, lam_d = plan.pca_batch(frames.cuda(), n, ws, 2, T - 1)
        img_d, lam_d = img_d.cpu(), lam_d.cpu()
        img_h, lam_h = plan.pca_batch_host(host, n, ws, 2, T - 1)
        assert plan.status() == 0
    assert torch.equal(img_h, img_d) and torch.equal(lam_h, lam_d)
