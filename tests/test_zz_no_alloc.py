"""The allocation-free covariance entry point (dh_covariance_noalloc).

Some callers cannot allocate device memory while they run (a frame-grabber callback, a
real-time acquisition thread, code whose memory belongs to another allocator); this entry
point gives them the window covariance with its scratch in a fixed device array inside the
library. Here it is called through the C ABI, twice in a row, and checked against the
covariance the regular plan-based path computes for the same holograms, and against the
oracle's covariance of the oracle's own holograms (rounded to FP32, the entry point's input
type). The sizes include two that fill the 2 MiB scratch exactly: 16 partial 128 x 128
matrices (T = 64 at 512 x 512) and 64 partial 64 x 64 ones (T = 32 at 1024 x 1024).

This file sorts last on purpose: a run that stops at the first failure has already run
every other test before it gets here. It passes alone in a fresh process too.
"""

import ctypes

import numpy as np
import pytest
import torch

import oracle
from dh_synth import speckle_window

pytestmark = pytest.mark.gpu

LAM, Z, PITCH = 785e-9, 0.35, 20e-6


def _noalloc_twice(lib, _lib, planes, npix, T):
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):  # two calls in a row share the library's scratch array
        C = torch.full((T, T, 2), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.dh_covariance_noalloc(ctypes.c_void_p(planes.data_ptr()), npix, T,
                                       ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(stream))
        assert rc == 0, _lib.STATUS_NAMES.get(rc, rc)
        torch.cuda.synchronize()
        outs.append(torch.view_as_complex(C).cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    return outs


SIZES = [(256, 256, 32), (128, 64, 16), (256, 128, 64), (512, 512, 64), (1024, 1024, 32)]


@pytest.mark.parametrize("nx,ny,T", SIZES)
def test_noalloc_covariance_matches_oracle(nx, ny, T):
    """The oracle renders the frames (Eq. 1, FP64); its holograms, rounded to FP32, are the
    entry point's input; the expected C is the oracle's covariance of those same FP32 values,
    so the only difference left is the entry point's FP32 products (FP64 accumulation)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2004_00923_b300 import _lib

    lib = _lib.load()
    frames = speckle_window(nx, ny, T, seed=nx + T + 5).numpy()
    H = oracle.render(frames, LAM, Z, PITCH).reshape(T, -1)
    H32 = H.real.astype(np.float32) + 1j * H.imag.astype(np.float32)
    C_ref = oracle.covariance(H32.astype(np.complex128))
    planes = np.empty((2 * T, nx * ny), dtype=np.float32)
    planes[0::2], planes[1::2] = H32.real, H32.imag
    outs = _noalloc_twice(lib, _lib, torch.from_numpy(planes).cuda(), nx * ny, T)
    err = np.linalg.norm(outs[0] - C_ref) / np.linalg.norm(C_ref)
    print(f"{nx}x{ny} T={T}: C against the oracle {err:.2e}")
    assert err <= 1e-6


@pytest.mark.parametrize("nx,ny,T", SIZES)
def test_noalloc_covariance_matches_plan_path(nx, ny, T):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as dh
    from paper_2004_00923_b300 import _lib

    lib = _lib.load()
    frames = torch.from_numpy(speckle_window(nx, ny, T, seed=nx + T).numpy()).cuda()
    with dh.Plan(nx, ny, LAM, Z, PITCH, T=T, precision="fp32") as plan:
        plan.render_stack(frames)
        plan.pca_windows(0, T, 1, 2, T - 1)
        C_ref = plan.debug_covariance(0).cpu().numpy()
        holo = [plan.debug_hologram(t) for t in range(T)]
    # caller-held planes [2T][npix]: row 2t = Re H_t, row 2t+1 = Im H_t
    planes = torch.empty((2 * T, nx * ny), dtype=torch.float32, device="cuda")
    for t, h in enumerate(holo):
        planes[2 * t] = h.real.reshape(-1)
        planes[2 * t + 1] = h.imag.reshape(-1)
    outs = _noalloc_twice(lib, _lib, planes, nx * ny, T)
    # same FP32-product / FP64-accumulation arithmetic as the plan's plain path
    assert np.linalg.norm(outs[0] - C_ref) <= 1e-6 * np.linalg.norm(C_ref)


def test_noalloc_rejects_sizes_beyond_its_limits():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2004_00923_b300 import _lib

    lib = _lib.load()
    x = torch.zeros((2 * 32, 1024), dtype=torch.float32, device="cuda")
    C = torch.zeros((32, 32, 2), dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p, c = ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(C.data_ptr())
    assert lib.dh_covariance_noalloc(p, 1024, 128, c, s) == 2   # T beyond the kernels
    assert lib.dh_covariance_noalloc(p, 1000, 32, c, s) == 1    # npix not a multiple of 32
    assert lib.dh_covariance_noalloc(p, 1 << 29, 32, c, s) == 2  # beyond 2^28 pixels
    assert lib.dh_covariance_noalloc(None, 1024, 32, c, s) == 1
    # misaligned caller pointers are rejected on the host before anything launches
    p4 = ctypes.c_void_p(x.data_ptr() + 4)
    c4 = ctypes.c_void_p(C.data_ptr() + 4)
    assert lib.dh_covariance_noalloc(p4, 1024, 32, c, s) == 1
    assert lib.dh_covariance_noalloc(p, 1024, 32, c4, s) == 1
