"""12-bit packed camera frames (Mono12p) through the C ABI: the device unpack against the
frames it came from, bitwise, and dh_pca_batch_host_packed12 against dh_pca_batch_host on the
same frames, bitwise (after the unpack both run the same device work)."""
import ctypes

import numpy as np
import pytest
import torch

from dh_synth import SpeckleParams, SpeckleStream
from parity_helpers import LAM, PITCH, Z

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


@pytest.mark.parametrize("F,ny,nx", [(1, 16, 16), (5, 64, 32), (3, 1024, 1024), (2, 2048, 2048)])
def test_unpack_is_bitwise(dh, F, ny, nx):
    rng = np.random.default_rng(F * 1000 + nx)
    f = rng.integers(0, 4096, size=(F, ny, nx), dtype=np.uint16)
    f[0, 0, :4] = [0, 4095, 0x800, 0x7FF]  # extremes of the 12-bit range
    packed = dh.pack_mono12p(f).cuda()
    out = dh.unpack_mono12p(packed, ny, nx)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), f)


@pytest.mark.parametrize("T,ws", [(32, 32), (16, 8)])
def test_packed_batch_equals_uint16_batch(dh, T, ws):
    n, nw = 256, 5
    nf = (nw - 1) * ws + T
    frames = SpeckleStream(SpeckleParams(n, n), seed=41).next(nf).numpy()
    assert frames.max() < 4096  # the generator's frames are 12-bit
    f16 = torch.from_numpy(frames).pin_memory()
    fp = dh.pack_mono12p(frames).pin_memory()
    with dh.Plan(n, n, LAM, Z, PITCH, T=T, precision="fp16", max_frames=nf, max_windows=nw) as plan:
        img_a, eig_a = plan.pca_batch_host(f16, nw, ws, 2, T - 1)
        img_a, eig_a = img_a.clone(), eig_a.clone()
        img_b, eig_b = plan.pca_batch_host_packed12(fp, nw, ws, 2, T - 1)
        assert plan.status() == 0
    assert torch.equal(img_a, img_b)
    assert torch.equal(eig_a, eig_b)


def test_argument_errors(dh):
    lib = dh._lib.load()
    src = torch.zeros(64 * 3 // 2 + 16, dtype=torch.uint8, device="cuda")
    dst = torch.zeros(64 + 16, dtype=torch.uint16, device="cuda")
    p, q = src.data_ptr(), dst.data_ptr()
    assert lib.dh_unpack_mono12p(p, 96, 64, 1, q, 64, None) == 0
    assert lib.dh_unpack_mono12p(p, 94, 64, 1, q, 64, None) == 1       # stride below 3/2 npix
    assert lib.dh_unpack_mono12p(p, 98, 64, 1, q, 64, None) == 1       # stride not a multiple of 4
    assert lib.dh_unpack_mono12p(p + 2, 96, 64, 1, q, 64, None) == 1   # source not 4-byte aligned
    assert lib.dh_unpack_mono12p(p, 96, 64, 1, q + 8, 64, None) == 1   # destination not 16-byte aligned
    assert lib.dh_unpack_mono12p(p, 96, 60, 1, q, 64, None) == 1       # npix not a multiple of 8
    torch.cuda.synchronize()
    with dh.Plan(64, 64, LAM, Z, PITCH, T=16, precision="fp16", max_frames=16, max_windows=1) as plan:
        img = torch.empty((1, 64, 64), dtype=torch.float32)
        fr = torch.zeros((16, 64 * 64 * 3 // 2), dtype=torch.uint8)
        rc = lib.dh_pca_batch_host_packed12(plan._h, fr.data_ptr(), 64 * 64 * 3 // 2 - 4, 1, 16, 2, 15,
                                            img.data_ptr(), None, None)
        assert rc == 1  # stride below the frame's bytes
        rc = lib.dh_pca_batch_host_packed12(plan._h, fr.data_ptr(), 64 * 64 * 3 // 2 + 2, 1, 16, 2, 15,
                                            img.data_ptr(), None, None)
        assert rc == 1  # not a multiple of 4
