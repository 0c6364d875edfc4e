"""Display normalisation (each image divided by its mean) and 8-bit display codes, through
the C ABI, against the oracle; the display codes are decided in FP32 on both sides from the
same mean, so they must agree exactly. Also the headless PGM output."""

import numpy as np
import pytest
import torch

import oracle
from dh_synth import SpeckleParams, SpeckleStream
from parity_helpers import LAM, PITCH, Z, to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


def test_normalize_pca_images(dh, tmp_path):
    T = 32
    frames = SpeckleStream(SpeckleParams(256, 128), seed=90).next(3 * T).numpy()
    with dh.Plan(256, 128, LAM, Z, PITCH, T=T, precision="fp16", max_frames=3 * T,
                 max_windows=3) as plan:
        img, _ = plan.pca_batch(to_gpu(frames), 3, T, 2, T - 1)
        norm, disp, means = dh.normalize_images(img, display=True, gain=100.0)
        torch.cuda.synchronize()
    M = img.double().cpu().numpy()
    for w in range(3):
        N_ref, mean_ref = oracle.normalize(M[w])
        assert abs(means[w].item() - mean_ref) <= 1e-12 * mean_ref
        n = norm[w].double().cpu().numpy()
        assert np.max(np.abs(n - N_ref) / np.maximum(N_ref, 1e-30)) <= 2e-7
        codes = oracle.display_u8(img[w].cpu().numpy(), means[w].item(), 100.0)
        assert np.array_equal(disp[w].cpu().numpy(), codes)
    path = tmp_path / "window0.pgm"
    dh.save_pgm(str(path), disp[0])
    data = path.read_bytes()
    header = b"P5\n256 128\n255\n"
    assert data.startswith(header) and data[len(header):] == disp[0].cpu().numpy().tobytes()


def test_normalize_in_place_and_repeatable(dh):
    x = torch.rand((5, 64, 64), device="cuda", dtype=torch.float32) * 10 + 0.1
    ref = x.clone()
    _, _, m1 = dh.normalize_images(x, normalized=False)
    n, _, m2 = dh.normalize_images(x, in_place=True)
    torch.cuda.synchronize()
    assert torch.equal(m1, m2)  # fixed-order reduction
    assert n.data_ptr() == x.data_ptr()
    assert torch.allclose(x.mean(dim=(1, 2)).double(), torch.ones(5, dtype=torch.float64,
                                                                 device="cuda"), rtol=1e-6)
    assert torch.allclose(x * m1.view(5, 1, 1).float(), ref, rtol=1e-6)
