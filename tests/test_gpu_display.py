"""Display normalisation (each image divided by its mean) and 8-bit display codes, through
the C ABI, against the oracle. The oracle takes the image alone: its own FP64 mean and FP64
code decisions. The kernel decides each code in FP32 (value * float(gain / mean)), within
about 2 FP32 roundings (~1.2e-7 relative, < 4e-5 of a code at 255) of the FP64 value, so the
codes agree exactly except where the FP64 value lies within TIE_DIST of a rounding
half-integer; there a difference of 1 is allowed, and the number of such pixels is counted
and bounded. Also the headless PGM output."""

import numpy as np
import pytest
import torch

import oracle
from dh_synth import SpeckleParams, SpeckleStream
from parity_helpers import LAM, PITCH, Z, to_gpu

pytestmark = pytest.mark.gpu

# distance (in code units) from a rounding half-integer within which FP32 and FP64 decisions
# may differ: 2.5 x the FP32 bound above at the top code
TIE_DIST = 1e-4


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
        codes = oracle.display_u8(M[w], 100.0)
        v = oracle.display_value(M[w], 100.0)
        near_tie = (np.abs(v - np.floor(v) - 0.5) < TIE_DIST) & (v < 255.5)
        got = disp[w].cpu().numpy().astype(np.int32)
        diff = np.abs(got - codes.astype(np.int32))
        assert np.all(diff[~near_tie] == 0), int(np.count_nonzero(diff[~near_tie]))
        assert np.all(diff[near_tie] <= 1)
        # the tie band is 2e-4 of a code wide: expect about 2e-4 of the pixels in it
        n_tie = int(np.count_nonzero(near_tie))
        print(f"window {w}: {n_tie} of {M[w].size} pixels near a tie, "
              f"{int(np.count_nonzero(diff))} codes differ")
        assert n_tie <= 1e-3 * M[w].size + 4
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
