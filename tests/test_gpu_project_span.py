"""Grouped projection of overlapping windows (DH_OPT_PROJECTION = 0, csrc/project_span.cu).

Windows with slot stride s < T (s a multiple of 4) are projected in groups that share each
pixel tile's load, and each window's power is its energy minus its discarded components'
power (Eq. 7 through the unitarity of V). Checked against the per-window projection of Eq. 7
(the same holograms and eigenvectors: FP32 rounding apart, bounded relative to the window's
energy / kept power ratio) and against the FP64 oracle, over
ragged last groups, one or both halves of a group's windows, 1-4 discarded components
(4 or 8 operand columns per window), strides 4/8/12/16, a start slot off zero and
non-square frames.
"""

import numpy as np
import pytest
import torch

from dh_synth import SpeckleParams, SpeckleStream
from parity_helpers import LAM, PITCH, Z, check_window, rel, to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


# nx, ny, T, stride, windows, k0, k1, first slot
CASES = [
    (128, 128, 16, 8, 23, 2, 15, 0),    # groups of 8: two full, a ragged one of 7
    (128, 128, 32, 8, 11, 2, 31, 5),    # last group of 3 (its second half empty)
    (128, 128, 64, 8, 10, 2, 63, 0),    # last group of 2
    (256, 128, 32, 4, 13, 1, 29, 3),    # 3 discarded components: 8 columns per window
    (128, 256, 64, 16, 5, 0, 63, 0),    # nothing discarded (power = energy), groups of 5
    (128, 128, 64, 4, 20, 4, 63, 0),    # 4 discarded
    (128, 128, 32, 12, 6, 2, 31, 2),    # stride 12
    (128, 128, 16, 8, 3, 2, 15, 0),     # one group of 3 (the smallest span: 64 rows)
]


@pytest.mark.parametrize("nx,ny,T,s,n,k0,k1,first", CASES)
def test_grouped_equals_per_window_and_oracle(dh, nx, ny, T, s, n, k0, k1, first):
    F = first + (n - 1) * s + T
    frames = SpeckleStream(SpeckleParams(nx, ny), seed=60 + T + s + n).next(F).numpy()
    with dh.Plan(nx, ny, LAM, Z, PITCH, T=T, precision="fp16", max_frames=F, max_windows=n) as plan:
        plan.render_frames(to_gpu(frames))
        img_g, lam_g = plan.pca_windows(first, s, n, k0, k1)
        img_g, lam_g = img_g.cpu().numpy(), lam_g.cpu().numpy()
        C = [plan.debug_covariance(w).cpu().numpy() for w in range(n)]
        prof = {}
        plan.profile(True)
        plan.pca_windows(first, s, n, k0, k1)
        prof = plan.profile_read()
        plan.profile(False)
        assert prof["project_span"][0] == 1 and prof["project_tc"][0] == 0
        plan.set_projection(False)
        img_w, lam_w = plan.pca_windows(first, s, n, k0, k1)
        img_w, lam_w = img_w.cpu().numpy(), lam_w.cpu().numpy()
        assert plan.status() == 0
    assert np.array_equal(lam_g, lam_w)  # same covariance and eigensolver
    for w in range(n):
        # the complement's rounding (FP32 sums, V to ~22 bits in hi + lo) is relative to the
        # window's energy, not to the kept power: the bound scales with their ratio
        lam = lam_g[w]
        ratio = lam.sum() / lam[k0:k1 + 1].sum()
        e = rel(img_g[w], img_w[w])
        assert e <= 1.5e-6 * ratio, (w, e, ratio)
        assert img_g[w].min() >= 0.0
    for w in (0, n // 2, n - 1):
        f0 = first + w * s
        check_window(img_g[w], lam_g[w], C[w], frames[f0:f0 + T], k0, k1, "fp16")


def test_grouped_not_used_where_it_does_not_apply(dh):
    """Per-window projection for: non-overlapping windows, a stride not a multiple of 4,
    BF16 storage, more than 4 discarded components, frames fewer than 128 rows high."""
    frames = to_gpu(SpeckleStream(SpeckleParams(128, 128), seed=70).next(96).numpy())
    small = to_gpu(SpeckleStream(SpeckleParams(128, 64), seed=71).next(96).numpy())
    for prec, fr, ny, s, k0, k1 in [("fp16", frames, 128, 32, 2, 31), ("fp16", frames, 128, 6, 2, 31),
                                    ("bf16", frames, 128, 8, 2, 31), ("fp16", frames, 128, 8, 3, 29),
                                    ("fp16", small, 64, 8, 2, 31)]:
        with dh.Plan(128, ny, LAM, Z, PITCH, T=32, precision=prec, max_frames=96, max_windows=4) as plan:
            plan.render_frames(fr)
            plan.profile(True)
            plan.pca_windows(0, s, 2, k0, k1)
            prof = plan.profile_read()
            plan.profile(False)
            assert prof["project_span"][0] == 0 and prof["project_tc"][0] == 1, (prec, s, k0, k1)


def test_grouped_in_graph_and_views(dh):
    """Views of one store (16/32/64 frames, stride 8) project grouped; graph replays are
    bitwise equal to the eager call."""
    F = 160
    frames = to_gpu(SpeckleStream(SpeckleParams(128, 128), seed=72).next(F).numpy())
    base = dh.Plan(128, 128, LAM, Z, PITCH, T=16, precision="fp16", max_frames=F, max_windows=19)
    base.render_frames(frames)
    plans = {16: base, 32: base.view(32, 17), 64: base.view(64, 13)}
    eager = {}
    for T, p in plans.items():
        n = (F - T) // 8 + 1
        img, _ = p.pca_windows(0, 8, n, 2, T - 1)
        eager[T] = img.clone()
    s = torch.cuda.Stream()
    outs = {T: torch.empty_like(eager[T]) for T in plans}
    torch.cuda.synchronize()
    with dh.capture(s) as g:
        for T, p in plans.items():
            n = (F - T) // 8 + 1
            p.pca_windows(0, 8, n, 2, T - 1, outs[T], None, want_eigvals=False, stream=s)
    for _ in range(2):
        g.launch(s)
        s.synchronize()
        for T in plans:
            assert torch.equal(outs[T], eager[T]), T
    g.close()
    for T in (32, 64):
        plans[T].close()
    base.close()
