"""Sliding windows of several lengths over one rendering, and CUDA graphs of library calls.

Each frame is rendered once (Eq. 1 is per frame) into a base plan's hologram store; views of
that store run Eqs. 4-7 for 16-, 32- and 64-frame windows at stride 8. Every window is
checked against the FP64 oracle run on that window's own frames, a view's windows are
bitwise those of a stand-alone plan of the same length, and a captured graph replays the
whole step bitwise.
"""

import numpy as np
import pytest
import torch

from dh_synth import SpeckleParams, SpeckleStream
from parity_helpers import LAM, PITCH, Z, check_window, to_gpu

pytestmark = pytest.mark.gpu

LENGTHS = (16, 32, 64)
STRIDE = 8


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


def counts(n_frames):
    return {T: (n_frames - T) // STRIDE + 1 for T in LENGTHS}


class Sliding:
    """A base plan (T = 16) plus views for 32 and 64 over one store, with output buffers."""

    def __init__(self, dh, nx, ny, n_frames, prec):
        self.n = counts(n_frames)
        self.base = dh.Plan(nx, ny, LAM, Z, PITCH, T=16, precision=prec, max_frames=n_frames,
                            max_windows=self.n[16])
        self.plans = {16: self.base, 32: self.base.view(32, self.n[32]),
                      64: self.base.view(64, self.n[64])}
        self.images = {T: torch.empty((self.n[T], ny, nx), dtype=torch.float32, device="cuda")
                       for T in LENGTHS}
        self.lam = {T: torch.empty((self.n[T], T), dtype=torch.float64, device="cuda")
                    for T in LENGTHS}

    def step(self, frames_dev):
        self.base.render_frames(frames_dev)
        for T in LENGTHS:
            self.plans[T].pca_windows(0, STRIDE, self.n[T], 2, T - 1, self.images[T], self.lam[T])

    def results(self):
        torch.cuda.synchronize()
        return {T: (self.images[T].cpu().numpy(), self.lam[T].cpu().numpy()) for T in LENGTHS}

    def close(self):
        for p in self.plans.values():
            p.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_sliding_lengths_share_one_rendering(dh, prec):
    """96 frames of 128x128: 11 + 9 + 5 windows, every one against the oracle."""
    frames = SpeckleStream(SpeckleParams(128, 128), seed=21).next(96).numpy()
    sl = Sliding(dh, 128, 128, 96, prec)
    sl.step(to_gpu(frames))
    res = sl.results()
    for T in LENGTHS:
        C = [sl.plans[T].debug_covariance(w).cpu().numpy() for w in range(sl.n[T])]
        img, lam = res[T]
        for w in range(sl.n[T]):
            check_window(img[w], lam[w], C[w], frames[w * STRIDE:w * STRIDE + T], 2, T - 1, prec)
    assert sl.base.status() == 0
    sl.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_view_equals_own_plan_bitwise(dh, prec):
    """A view's windows are computed exactly as by a plan of that length that renders the
    same frames itself."""
    frames = SpeckleStream(SpeckleParams(256, 128), seed=22).next(80).numpy()
    sl = Sliding(dh, 256, 128, 80, prec)
    f = to_gpu(frames)
    sl.step(f)
    res = sl.results()
    for T in (32, 64):
        with dh.Plan(256, 128, LAM, Z, PITCH, T=T, precision=prec, max_frames=80,
                     max_windows=sl.n[T]) as own:
            img, lam = own.pca_batch(f, sl.n[T], STRIDE, 2, T - 1)
            torch.cuda.synchronize()
            assert np.array_equal(img.cpu().numpy(), res[T][0])
            assert np.array_equal(lam.cpu().numpy(), res[T][1])
    sl.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_graph_replay_matches_eager(dh, prec):
    """The whole step (render + three window lengths, with the eigensolver forked onto each
    plan's own stream) captured once and replayed: bitwise the eager results, and replays
    read the frame buffer as it is at launch time."""
    gen = SpeckleStream(SpeckleParams(128, 128), seed=23)
    fa, fb = gen.next(72).numpy(), gen.next(72).numpy()
    eager = {}
    for key, fr in (("a", fa), ("b", fb)):
        sl = Sliding(dh, 128, 128, 72, prec)
        sl.step(to_gpu(fr))
        eager[key] = sl.results()
        sl.close()

    sl = Sliding(dh, 128, 128, 72, prec)
    buf = to_gpu(fa)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with dh.capture(s) as g:
        sl.step(buf)
    for key, fr in (("a", fa), ("b", fb), ("a", fa)):
        buf.copy_(torch.from_numpy(fr))
        torch.cuda.synchronize()
        g.launch(s)
        s.synchronize()
        got = sl.results()
        for T in LENGTHS:
            assert np.array_equal(got[T][0], eager[key][T][0]), (key, T)
            assert np.array_equal(got[T][1], eager[key][T][1]), (key, T)
    g.close()
    sl.close()


def test_view_rules(dh):
    """Views render nothing, pin their base's storage and slot count, and keep the store
    alive after the base's handle is closed."""
    from paper_2004_00923_b300 import _lib
    lib = _lib.load()
    frames = to_gpu(SpeckleStream(SpeckleParams(64, 64), seed=24).next(48).numpy())
    base = dh.Plan(64, 64, LAM, Z, PITCH, T=16, precision="fp16", max_frames=48, max_windows=2)
    v = base.view(32, max_windows=2)
    with pytest.raises(dh.DHError) as e:
        v.render_frames(frames)
    assert e.value.code == 7
    with pytest.raises(dh.DHError) as e:
        v.pca_batch(frames, 1, 8, 2, 31)
    assert e.value.code == 7
    assert lib.dh_plan_set_precision(base._h, 0) == 7       # storage pinned by the view
    assert lib.dh_plan_reserve(base._h, 64, 2) == 7         # slot count pinned by the view
    assert lib.dh_plan_reserve(base._h, 48, 3) == 0         # windows of the base may change
    assert lib.dh_plan_reserve(v._h, 48, 3) == 0            # and of the view
    with pytest.raises(dh.DHError) as e:
        base.view(128)                                     # unsupported window length
    assert e.value.code == 2
    base.render_frames(frames)
    img_before, lam_before = v.pca_windows(0, 16, 2, 2, 31)
    torch.cuda.synchronize()
    base.close()                                           # the view still holds the store
    img_after, lam_after = v.pca_windows(0, 16, 2, 2, 31)
    torch.cuda.synchronize()
    assert torch.equal(img_before, img_after) and torch.equal(lam_before, lam_after)
    v.close()


@pytest.mark.parametrize("prec", ["fp16"])
def test_views_run_concurrently_in_a_batch(dh, prec):
    """One batch: render, then the three lengths' windows on concurrent branches (views of one
    store); bitwise the sequential calls' results."""
    frames = SpeckleStream(SpeckleParams(128, 128), seed=25).next(96).numpy()
    f = to_gpu(frames)
    sl = Sliding(dh, 128, 128, 96, prec)
    sl.step(f)
    ref = sl.results()
    items = [{"plan": sl.base, "frames": f}] + [
        {"plan": sl.plans[T], "n_windows": sl.n[T], "first_slot": 0, "slot_stride": STRIDE,
         "k0": 2, "k1": T - 1, "images": sl.images[T], "eigvals": sl.lam[T]} for T in (64, 32, 16)]
    for T in LENGTHS:
        sl.images[T].zero_()
    dh.run_batch(items)
    got = sl.results()
    for T in LENGTHS:
        assert np.array_equal(got[T][0], ref[T][0]) and np.array_equal(got[T][1], ref[T][1])
    sl.close()


def test_batch_orders_a_rerender_after_its_readers(dh):
    """render A; windows (views); render B into the same slots; windows again: the first
    windows see A and the second see B (the second render waits for the first readers)."""
    gen = SpeckleStream(SpeckleParams(64, 64), seed=26)
    fa, fb = to_gpu(gen.next(48).numpy()), to_gpu(gen.next(48).numpy())
    base = dh.Plan(64, 64, LAM, Z, PITCH, T=16, precision="fp16", max_frames=48, max_windows=5)
    v32 = base.view(32, 3)
    out = {k: torch.empty((3, 64, 64), dtype=torch.float32, device="cuda") for k in ("a", "b")}
    items = [{"plan": base, "frames": fa},
             {"plan": v32, "n_windows": 3, "first_slot": 0, "slot_stride": 8, "k0": 2, "k1": 31,
              "images": out["a"]},
             {"plan": base, "frames": fb},
             {"plan": v32, "n_windows": 3, "first_slot": 0, "slot_stride": 8, "k0": 2, "k1": 31,
              "images": out["b"]}]
    dh.run_batch(items)
    torch.cuda.synchronize()
    for key, fr in (("a", fa), ("b", fb)):
        with dh.Plan(64, 64, LAM, Z, PITCH, T=32, precision="fp16", max_frames=48, max_windows=3) as own:
            img, _ = own.pca_batch(fr, 3, 8, 2, 31)
            torch.cuda.synchronize()
            assert torch.equal(img, out[key]), key
    v32.close()
    base.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_band_covariance_serves_every_length(dh, prec):
    """dh_band_gram once over the store, then 16/32/64-frame windows at stride 8 (and one
    window at an odd offset) take C from it: equal to the per-window Gram within FP32
    accumulation (3e-6), and the windows' images and eigenvalues match the oracle."""
    F = 200
    frames = SpeckleStream(SpeckleParams(128, 128), seed=27).next(F).numpy()
    base = dh.Plan(128, 128, LAM, Z, PITCH, T=16, precision=prec, max_frames=F, max_windows=24)
    base.render_frames(to_gpu(frames))
    base.band_gram(0, F)
    for T in LENGTHS:
        n = (F - T) // STRIDE + 1
        band_plan = base if T == 16 else base.view(T, n)
        ref_plan = base.view(T, n)
        band_plan.set_covariance_source("band")
        img_b, lam_b = band_plan.pca_windows(0, STRIDE, n, 2, T - 1)
        Cb = [band_plan.debug_covariance(w).cpu().numpy() for w in range(n)]
        img_r, lam_r = ref_plan.pca_windows(0, STRIDE, n, 2, T - 1)
        Cr = [ref_plan.debug_covariance(w).cpu().numpy() for w in range(n)]
        for w in range(n):
            assert np.linalg.norm(Cb[w] - Cr[w]) <= 3e-6 * np.linalg.norm(Cr[w]), (T, w)
        if prec == "fp16":
            img_b, lam_b = img_b.cpu().numpy(), lam_b.cpu().numpy()
            for w in (0, n // 2, n - 1):
                check_window(img_b[w], lam_b[w], Cb[w], frames[w * STRIDE:w * STRIDE + T], 2, T - 1,
                             prec)
        # a window at an offset that is not a multiple of 8, inside the band
        img1, _ = band_plan.pca_windows(37, 1, 1, 2, T - 1)
        C1 = band_plan.debug_covariance(0).cpu().numpy()
        ref1, _ = ref_plan.pca_windows(37, 1, 1, 2, T - 1)
        C1r = ref_plan.debug_covariance(0).cpu().numpy()
        assert np.linalg.norm(C1 - C1r) <= 3e-6 * np.linalg.norm(C1r)
        if band_plan is not base:
            band_plan.close()
        ref_plan.close()
    assert base.status() == 0
    base.close()


def test_band_rules(dh):
    frames = to_gpu(SpeckleStream(SpeckleParams(64, 64), seed=28).next(96).numpy())
    base = dh.Plan(64, 64, LAM, Z, PITCH, T=32, precision="fp16", max_frames=96, max_windows=4)
    base.render_frames(frames)
    base.set_covariance_source("band")
    with pytest.raises(dh.DHError) as e:      # no band yet
        base.pca_windows(0, 8, 2, 2, 31)
    assert e.value.code == 7
    base.band_gram(0, 64)
    base.pca_windows(0, 8, 2, 2, 31)          # frames 0..39: inside
    with pytest.raises(dh.DHError) as e:      # frames 40..71 reach past the band
        base.pca_windows(40, 8, 1, 2, 31)
    assert e.value.code == 7
    base.close()
    with dh.Plan(64, 64, LAM, Z, PITCH, T=16) as p32:
        with pytest.raises(dh.DHError) as e:
            p32.band_gram(0, 16)
        assert e.value.code == 7
