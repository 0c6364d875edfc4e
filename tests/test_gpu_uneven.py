"""A batch of several frame sizes and window lengths in one call (dh_batch_run).

Three frame sizes, each with its own reconstruction distance; windows alternate between 32
and 64 frames and carry their own Doppler spread. Every window is checked against the FP64
oracle run with its size's distance, the batch is bitwise the same as the sizes run one
after the other through the single-plan calls, and a captured graph of the batch replays it
bitwise.
"""

import numpy as np
import pytest
import torch

from dh_synth import uneven_batch
from parity_helpers import LAM, PITCH, check_window

pytestmark = pytest.mark.gpu

SIZES = ((64, 4), (128, 3), (256, 2))
STRIDE = 96  # a 32-frame window and a 64-frame window end to end


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


class Uneven:
    """Per size: a 32-frame base plan (rendering) and a 64-frame view, with outputs."""

    def __init__(self, dh, groups, prec):
        self.groups = groups
        self.frames = [g.frames.cuda() for g in groups]
        self.sizes = []
        for g in groups:
            n = {T: len(g.starts(T)) for T in (32, 64)}
            base = dh.Plan(g.n, g.n, LAM, g.z, PITCH, T=32, precision=prec,
                           max_frames=g.frames.shape[0], max_windows=max(n[32], 1))
            plans = {32: base}
            if n[64]:
                plans[64] = base.view(64, n[64])
            out = {T: (torch.empty((n[T], g.n, g.n), dtype=torch.float32, device="cuda"),
                       torch.empty((n[T], T), dtype=torch.float64, device="cuda"))
                   for T in plans}
            self.sizes.append((g, n, plans, out))

    def items(self):
        items = []
        for (g, n, plans, out), f in zip(self.sizes, self.frames):
            for i, T in enumerate(sorted(plans)):
                it = {"plan": plans[T], "n_windows": n[T], "first_slot": g.starts(T)[0],
                      "slot_stride": STRIDE, "k0": 2, "k1": T - 1,
                      "images": out[T][0], "eigvals": out[T][1]}
                if i == 0:
                    it["frames"] = f
                items.append(it)
        return items

    def one_by_one(self):
        for (g, n, plans, out), f in zip(self.sizes, self.frames):
            plans[32].render_frames(f)
            for T in sorted(plans):
                plans[T].pca_windows(g.starts(T)[0], STRIDE, n[T], 2, T - 1, out[T][0], out[T][1])

    def results(self):
        torch.cuda.synchronize()
        return [{T: (o[0].cpu().numpy(), o[1].cpu().numpy()) for T, o in out.items()}
                for (_, _, _, out) in self.sizes]

    def close(self):
        for (_, _, plans, _) in self.sizes:
            for p in plans.values():
                p.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_uneven_batch_matches_oracle(dh, prec):
    groups = uneven_batch(SIZES, seed=31)
    u = Uneven(dh, groups, prec)
    dh.run_batch(u.items())
    res = u.results()
    for (g, n, plans, _), r in zip(u.sizes, res):
        fr = g.frames.numpy()
        for T in plans:
            C = [plans[T].debug_covariance(w).cpu().numpy() for w in range(n[T])]
            img, lam = r[T]
            for w, s in enumerate(g.starts(T)):
                check_window(img[w], lam[w], C[w], fr[s:s + T], 2, T - 1, prec, z=g.z)
        assert plans[32].status() == 0
    u.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_batch_equals_one_by_one_and_graph(dh, prec):
    """Alone (each size through the single-plan calls, one after the other) and in the mix
    (one batch, sizes on concurrent branches; also as a replayed graph): bitwise equal."""
    groups = uneven_batch(SIZES, seed=32)
    u = Uneven(dh, groups, prec)
    u.one_by_one()
    alone = u.results()
    for (_, _, _, out) in u.sizes:
        for o in out.values():
            o[0].fill_(float("nan"))
            o[1].fill_(float("nan"))
    dh.run_batch(u.items())
    mixed = u.results()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with dh.capture(s) as g:
        dh.run_batch(u.items())
    for (_, _, _, out) in u.sizes:
        for o in out.values():
            o[0].zero_()
    torch.cuda.synchronize()
    g.launch(s)
    s.synchronize()
    graphed = u.results()
    for a, b, c in zip(alone, mixed, graphed):
        for T in a:
            for k in (0, 1):
                assert np.array_equal(a[T][k], b[T][k]), T
                assert np.array_equal(a[T][k], c[T][k]), T
    g.close()
    u.close()


def test_batch_rejects_bad_items_before_launching(dh):
    groups = uneven_batch(((64, 2),), seed=33)
    u = Uneven(dh, groups, "fp16")
    items = u.items()
    bad = dict(items[1], k1=64)  # k1 >= T of the 64-frame view
    with pytest.raises(dh.DHError) as e:
        dh.run_batch([items[0], bad])
    assert e.value.code == 1
    with pytest.raises(dh.DHError) as e:
        dh.run_batch([dict(items[0], n_windows=5)])  # more windows than reserved
    assert e.value.code == 1
    u.close()
