"""The autotuner's candidates and its persistent cache, through the C ABI.

Every candidate must pass parity: the alternative FFT radix (a different rounding) against
the FP64 oracle at the render tolerance, schedules bitwise against each other, the covariance
split-K units (a different order of the FP64 partial sums) against the oracle at the stated
window tolerances. The cache: a tuned plan's picks are written as JSON and a second plan of
the same shape takes them from the file without measuring; unreadable files and rejected
values change nothing."""

import json
import os

import numpy as np
import pytest
import torch

import oracle
from dh_synth import SpeckleParams, SpeckleStream, speckle_window
from parity_helpers import LAM, PITCH, Z, check_window, rel, to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


ALT = [(512, 16), (1024, 16), (2048, 16), (4096, 32)]


@pytest.mark.parametrize("n,radix", ALT)
def test_alternative_radix_matches_oracle(dh, n, radix):
    frames = SpeckleStream(SpeckleParams(n, n), seed=n + radix).next(2).numpy()
    H = oracle.render(frames, LAM, Z, PITCH)
    with dh.Plan(n, n, LAM, Z, PITCH, T=16, precision="fp32", max_frames=16) as plan:
        plan.set_fft_radix(radix)
        assert plan.render_schedule()["radix"] == radix
        plan.render_frames(to_gpu(frames))
        for t in range(2):
            e = rel(plan.debug_hologram(t).cpu().numpy(), H[t])
            print(f"{n}^2 radix {radix} frame {t}: {e:.2e}")
            assert e <= 3e-6
        assert plan.status() == 0


@pytest.mark.parametrize("n,radix", ALT)
def test_alternative_radix_schedules_bitwise_equal(dh, n, radix):
    """Chunks and the persistent ring with the alternative radix: bitwise the same holograms."""
    F = 5 if n <= 1024 else 3
    frames = to_gpu(SpeckleStream(SpeckleParams(n, n), seed=3 * n).next(F).numpy())
    out = []
    for sched in ((False, 0, 0), (True, 3, 1)):
        with dh.Plan(n, n, LAM, Z, PITCH, T=16, precision="fp16", max_frames=16) as plan:
            plan.set_fft_radix(radix)
            plan.set_render_schedule(*sched)
            plan.render_frames(frames)
            out.append([plan.debug_hologram(t).cpu() for t in range(F)])
            assert plan.status() == 0
    for a, b in zip(*out):
        assert torch.equal(a, b)


def test_radix_option_rejects_what_is_not_instantiated(dh):
    with dh.Plan(256, 256, LAM, Z, PITCH, T=16) as plan:
        with pytest.raises(dh.DHError) as e:
            plan.set_fft_radix(32)  # 256: only its default radix 16
        assert e.value.code == 2
        with pytest.raises(dh.DHError) as e:
            plan.set_fft_radix(8)
        assert e.value.code == 1
        plan.set_fft_radix(16)  # its default: accepted
        assert plan.render_schedule()["radix"] == 16


@pytest.mark.parametrize("units", [0, 1, 2, 8])
def test_covariance_split_k_units_match_oracle(dh, units):
    """The default split-K units of a 256^2 frame (4) and a quarter, half and twice it: every window
    at the stated tolerances, and the covariance the same up to the order of its sums."""
    T, n = 32, 3
    frames = np.concatenate([speckle_window(256, 256, T, seed=50 + w).numpy() for w in range(n)])
    Cs = []
    for u in (0, units):
        with dh.Plan(256, 256, LAM, Z, PITCH, T=T, precision="fp16", max_frames=n * T,
                     max_windows=n) as plan:
            plan.set_gram_units(u)
            assert plan.render_schedule()["gram_units"] == u
            img, lam = plan.pca_batch(to_gpu(frames), n, T, 2, T - 1)
            img, lam = img.cpu(), lam.cpu()
            C = [plan.debug_covariance(w).cpu().numpy() for w in range(n)]
            assert plan.status() == 0
        Cs.append(C)
    for w in range(n):
        check_window(img[w].numpy().astype(np.float64), lam[w].numpy(), Cs[1][w],
                     frames[w * T:(w + 1) * T], 2, T - 1, "fp16", label=f"units {units}")
        assert rel(Cs[1][w], Cs[0][w]) <= 1e-6


def test_split_k_units_option_range(dh):
    with dh.Plan(256, 256, LAM, Z, PITCH, T=32, precision="fp16") as plan:
        for bad, code in ((3, 1), (-2, 1), (512, 2)):  # 512 does not divide 256^2 / 256
            with pytest.raises(dh.DHError) as e:
                plan.set_gram_units(bad)
            assert e.value.code == code
    with dh.Plan(256, 256, LAM, Z, PITCH, T=32, precision="fp32") as plan:
        with pytest.raises(dh.DHError) as e:
            plan.set_gram_units(8)  # the CUDA-core covariance has no split-K option
        assert e.value.code == 7


def test_autotune_cache_round_trip(dh, tmp_path):
    path = str(tmp_path / "tune.json")
    frames = to_gpu(SpeckleStream(SpeckleParams(512, 512), seed=11).next(32).numpy())
    with dh.Plan(512, 512, LAM, Z, PITCH, T=16, precision="fp16", max_frames=64, max_windows=4) as a:
        pick = a.autotune(32, cache=path)
        assert pick["from_cache"] is False
        a.render_frames(frames)
        holo_a = [a.debug_hologram(t).cpu() for t in (0, 31)]
    doc = json.load(open(path))
    assert doc["version"] == 1
    (key, entry), = doc["entries"].items()
    assert "nx=512,ny=512,T=16,prec=fp16" in key
    assert entry["render_fft"] in (1, 2) and entry["fft_radix"] in (0, 16, 32)
    with dh.Plan(512, 512, LAM, Z, PITCH, T=16, precision="fp16", max_frames=64, max_windows=4) as b:
        again = b.autotune(32, cache=path)
        assert again.pop("from_cache") is True
        assert again == {k: v for k, v in pick.items() if k != "from_cache"}
        b.render_frames(frames)
        holo_b = [b.debug_hologram(t).cpu() for t in (0, 31)]
    for x, y in zip(holo_a, holo_b):
        assert torch.equal(x, y)
    # another shape adds its own entry and keeps the first
    with dh.Plan(256, 256, LAM, Z, PITCH, T=16, precision="fp16", max_frames=32, max_windows=2) as c:
        assert c.autotune(16, cache=path)["from_cache"] is False
    assert len(json.load(open(path))["entries"]) == 2


def test_autotune_cache_refuses_bad_files(dh, tmp_path):
    bad = tmp_path / "bad.json"
    bad.write_text('{"version": 1, "entries": {')
    with dh.Plan(256, 256, LAM, Z, PITCH, T=16, precision="fp16") as plan:
        before = plan.render_schedule()
        with pytest.raises(dh.DHError) as e:
            plan.autotune(16, cache=str(bad))
        assert e.value.code == 1
        assert bad.read_text() == '{"version": 1, "entries": {'  # left as it was
        # an entry with a value the options reject: nothing is applied
        lib = plan._lib
        key = None
        good = tmp_path / "good.json"
        assert lib.dh_plan_tune_save(plan._h, os.fsencode(str(good))) == 0
        doc = json.load(open(good))
        key = next(iter(doc["entries"]))
        doc["entries"][key]["fft_radix"] = 7
        good.write_text(json.dumps(doc))
        with pytest.raises(dh.DHError) as e:
            plan.autotune(16, cache=str(good))
        assert e.value.code == 1
        assert plan.render_schedule() == before


def test_autotune_cache_keeps_other_entries_readable(dh, tmp_path):
    """Saving rewrites every other entry of the file: a key holding an escaped control
    character is escaped again, a huge number stays a number and a non-finite one (which JSON
    cannot hold) is dropped, so the file stays strict JSON and keeps the other entries."""
    path = tmp_path / "shared.json"
    path.write_text('{"version": 1, "entries": {"other\\nkey": {"render_ring": 8, '
                    '"big": 1e300, "bad": NaN}}}')
    with dh.Plan(256, 256, LAM, Z, PITCH, T=16, precision="fp16") as plan:
        assert plan._lib.dh_plan_tune_save(plan._h, os.fsencode(str(path))) == 0

    def no_constants(name):
        raise ValueError(f"non-JSON constant {name}")

    doc = json.loads(path.read_text(), parse_constant=no_constants)
    assert doc["entries"]["other\nkey"] == {"render_ring": 8, "big": 1e300}
    assert len(doc["entries"]) == 2
