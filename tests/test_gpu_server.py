"""The serving runtime (dh_server_*): camera streams admitted against an HBM budget, frames
pushed from host memory in chunks as they arrive, windows finished concurrently.

Each stream's windows, computed in the mix with the other streams' pushes interleaved, are
bitwise those of a single plan run alone over the same frames, and match the FP64 oracle;
admission, frame gaps and output backpressure behave as declared in the header.
"""

import numpy as np
import pytest
import torch

from dh_synth import SpeckleParams, SpeckleStream
from parity_helpers import LAM, PITCH, Z, check_window

pytestmark = pytest.mark.gpu

GiB = 1 << 30


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


# (nx, ny, T, precision, frames, seed)
STREAMS = [(128, 128, 32, "fp16", 96, 41), (256, 128, 16, "fp32", 64, 42),
           (64, 64, 64, "fp16", 128, 43)]


def alone(dh, nx, ny, T, prec, frames_np):
    nw = frames_np.shape[0] // T
    with dh.Plan(nx, ny, LAM, Z, PITCH, T=T, precision=prec, max_frames=frames_np.shape[0],
                 max_windows=nw) as plan:
        img, lam = plan.pca_batch(torch.from_numpy(frames_np).cuda(), nw, T, 2, T - 1)
        torch.cuda.synchronize()
        return img.cpu(), lam.cpu()


def test_server_mix_equals_alone(dh):
    srv = dh.Server(8 * GiB)
    frames, ids = [], []
    for nx, ny, T, prec, F, seed in STREAMS:
        f = SpeckleStream(SpeckleParams(nx, ny), seed=seed).next(F)
        frames.append(f.pin_memory())
        ids.append(srv.add_stream(nx, ny, LAM, Z, PITCH, T, prec, 2, T - 1, ring_windows=8))
    # interleave the streams' pushes, in chunks of 1..7 frames
    rng = np.random.default_rng(0)
    pos = [0] * len(STREAMS)
    got = {}
    while any(p < f.shape[0] for p, f in zip(pos, frames)):
        for i, f in enumerate(frames):
            if pos[i] < f.shape[0]:
                n = int(min(rng.integers(1, 8), f.shape[0] - pos[i]))
                srv.push(ids[i], f[pos[i]:pos[i] + n], pos[i])
                pos[i] += n
        for r in srv.poll():
            got[(r["stream"], r["window"])] = r
    srv.drain()
    for r in srv.poll(256):
        got[(r["stream"], r["window"])] = r
    for i, (nx, ny, T, prec, F, _) in enumerate(STREAMS):
        img, lam = alone(dh, nx, ny, T, prec, frames[i].numpy())
        for w in range(F // T):
            r = got[(ids[i], w)]
            assert torch.equal(r["image"], img[w]), (i, w)
            assert torch.equal(r["eigvals"], lam[w]), (i, w)
            assert r["t_done"] >= r["t_ready"]
        # and window 0 of each stream against the oracle
        w0 = got[(ids[i], 0)]
        C = None
        with dh.Plan(nx, ny, LAM, Z, PITCH, T=T, precision=prec) as plan:
            plan.render_stack(torch.from_numpy(frames[i][:T].numpy()).cuda())
            plan.pca_window(2, T - 1)
            C = plan.debug_covariance(0).cpu().numpy()
        check_window(w0["image"].numpy(), w0["eigvals"].numpy(), C, frames[i][:T].numpy(),
                     2, T - 1, prec)
    srv.close()


def test_admission_against_budget(dh):
    b = dh.Server.stream_bytes(256, 256, 32, "fp16", ring_windows=4)
    assert b > 0
    srv = dh.Server(int(2.5 * b))
    a = srv.add_stream(256, 256, LAM, Z, PITCH, 32, "fp16", ring_windows=4)
    srv.add_stream(256, 256, LAM, Z, PITCH, 32, "fp16", ring_windows=4)
    assert srv.used_bytes == 2 * b  # the charge is what the estimate said
    with pytest.raises(dh.DHError) as e:
        srv.add_stream(256, 256, LAM, Z, PITCH, 32, "fp16", ring_windows=4)
    assert e.value.code == 3  # denied, nothing allocated
    assert srv.used_bytes == 2 * b
    srv.remove_stream(a)
    assert srv.used_bytes == b
    srv.add_stream(256, 256, LAM, Z, PITCH, 32, "fp16", ring_windows=4)  # room again
    srv.close()


def test_plan_footprint_is_what_a_plan_allocates(dh):
    from paper_2004_00923_b300 import _lib
    lib = _lib.load()
    for nx, ny, T, prec, F, W in [(1024, 1024, 32, "fp16", 64, 1), (256, 128, 16, "fp32", 96, 5),
                                  (2048, 2048, 64, "bf16", 128, 2), (64, 64, 64, "fp16", 64, 1)]:
        with dh.Plan(nx, ny, LAM, Z, PITCH, T=T, precision=prec, max_frames=F,
                     max_windows=W) as plan:
            assert lib.dh_plan_footprint(nx, ny, T, dh.PREC[prec], F, W) == plan.device_bytes


def test_frame_gap_and_backpressure(dh):
    srv = dh.Server(4 * GiB)
    T = 16
    sid = srv.add_stream(64, 64, LAM, Z, PITCH, T, "fp16", ring_windows=2)
    f = SpeckleStream(SpeckleParams(64, 64), seed=44).next(4 * T).pin_memory()
    with pytest.raises(dh.DHError) as e:
        srv.push(sid, f[:4], 3)  # the stream expects frame 0
    assert e.value.code == 6
    srv.push(sid, f[:T], 0)        # window 0
    srv.push(sid, f[T:2 * T], T)   # window 1: both output slots now taken
    srv.drain()
    with pytest.raises(dh.DHError) as e:
        srv.push(sid, f[2 * T:3 * T], 2 * T)  # window 2 needs slot 0, not yet released
    assert e.value.code == 7
    res = srv.poll(copy=False)
    assert sorted(r["window"] for r in res) == [0, 1]
    srv.release(sid, 0)
    srv.push(sid, f[2 * T:3 * T], 2 * T)  # the refused frames again, now accepted
    srv.drain()
    assert [r["window"] for r in srv.poll()] == [2]
    srv.close()


OPTS = {"schedule": 0, "ring": 1, "lag": 2, "fft": 7, "radix": 8, "gram_units": 9}


def test_restart_from_tune_cache(dh, tmp_path):
    """A server autotunes a stream once and saves the picks; a restarted server (a new one
    on the same cache file) admits the same stream with the same plan options without
    measuring, and its windows equal a stand-alone plan given those options, bitwise."""
    cache = str(tmp_path / "tune.json")
    nx, ny, T = 256, 256, 32
    srv = dh.Server(4 * GiB)
    srv.set_tune_cache(cache, autotune=True)
    sid = srv.add_stream(nx, ny, LAM, Z, PITCH, T, "fp16", 2, T - 1, ring_windows=2)
    first = {k: srv.stream_option(sid, o) for k, o in OPTS.items()}
    srv.close()
    with open(cache) as fh:
        text = fh.read()
    assert '"entries"' in text and str(nx) in text
    # restart: load only, never measure (the file is left as it is)
    srv = dh.Server(4 * GiB)
    srv.set_tune_cache(cache, autotune=False)
    sid = srv.add_stream(nx, ny, LAM, Z, PITCH, T, "fp16", 2, T - 1, ring_windows=2)
    assert {k: srv.stream_option(sid, o) for k, o in OPTS.items()} == first
    with open(cache) as fh:
        assert fh.read() == text
    f = SpeckleStream(SpeckleParams(nx, ny), seed=77).next(T).pin_memory()
    srv.push(sid, f, 0)
    srv.drain()
    res = srv.poll(4)
    assert len(res) == 1
    with dh.Plan(nx, ny, LAM, Z, PITCH, T=T, precision="fp16", max_frames=2 * T) as plan:
        for k, o in OPTS.items():
            assert plan._lib.dh_plan_set_option(plan._h, o, first[k]) == 0, k
        img, lam = plan.pca_batch(f.cuda(), 1, T, 2, T - 1)
        torch.cuda.synchronize()
    assert torch.equal(res[0]["image"], img[0].cpu())
    assert torch.equal(res[0]["eigvals"], lam[0].cpu())
    srv.close()


def test_tune_cache_unreadable_file_refuses_admission(dh, tmp_path):
    bad = tmp_path / "bad.json"
    bad.write_text("not json")
    srv = dh.Server(4 * GiB)
    srv.set_tune_cache(str(bad))
    with pytest.raises(dh.DHError) as e:
        srv.add_stream(128, 128, LAM, Z, PITCH, 16, "fp16", 2, 15, ring_windows=1)
    assert e.value.code == 1
    assert srv.used_bytes == 0
    assert bad.read_text() == "not json"
    srv.close()
