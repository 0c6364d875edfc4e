"""Failure detection on the GPU without a fault: a bounded device-side wait that runs out.

DH_OPT_TEST_STALL makes every CTA of the persistent render wait a few microseconds on a
device word that nothing sets. The wait gives up, the CTA raises DH_FLAG_WAIT_TIMEOUT and
skips its work, the kernel ends on its own, and the next dh_plan_status returns
DH_ERR_TIMEOUT through the C ABI. The same plan then renders correctly (the context stays
usable). A status read waits only for the plan's own streams: it returns while a long
kernel is still running on another stream.
"""

import ctypes
import time

import numpy as np
import pytest
import torch

import oracle
from dh_synth import SpeckleParams, SpeckleStream
from parity_helpers import LAM, PITCH, Z, rel, to_gpu

pytestmark = pytest.mark.gpu

DH_OK, DH_ERR_TIMEOUT, FLAG_WAIT_TIMEOUT = 0, 5, 0x8


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


def _status(plan):
    flags = ctypes.c_uint32(0)
    rc = plan._lib.dh_plan_status(plan._h, ctypes.byref(flags))
    return rc, int(flags.value)


def test_bounded_wait_runs_out_and_reports_timeout(dh):
    n, F = 256, 8
    frames = SpeckleStream(SpeckleParams(n, n), seed=31).next(F).numpy()
    with dh.Plan(n, n, LAM, Z, PITCH, T=16, precision="fp16", max_frames=16) as plan:
        plan.set_render_schedule(True, ring=4, lag=2)  # the persistent render at 256^2
        assert plan.status() == 0
        plan.set_test_stall(20000)  # ~10 us at 2 GHz, on a word nothing sets
        t0 = time.perf_counter()
        plan.render_frames(to_gpu(frames))
        rc, flags = _status(plan)
        dt = time.perf_counter() - t0
        assert rc == DH_ERR_TIMEOUT, rc
        assert flags & FLAG_WAIT_TIMEOUT
        assert dt < 5.0, dt  # the kernel ended by itself, long before any full wait budget
        # the flag was cleared by the read, and the context is still usable
        plan.set_test_stall(0)
        plan.render_frames(to_gpu(frames))
        rc, flags = _status(plan)
        assert (rc, flags) == (DH_OK, 0)
        H = oracle.render(frames, LAM, Z, PITCH)
        for t in (0, F - 1):
            h = plan.debug_hologram(t).cpu().numpy()
            assert rel(h, H[t]) < 1e-3, t


def test_stall_option_range(dh):
    with dh.Plan(64, 64, LAM, Z, PITCH, T=16) as plan:
        for bad in (-1, 100000001):
            with pytest.raises(RuntimeError):
                plan.set_test_stall(bad)
        v = ctypes.c_int(-1)
        plan.set_test_stall(123)
        assert plan._lib.dh_plan_get_option(plan._h, 6, ctypes.byref(v)) == 0 and v.value == 123


def test_status_read_does_not_wait_for_other_streams(dh):
    """A long kernel (~0.5 s of clock cycles) on an unrelated stream: the plan's status read
    returns well before it ends."""
    n = 128
    frames = SpeckleStream(SpeckleParams(n, n), seed=32).next(16).numpy()
    with dh.Plan(n, n, LAM, Z, PITCH, T=16, precision="fp16") as plan:
        plan.render_frames(to_gpu(frames))
        plan.pca_windows(0, 16, 1, 2, 15)
        assert plan.status() == 0
        plan.render_frames(to_gpu(frames))
        other = torch.cuda.Stream()
        with torch.cuda.stream(other):
            torch.cuda._sleep(1_000_000_000)  # >= 0.49 s at the 2032 MHz maximum SM clock
        t0 = time.perf_counter()
        assert plan.status() == 0
        dt = time.perf_counter() - t0
        long_done = other.query()
        other.synchronize()
        assert not long_done, "the unrelated kernel ended before the status read returned"
        assert dt < 0.25, dt


def test_covariance_abort_path_ends_and_reports_timeout(dh):
    """The 16-bit tensor-core covariance with its waiter warp timed out from the first stage:
    the MMA warp still completes its loop (the waiter releases each stage once the MMAs of the
    stage a ring before have completed), the launch ends by itself, the call reports
    DH_ERR_TIMEOUT, and the next call on the same plan is correct."""
    n, T, nw = 256, 32, 4
    frames = SpeckleStream(SpeckleParams(n, n), seed=33).next(nw * T).numpy()
    with dh.Plan(n, n, LAM, Z, PITCH, T=T, precision="fp16", max_frames=nw * T, max_windows=nw) as plan:
        plan.set_render_schedule(False)  # the chunked render: the stall reaches only the covariance
        assert plan.status() == 0
        plan.set_test_stall(20000)
        t0 = time.perf_counter()
        plan.pca_batch(to_gpu(frames), nw, T, 2, T - 1)
        rc, flags = _status(plan)
        dt = time.perf_counter() - t0
        assert rc == DH_ERR_TIMEOUT, rc
        assert flags & FLAG_WAIT_TIMEOUT
        assert dt < 5.0, dt
        plan.set_test_stall(0)
        images, _ = plan.pca_batch(to_gpu(frames), nw, T, 2, T - 1)
        rc, flags = _status(plan)
        assert (rc, flags) == (DH_OK, 0)
        M, _, _, _ = oracle.pca_window(frames[:T], LAM, Z, PITCH, 2, T - 1)
        assert rel(images[0].double().cpu().numpy(), M) < 1e-3
