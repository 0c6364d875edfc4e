"""The library's rate measurements (dh_measure_fma_rate, dh_measure_mma_issue): they run,
give finite positive rates below the hardware's nominal ones, and the tensor-core issue forms
order as the covariance and projection kernels' design assumes (a wait in the issuing warp
costs issue rate; a waiter warp recovers most of it)."""
import ctypes
import math

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dh():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2004_00923_b300 as m
    return m


def test_fma_rates_are_finite_and_below_nominal(dh):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 128 * 2 * 2.1e9 / 1e12  # FP32 lanes x 2 flops x a clock above the maximum
    for kind, iters in (("fp32", 2048), ("fp32x2", 1024), ("fp64", 64)):
        r = dh.measure_fma_rate(kind, iters=iters, blocks_per_sm=4)
        assert math.isfinite(r["tflops"]) and r["tflops"] > 0
        assert r["tflops"] < nominal


def test_mma_issue_forms(dh):
    rates = {f: dh.measure_mma_issue(f, stages=1024)
             for f in ("back-to-back", "mbarrier-wait", "waiter-warp")}
    print({f: round(r["cycles_per_mma"], 1) for f, r in rates.items()})
    for r in rates.values():
        assert math.isfinite(r["cycles_per_mma"]) and r["cycles_per_mma"] > 0
        assert 0 < r["tflops"] < 2500  # below the dense FP16 peak of the part
    # an M = N = 128, K = 16 MMA is 2^18 multiply-adds: at least ~32 cycles on one SM
    assert rates["back-to-back"]["cycles_per_mma"] > 30
    # the waiter warp keeps the issue rate closer to back-to-back than the in-warp wait
    assert rates["waiter-warp"]["cycles_per_mma"] < rates["mbarrier-wait"]["cycles_per_mma"]


def test_mma_issue_rejects_bad_arguments(dh):
    lib = dh._lib.load()
    ms, c, f = ctypes.c_float(0), ctypes.c_double(0), ctypes.c_double(0)
    assert lib.dh_measure_mma_issue(3, 16, ctypes.byref(ms), ctypes.byref(c), ctypes.byref(f), None) == 1
    assert lib.dh_measure_mma_issue(0, 0, ctypes.byref(ms), ctypes.byref(c), ctypes.byref(f), None) == 1
    assert lib.dh_measure_mma_issue(0, 16, None, ctypes.byref(c), ctypes.byref(f), None) == 1
