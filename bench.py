#!/usr/bin/env python
"""Benchmark of the retinal-holography PCA path (Puyo et al., arXiv 2004.00923).

One step = the whole hot path (Fresnel rendering, covariance, eigendecomposition,
projection + power image) over one batch: 2048 synthetic 1024x1024 uint16 frames cut into
64 non-overlapping 32-frame windows, holograms stored FP16, k0..k1 = 2..31.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0. Under torchrun each rank processes its own 64 windows
(weak scaling, no collective on the data path); the step time is the max over ranks.
`--impl reference` times the FP64 CPU oracle (the reference arm of this workload) on the
host cores, one window per step.
"""

from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCA windows/s @1024²×32 vs plain FP32, ≤1e-3 rel err; %HBM roofline; p99 ms"
UNIT = "windows/s"
NX = NY = 1024
T = 32
NWIN = 64
K0, K1 = 2, 31
LAM, Z, PITCH = 785e-9, 0.35, 20e-6
PAPER_WINDOWS_PER_S = 20.0  # the paper's PCA rate at 1024^2 x 32 (Titan RTX)
WORKLOAD = "1024x1024 uint16 frames, 64 non-overlapping 32-frame windows per step, FP16 holograms"


# --------------------------------------------------------------------------- helpers
def print_line(line: dict) -> None:
    print(json.dumps(line), flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(ws):
    if ws > 1 and not torch.distributed.is_initialized():
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        torch.distributed.init_process_group(backend=backend)


def barrier(ws):
    if ws > 1:
        torch.distributed.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    """Largest value of x over all ranks (the slowest rank sets the step time)."""
    if ws == 1:
        return x
    dev = "cuda" if torch.cuda.is_available() and torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, ws: int, ms_per_step_max: float) -> float:
    """Units all ranks processed per second, over the slowest rank's step time."""
    return units_per_rank * ws / (ms_per_step_max / 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms from before the timed region
    to after it; the samples stamped between begin() and end() (the timed region, host clock)
    are the ones reported, all of them if none falls inside."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.t_begin = self.t_end = None

    def begin(self):
        self.t_begin = datetime.datetime.now()

    def end(self):
        self.t_end = datetime.datetime.now()

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="dh_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def stamp(r):
            try:
                return datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                return None
        inside = rows
        if self.t_begin is not None and self.t_end is not None:
            kept = [r for r in rows if stamp(r) is not None and self.t_begin <= stamp(r) <= self.t_end]
            if kept:
                inside = kept
        sm = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in inside if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(inside),
                "in_timed_region": inside is not rows}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    return 6400.0, 1800.0, "fallback"


def traffic_record(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when the
    summary is absent or the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["sha256"]:
        return None
    return float(rec["bytes_per_launch"])


# Algorithmic DRAM bytes of one step, per kernel (minimum traffic of the store-H schedule:
# the row-pass intermediate stays in L2 by construction and is not counted).
def algorithmic_bytes(npix, frames, windows, T, hbytes):
    return {
        "render_rows": frames * npix * 2,                    # uint16 frames in
        "render_cols": frames * npix * 2 * hbytes,           # Re/Im planes out
        "render_fused": frames * npix * (2 + 2 * hbytes),    # both, one persistent launch
        "gram_tc": windows * T * npix * 2 * hbytes,          # H read once per window
        "gram_raw": windows * T * npix * 2,                  # uint16 frames read once per window
        "gram_simt": windows * T * npix * 2 * hbytes,
        "project_tc": windows * (T * npix * 2 * hbytes + npix * 4),  # H read + image out
        "project_simt": windows * (T * npix * 2 * hbytes + npix * 4),
    }


# --------------------------------------------------------------------------- arms
def run_reference(args, ws, rank):
    """The FP64 CPU oracle, as it stands, on the host cores: one 1024^2 x 32 window/step."""
    if rank != 0:
        return 0
    import oracle
    from dh_synth import SpeckleParams, SpeckleStream
    frames = SpeckleStream(SpeckleParams(NX, NY), seed=1000, device="cpu").next(T).numpy()
    for _ in range(args.warmup):
        oracle.pca_window(frames, LAM, Z, PITCH, K0, K1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.pca_window(frames, LAM, Z, PITCH, K0, K1)
        times.append(time.perf_counter() - t0)
    sec = sum(times) / len(times)
    value = 1.0 / sec
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_WINDOWS_PER_S,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (one window of it per step)", "nx": NX, "ny": NY,
                   "T": T, "k0": K0, "k1": K1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "1 window of 1024x1024x32 per step (FP64 C oracle, OpenMP)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, ws, rank, local):
    import paper_2004_00923_b300 as dh
    from dh_synth import SpeckleParams, SpeckleStream

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    nwin = args.windows
    nframes = nwin * T
    # config-1 stream: seed 1000 * config + rank, 2048 frames resident in HBM (4 GiB > L2)
    frames = SpeckleStream(SpeckleParams(NX, NY), seed=1000 + rank, device=dev).next(nframes)
    npix = NX * NY

    # pipelined steps use two halves of hologram slots: batch k+1 renders into one half while
    # batch k's covariance, eigensolver and projection read the other
    pipeline = args.pipeline and args.covariance != "raw"
    plan = dh.Plan(NX, NY, LAM, Z, PITCH, T=T, precision=args.precision,
                   max_frames=nframes * (2 if pipeline else 1), max_windows=nwin)
    plan.set_covariance_source(args.covariance)
    if args.residual:
        plan.set_residual(True)
    if args.render_fft != "auto":
        plan.set_render_fft(args.render_fft)
    if args.render_schedule == "auto":
        tuned = plan.autotune(256)  # setup, outside the timed region
    else:
        plan.set_render_schedule(args.render_schedule == "persistent", args.render_ring, args.render_lag)
        tuned = plan.render_schedule()
    images = torch.empty((nwin, NY, NX), dtype=torch.float32, device=dev)
    eig = torch.empty((nwin, T), dtype=torch.float64, device=dev)

    def step(p):
        p.pca_batch(frames, nwin, T, K0, K1, images, eig)

    s_render, s_pca = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev_rendered = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    done_marks = []

    def pipelined(k_first, n):
        """Steps k_first .. k_first + n - 1: render of step k on one stream, Eqs. 4-7 of step k
        on another; half k % 2 is re-rendered only after its previous PCA (step k - 2)."""
        for k in range(k_first, k_first + n):
            h = k % 2
            s_render.wait_event(ev_done[h])
            plan.render_frames(frames, first_slot=h * nframes, stream=s_render)
            ev_rendered[h].record(s_render)
            s_pca.wait_event(ev_rendered[h])
            plan.pca_windows(h * nframes, T, nwin, K0, K1, images, eig, stream=s_pca)
            mark = torch.cuda.Event(enable_timing=True)
            mark.record(s_pca)
            done_marks.append(mark)
            ev_done[h].record(s_pca)

    if pipeline:
        pipelined(0, max(args.warmup, 0))
    else:
        for _ in range(max(args.warmup, 0)):
            step(plan)
    torch.cuda.synchronize()

    # ---------------------------------------------------------------- timed region
    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.begin()
    if pipeline:
        start.record(stream)
        s_render.wait_stream(stream)
        s_pca.wait_stream(stream)
        done_marks.clear()
        pipelined(args.warmup, args.steps)
        stream.wait_stream(s_render)
        stream.wait_stream(s_pca)
        end.record(stream)
        torch.cuda.synchronize()
        step_ms = [start.elapsed_time(done_marks[0])] + [
            done_marks[k - 1].elapsed_time(done_marks[k]) for k in range(1, len(done_marks))]
    else:
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        start.record(stream)
        for k in range(args.steps):
            step(plan)
            marks[k].record(stream)
        end.record(stream)
        torch.cuda.synchronize()
        step_ms = [start.elapsed_time(marks[0])] + [marks[k - 1].elapsed_time(marks[k])
                                                    for k in range(1, args.steps)]
    clocks.end()
    barrier(ws)
    clock_info = clocks.stop()
    ms = start.elapsed_time(end) / args.steps
    ms_max = max_over_ranks(ms, ws)
    value = whole_job_rate(nwin, ws, ms_max)
    flags = plan.status()
    # per-kernel breakdown: the same number of steps again, one after another with the
    # library's tracer on (overlapped steps would mix their event intervals); not timed
    plan.profile(True)
    for _ in range(args.steps):
        step(plan)
    prof = plan.profile_read()
    plan.profile(False)

    # ---------------------------------------------------------------- measured FMA rates
    rates = None if args.no_peaks else measure_rates(local)
    if rates is not None:
        rates["library_fft2"] = library_fft2(NX)

    # ---------------------------------------------------------------- roofline
    hbm, bf16_peak, peak_kind = measured_peaks()
    hbytes = 2 if args.precision in ("fp16", "bf16") else 4
    per_kernel, launches_total = kernel_table(prof)
    steps = args.steps
    alg = {k: v * steps for k, v in algorithmic_bytes(npix, nframes, nwin, T, hbytes).items()}
    fl = render_flops(npix, NX, NY, nframes) * steps
    roofline = roofline_of(per_kernel, alg, hbm, peak_kind, ms / 1e3,
                           {k: fl for k in RENDER_KERNELS}, alg_steps=steps,
                           fp32_peak=rates["fp32_peak_tflops"] if rates else None)
    if rates is not None:
        rk = per_kernel.get("render_fused")
        if rk and rk["launches"]:
            rates["library_fft2"]["render_us_per_frame"] = rk["ms_total"] * 1e3 / (rk["launches"] * nframes)

    # ---------------------------------------------------------------- end to end (host buffers)
    # dh_pca_batch_host: pinned host frames in, host images and eigenvalues out; the library
    # overlaps the frame copies with the computation of earlier groups of windows
    e2e, e2e_packed = None, None
    if not args.no_e2e and not args.residual:  # the host-buffer call has no residual mode
        host_frames = torch.empty(frames.shape, dtype=torch.uint16, pin_memory=True)
        host_frames.copy_(frames)
        host_images = torch.empty(images.shape, dtype=torch.float32, pin_memory=True)
        host_eig = torch.empty(eig.shape, dtype=torch.float64, pin_memory=True)

        def e2e_step():
            plan.pca_batch_host(host_frames, nwin, T, K0, K1, host_images, host_eig, sync=False)

        e2e_step()
        torch.cuda.synchronize()
        n_e2e = max(2, min(args.steps, 5))
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        torch.cuda.synchronize()
        e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / n_e2e, ws)
        e2e = {"value": whole_job_rate(nwin, ws, e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(host_frames.numel() * 2),
               "d2h_bytes_per_step": int(host_images.numel() * 4 + host_eig.numel() * 8),
               "ms_per_step": e_ms, "call": "dh_pca_batch_host (copies overlapped with compute)"}
        ref_images = host_images.clone()
        del host_frames

        # the same with the frames as a 12-bit camera delivers them packed (Mono12p: two
        # pixels in three bytes), expanded on the device: 3/4 of the bytes over the host link.
        # The packing is the synthetic camera's output format, made once before timing.
        v = (frames.view(torch.int16).to(torch.int32) & 0xFFFF).view(frames.shape[0], -1, 2)
        if int(v.max()) < 4096:
            lo, hi = v[..., 0], v[..., 1]
            packed = torch.stack((lo & 0xFF, (lo >> 8) | ((hi & 0xF) << 4), hi >> 4), dim=-1)
            host_packed = torch.empty((frames.shape[0], packed.shape[1] * 3), dtype=torch.uint8,
                                      pin_memory=True)
            host_packed.copy_(packed.to(torch.uint8).view(frames.shape[0], -1))
            del lo, hi, packed

            def e2e_packed_step():
                plan.pca_batch_host_packed12(host_packed, nwin, T, K0, K1, host_images, host_eig, sync=False)

            e2e_packed_step()
            torch.cuda.synchronize()
            same = bool(torch.equal(host_images, ref_images))
            barrier(ws)
            t0 = time.perf_counter()
            for _ in range(n_e2e):
                e2e_packed_step()
            torch.cuda.synchronize()
            p_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / n_e2e, ws)
            e2e_packed = {"value": whole_job_rate(nwin, ws, p_ms), "unit": UNIT,
                          "h2d_bytes_per_step": int(host_packed.numel()),
                          "d2h_bytes_per_step": int(host_images.numel() * 4 + host_eig.numel() * 8),
                          "ms_per_step": p_ms, "format": "Mono12p (12-bit packed, 2 pixels in 3 bytes)",
                          "call": "dh_pca_batch_host_packed12 (copies overlapped, expanded on the device)",
                          "images_bitwise_equal_to_uint16_call": same}
            del host_packed
        del ref_images, v

    # ---------------------------------------------------------------- plain FP32 GPU path
    plain = None
    if not args.no_plain and args.precision != "fp32":
        p32 = dh.Plan(NX, NY, LAM, Z, PITCH, T=T, precision="fp32", max_frames=nframes,
                      max_windows=nwin)
        step(p32)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n32 = max(2, min(args.steps, 5))
        a.record(stream)
        for _ in range(n32):
            step(p32)
        b.record(stream)
        torch.cuda.synchronize()
        ms32 = max_over_ranks(a.elapsed_time(b) / n32, ws)
        plain = {"value": whole_job_rate(nwin, ws, ms32), "unit": UNIT, "ms_per_step": ms32}
        p32.close()
        step(plan)  # the headline plan's images again for the parity sample below
        torch.cuda.synchronize()

    # ---------------------------------------------------------------- oracle sample (rank 0)
    cpu_baseline, parity = None, None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        f0 = frames[:T].cpu().numpy()
        t0 = time.perf_counter()
        M, lam_ref, C_ref, _ = oracle.pca_window(f0, LAM, Z, PITCH, K0, K1)
        sec = time.perf_counter() - t0
        cpu_baseline = {"value": 1.0 / sec, "unit": UNIT, "cores": oracle.num_threads(),
                        "kind": "oracle",
                        "sample": "window 0 of the step (1024x1024x32), FP64 C oracle, OpenMP"}
        img0 = images[0].double().cpu().numpy()
        lam0 = eig[0].cpu().numpy()
        C0 = plan.debug_covariance(0).cpu().numpy()  # the last step's window 0
        parity = {"window": 0,
                  "image_rel_l2": float(np.linalg.norm(img0 - M) / np.linalg.norm(M)),
                  "eig_normwise": float(np.max(np.abs(lam0 - lam_ref)) / lam_ref[0]),
                  "C_rel_fro": float(np.linalg.norm(C0 - C_ref) / np.linalg.norm(C_ref)),
                  "tolerance_image": 1e-3 if args.precision != "fp32" else 1e-4,
                  "tolerance_eig": 1e-5}

    # ---------------------------------------------------------------- p50 / p99 latency
    # the metric's third term: a short replay of the serving mix at the stream clock, after
    # the headline plan's memory is given back
    latency = None
    plan.close()
    torch.cuda.synchronize()
    if args.latency_seconds > 0:
        frames = None  # the step's 4 GiB of input frames
        torch.cuda.empty_cache()
        latency = serve_latency(args, ws, rank, local)

    # ---------------------------------------------------------------- the other workloads
    # short runs (3 timed steps each, their window-0 parity samples against the oracle), so
    # that the sliding, uneven and Fourier workloads are measured in the same line
    workloads = None
    if not args.no_workloads:
        workloads = {}
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup, sub.frames = 3, 1, 0
        for name, fn in (("sliding", run_sliding), ("uneven", run_uneven), ("fourier", run_fourier)):
            got = []
            fn(sub, ws, rank, local, emit=got.append)
            torch.cuda.empty_cache()
            if got:
                w = got[0]
                par = w.get("parity") or {}
                errs = [v.get("image_rel_l2") for v in par.values() if isinstance(v, dict)]
                workloads[name] = {
                    "metric": w["metric"], "value": w["value"], "unit": w["unit"],
                    "ms_per_step": w["ms_per_step"], "steps": w["steps"],
                    "parity_image_rel_l2_max": max(e for e in errs if e is not None) if errs else None,
                    "device_flags": w.get("device_flags"), "workload": w["config"].get("workload"),
                    "render_schedule": w["config"].get("render_schedule")}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": value / PAPER_WINDOWS_PER_S,
            "dtype": "mixed: f32 FFT, f16 tensor-core products (f32 accumulate), f64 eig",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "T": T,
                       "windows_per_step": nwin, "frames_per_step": nframes, "k0": K0, "k1": K1,
                       "precision": args.precision,
                       "l2": "no flush: 4 GiB of input frames per step exceed the 126 MB L2",
                       "render_schedule": tuned,
                       "covariance": "raw (C = I^T I)" if args.residual else args.covariance,
                       "storage": "mean-residual" if args.residual else "plain",
                       "pipelined_steps": pipeline,
                       "parallelism": f"replicas x{ws}"},
            "frames_per_s": value * T,
            "step_ms": {"p50": statistics.median(step_ms), "max": max(step_ms)},
            "roofline": roofline,
            "cpu_baseline": cpu_baseline,
            "e2e": e2e,
            "e2e_packed12": e2e_packed,
            "plain_fp32": plain,
            "speedup_vs_plain_fp32": (value / plain["value"]) if plain else None,
            "parity": parity,
            "latency_ms": latency,
            "workloads": workloads,
            "measured_rates": rates,
            "gpu_launches": launches_total,
            "device_flags": flags,
            "clocks": clock_info,
        }
        print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- shared pieces
def kernel_table(prof: dict) -> tuple[dict, int]:
    """{kernel: launches, ms_total, share} from a plan's tracer read, and total launches."""
    per_kernel, launches = {}, 0
    for name, (n, tot) in prof.items():
        if n:
            launches += n
            per_kernel[name] = {"launches": n, "ms_total": tot, "share": 0.0}
    tot_ms = sum(v["ms_total"] for v in per_kernel.values()) or 1.0
    for v in per_kernel.values():
        v["share"] = v["ms_total"] / tot_ms
    return per_kernel, launches


def merge_tables(tables: list[dict]) -> dict:
    out = {}
    for t in tables:
        for k, v in t.items():
            o = out.setdefault(k, {"launches": 0, "ms_total": 0.0, "share": 0.0})
            o["launches"] += v["launches"]
            o["ms_total"] += v["ms_total"]
    tot = sum(v["ms_total"] for v in out.values()) or 1.0
    for v in out.values():
        v["share"] = v["ms_total"] / tot
    return out


RENDER_KERNELS = ("render_rows", "render_cols", "render_fused")


def render_flops(npix: int, nx: int, ny: int, frames: int) -> float:
    """Algorithmic FP32 flops of Eq. 1 for `frames` frames: 5 N log2 N per 1-D FFT on both
    axes (the conventional radix-2 count) plus the two chirps (2 flops for the uint16 x
    complex input chirp, 6 for the complex output chirp) per pixel."""
    return frames * npix * (5 * np.log2(nx) + 5 * np.log2(ny) + 8)


def fp32_peak_tflops() -> float:
    """Nominal FP32 FMA peak: SMs x 128 FP32 lanes x 2 flops x the maximum SM clock (2032 MHz)."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * 128 * 2 * 2.032e9 / 1e12


def measure_rates(local) -> dict:
    """FP32 (scalar and paired FMA) and FP64 FMA throughput measured now, on this GPU, by the
    library's rate kernel (dh_measure_fma_rate), with the SM clock sampled meanwhile; no clock
    or power setting is touched. The FP32 peak is the larger of the two FP32 forms."""
    import paper_2004_00923_b300 as dh
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    clocks.begin()
    out = {}
    for kind, iters in (("fp32", 32768), ("fp32x2", 16384), ("fp64", 512)):
        best = None
        for _ in range(3):
            r = dh.measure_fma_rate(kind, iters=iters, blocks_per_sm=4)
            if best is None or r["tflops"] > best["tflops"]:
                best = r
        out[kind] = {"tflops": best["tflops"], "ms": best["ms"]}
    # tensor-core issue rate of the covariance / projection MMA shape, three issue forms
    out["mma_issue"] = {f: dh.measure_mma_issue(f, stages=4096)
                        for f in ("back-to-back", "mbarrier-wait", "waiter-warp")}
    clocks.end()
    info = clocks.stop()
    out["fp32_peak_tflops"] = max(out["fp32"]["tflops"], out["fp32x2"]["tflops"])
    out["fp64_peak_tflops"] = out["fp64"]["tflops"]
    out["clocks"] = info
    out["how"] = ("dh_measure_fma_rate: 4 x SMs CTAs x 256 threads x 8 independent FMA chains, "
                  "best of 3 timed launches (CUDA events) after a warm-up; dh_measure_mma_issue: "
                  "one CTA per SM, 4096 stages of four M = N = 128, K = 16 FP16 MMAs")
    return out


def library_fft2(n: int, batch: int = 256) -> dict:
    """Context for the render: cuFFT's batched 2D FFT of complex64 n x n frames (through
    torch.fft.fft2, the library's own code path), the transform of Eq. 1 alone (no uint16
    conversion, chirps or 16-bit output). Best of 3 timings of 5 calls each (CUDA events)."""
    x = torch.randn(batch, n, n, dtype=torch.complex64, device="cuda")
    for _ in range(3):
        y = torch.fft.fft2(x)
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            y = torch.fft.fft2(x)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        best = ms if best is None else min(best, ms)
    del x, y
    torch.cuda.empty_cache()
    return {"us_per_frame": best * 1e3 / batch, "frames": batch,
            "what": f"cuFFT batched 2D FFT of complex64 {n}x{n} frames (torch.fft.fft2), the "
                    "transform of Eq. 1 alone: context for the render, not part of the step"}


def roofline_of(per_kernel: dict, alg: dict, hbm: float, peak_kind: str, step_s: float,
                flops: dict | None = None, alg_steps: int = 1, fp32_peak: float | None = None) -> dict:
    """Roofline of the kernel with the most device time among those with algorithmic bytes;
    `alg` (and `flops`) and `per_kernel` cover the same traced steps. The FFT kernels of
    Eq. 1 are bound by FP32 arithmetic (their DRAM traffic is the algorithmic minimum at a
    fraction of the HBM rate), so with `flops` they are reported against the FP32 peak, with
    the HBM view beside it; the contractions are reported against the measured copy rate."""
    dom = max((k for k in per_kernel if k in alg), key=lambda k: per_kernel[k]["ms_total"])
    d = per_kernel[dom]
    launch_s = d["ms_total"] / d["launches"] / 1e3
    gbs = alg[dom] / d["launches"] / launch_s / 1e9
    out = {"bound": "hbm", "kernel": dom, "achieved": gbs, "peak": hbm, "unit": "GB/s",
           "frac": gbs / hbm, "traffic": traffic_record(dom),
           "peak_kind": f"{peak_kind} copy bandwidth"}
    if flops and dom in flops:
        tf = flops[dom] / d["launches"] / launch_s / 1e12
        if fp32_peak:
            peak, kind = fp32_peak, "measured FP32 FMA rate of this run (dh_measure_fma_rate)"
        else:
            peak, kind = fp32_peak_tflops(), "nominal FP32 FMA peak: SMs x 128 lanes x 2 flops x 2032 MHz"
        out = {"bound": "alu", "kernel": dom, "achieved": tf, "peak": peak, "unit": "TFLOP/s",
               "frac": tf / peak, "traffic": traffic_record(dom), "peak_kind": kind,
               "nominal_fp32_tflops": fp32_peak_tflops(),
               "hbm_view": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm}}
    # `alg` covers `alg_steps` traced steps; the fraction is per step
    out["step_hbm_frac"] = sum(alg[k] for k in per_kernel if k in alg) / alg_steps / step_s / 1e9 / hbm
    out["kernels"] = per_kernel
    return out


def oracle_parity(frames_np, images_np, lam_np, k0, k1, tol_img):
    import oracle
    t0 = time.perf_counter()
    M, lam_ref, _, _ = oracle.pca_window(frames_np, LAM, Z, PITCH, k0, k1)
    sec = time.perf_counter() - t0
    return sec, {"image_rel_l2": float(np.linalg.norm(images_np - M) / np.linalg.norm(M)),
                 "eig_normwise": float(np.max(np.abs(lam_np - lam_ref)) / lam_ref[0]),
                 "tolerance_image": tol_img, "tolerance_eig": 1e-5}


def timed_graph(graph, stream, steps, ws, local):
    """Replay `graph` `steps` times between CUDA events on `stream`, with clocks sampled."""
    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    clocks.begin()
    ev[0].record(stream)
    for k in range(steps):
        graph.launch(stream)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    clocks.end()
    barrier(ws)
    clock_info = clocks.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    return ev[0].elapsed_time(ev[-1]) / steps, step_ms, clock_info


# --------------------------------------------------------------------------- sliding windows
SLIDE_FRAMES, SLIDE_STRIDE, SLIDE_LENGTHS = 2048, 8, (16, 32, 64)


def span_bytes(F, npix):
    """Hologram bytes the grouped projection reads per step: groups of 8 windows at stride 8,
    each group's span of T + 56 frames once (4 bytes a pixel: Re, Im FP16)."""
    total = 0
    for L in SLIDE_LENGTHS:
        n = (F - L) // SLIDE_STRIDE + 1
        for g0 in range(0, n, 8):
            gw = min(8, n - g0)
            total += (L + (gw - 1) * SLIDE_STRIDE) * npix * 4
    return total


def tune_plan(plan, args, n_frames: int = 256) -> dict:
    """The render and covariance options of a workload's rendering plan, set up outside the
    timed region: the library's autotuner (dh_plan_autotune: DFT arithmetic, FFT radix, render
    schedule, split-K units) unless the command line fixes the render schedule."""
    if args.render_schedule == "auto":
        return plan.autotune(n_frames)
    plan.set_render_schedule(args.render_schedule == "persistent", args.render_ring, args.render_lag)
    return plan.render_schedule()


def run_sliding(args, ws, rank, local, emit=None):
    """16-, 32- and 64-frame windows at stride 8 over 2048 frames of 1024^2: each frame is
    rendered once into a FP16 store read by all three window lengths (views), and the whole
    step is one CUDA graph."""
    import paper_2004_00923_b300 as dh
    from dh_synth import SpeckleParams, SpeckleStream

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    F = args.frames or SLIDE_FRAMES
    n = {L: (F - L) // SLIDE_STRIDE + 1 for L in SLIDE_LENGTHS}
    frames = SpeckleStream(SpeckleParams(NX, NY), seed=2000 + rank, device=dev).next(F)
    base = dh.Plan(NX, NY, LAM, Z, PITCH, T=16, precision="fp16", max_frames=F, max_windows=n[16])
    tuned = tune_plan(base, args)  # before the views: the base plan renders for all of them
    plans = {16: base, 32: base.view(32, n[32]), 64: base.view(64, n[64])}
    images = {L: torch.empty((n[L], NY, NX), dtype=torch.float32, device=dev) for L in SLIDE_LENGTHS}
    eig = {L: torch.empty((n[L], L), dtype=torch.float64, device=dev) for L in SLIDE_LENGTHS}

    def step():
        base.render_frames(frames)
        for L in SLIDE_LENGTHS:
            plans[L].pca_windows(0, SLIDE_STRIDE, n[L], 2, L - 1, images[L], eig[L])

    # one traced eager step for the per-kernel breakdown (captured launches are not traced)
    step()
    torch.cuda.synchronize()
    for p in plans.values():
        p.profile(True)
    step()
    tables = []
    for p in plans.values():
        tables.append(kernel_table(p.profile_read())[0])
        p.profile(False)
    per_kernel = merge_tables(tables)
    launches = sum(v["launches"] for v in per_kernel.values())

    # timed form: render, the banded covariance of the whole sequence (each frame read three
    # times instead of once per window holding it), then one batch with the three window
    # lengths (views of one store) running concurrently, longest first
    if args.band:
        for p in plans.values():
            p.set_covariance_source("band")
    for p in plans.values():
        p.set_projection(args.projection == "grouped")
    items = [{"plan": plans[L], "n_windows": n[L], "first_slot": 0, "slot_stride": SLIDE_STRIDE,
              "k0": 2, "k1": L - 1, "images": images[L], "eigvals": eig[L]} for L in (64, 32, 16)]

    def timed_step():
        base.render_frames(frames)
        if args.band:
            base.band_gram(0, F)
        dh.run_batch(items)

    # traced once more in the timed form's covariance and projection modes, stage by stage
    if args.band or args.projection == "grouped":
        for p in plans.values():
            p.profile(True)
        base.render_frames(frames)
        if args.band:
            base.band_gram(0, F)
        for L in SLIDE_LENGTHS:
            plans[L].pca_windows(0, SLIDE_STRIDE, n[L], 2, L - 1, images[L], eig[L])
        per_kernel = merge_tables([kernel_table(p.profile_read())[0] for p in plans.values()])
        for p in plans.values():
            p.profile(False)
        launches = sum(v["launches"] for v in per_kernel.values())
    s = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    with dh.capture(s) as g:
        timed_step()
    for _ in range(max(args.warmup, 0)):
        g.launch(s)
    ms, step_ms, clock_info = timed_graph(g, s, args.steps, ws, local)
    ms_max = max_over_ranks(ms, ws)
    nwin = sum(n.values())
    value = whole_job_rate(nwin, ws, ms_max)
    flags = base.status() | plans[32].status() | plans[64].status()

    hbm, _, peak_kind = measured_peaks()
    npix = NX * NY
    gram = sum(n[L] * L * npix * 4 for L in SLIDE_LENGTHS)
    alg = {"render_rows": F * npix * 2, "render_cols": F * npix * 4, "render_fused": F * npix * 6,
           "gram_tc": gram, "project_tc": gram + nwin * npix * 4,
           "band_gram": 3 * F * npix * 4,
           "project_span": span_bytes(F, npix) + nwin * npix * 4}  # each frame read as block b (twice) and as b + 1
    fl = render_flops(npix, NX, NY, F)
    roofline = roofline_of(per_kernel, alg, hbm, peak_kind, ms / 1e3, {k: fl for k in RENDER_KERNELS})

    parity, cpu = None, None
    if rank == 0 and not args.no_cpu_baseline:
        parity, secs = {}, 0.0
        fr = frames[:64].cpu().numpy()
        for L in SLIDE_LENGTHS:
            sec, par = oracle_parity(fr[:L], images[L][0].double().cpu().numpy(),
                                     eig[L][0].cpu().numpy(), 2, L - 1, 1e-3)
            parity[f"T{L}_window0"] = par
            secs += sec
        import oracle
        cpu = {"value": 3 / secs, "unit": "windows/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": "window 0 of each length (16, 32, 64), FP64 C oracle"}
    if rank == 0:
        line = {
            "metric": "sliding PCA windows/s (16/32/64-frame windows, stride 8) @1024²",
            "value": value, "unit": "windows/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "mixed: f32 FFT, f16 tensor-core products (f32 accumulate), f64 eig",
            "data": "synthetic",
            "config": {"workload": f"sliding: {F} frames of 1024x1024 uint16, 16/32/64-frame "
                                   "windows at stride 8, each frame rendered once (FP16), "
                                   "the lengths run concurrently, one CUDA graph per step",
                       "covariance": "banded Gram of the store (dh_band_gram)" if args.band
                       else "one Gram per window",
                       "projection": "grouped: 8 windows per tile load, energy minus discarded "
                                     "components" if args.projection == "grouped"
                       else "per window (Eq. 7 over the kept components)",
                       "windows_per_step": n, "k0": 2, "k1": "T-1",
                       "render_schedule": tuned,
                       "l2": "no flush: 4 GiB of frames and 8 GiB of holograms per step",
                       "parallelism": f"replicas x{ws}"},
            "frames_per_s": F * ws / (ms_max / 1e3),
            "step_ms": {"p50": statistics.median(step_ms), "max": max(step_ms)},
            "roofline": roofline, "cpu_baseline": cpu, "parity": parity,
            "gpu_launches": launches, "device_flags": flags, "clocks": clock_info,
        }
        (emit or print_line)(line)
    g.close()
    for p in plans.values():
        p.close()
    return 0


# --------------------------------------------------------------------------- Fourier mode
FOURIER_FRAMES, FOURIER_BINS = 2048, (7, 23)  # the paper's n_1 = 8, n_2 = 24, from 0
PAPER_FFT_GVOXEL_S = 17.0  # Table 1, FFT row: output voxels of 32 x 1024^2 windows per s


def run_fourier(args, ws, rank, local, emit=None):
    """Eqs. 8-9 with a new 32-frame window per frame (stride 1) over 2048 frames of 1024^2:
    each frame rendered once (FP16), then the DFT-bin power image of all 2017 windows."""
    import paper_2004_00923_b300 as dh
    from dh_synth import SpeckleParams, SpeckleStream

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    F = args.frames or FOURIER_FRAMES
    nwin = F - T + 1
    k0, k1 = FOURIER_BINS
    frames = SpeckleStream(SpeckleParams(NX, NY), seed=5000 + rank, device=dev).next(F)
    plan = dh.Plan(NX, NY, LAM, Z, PITCH, T=T, precision=args.precision, max_frames=F)
    tuned = tune_plan(plan, args)
    images = torch.empty((nwin, NY, NX), dtype=torch.float32, device=dev)

    def step():
        plan.render_frames(frames)
        plan.fourier_windows(0, 1, nwin, k0, k1, images)

    step()
    torch.cuda.synchronize()
    plan.profile(True)
    step()
    per_kernel, launches = kernel_table(plan.profile_read())
    plan.profile(False)
    s = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    with dh.capture(s) as g:
        step()
    for _ in range(max(args.warmup, 0)):
        g.launch(s)
    ms, step_ms, clock_info = timed_graph(g, s, args.steps, ws, local)
    ms_max = max_over_ranks(ms, ws)
    value = whole_job_rate(nwin, ws, ms_max)
    flags = plan.status()
    hbm, _, peak_kind = measured_peaks()
    npix = NX * NY
    hb = 2 if args.precision in ("fp16", "bf16") else 4
    hread = nwin * T * npix * 2 * hb
    alg = {"render_rows": F * npix * 2, "render_cols": F * npix * 2 * hb,
           "render_fused": F * npix * (2 + 2 * hb),
           "project_tc": hread + nwin * npix * 4, "project_simt": hread + nwin * npix * 4}
    fl = render_flops(npix, NX, NY, F)
    roofline = roofline_of(per_kernel, alg, hbm, peak_kind, ms / 1e3, {k: fl for k in RENDER_KERNELS})
    parity, cpu = None, None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        parity, secs = {}, 0.0
        for w in (0, nwin // 2, nwin - 1):
            fr = frames[w:w + T].cpu().numpy()
            t0 = time.perf_counter()
            M = oracle.fourier_window(fr, LAM, Z, PITCH, k0, k1)
            secs += time.perf_counter() - t0
            im = images[w].double().cpu().numpy()
            parity[f"window{w}"] = {"image_rel_l2": float(np.linalg.norm(im - M) / np.linalg.norm(M)),
                                    "tolerance_image": 1e-3 if hb == 2 else 1e-4}
        cpu = {"value": 3 / secs, "unit": "windows/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": "windows 0, 1008 and 2016 (1024x1024x32), FP64 C oracle"}
    gvox = value * T * npix / 1e9
    if rank == 0:
        line = {
            "metric": "Fourier-demodulation windows/s (Eqs. 8-9, stride-1 32-frame windows) @1024²",
            "value": value, "unit": "windows/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": gvox / PAPER_FFT_GVOXEL_S,
            "dtype": ("mixed: f32 FFT, f16 tensor-core products (f32 accumulate)"
                      if hb == 2 else "f32"),
            "data": "synthetic",
            "config": {"workload": f"fourier: {F} frames of 1024x1024 uint16, a 32-frame window "
                                   f"per frame ({nwin} windows), DFT bins 7..23, one CUDA graph "
                                   "per step", "precision": args.precision,
                       "render_schedule": tuned,
                       "l2": "no flush: 4 GiB of frames and 8 GiB of holograms per step",
                       "parallelism": f"replicas x{ws}"},
            "output_gvoxel_per_s": gvox,
            "vs_baseline_note": "output voxels/s over the paper's ~17 Gvoxel/s (Table 1, FFT)",
            "frames_per_s": F * ws / (ms_max / 1e3),
            "step_ms": {"p50": statistics.median(step_ms), "max": max(step_ms)},
            "roofline": roofline, "cpu_baseline": cpu, "parity": parity,
            "gpu_launches": launches, "device_flags": flags, "clocks": clock_info,
        }
        (emit or print_line)(line)
    g.close()
    plan.close()
    return 0


# --------------------------------------------------------------------------- uneven sizes
UNEVEN_SIZES = ((512, 40), (1024, 16), (2048, 4))


def run_uneven(args, ws, rank, local, emit=None):
    """512^2 x 40, 1024^2 x 16 and 2048^2 x 4 windows, alternating 32/64 frames, per-size z,
    per-window Doppler spread: one dh_batch_run (sizes on concurrent branches) per step,
    captured in one CUDA graph."""
    import paper_2004_00923_b300 as dh
    from dh_synth import uneven_batch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    groups = uneven_batch(UNEVEN_SIZES, seed=3000 + rank, device=dev)
    stride = 96
    sizes, items, plans_all, tuned = [], [], [], {}
    for g in groups:
        n = {L: len(g.starts(L)) for L in (32, 64)}
        base = dh.Plan(g.n, g.n, LAM, g.z, PITCH, T=32, precision=args.precision,
                       max_frames=g.frames.shape[0], max_windows=n[32])
        tuned[f"{g.n}x{g.n}"] = tune_plan(base, args, min(256, g.frames.shape[0]))
        plans = {32: base, 64: base.view(64, n[64])}
        out = {L: (torch.empty((n[L], g.n, g.n), dtype=torch.float32, device=dev),
                   torch.empty((n[L], L), dtype=torch.float64, device=dev)) for L in plans}
        for i, L in enumerate((32, 64)):
            it = {"plan": plans[L], "n_windows": n[L], "first_slot": g.starts(L)[0],
                  "slot_stride": stride, "k0": 2, "k1": L - 1, "images": out[L][0],
                  "eigvals": out[L][1]}
            if i == 0:
                it["frames"] = g.frames
            items.append(it)
        sizes.append((g, n, plans, out))
        plans_all += list(plans.values())

    dh.run_batch(items)
    torch.cuda.synchronize()
    # traced run with one batch call per item: the branches then run one after the other, so
    # each kernel's event interval is its own time (concurrent branches would overlap them)
    for p in plans_all:
        p.profile(True)
    for it in items:
        dh.run_batch([it])
    per_kernel = merge_tables([kernel_table(p.profile_read())[0] for p in plans_all])
    for p in plans_all:
        p.profile(False)
    launches = sum(v["launches"] for v in per_kernel.values())

    s = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    with dh.capture(s) as gr:
        dh.run_batch(items)
    for _ in range(max(args.warmup, 0)):
        gr.launch(s)
    ms, step_ms, clock_info = timed_graph(gr, s, args.steps, ws, local)
    ms_max = max_over_ranks(ms, ws)
    nwin = sum(sum(n.values()) for _, n, _, _ in sizes)
    nframes = sum(g.frames.shape[0] for g in groups)
    value = whole_job_rate(nwin, ws, ms_max)
    flags = 0
    for p in plans_all:
        flags |= p.status()

    hbm, _, peak_kind = measured_peaks()
    hb = 2 if args.precision in ("fp16", "bf16") else 4
    alg = {"render_rows": 0, "render_cols": 0, "render_fused": 0, "gram_tc": 0, "gram_simt": 0,
           "project_tc": 0, "project_simt": 0}
    fl = 0.0
    for g, n, _, _ in sizes:
        npix = g.n * g.n
        F = g.frames.shape[0]
        fl += render_flops(npix, g.n, g.n, F)
        alg["render_rows"] += F * npix * 2
        alg["render_cols"] += F * npix * 2 * hb
        alg["render_fused"] += F * npix * (2 + 2 * hb)
        hread = sum(n[L] * L * npix * 2 * hb for L in n)
        for k in ("gram_tc", "gram_simt"):
            alg[k] += hread
        for k in ("project_tc", "project_simt"):
            alg[k] += hread + sum(n.values()) * npix * 4
    roofline = roofline_of(per_kernel, alg, hbm, peak_kind, ms / 1e3, {k: fl for k in RENDER_KERNELS})

    parity, cpu = None, None
    tol = 1e-3 if args.precision != "fp32" else 1e-4
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        parity, secs, nsamp = {}, 0.0, 0
        for g, n, plans, out in sizes:
            picks = [(32, 0)] + ([(64, 0)] if g.n == 512 else [])
            for L, w in picks:
                s0 = g.starts(L)[w]
                fr = g.frames[s0:s0 + L].cpu().numpy()
                t0 = time.perf_counter()
                M, lam_ref, _, _ = oracle.pca_window(fr, LAM, g.z, PITCH, 2, L - 1)
                secs += time.perf_counter() - t0
                nsamp += 1
                img = out[L][0][w].double().cpu().numpy()
                lam = out[L][1][w].cpu().numpy()
                parity[f"{g.n}x{g.n}_T{L}_w{w}"] = {
                    "image_rel_l2": float(np.linalg.norm(img - M) / np.linalg.norm(M)),
                    "eig_normwise": float(np.max(np.abs(lam - lam_ref)) / lam_ref[0]),
                    "tolerance_image": tol, "tolerance_eig": 1e-5}
        cpu = {"value": nsamp / secs, "unit": "windows/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": "window 0 (32 frames) of each size and one 64-frame "
                                           "window at 512^2, FP64 C oracle"}
    if rank == 0:
        line = {
            "metric": "uneven-size PCA windows/s (512²×40, 1024²×16, 2048²×4; T 32/64)",
            "value": value, "unit": "windows/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("mixed: f32 FFT, f16 tensor-core products (f32 accumulate), f64 eig"
                      if args.precision != "fp32" else "f32 (f64 covariance reduction and eig)"),
            "data": "synthetic",
            "config": {"workload": "uneven: 512^2 x 40, 1024^2 x 16, 2048^2 x 4 windows, "
                                   "alternating 32/64 frames, per-size z ~ U(0.25, 0.45) m, "
                                   "sigma_D ~ U(0.1, 1.0) per window, one batch per step "
                                   "(one CUDA graph)",
                       "precision": args.precision,
                       "sizes": [{"n": g.n, "z": g.z, "windows": n, "frames": g.frames.shape[0]}
                                 for g, n, _, _ in sizes],
                       "render_schedule": tuned,
                       "l2": "no flush: 4 GiB of frames per step",
                       "parallelism": f"replicas x{ws}"},
            "frames_per_s": nframes * ws / (ms_max / 1e3),
            "step_ms": {"p50": statistics.median(step_ms), "max": max(step_ms)},
            "roofline": roofline, "cpu_baseline": cpu, "parity": parity,
            "gpu_launches": launches, "device_flags": flags, "clocks": clock_info,
        }
        (emit or print_line)(line)
    gr.close()
    for p in plans_all:
        p.close()
    return 0


# --------------------------------------------------------------------------- serving loop
SERVE_STREAMS = [(1024, 500.0)] * 4 + [(2048, 125.0)]  # (frame side, frames per second)
SERVE_T, SERVE_BUDGET, SERVE_POOL, SERVE_CHUNK, SERVE_RING = 32, 40 * 10**9, 256, 4, 8


def pct(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if xs else None


class ServeReplay:
    """The serving mix (4 camera streams of 1024^2 at 500 fps and 1 of 2048^2 at 125 fps,
    32-frame windows) on one dh.Server, fed from pinned host frame pools of `pool` frames per
    stream. run(seconds, clocked) replays that much stream time: frames are pushed in
    4-frame grabber chunks as they arrive (clocked) or as fast as the loop accepts them, every
    finished window is polled back to the host and its latency recorded."""

    def __init__(self, dh, dev, rank, pool=SERVE_POOL):
        from dh_synth import SpeckleParams, SpeckleStream
        self.dh = dh
        self.pool = pool
        self.srv = dh.Server(SERVE_BUDGET)
        self.pools, self.ids, self.fps = [], [], []
        for i, (n, rate) in enumerate(SERVE_STREAMS):
            gen = SpeckleStream(SpeckleParams(n, n), seed=4000 + 10 * rank + i, device=dev)
            pl = torch.empty((pool, n, n), dtype=torch.uint16, pin_memory=True)
            for k in range(0, pool, 32):
                pl[k:k + 32].copy_(gen.next(min(32, pool - k)))
            self.pools.append(pl)
            self.ids.append(self.srv.add_stream(n, n, LAM, Z, PITCH, SERVE_T, "fp16", 2, SERVE_T - 1,
                                                ring_windows=SERVE_RING))
            self.fps.append(rate)
        torch.cuda.synchronize()
        self.pushed = [0] * len(self.ids)  # frames each stream has received so far

    def frames_of(self, i, k, cnt):
        j = k % self.pool
        return self.pools[i][j:j + cnt]

    def run(self, seconds, clocked):
        """Returns (windows, wall seconds, latencies per stream, latencies from the push,
        push lateness)."""
        srv, ids, fps, dh = self.srv, self.ids, self.fps, self.dh
        start = list(self.pushed)
        nxt = [0] * len(ids)  # frames pushed in this pass
        lat = {sid: [] for sid in ids}       # from the scheduled arrival of the last frame
        lat_push = {sid: [] for sid in ids}  # from the push of the last frame
        sched = {}
        late = []
        total = 0
        per_stream_frames = [int(seconds * r) // SERVE_T * SERVE_T for r in fps]
        t0 = time.perf_counter()
        off = srv.clock() - time.perf_counter()  # server clock minus perf_counter

        def collect():
            nonlocal total
            for r in srv.poll(64):
                key = (r["stream"], r["window"])
                t_arr = sched.pop(key, r["t_ready"])
                lat[r["stream"]].append((r["t_done"] - t_arr) * 1e3)
                lat_push[r["stream"]].append((r["t_done"] - r["t_ready"]) * 1e3)
                total += 1

        while any(nx < F for nx, F in zip(nxt, per_stream_frames)):
            if clocked:
                # the next chunk due: stream i's chunk ends with frame nxt+CHUNK-1
                due = [(t0 + (nxt[i] + SERVE_CHUNK) / fps[i], i)
                       for i in range(len(ids)) if nxt[i] < per_stream_frames[i]]
                t_due, i = min(due)
                while True:
                    now = time.perf_counter()
                    if now >= t_due:
                        break
                    collect()
                    if t_due - time.perf_counter() > 0.0005:
                        time.sleep(0.0002)
                late.append(time.perf_counter() - t_due)
                k_end = start[i] + nxt[i] + SERVE_CHUNK
                if k_end % SERVE_T == 0:  # this chunk completes window k_end / T - 1
                    sched[(ids[i], k_end // SERVE_T - 1)] = t_due + off
            else:
                i = min(range(len(ids)), key=lambda j: nxt[j] / per_stream_frames[j]
                        if nxt[j] < per_stream_frames[j] else 2.0)
            while True:
                try:
                    k = start[i] + nxt[i]
                    srv.push(ids[i], self.frames_of(i, k, SERVE_CHUNK), k)
                    break
                except dh.DHError as e:
                    if e.code != 7:  # only output backpressure is waited out
                        raise
                    collect()
            nxt[i] += SERVE_CHUNK
            collect()
        srv.drain()
        collect()
        wall = time.perf_counter() - t0
        for i in range(len(ids)):
            self.pushed[i] = start[i] + nxt[i]
        return total, wall, lat, lat_push, late

    def latency_summary(self, lat, seconds):
        all_lat = [x for v in lat.values() for x in v]
        by_size = {}
        for (n, _), sid in zip(SERVE_STREAMS, self.ids):
            by_size.setdefault(f"{n}x{n}", []).extend(lat[sid])
        return {"p50": pct(all_lat, 50), "p99": pct(all_lat, 99),
                "max": max(all_lat) if all_lat else None, "windows": len(all_lat),
                "expected_windows": sum(int(seconds * r) // SERVE_T for _, r in SERVE_STREAMS),
                "by_size": {k: {"p50": pct(v, 50), "p99": pct(v, 99), "max": max(v) if v else None}
                            for k, v in by_size.items()},
                "from": "scheduled arrival of the window's last frame at the stream clock -> "
                        "image and eigenvalues in host memory",
                "target_p99": 64.0}

    def close(self):
        self.srv.close()


def serve_latency(args, ws, rank, local):
    """The third term of the headline metric: p50/p99 window latency of a short replay of
    the serving mix at the stream clock (`--latency-seconds` of stream time, after one
    clock-free second of warm-up); the max of each percentile over ranks."""
    import paper_2004_00923_b300 as dh
    dev = torch.device("cuda", local)
    rep = ServeReplay(dh, dev, rank, pool=64)
    try:
        rep.run(1.0, clocked=False)
        n_win, wall, lat, _, late = rep.run(args.latency_seconds, clocked=True)
        out = rep.latency_summary(lat, args.latency_seconds)
    finally:
        rep.close()
    for key in ("p50", "p99", "max"):
        if out[key] is not None:
            out[key] = max_over_ranks(out[key], ws)
    out["stream_seconds"] = args.latency_seconds
    out["windows_per_s"] = n_win / wall
    out["push_lateness_p99_ms"] = pct(late, 99) * 1e3 if late else None
    out["streams"] = [{"n": n, "fps": r} for n, r in SERVE_STREAMS]
    return out


def run_serving(args, ws, rank, local):
    """4 camera streams of 1024^2 at 500 fps and 1 of 2048^2 at 125 fps, 32-frame windows,
    replayed at the stream clock from pinned host frame pools for `--serve-seconds` of stream
    time: frames are pushed in 4-frame grabber chunks as they arrive, every finished window
    is polled back to the host, and its latency (push of its last frame -> image in host
    memory) is recorded. Then an admission pass against the 40 GB budget and a saturation
    pass (no clock) for the loop's capacity."""
    import paper_2004_00923_b300 as dh

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rep = ServeReplay(dh, dev, rank)
    srv, ids, pools = rep.srv, rep.ids, rep.pools
    used_served = srv.used_bytes
    run = rep.run

    # warm-up: one clock-free second of every stream
    run(1.0, clocked=False)
    clocks = ClockSampler(local)
    clocks.start()
    clocks.begin()
    n_win, wall, lat, lat_push, late = run(args.serve_seconds, clocked=True)
    clocks.end()
    clock_info = clocks.stop()
    n_sat, wall_sat, _, lat_sat, _ = run(min(10.0, args.serve_seconds), clocked=False)

    # admission: add 1024^2 streams until the budget refuses one, then give them back
    extra, refused = [], None
    while refused is None and len(extra) < 256:
        try:
            extra.append(srv.add_stream(1024, 1024, LAM, Z, PITCH, SERVE_T, "fp16", 2,
                                        SERVE_T - 1, ring_windows=SERVE_RING))
        except dh.DHError as e:
            refused = e.code
    used_full = srv.used_bytes
    for sid in extra:
        srv.remove_stream(sid)

    all_lat = [x for v in lat.values() for x in v]
    all_push = [x for v in lat_push.values() for x in v]
    by_size = {}
    for (n, _), sid in zip(SERVE_STREAMS, ids):
        by_size.setdefault(f"{n}x{n}", []).extend(lat[sid])
    sat_lat = [x for v in lat_sat.values() for x in v]

    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        parity = {}
        for i in (0, len(ids) - 1):
            n = SERVE_STREAMS[i][0]
            with dh.Plan(n, n, LAM, Z, PITCH, T=SERVE_T, precision="fp16") as plan:
                img, lam = plan.pca_batch(pools[i][:SERVE_T].to(dev), 1, SERVE_T, 2, SERVE_T - 1)
                M, lam_ref, _, _ = oracle.pca_window(pools[i][:SERVE_T].numpy(), LAM, Z, PITCH,
                                                     2, SERVE_T - 1)
                im = img[0].double().cpu().numpy()
                parity[f"stream{i}_{n}x{n}_window0"] = {
                    "image_rel_l2": float(np.linalg.norm(im - M) / np.linalg.norm(M)),
                    "eig_normwise": float(np.max(np.abs(lam[0].cpu().numpy() - lam_ref)) / lam_ref[0]),
                    "tolerance_image": 1e-3, "tolerance_eig": 1e-5}
    value = n_win / wall
    if rank == 0:
        line = {
            "metric": "serving windows/s and p50/p99 window latency (4×1024²@500 fps + "
                      "1×2048²@125 fps, T=32)",
            "value": value, "unit": "windows/s", "n_gpus": ws, "steps": 1, "warmup": 1,
            "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "mixed: f32 FFT, f16 tensor-core products (f32 accumulate), f64 eig",
            "data": "synthetic",
            "config": {"workload": f"serving: {args.serve_seconds:g} s of stream time, frames "
                                   f"pushed from pinned host pools ({SERVE_POOL} per stream) "
                                   f"in {SERVE_CHUNK}-frame chunks at the stream clock",
                       "streams": [{"n": n, "fps": r} for n, r in SERVE_STREAMS], "T": SERVE_T,
                       "k0": 2, "k1": SERVE_T - 1, "ring_windows": SERVE_RING,
                       "hbm_budget_bytes": SERVE_BUDGET, "parallelism": f"replicas x{ws}"},
            "windows": n_win,
            "expected_windows": sum(int(args.serve_seconds * r) // SERVE_T for _, r in SERVE_STREAMS),
            "latency_ms": {"p50": pct(all_lat, 50), "p99": pct(all_lat, 99), "max": max(all_lat),
                           "by_size": {k: {"p50": pct(v, 50), "p99": pct(v, 99), "max": max(v)}
                                       for k, v in by_size.items()},
                           "from": "scheduled arrival of the window's last frame at the "
                                   "stream clock -> image and eigenvalues in host memory",
                           "target_p99": 64.0},
            "latency_from_push_ms": {"p50": pct(all_push, 50), "p99": pct(all_push, 99),
                                     "max": max(all_push)},
            "push_lateness_ms": {"p50": pct(late, 50) * 1e3, "p99": pct(late, 99) * 1e3,
                                 "max": max(late) * 1e3},
            "saturation": {"windows_per_s": n_sat / wall_sat, "windows": n_sat,
                           "latency_from_push_ms": {"p50": pct(sat_lat, 50), "p99": pct(sat_lat, 99)},
                           "note": "same streams pushed as fast as the loop accepts them"},
            "admission": {"budget_bytes": SERVE_BUDGET, "served_streams_bytes": used_served,
                          "stream_bytes": {"1024x1024": dh.Server.stream_bytes(1024, 1024, SERVE_T, "fp16", SERVE_RING),
                                           "2048x2048": dh.Server.stream_bytes(2048, 2048, SERVE_T, "fp16", SERVE_RING)},
                          "extra_1024_streams_admitted": len(extra), "refusal_code": refused,
                          "used_bytes_at_refusal": used_full},
            "e2e": {"value": value, "unit": "windows/s",
                    "h2d_bytes_per_step": int(sum(int(args.serve_seconds * r) * n * n * 2
                                                  for n, r in SERVE_STREAMS)),
                    "d2h_bytes_per_step": int(sum(int(args.serve_seconds * r) // SERVE_T * (n * n * 4 + SERVE_T * 8)
                                                  for n, r in SERVE_STREAMS)),
                    "note": "the serving loop is end to end: host frames in, host images out"},
            "parity": parity, "clocks": clock_info,
        }
        print(json.dumps(line), flush=True)
    rep.close()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp16", "bf16", "fp32"], default="fp16")
    ap.add_argument("--windows", type=int, default=NWIN,
                    help="windows per step (default 64; smaller only for profiler captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--render-schedule", choices=["auto", "persistent", "chunks"], default="auto",
                    help="Eq. 1 schedule of the headline plan: auto = the library's autotuner "
                         "(dh_plan_autotune); else DH_OPT_RENDER_SCHEDULE with ring and lag")
    ap.add_argument("--pipeline", action=argparse.BooleanOptionalAction, default=False,
                    help="overlap the render of batch k+1 with Eqs. 4-7 of batch k (two halves of "
                         "hologram slots, two streams; measured no faster: the persistent render "
                         "holds every SM's registers); default: batches back to back")
    ap.add_argument("--band", action=argparse.BooleanOptionalAction, default=True,
                    help="sliding workload: windows take C from the store's banded Gram "
                         "(dh_band_gram) instead of one Gram per window")
    ap.add_argument("--frames", type=int, default=0,
                    help="sliding and fourier workloads: frames per step (default 2048; smaller for "
                         "ncu captures)")
    ap.add_argument("--projection", choices=["grouped", "per-window"], default="grouped",
                    help="sliding workload: DH_OPT_PROJECTION (grouped = 0, per-window = 1)")
    ap.add_argument("--covariance", choices=["holograms", "raw"], default="holograms",
                    help="Eq. 4 from the holograms (as written, default) or exactly from the uint16 "
                         "frames (DH_OPT_COVARIANCE = 1, C = I^T I)")
    ap.add_argument("--render-ring", type=int, default=0, help="DH_OPT_RENDER_RING (0 = automatic)")
    ap.add_argument("--render-lag", type=int, default=0, help="DH_OPT_RENDER_LAG (0 = automatic)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="stream time replayed by --workload serving")
    ap.add_argument("--latency-seconds", type=float, default=10.0,
                    help="headline line: stream time of the serving replay that gives the p50/p99 "
                         "window latency (0 = skip)")
    ap.add_argument("--render-fft", choices=["auto", "cuda", "tensor"], default="auto",
                    help="headline: DH_OPT_RENDER_FFT (tensor: the 32-point DFT stages on the tensor "
                         "cores); with --render-schedule auto the autotuner may still change it")
    ap.add_argument("--residual", action="store_true",
                    help="headline: mean-residual storage of the 16-bit holograms (DH_OPT_RESIDUAL)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="headline line: skip the short sliding / uneven / Fourier runs")
    ap.add_argument("--no-peaks", action="store_true",
                    help="headline line: skip the FP32/FP64 FMA-rate measurement")
    ap.add_argument("--workload", choices=["paper", "sliding", "uneven", "serving", "fourier"],
                    default="paper",
                    help="paper: the headline 64 x 1024^2 x 32 step (default); sliding: "
                         "16/32/64-frame windows at stride 8 over 2048 frames; uneven: "
                         "512^2/1024^2/2048^2 windows of 32/64 frames in one batch; serving: "
                         "4 x 1024^2 @ 500 fps + 1 x 2048^2 @ 125 fps camera streams; fourier: "
                         "Eqs. 8-9 with stride-1 32-frame windows over 2048 frames")
    args = ap.parse_args(argv)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    dist_init(ws)
    try:
        if args.workload == "sliding":
            return run_sliding(args, ws, rank, local)
        if args.workload == "uneven":
            return run_uneven(args, ws, rank, local)
        if args.workload == "serving":
            return run_serving(args, ws, rank, local)
        if args.workload == "fourier":
            return run_fourier(args, ws, rank, local)
        return run_ours(args, ws, rank, local)
    finally:
        if ws > 1 and torch.distributed.is_initialized():
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
