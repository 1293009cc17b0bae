#!/usr/bin/env python3
"""Gridded + degridded visibilities per second for W-projection imaging on GB300.

One step is one pass of the whole hot path over the full W-projection workload (351 baselines x
2000 integrations x 64 channels 2-4 GHz x 4 pols = 179.7M visibilities, 64 w-planes with CF
supports 8-64, oversampling 20, 4096 x 4096 x 4 grid):

    plan_update          per-sample FP64 index, w-plane, CF, pixel/offset; tiled counting sort
    grid_visibilities    G (Eq. IMAGE-MOD) into a zeroed grid, FP64 sum of weights
    grid_normalize       taper / weight correction of the gridded plane (after the caller's FFT)
    degrid_visibilities  D (Eq. ME-MOD-GRIDDED) from a model grid

value = (gridded + degridded visibilities) / step time, summed over ranks.  The inputs (1.44 GB of
visibilities, 0.72 GB of weights, a 0.54 GB model grid) are larger than the 129 MB L2, so no
extra flush is needed between steps.  `--impl reference` times the FP64 CPU oracle on a bounded
sample of the same workload instead.

Multi-GPU (torchrun): every rank takes its own slice of integrations of a track N times as long
(the same per-rank size, weak scaling) and the gridded planes are summed with one all-reduce per
step, which is the accumulation of Eq. ResIm over time.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

CONFIG = "wproj"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-int", type=int, default=None, help="integrations per rank (default: the full 2000)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-every", type=int, default=None,
                    help="oracle sample: every k-th integration (default 40 for cpu_baseline, 200 per reference step)")
    ap.add_argument("--config", choices=["wproj", "awproj"], default="wproj",
                    help="wproj: the W-projection workload (default); awproj: the batched AW-projection workload "
                         "(20 PA bins x 32 w-planes x 16 sub-bands, CFs as sums of outer products)")
    ap.add_argument("--mosaic", action="store_true",
                    help="give every row its own phase centre (a two-field mosaic with pointing offsets)")
    ap.add_argument("--full-pol", action="store_true",
                    help="with --config awproj: full-polarisation A-terms (sparse Mueller CFs; 4 PA bins x 4 "
                         "sub-bands so that the 12-element CF set builds in seconds)")
    ap.add_argument("--no-aw", action="store_true",
                    help="skip the batched AW-projection step that the default W-projection line reports "
                         "under the key awproj")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default kernel configuration of every support instead of timing them all")
    ap.add_argument("--kernel-config", default=None, metavar="S:C,...",
                    help="fix the kernel configuration C (0-3) of support S instead of autotuning, e.g. to "
                         "profile a reduced workload with the kernels the full one tunes to")
    ap.add_argument("--minor-cycle", action="store_true",
                    help="time the Hogbom minor cycle on a 4096^2 image (one JSON line, HBM roofline)")
    ap.add_argument("--calibrate", action="store_true",
                    help="time the G-Jones solve on the W-projection workload with degridded model visibilities")
    ap.add_argument("--forward-model", action="store_true",
                    help="time ten major cycles of the differentiable forward model (1024^2 sky, 5.01M "
                         "visibilities) and its chi^2 gradient")
    ap.add_argument("--precision-sweep", action="store_true",
                    help="CF storage / accumulation variants against the FP64 oracle (one JSON line each)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


WORKLOAD_OVERRIDES = {}


def rank_workload(world: int, rank: int, n_int: int, device: str, with_vis=True):
    """Rank `rank`'s slice of a track of world * n_int integrations (time-major rows)."""
    full = synth.make_workload(CONFIG, with_vis=False, n_int=n_int * world, **WORKLOAD_OVERRIDES)
    r0, r1 = rank * n_int * full.n_bl, (rank + 1) * n_int * full.n_bl
    wl = dataclasses.replace(full, uvw_m=full.uvw_m[r0:r1].copy(), pa_rad=full.pa_rad[r0:r1].copy(),
                             pa_bin=full.pa_bin[r0:r1].copy(), n_int=n_int)
    if with_vis:
        synth.fill_visibilities(wl, device=device)
    return wl


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# Sources that do not take part in a gridding or degridding launch (minor cycle, calibration,
# peak probe, plain FP64 baseline, no-allocation entry point): changing them leaves the DRAM
# counters of the gridding and degridding kernels valid.
NOT_GD_SOURCES = ("clean.cu", "gcal.cu", "probe.cu", "plain_fp64.cu", "noalloc.cu")


def csrc_hash() -> str:
    """SHA-256 over the library's CUDA / C++ sources that build or launch the gridding and
    degridding kernels (names and contents, sorted)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2508_17187_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h", ".cpp")) and name not in NOT_GD_SOURCES:
            h.update(name.encode())
            h.update(open(os.path.join(d, name), "rb").read())
    return h.hexdigest()


def measured_traffic(op: str, variant: bool = False):
    """DRAM bytes per full-size launch of `op` from the committed ncu summary, or None when the
    kernels have changed since the counters were taken or the step is a variant of the workload
    (mosaic phases, full polarisation) that the counters were not taken on."""
    if variant:
        return None
    try:
        with open(os.path.join(ROOT, "profiles", f"dram_traffic_{CONFIG}.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("csrc_sha256") != csrc_hash():
        return None
    return rec.get("per_launch_bytes", {}).get(op)


def measure_fma_peak(lib, sms: int, dev: str, seconds: float = 0.5) -> dict:
    """FP32 FMA rate from the library's probe kernel (8 CTAs of 256 threads per SM, 8 independent
    FMA chains a thread), timed with CUDA events on the launching stream: one launch as the burst
    figure, back-to-back launches over about `seconds` as the sustained one."""
    import ctypes

    import torch
    n_blocks = sms * 8
    out = torch.empty(n_blocks * 256, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    flop = ctypes.c_double()

    def launch(iters):
        st = lib.awg_fp32_fma_probe(ctypes.c_void_p(out.data_ptr()), n_blocks, iters, sp, ctypes.byref(flop))
        if st != 0:
            raise RuntimeError("awg_fp32_fma_probe failed: " + lib.awg_last_error().decode())
        return flop.value

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = 1 << 14
    launch(iters)
    while True:   # grow the launch to about 50 ms
        e0.record(stream)
        f = launch(iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if ms >= 40.0 or iters >= (1 << 26):
            break
        iters = int(iters * max(2.0, 50.0 / max(ms, 1e-3)))
    burst = f / (ms / 1e3) / 1e12
    reps = max(1, int(seconds * 1e3 / ms))
    e0.record(stream)
    for _ in range(reps):
        f = launch(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    sustained = f * reps / (e0.elapsed_time(e1) / 1e3) / 1e12
    return {"burst_tflops": burst, "sustained_tflops": sustained, "launch_ms": ms, "launches": reps + 2}


def fp32_alu_peak_tflops(sms: int, mhz: float) -> float:
    """Non-tensor FP32 FMA peak: SMs x 128 FP32 lanes x 2 FLOP per FMA x SM clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def run_cpu_baseline(wl, every: int, single_thread: bool = False):
    """Time the FP64 oracle (G and D, OpenMP over all cores) on every `every`-th integration, and
    with single_thread also on one thread over a tenth of that sample."""
    from oracle import cf as ocf
    from oracle import index as oindex
    from oracle import ops as oops
    rows = np.concatenate([np.arange(t * wl.n_bl, (t + 1) * wl.n_bl) for t in range(0, wl.n_int, every)])
    op = ocf.CFParams(grid_n=wl.grid_n, cell_rad=wl.cell_rad, oversampling=wl.oversampling,
                      ps_support=wl.ps_support, use_w=wl.use_w, n_wplanes=wl.n_wplanes,
                      w_max_lambda=wl.w_max_lambda, max_support=wl.max_support)
    idx = oindex.sample_index(op, wl.uvw_m[rows], wl.freq_hz)
    tabs = ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist()))
    buf, off, _ = ocf.flatten_cf_set(op, tabs)
    vis = np.asarray(wl.vis)[rows].reshape(-1, wl.n_pol)
    wt = np.asarray(wl.weight)[rows].reshape(-1, wl.n_pol)
    threads = oops.default_threads()
    t0 = time.perf_counter()
    g, sw = oops.grid(idx, buf, off, wl.oversampling, wl.grid_n, vis, wt, nthreads=threads)
    t1 = time.perf_counter()
    d = oops.degrid(idx, buf, off, wl.oversampling, g, nthreads=threads)
    t2 = time.perf_counter()
    n_vis = int(idx.valid.size) * wl.n_pol
    out = {"value": 2 * n_vis / (t2 - t0), "unit": "visibilities/s", "cores": threads, "kind": "oracle",
           "cpu_model": cpu_model(),
           "sample": f"every {every}th integration: {len(rows)} rows x {wl.n_chan} channels x {wl.n_pol} pols "
                     f"= {n_vis} visibilities, gridded then degridded (grid {t1 - t0:.2f} s, degrid {t2 - t1:.2f} s)",
           "seconds": t2 - t0, "rows": rows, "grid": g, "sumwt": sw, "degrid": d,
           "support": idx.support[idx.valid]}
    if single_thread and len(rows) >= 10 * wl.n_bl:
        # one thread on the first tenth of the sample's integrations
        sub = rows[:len(rows) // 10 // wl.n_bl * wl.n_bl]
        idx1 = oindex.sample_index(op, wl.uvw_m[sub], wl.freq_hz)
        v1 = np.asarray(wl.vis)[sub].reshape(-1, wl.n_pol)
        w1 = np.asarray(wl.weight)[sub].reshape(-1, wl.n_pol)
        t0 = time.perf_counter()
        g1, _ = oops.grid(idx1, buf, off, wl.oversampling, wl.grid_n, v1, w1, nthreads=1)
        oops.degrid(idx1, buf, off, wl.oversampling, g1, nthreads=1)
        t1 = time.perf_counter()
        n1 = int(idx1.valid.size) * wl.n_pol
        out["single_thread"] = {"value": 2 * n1 / (t1 - t0), "unit": "visibilities/s",
                                "sample": f"{len(sub)} rows of the sample ({n1} visibilities), 1 thread"}
    return out


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    import subprocess
    try:
        for ln in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def sample_accuracy(cf, wl, vis, wt, cb, dev) -> dict:
    """The library against the oracle on the baseline's sample: the gridded plane and the
    degridding of the oracle's own FP64 plane (relative RMS over their full extent), and the
    dirty image over the inner half of the field (where T >= 0.25; the error measure of the 1e-5
    accuracy target).  The library's image is its whole path: gridding, the inverse FFT on the
    GPU and grid_normalize with the library's sum of weights; the oracle's is
    oracle.image.dirty_image of its FP64 grid with its own sum of weights and taper."""
    import torch

    import paper_2508_17187_gb300 as awg
    from oracle import image as oimage
    rows = torch.as_tensor(cb["rows"], device=dev)
    N, P = wl.grid_n, wl.n_pol
    plan = awg.plan_create(cf, torch.as_tensor(wl.uvw_m, device=dev)[rows], torch.as_tensor(wl.freq_hz, device=dev))
    g = torch.zeros((N, N, P), dtype=torch.complex64, device=dev)
    sw = torch.zeros(P, dtype=torch.float64, device=dev)
    awg.grid_visibilities(cf, plan, vis[rows].contiguous(), wt[rows].contiguous(), g, sw)
    g_o = torch.as_tensor(cb["grid"], device=dev)
    out = torch.empty((len(cb["rows"]), wl.n_chan, P), dtype=torch.complex64, device=dev)
    awg.degrid_visibilities(cf, plan, g_o.to(torch.complex64).contiguous(), out)
    d_o = torch.as_tensor(cb["degrid"], device=dev).reshape(out.shape)

    def rel(a, b):
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

    x = torch.fft.ifftshift(g, dim=(0, 1))
    img = torch.fft.fftshift(torch.fft.ifft2(x, dim=(0, 1), norm="forward"), dim=(0, 1)).contiguous()
    awg.grid_normalize(cf, img, sw, direction=0)
    q = slice(N // 4, 3 * N // 4)
    img_lib = img.real[q, q].double().cpu().numpy()
    img_o = oimage.dirty_image(cb["grid"], cb["sumwt"], wl.ps_support)[q, q]
    img_err = float(np.linalg.norm(img_lib - img_o) / np.linalg.norm(img_o))
    err = {"grid_rel_rms": rel(g.to(torch.complex128), g_o), "degrid_rel_rms": rel(out.to(torch.complex128), d_o),
           "image_rel_rms_inner_half": img_err,
           "sumwt_rel": float(np.max(np.abs(sw.cpu().numpy() - cb["sumwt"]) / np.abs(cb["sumwt"]))),
           "sample": "the cpu_baseline sample, FP64 oracle vs the library (image: library gridding + GPU FFT + "
                     "grid_normalize vs oracle dirty_image with the oracle's taper and sum of weights)"}
    plan.close()
    return err


def plain_fp64_on_sample(wl, vis, wt, cb, dev) -> dict:
    """The plain FP64 GPU baseline (one launch per channel, full CF tables, FP64 grid) on the
    cpu_baseline sample: its throughput and its error against the oracle."""
    import ctypes

    import torch

    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300 import _lib
    lib = _lib.load()
    cf = awg.cf_set_create(**cf_kwargs(wl), separable=False)
    rows = torch.as_tensor(cb["rows"], device=dev)
    uvw = torch.as_tensor(wl.uvw_m, device=dev)[rows].contiguous()
    v, w = vis[rows].contiguous(), wt[rows].contiguous()
    R, C, P, N = len(cb["rows"]), wl.n_chan, wl.n_pol, wl.grid_n
    fr = np.ascontiguousarray(wl.freq_hz)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    g64 = torch.zeros((N, N, P), dtype=torch.complex128, device=dev)
    sw = torch.zeros(P, dtype=torch.float64, device=dev)
    out = torch.empty_like(v)
    g_o = torch.as_tensor(cb["grid"], device=dev)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    rc = lib.grid_visibilities_plain_fp64(cf.handle, vp(uvw), R, fr.ctypes.data_as(ctypes.c_void_p), C, 0, C, None,
                                          None, vp(v), vp(w), P, vp(g64), vp(sw), st)
    e[1].record()
    assert rc == 0, lib.awg_last_error()
    g_err = float(torch.linalg.vector_norm(g64 - g_o) / torch.linalg.vector_norm(g_o))
    g64.copy_(g_o)
    e[2].record()
    rc = lib.degrid_visibilities_plain_fp64(cf.handle, vp(uvw), R, fr.ctypes.data_as(ctypes.c_void_p), C, 0, C, None,
                                            None, vp(g64), vp(out), P, st)
    e[3].record()
    assert rc == 0, lib.awg_last_error()
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1]) + e[2].elapsed_time(e[3])
    d_o = torch.as_tensor(cb["degrid"], device=dev).reshape(out.shape)
    d_err = float(torch.linalg.vector_norm(out.to(torch.complex128) - d_o) / torch.linalg.vector_norm(d_o))
    n_vis = R * C * P
    cf.close()
    # its ceiling: the FP64 FMA rate of this GPU (8 FLOP per tap and pol, as for the FP32 path)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    o64 = torch.empty(sms * 8 * 256, dtype=torch.float64, device=dev)
    fl = ctypes.c_double()
    for _ in range(2):   # warm-up, then the timed launch
        e[0].record()
        assert lib.awg_fp64_fma_probe(vp(o64), sms * 8, 1 << 12, st, ctypes.byref(fl)) == 0
        e[1].record()
    torch.cuda.synchronize()
    fp64_peak = fl.value / (e[0].elapsed_time(e[1]) / 1e3) / 1e12
    taps = float(np.sum(cb["support"].astype(np.float64) ** 2))
    fp64_tflops = 2 * 8.0 * P * taps / (ms / 1e3) / 1e12
    return {"value": 2 * n_vis / (ms / 1e3), "unit": "visibilities/s", "grid_rel_rms": g_err, "degrid_rel_rms": d_err,
            "tflops": fp64_tflops, "fp64_fma_peak_tflops": fp64_peak, "frac_of_fp64_peak": fp64_tflops / fp64_peak,
            "sample": "the cpu_baseline sample: one FP64 launch per channel over full CF tables (CUDA events)"}


def reference_arm(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    # only the sampled integrations get visibilities (CPU DFT of the sky), the rest is never read
    full = rank_workload(1, 0, args.n_int or synth.CONFIGS[CONFIG]["n_int"], "cpu", with_vis=False)
    every = args.cpu_sample_every or 200
    ints = np.arange(0, full.n_int, every)
    rows = np.concatenate([np.arange(t * full.n_bl, (t + 1) * full.n_bl) for t in ints])
    wl = dataclasses.replace(full, uvw_m=full.uvw_m[rows].copy(), pa_rad=full.pa_rad[rows].copy(),
                             pa_bin=full.pa_bin[rows].copy(), n_int=len(ints))
    synth.fill_visibilities(wl, device="cpu")
    times = []
    info = None
    for i in range(args.warmup + args.steps):
        info = run_cpu_baseline(wl, 1)
        info["sample"] = info["sample"].replace("every 1th integration", f"every {every}th integration")
        if i >= args.warmup:
            times.append(info["seconds"])
    per_step = statistics.mean(times)
    value = info["value"] * info["seconds"] / per_step
    line = {"impl": "reference", "metric": "gridded+degridded visibilities/s", "value": value,
            "unit": "visibilities/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "W-projection, VLA A-array-like, 351 bl x 2000 int x 64 ch x 4 pol, "
                                   "64 w-planes, supports 8-64, OS 20, 4096^2 x 4 grid (bounded sample per step)"},
            "cpu_baseline": {"kind": "oracle", "cores": info["cores"], "sample": info["sample"], "value": value,
                             "unit": "visibilities/s"},
            "e2e": {"value": value, "unit": "visibilities/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def minor_cycle_bench(args):
    """Hogbom minor cycle on a 4096 x 4096 FP32 residual with an 8192 x 8192 PSF (every shift
    covered): iterations per second, and the HBM roofline of one iteration, whose algorithmic
    traffic is the window search (4 B per window pixel) plus the subtraction (residual read and
    written, PSF read: 12 B per image pixel)."""
    import torch

    import paper_2508_17187_gb300 as awg
    N, n_iter = 4096, 1000
    Np = 2 * N
    g = torch.Generator(device="cuda").manual_seed(7)
    r = torch.hypot(*torch.meshgrid(torch.arange(Np, device="cuda", dtype=torch.float32) - Np // 2,
                                    torch.arange(Np, device="cuda", dtype=torch.float32) - Np // 2, indexing="ij"))
    psf = (torch.exp(-r ** 2 / 8.0) + 0.15 * torch.cos(r / 2.5) * torch.exp(-r / 400.0)).contiguous()
    del r
    base = torch.randn((N, N), device="cuda", generator=g) * 0.01
    ys = torch.randint(N // 8, 7 * N // 8, (300,), generator=g, device="cuda")
    xs = torch.randint(N // 8, 7 * N // 8, (300,), generator=g, device="cuda")
    amp = torch.rand(300, generator=g, device="cuda") * 0.8 + 0.2
    for y, x, a in zip(ys.tolist(), xs.tolist(), amp.tolist()):
        base += a * psf[Np // 2 - y:Np // 2 - y + N, Np // 2 - x:Np // 2 - x + N]
    window = (N // 4, 3 * N // 4, N // 4, 3 * N // 4)
    res, model = base.clone(), torch.zeros_like(base)
    ws = awg.CleanWorkspace()
    for _ in range(3):                       # warm-up
        res.copy_(base)
        model.zero_()
        awg.clean_hogbom(res, model, psf, 50, 0.1, 0.0, window, ws)
    torch.cuda.synchronize()
    res.copy_(base)
    model.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    awg.clean_hogbom(res, model, psf, n_iter, 0.1, 0.0, window, ws)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    per_it = ms / n_iter
    nbytes = (window[1] - window[0]) * (window[3] - window[2]) * 4 + N * N * 12
    achieved = nbytes / (per_it / 1e3) / 1e9
    peak = measured_peaks().get("hbm_gbs")
    line = {"metric": "Hogbom minor-cycle iterations/s", "value": n_iter / (ms / 1e3), "unit": "iterations/s",
            "higher_is_better": True, "n_gpus": 1, "steps": n_iter, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "4096x4096 residual, 8192x8192 PSF, 300 sources, inner-half search window, gain 0.1"},
            "components": ws.components(), "us_per_iteration": per_it * 1e3,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if peak else None, "traffic": None,
                         "bytes_per_iteration": nbytes, "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)"}}
    print(json.dumps(line), flush=True)
    return 0


def calibrate_bench(args):
    """G-Jones calibration (Eq. VAvg, Eq. CalUpdateDir, Eq. CalUpdateModel) of the full W-projection
    workload: model visibilities from degridding a point-source model grid (Eq. VMod), observed data =
    per-antenna gains x model + 1% noise, solution intervals of 10 integrations x 16 channels for
    both parallel hands (200 x 4 x 2 solutions of 27 antennas).  Reports visibilities/s of the
    solve and the HBM roofline of its averaging pass (20 B per parallel-hand sample: V, M, w)."""
    import torch

    import paper_2508_17187_gb300 as awg
    n_int = args.n_int or synth.CONFIGS["wproj"]["n_int"]
    wl = rank_workload(1, 0, n_int, "cuda")
    N, P, R, C = wl.grid_n, wl.n_pol, wl.n_rows, wl.n_chan
    cf = awg.cf_set_create(**cf_kwargs(wl))
    uvw, freq = torch.as_tensor(wl.uvw_m, device="cuda"), torch.as_tensor(wl.freq_hz, device="cuda")
    plan = awg.plan_create(cf, uvw, freq)
    model = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    ii = ((torch.as_tensor(wl.sky_m) / wl.cell_rad).round().long() + N // 2).clamp(0, N - 1).cuda()
    jj = ((torch.as_tensor(wl.sky_l) / wl.cell_rad).round().long() + N // 2).clamp(0, N - 1).cuda()
    for p in (0, P - 1):
        model[ii, jj, p] = torch.as_tensor(wl.sky_flux, dtype=torch.complex64, device="cuda")
    awg.grid_normalize(cf, model, None, direction=1)
    mgrid = torch.fft.fftshift(torch.fft.fft2(torch.fft.ifftshift(model, dim=(0, 1)), dim=(0, 1)), dim=(0, 1)).contiguous()
    del model
    M = torch.empty((R, C, P), dtype=torch.complex64, device="cuda")
    awg.degrid_visibilities(cf, plan, mgrid, M)
    a1, a2 = synth.baseline_antennas(27)
    n_bl, sol_int, sol_chan = len(a1), 10, 16
    n_ts, n_fs = -(-n_int // sol_int), -(-C // sol_chan)
    g = torch.as_tensor(synth.antenna_gains((n_ts, n_fs, 2, 27), seed=5), device="cuda")
    rows = torch.arange(R, device="cuda")
    t_of = (rows // n_bl) // sol_int
    b_of = rows % n_bl
    A1, A2 = torch.as_tensor(a1, device="cuda")[b_of], torch.as_tensor(a2, device="cuda")[b_of]
    f_of = torch.arange(C, device="cuda") // sol_chan
    V = M.clone()
    gen = torch.Generator(device="cuda").manual_seed(1)
    sigma = 0.01 * float(M.abs().mean())
    for q, p in enumerate((0, P - 1)):
        fac = g[t_of[:, None], f_of[None, :], q, A1[:, None]] * torch.conj(g[t_of[:, None], f_of[None, :], q, A2[:, None]])
        V[:, :, p] = (M[:, :, p].to(torch.complex128) * fac).to(torch.complex64)
        del fac
    V += sigma * torch.complex(torch.randn(V.shape, device="cuda", generator=gen),
                               torch.randn(V.shape, device="cuda", generator=gen))
    W = wl.weight
    ant1, ant2 = torch.as_tensor(a1, device="cuda"), torch.as_tensor(a2, device="cuda")
    for _ in range(max(3, args.warmup)):
        G, its = awg.gcal_solve(V, M, W, ant1, ant2, 27, sol_int, sol_chan, alpha=0.5, delta=1e-10, max_iter=200)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        G, its = awg.gcal_solve(V, M, W, ant1, ant2, 27, sol_int, sol_chan, alpha=0.5, delta=1e-10, max_iter=200)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    gt = g * torch.conj(g[..., :1]) / g[..., :1].abs()
    err = float((G - gt).abs().max())
    nbytes = R * C * 2 * (8 + 8 + 4)
    peak = measured_peaks().get("hbm_gbs")
    achieved = nbytes / (ms / 1e3) / 1e9
    line = {"metric": "calibrated visibilities/s (G-Jones solve)", "value": R * C * P / (ms / 1e3),
            "unit": "visibilities/s", "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "dtype": "f32 (compensated interval sums), f64 gain iteration", "data": "synthetic",
            "config": {"workload": f"W-projection data {R} rows x {C} channels x {P} pols, model from degridding; "
                                   f"solution intervals {sol_int} integrations x {sol_chan} channels, 2 hands, 27 antennas",
                       "solutions": n_ts * n_fs * 2},
            "iterations_max": int(its.max()), "iterations_mean": float(its.float().mean()),
            "max_gain_error": err,
            "roofline": {"bound": "hbm", "kernel": "gcal_solve (averaging pass + gain iterations)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if peak else None, "traffic": None,
                         "bytes_per_step": nbytes, "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)"}}
    print(json.dumps(line), flush=True)
    return 0


def forward_model_bench(args):
    """Differentiable forward model: 1024^2 FP32 sky -> taper, F -> D to 5.01M visibilities (351
    baselines x 223 integrations x 64 channels, 1 pol, W-projection supports 8-32).

    One step is ten steepest-descent major cycles (Eq. ResIm, Eq. ModelUpdate) from an empty model,
    through the public `autograd.major_cycle`: each cycle grids the data residual for the residual
    image and degrids the updated model once, the residual V - D F I formed in place, which gives
    the cycle's chi^2 and the next cycle's residual; with the first residual a step moves
    21 x 5.01M visibilities through the library.
    The step size 1 / lambda_max (power iteration) is found once, before the timed region.  The
    line also times the chi^2 gradient through autograd (forward: taper, F, DegridFn; backward:
    gridding, F^H) and each operator alone; the roofline is that of the slower operator's launches
    (FP32 FMA, 8 S^2 FLOP per visibility) against the sustained FP32 FMA probe rate."""
    import torch

    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300 import _lib
    from paper_2508_17187_gb300 import autograd as ag
    lib = _lib.load()
    n_cycles = 10
    wl = synth.make_workload("autograd", vis_device="cuda")
    N, P, R, C = wl.grid_n, wl.n_pol, wl.n_rows, wl.n_chan
    vis, wt = wl.vis, wl.weight
    cf = awg.cf_set_create(**cf_kwargs(wl))
    uvw, freq = torch.as_tensor(wl.uvw_m, device="cuda"), torch.as_tensor(wl.freq_hz, device="cuda")
    tuned = None
    if not args.no_autotune:
        tuned, _ = cf.autotune(uvw, freq, n_pol=P)
    plan = awg.plan_create(cf, uvw, freq)
    kept, dropped, sum_taps = plan.stats()
    fm = ag.ForwardModel(cf, plan, n_pol=P)
    mask = ag.inner_mask(N)
    gain = 1.0 / ag.largest_eigenvalue(fm, wt, mask)
    stream = torch.cuda.current_stream()

    # chi^2 gradient through autograd (one D forward, one G backward)
    sky = torch.as_tensor(synth.gaussian_blob_sky(N, wl.cell_rad, wl.sky_l, wl.sky_m, wl.sky_flux),
                          device="cuda").float()[..., None] * 0.5

    def gradient():
        x = sky.clone().requires_grad_(True)
        (g,) = torch.autograd.grad(ag.chi2(fm(x), vis, wt), x)
        return g

    # each operator alone, on the launching stream
    grid = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda")
    sumwt = torch.zeros(P, dtype=torch.float64, device="cuda")
    mgrid = ag.image_to_grid(sky, fm.inv_taper2d).contiguous()
    vis_out = torch.empty_like(vis)

    # the workload's inputs (60 MB) fit in the 129 MB L2: every timed repetition starts after a
    # 256 MB write, outside its events
    l2_flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def timed(fn, reps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda.synchronize()
        for b, e in evs:
            l2_flush.zero_()
            b.record(stream)
            fn()
            e.record(stream)
        torch.cuda.synchronize()
        return sum(b.elapsed_time(e) for b, e in evs) / reps

    def op_grid():
        grid.zero_()
        sumwt.zero_()
        awg.grid_visibilities(cf, plan, vis, wt, grid, sumwt)

    def op_degrid():
        awg.degrid_visibilities(cf, plan, mgrid, vis_out)

    for _ in range(max(3, args.warmup)):
        op_grid()
        op_degrid()
        gradient()
        ag.major_cycle(fm, vis, wt, n_iter=1, gain=gain, mask=mask)
    reps = max(args.steps, 5)
    g_ms, d_ms = timed(op_grid, reps), timed(op_degrid, reps)
    grad_ms = timed(gradient, reps)

    hist = []

    def cycles():
        _, h = ag.major_cycle(fm, vis, wt, n_iter=n_cycles, gain=gain, mask=mask)
        hist[:] = h

    launches0 = lib.awg_kernel_launches()
    with ClockSampler(0) as clocks:
        ms = timed(cycles, args.steps)
    launches = lib.awg_kernel_launches() - launches0

    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    cs = clocks.summary()
    fma = measure_fma_peak(lib, sms, "cuda")
    peak_tf = fma["sustained_tflops"]
    flop = 8.0 * P * sum_taps
    n_vis = R * C * P
    ops = {name: {"ms": t, "visibilities_per_s": n_vis / (t / 1e3), "tflops": flop / (t / 1e3) / 1e12,
                  "frac_of_fp32_peak": flop / (t / 1e3) / 1e12 / peak_tf}
           for name, t in (("grid", g_ms), ("degrid", d_ms))}
    dom = "grid" if g_ms >= d_ms else "degrid"
    achieved = ops[dom]["tflops"]
    vis_per_step = (2 * n_cycles + 1) * n_vis
    line = {"metric": "major cycles/s (differentiable forward model)", "value": n_cycles / (ms / 1e3),
            "unit": "major cycles/s", "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"differentiable forward model: {N}x{N} FP32 sky -> F -> D to {n_vis} "
                                   f"visibilities ({wl.n_bl} baselines x {wl.n_int} integrations x {C} channels, "
                                   f"{P} pol), W-projection supports 8-{wl.max_support}; one step = {n_cycles} "
                                   "major cycles (1 D + 1 G each, plus the first residual)",
                       "kept_samples": kept, "dropped_samples": dropped, "mean_taps": sum_taps / max(kept, 1),
                       "step_size": gain, "l2": "flushed: a 256 MB write before every timed repetition",
                       "kernel_config_per_support": tuned,
                       "residual": "formed by degridding in place (AWG_DEGRID_SUBTRACT)"},
            "visibilities_per_s": vis_per_step / (ms / 1e3),
            "ms_per_major_cycle": ms / n_cycles,
            "gradient_ms": grad_ms,
            "chi2_first_last": [hist[0], hist[-1]] if hist else None,
            "ops": ops,
            "roofline": {"bound": "alu", "kernel": f"{dom}_visibilities (all supports)", "achieved": achieved,
                         "peak": peak_tf, "unit": "TFLOP/s", "frac": achieved / peak_tf, "traffic": None,
                         "peak_basis": "measured: sustained FP32 FMA rate of awg_fp32_fma_probe"},
            "clocks": {k: cs[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)
    return 0


def precision_sweep(args):
    """Per-variant dirty-image and degridding error against the FP64 oracle, and throughput.

    Workload: the W-projection configuration with `--n-int` integrations (default 100, 9M
    visibilities) so that the oracle's FP64 gridding of every sample takes seconds.  Image error:
    relative RMS of the dirty image over the inner half of the field (where the PS taper is above
    0.25); degridding error: relative RMS of D applied to one common model grid."""
    import ctypes

    import torch

    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300 import _lib
    from oracle import cf as ocf
    from oracle import image as oimage
    from oracle import index as oindex
    from oracle import ops as oops
    lib = _lib.load()
    n_int = args.n_int or 100
    wl = rank_workload(1, 0, n_int, "cuda")
    N, P, R, C = wl.grid_n, wl.n_pol, wl.n_rows, wl.n_chan
    op = ocf.CFParams(grid_n=N, cell_rad=wl.cell_rad, oversampling=wl.oversampling, ps_support=wl.ps_support,
                      use_w=True, n_wplanes=wl.n_wplanes, w_max_lambda=wl.w_max_lambda, max_support=wl.max_support)
    idx = oindex.sample_index(op, wl.uvw_m, wl.freq_hz)
    buf, off, _ = ocf.flatten_cf_set(op, ocf.cf_set(op, which=set(np.unique(idx.cf[idx.valid]).tolist())))
    vis_h = wl.vis.cpu().numpy().reshape(-1, P)
    wt_h = wl.weight.cpu().numpy().reshape(-1, P)
    g_o, sw_o = oops.grid(idx, buf, off, op.oversampling, N, vis_h, wt_h)
    img_o = oimage.dirty_image(g_o, sw_o, wl.ps_support)[N // 4:3 * N // 4, N // 4:3 * N // 4]
    rng = np.random.default_rng(7)
    model = np.zeros((N, N, P))
    pts = rng.integers(N // 4, 3 * N // 4, (50, 2))
    model[pts[:, 0], pts[:, 1], :] = rng.uniform(0.1, 1.0, (50, 1))
    mgrid = oimage.model_to_grid(model, wl.ps_support)
    d_o = oops.degrid(idx, buf, off, op.oversampling, mgrid)
    mgrid_d = torch.as_tensor(mgrid.astype(np.complex64)).cuda()
    uvw = torch.as_tensor(wl.uvw_m).cuda()
    freq = torch.as_tensor(wl.freq_hz).cuda()
    base = dict(grid_n=N, cell_rad=wl.cell_rad, oversampling=wl.oversampling, ps_support=wl.ps_support, use_w=True,
                n_wplanes=wl.n_wplanes, w_max_lambda=wl.w_max_lambda, max_support=wl.max_support)
    variants = [("cf fp32 separable, grid fp32", dict(separable=True), 0),
                ("cf fp32 full tables, grid fp32", dict(separable=False), 0),
                ("cf bf16 full tables, grid fp32", dict(separable=False, cf_dtype=awg.AWG_CF_BF16), 0),
                ("cf fp32 separable, grid fp32 + Kahan flush", dict(separable=True), awg.AWG_GRID_KAHAN),
                ("cf fp32 separable, grid fp64 flush", dict(separable=True), awg.AWG_GRID_FP64)]
    n_vis = R * C * P

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for name, kw, flags in variants:
        cf = awg.cf_set_create(**base, **kw)
        plan = awg.plan_create(cf, uvw, freq)
        dt = torch.complex128 if flags & awg.AWG_GRID_FP64 else torch.complex64
        g = torch.zeros((N, N, P), dtype=dt, device="cuda")
        glo = torch.zeros((N, N, P), dtype=torch.complex64, device="cuda") if flags & awg.AWG_GRID_KAHAN else None
        sw = torch.zeros(P, dtype=torch.float64, device="cuda")

        def do_grid():
            g.zero_()
            sw.zero_()
            if glo is not None:
                glo.zero_()
            awg.grid_visibilities(cf, plan, wl.vis, wl.weight, g, sw, grid_lo=glo, flags=flags)
        ms = timed(do_grid)
        gh = g.to(torch.complex128) + (glo.to(torch.complex128) if glo is not None else 0)
        img = oimage.dirty_image(gh.cpu().numpy(), sw.cpu().numpy(), wl.ps_support)[N // 4:3 * N // 4, N // 4:3 * N // 4]
        err_img = float(np.linalg.norm(img - img_o) / np.linalg.norm(img_o))
        out = torch.empty_like(wl.vis)
        ms_d = timed(lambda: awg.degrid_visibilities(cf, plan, mgrid_d, out))
        err_d = float(np.linalg.norm(out.cpu().numpy().reshape(-1, P) - d_o) / np.linalg.norm(d_o))
        print(json.dumps({"variant": name, "image_rel_rms": err_img, "degrid_rel_rms": err_d,
                          "grid_visibilities_per_s": n_vis / (ms / 1e3), "degrid_visibilities_per_s": n_vis / (ms_d / 1e3),
                          "workload": f"W-projection, {n_int} integrations x 351 baselines x {C} channels x {P} pols"}),
              flush=True)
    # the plain FP64 per-channel launch on the same data
    cf = awg.cf_set_create(**base, separable=False)
    g64 = torch.zeros((N, N, P), dtype=torch.complex128, device="cuda")
    sw = torch.zeros(P, dtype=torch.float64, device="cuda")
    fr = np.ascontiguousarray(wl.freq_hz)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())

    def plain():
        g64.zero_()
        sw.zero_()
        rc = lib.grid_visibilities_plain_fp64(cf.handle, vp(uvw), R, fr.ctypes.data_as(ctypes.c_void_p), C, 0, C,
                                              None, None, vp(wl.vis), vp(wl.weight), P, vp(g64), vp(sw), st)
        assert rc == 0, lib.awg_last_error()
    ms = timed(plain, reps=1)
    img = oimage.dirty_image(g64.cpu().numpy(), sw.cpu().numpy(), wl.ps_support)[N // 4:3 * N // 4, N // 4:3 * N // 4]
    out = torch.empty_like(wl.vis)
    g64.copy_(mgrid_d.to(torch.complex128))
    ms_d = timed(lambda: lib.degrid_visibilities_plain_fp64(cf.handle, vp(uvw), R, fr.ctypes.data_as(ctypes.c_void_p),
                                                            C, 0, C, None, None, vp(g64), vp(out), P, st), reps=1)
    err_d = float(np.linalg.norm(out.cpu().numpy().reshape(-1, P) - d_o) / np.linalg.norm(d_o))
    print(json.dumps({"variant": "plain FP64 per-channel launches (baseline)",
                      "image_rel_rms": float(np.linalg.norm(img - img_o) / np.linalg.norm(img_o)),
                      "degrid_rel_rms": err_d, "grid_visibilities_per_s": n_vis / (ms / 1e3),
                      "degrid_visibilities_per_s": n_vis / (ms_d / 1e3)}), flush=True)
    return 0


WORKLOADS = {
    "wproj": "W-projection: 351 baselines x 2000 integrations x 64 channels (2-4 GHz) x 4 pols per rank, 64 w-planes, "
             "CF supports 8-64, oversampling 20, 4096x4096x4 c64 grid",
    "awproj": "batched AW-projection: 351 baselines x 2000 integrations x 64 channels (2-4 GHz) x 4 pols per rank, "
              "20 PA bins x 32 w-planes x 16 sub-bands = 10,240 A-term CFs (20,160 signed), supports 8-64, "
              "oversampling 20, 4096x4096x4 c64 grid",
}


def cf_kwargs(wl, full_pol=False) -> dict:
    """cf_set_create arguments of a workload (full_pol: squinted feeds, leakage 0.04, 12 Mueller
    elements)."""
    kw = dict(grid_n=wl.grid_n, cell_rad=wl.cell_rad, oversampling=wl.oversampling, ps_support=wl.ps_support,
              use_w=wl.use_w, n_wplanes=wl.n_wplanes, w_max_lambda=wl.w_max_lambda, max_support=wl.max_support)
    if wl.use_a:
        kw.update(use_a=True, n_pa_bins=wl.n_pa_bins, pa_bin_centers_rad=np.asarray(wl.pa_bin_centers),
                  n_subbands=wl.n_subbands, subband_freq_hz=np.asarray(wl.subband_freq_hz))
    if full_pol:
        kw.update(use_pol=True, squint_rad=2e-4, leakage=0.04 * np.exp(0.9j), mueller_threshold=0.01)
    return kw


def mosaic_row_phase(wl) -> np.ndarray:
    """Per-row (dl, dm) of a two-field mosaic: pointings on alternating integrations 30 / 20 cells
    from the image centre, plus a per-row pointing offset of up to 2 cells."""
    rng = np.random.default_rng(4)
    field = (np.arange(wl.n_rows) // wl.n_bl) % 2
    dl = np.where(field == 0, 30.0, -30.0) * wl.cell_rad
    dm = np.where(field == 0, -20.0, 20.0) * wl.cell_rad
    jit = rng.uniform(-2.0, 2.0, (wl.n_rows, 2)) * wl.cell_rad
    return np.stack([dl + jit[:, 0], dm + jit[:, 1]], -1)


def aw_side_measure(args, dev: str, peak_tf: float) -> dict:
    """The batched AW-projection step (Tab. AWP-CFSETUP AW-Projection: a CF per signed w-plane, PA bin
    and sub-band, each a few outer-product terms; the same 179.7M visibilities as the headline), timed
    like the headline (plan update, gridding, normalisation, degridding; CUDA events on the
    launching stream) so that the default line carries a measured AW figure.  Fractions are of the
    FP32 FMA peak by the method's FLOP (8 P S^2 per visibility and operator); executed_tflops counts
    what the fused kernels execute ((terms + P) / P of it)."""
    import torch

    import paper_2508_17187_gb300 as awg
    wl = synth.make_workload("awproj", vis_device=dev)
    P, N = wl.n_pol, wl.grid_n
    t0 = time.perf_counter()
    cf = awg.cf_set_create(**cf_kwargs(wl))
    cf_s = time.perf_counter() - t0
    uvw, freq = torch.as_tensor(wl.uvw_m, device=dev), torch.as_tensor(wl.freq_hz, device=dev)
    pa_bin = torch.as_tensor(wl.pa_bin, device=dev)
    chan_sb = torch.as_tensor(wl.chan_subband, device=dev)
    tuned = None
    if not args.no_autotune:
        tuned, _ = cf.autotune(uvw, freq, pa_bin, chan_sb, n_pol=P)
    plan = awg.plan_create(cf, uvw, freq, pa_bin, chan_sb)
    kept, dropped, sum_taps = plan.stats()
    grid = torch.zeros((N, N, P), dtype=torch.complex64, device=dev)
    model = torch.zeros_like(grid)
    sumwt = torch.zeros(P, dtype=torch.float64, device=dev)
    out = torch.empty_like(wl.vis)
    stream = torch.cuda.current_stream()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]

    def step(e=None):
        if e: e[0].record(stream)
        plan.update(uvw, freq, pa_bin, chan_sb)
        if e: e[1].record(stream)
        grid.zero_()
        sumwt.zero_()
        awg.grid_visibilities(cf, plan, wl.vis, wl.weight, grid, sumwt)
        if e: e[2].record(stream)
        awg.grid_normalize(cf, grid, sumwt, direction=0)
        if e: e[3].record(stream)
        awg.degrid_visibilities(cf, plan, model, out)
        if e: e[4].record(stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    for e in ev:
        step(e)
    torch.cuda.synchronize()
    ms = statistics.mean(e[0].elapsed_time(e[4]) for e in ev)
    g_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    d_ms = statistics.mean(e[3].elapsed_time(e[4]) for e in ev)
    n_vis = wl.n_rows * wl.n_chan * P
    flop = 8.0 * P * sum_taps
    mult = (cf.fused_terms + P) / P if cf.fused_terms else cf.rank
    ops = {k: {"ms": t, "visibilities_per_s": n_vis / (t / 1e3), "tflops": flop / (t / 1e3) / 1e12,
               "frac_of_fp32_peak": flop / (t / 1e3) / 1e12 / peak_tf,
               "executed_tflops": mult * flop / (t / 1e3) / 1e12} for k, t in (("grid", g_ms), ("degrid", d_ms))}
    return {"metric": "gridded+degridded visibilities/s", "value": 2 * n_vis / (ms / 1e3), "unit": "visibilities/s",
            "ms_per_step": ms, "steps": args.steps,
            "workload": f"batched AW-projection: {wl.n_bl} baselines x {wl.n_int} integrations x {wl.n_chan} channels "
                        f"x {P} pols, {cf.n_cf} CFs ({wl.n_wplanes} w-planes x {wl.n_pa_bins} PA bins x "
                        f"{wl.n_subbands} sub-bands), {cf.rank} terms each, supports up to {wl.max_support}, "
                        f"{N}x{N}x{P} grid",
            "cf_terms": cf.rank, "fused_terms": cf.fused_terms, "cf_build_s": cf_s, "kept_samples": kept,
            "mean_taps": sum_taps / max(kept, 1), "kernel_config_per_support": tuned, "ops": ops}


def main():
    global CONFIG
    args = parse()
    CONFIG = args.config
    if args.full_pol:
        if CONFIG != "awproj":
            raise SystemExit("--full-pol needs --config awproj")
        WORKLOAD_OVERRIDES.update(n_pa=4, n_sb=4)
    if args.impl == "reference":
        return reference_arm(args)
    if args.precision_sweep:
        return precision_sweep(args)
    if args.minor_cycle:
        return minor_cycle_bench(args)
    if args.calibrate:
        return calibrate_bench(args)
    if args.forward_model:
        return forward_model_bench(args)
    import torch
    import torch.distributed as dist

    import paper_2508_17187_gb300 as awg
    from paper_2508_17187_gb300 import _lib

    world, rank, local = dist_env()
    torch.cuda.set_device(local)   # before the process group, so NCCL binds this rank's GPU
    if world > 1:
        dist.init_process_group("nccl")
    dev = f"cuda:{local}"
    n_int = args.n_int or synth.CONFIGS[CONFIG]["n_int"]
    wl = rank_workload(world, rank, n_int, dev)
    N, P = wl.grid_n, wl.n_pol
    R, C = wl.n_rows, wl.n_chan
    lib = _lib.load()

    t_cf = time.perf_counter()
    cf = awg.cf_set_create(**cf_kwargs(wl, args.full_pol))
    t_cf = time.perf_counter() - t_cf
    uvw = torch.as_tensor(wl.uvw_m, device=dev)
    freq = torch.as_tensor(wl.freq_hz, device=dev)
    pa_bin = torch.as_tensor(wl.pa_bin, device=dev) if wl.use_a else None
    chan_sb = torch.as_tensor(wl.chan_subband, device=dev) if wl.use_a else None
    vis, wt = wl.vis, wl.weight
    tuned, t_tune, tune_ms = None, None, None
    if args.kernel_config:
        tuned = {}
        for item in args.kernel_config.split(","):
            sup, kcfg = (int(v) for v in item.split(":"))
            cf.choose(sup, kcfg)
            tuned[str(sup)] = kcfg
    elif not args.no_autotune:
        t_tune = time.perf_counter()
        tuned, tune_ms = cf.autotune(uvw, freq, pa_bin, chan_sb, n_pol=wl.n_pol)
        tune_ms = {S: [round(t, 3) for t in v] for S, v in tune_ms.items()}
        t_tune = time.perf_counter() - t_tune
    plan = awg.plan_create(cf, uvw, freq, pa_bin, chan_sb)
    if args.mosaic:
        plan.set_row_phase(torch.as_tensor(mosaic_row_phase(wl), device=dev), uvw, freq)
    kept, dropped, sum_taps = plan.stats()
    grid = torch.zeros((N, N, P), dtype=torch.complex64, device=dev)
    sumwt = torch.zeros(P, dtype=torch.float64, device=dev)
    # model grid for the degridding half: F of a taper-corrected model image (one cuFFT call here,
    # outside the timed region; the FFT is not part of the library)
    model = torch.zeros((N, N, P), dtype=torch.complex64, device=dev)
    ii = ((torch.as_tensor(wl.sky_m) / wl.cell_rad).round().long() + N // 2).clamp(0, N - 1)
    jj = ((torch.as_tensor(wl.sky_l) / wl.cell_rad).round().long() + N // 2).clamp(0, N - 1)
    for p in (0, P - 1):
        model[ii.to(dev), jj.to(dev), p] = torch.as_tensor(wl.sky_flux, dtype=torch.complex64, device=dev)
    awg.grid_normalize(cf, model, None, direction=1)
    mgrid = torch.fft.fftshift(torch.fft.fft2(torch.fft.ifftshift(model, dim=(0, 1)), dim=(0, 1)), dim=(0, 1))
    mgrid = mgrid.contiguous()
    del model
    vis_out = torch.empty_like(vis)
    stream = torch.cuda.current_stream()

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    op_ms = {"plan": [], "grid": [], "normalize": [], "degrid": []}

    def step(record=False):
        if record:
            ev[0].record(stream)
        plan.update(uvw, freq, pa_bin, chan_sb)
        if record:
            ev[1].record(stream)
        grid.zero_()
        sumwt.zero_()
        awg.grid_visibilities(cf, plan, vis, wt, grid, sumwt)
        if record:
            ev[2].record(stream)
        if world > 1:
            dist.all_reduce(torch.view_as_real(grid))
            dist.all_reduce(sumwt)
        awg.grid_normalize(cf, grid, sumwt, direction=0)
        if record:
            ev[3].record(stream)
        awg.degrid_visibilities(cf, plan, mgrid, vis_out)
        if record:
            ev[4].record(stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        step()
    barrier()
    # per-operator timing pass (events on the launching stream), outside the headline timing
    for _ in range(args.steps):
        step(record=True)
        torch.cuda.synchronize()
        op_ms["plan"].append(ev[0].elapsed_time(ev[1]))
        op_ms["grid"].append(ev[1].elapsed_time(ev[2]))
        op_ms["normalize"].append(ev[2].elapsed_time(ev[3]))
        op_ms["degrid"].append(ev[3].elapsed_time(ev[4]))
    barrier()
    launches0 = lib.awg_kernel_launches()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier()
        t_start.record(stream)
        for _ in range(args.steps):
            step()
        t_end.record(stream)
        barrier()
    launches = lib.awg_kernel_launches() - launches0
    ms = t_start.elapsed_time(t_end) / args.steps
    # the same step captured once as a CUDA graph and replayed (single rank: no collective inside)
    graph_ms = None
    if world == 1:
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            step()
        stream.wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        graph.replay()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            graph.replay()
        g1.record(stream)
        torch.cuda.synchronize()
        graph_ms = g0.elapsed_time(g1) / args.steps
        del graph
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    vis_per_step = 2 * R * C * P * world
    value = vis_per_step / (ms / 1e3)

    # end to end through the public API with host buffers: H2D of the step's inputs from pinned
    # memory, the step, D2H of its results (degridded visibilities, gridded plane, weight sums)
    e2e = None
    if not args.no_e2e:
        h_vis = vis.cpu().pin_memory()
        h_wt = wt.cpu().pin_memory()
        h_uvw = uvw.cpu().pin_memory()
        h_freq = freq.cpu().pin_memory()
        h_pa = pa_bin.cpu().pin_memory() if pa_bin is not None else None
        h_sb = chan_sb.cpu().pin_memory() if chan_sb is not None else None
        h_out = torch.empty(vis_out.shape, dtype=vis_out.dtype).pin_memory()
        h_grid = torch.empty(grid.shape, dtype=grid.dtype).pin_memory()
        h_sw = torch.empty(sumwt.shape, dtype=sumwt.dtype).pin_memory()

        # Two buffer sets and three streams: step k+1's inputs are copied in (s_in) while step k
        # computes, and step k's results are copied out (s_out) while step k+1 computes.  Each
        # copy waits for the compute that last used its buffers; every step still copies all its
        # inputs in and all its results out inside the timed region.
        s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        ins = [(vis, wt, uvw, freq, pa_bin, chan_sb),
               tuple(torch.empty_like(t) if t is not None else None for t in (vis, wt, uvw, freq, pa_bin, chan_sb))]
        outs = [(vis_out, grid, sumwt), (torch.empty_like(vis_out), torch.empty_like(grid), torch.empty_like(sumwt))]
        ev_in, ev_comp, ev_out = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))
        k_step = [0]

        def e2e_step():
            i = k_step[0] % 2
            k_step[0] += 1
            v, w, u, f, pa, sb = ins[i]
            vo, g, sw = outs[i]
            s_in.wait_event(ev_comp[i])
            with torch.cuda.stream(s_in):
                v.copy_(h_vis, non_blocking=True)
                w.copy_(h_wt, non_blocking=True)
                u.copy_(h_uvw, non_blocking=True)
                f.copy_(h_freq, non_blocking=True)
                if h_pa is not None:
                    pa.copy_(h_pa, non_blocking=True)
                    sb.copy_(h_sb, non_blocking=True)
                ev_in[i].record(s_in)
            stream.wait_event(ev_in[i])
            stream.wait_event(ev_out[i])
            plan.update(u, f, pa, sb)
            g.zero_()
            sw.zero_()
            awg.grid_visibilities(cf, plan, v, w, g, sw)
            if world > 1:
                dist.all_reduce(torch.view_as_real(g))
                dist.all_reduce(sw)
            awg.grid_normalize(cf, g, sw, direction=0)
            awg.degrid_visibilities(cf, plan, mgrid, vo)
            ev_comp[i].record(stream)
            s_out.wait_event(ev_comp[i])
            with torch.cuda.stream(s_out):
                h_out.copy_(vo, non_blocking=True)
                h_grid.copy_(g, non_blocking=True)
                h_sw.copy_(sw, non_blocking=True)
                ev_out[i].record(s_out)

        for _ in range(2):
            e2e_step()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_event(e0)
        for _ in range(args.steps):
            e2e_step()
        for x in ev_out:
            stream.wait_event(x)
        e1.record(stream)
        barrier()
        e_ms = e0.elapsed_time(e1) / args.steps
        if world > 1:
            tt = torch.tensor([e_ms], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e_ms = float(tt.item())
        h2d = vis.numel() * 8 + wt.numel() * 4 + uvw.numel() * 8 + freq.numel() * 8
        if pa_bin is not None:
            h2d += pa_bin.numel() * 4 + chan_sb.numel() * 4
        d2h = vis_out.numel() * 8 + grid.numel() * 8 + sumwt.numel() * 8
        e2e = {"value": vis_per_step / (e_ms / 1e3), "unit": "visibilities/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e_ms}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    peaks = measured_peaks()
    cs = clocks.summary()
    max_mhz = cs["sm_max_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    nominal_tf = fp32_alu_peak_tflops(sms, max_mhz)
    fma = measure_fma_peak(lib, sms, dev)
    # the kernels run inside a long step: the sustained probe rate is their ceiling
    peak_tf = fma["sustained_tflops"]
    # one complex MAC = 4 FP32 FMA = 8 FLOP per tap and pol product; a full-polarisation set applies
    # one CF per kept Mueller element instead of one per pol
    flop = 8.0 * (len(cf.mueller()) or P) * sum_taps
    g_ms = statistics.mean(op_ms["grid"])
    d_ms = statistics.mean(op_ms["degrid"])
    dom, dom_ms = ("grid", g_ms) if g_ms >= d_ms else ("degrid", d_ms)
    achieved = flop / (dom_ms / 1e3) / 1e12
    ops = {}
    for op_name, op_t in (("grid", g_ms), ("degrid", d_ms)):
        ops[op_name] = {"ms": op_t, "visibilities_per_s": R * C * P / (op_t / 1e3),
                        "cf_gmac_per_s": P * sum_taps / (op_t / 1e3) / 1e9,
                        "tflops": flop / (op_t / 1e3) / 1e12, "frac_of_fp32_peak": flop / (op_t / 1e3) / 1e12 / peak_tf}
    line = {
        "metric": "gridded+degridded visibilities/s", "value": value, "unit": "visibilities/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic VLA A-array-like uvw, 200 point sources + 1 mJy noise, natural weights",
        "config": {"workload": WORKLOADS[CONFIG] + (" (full polarisation: 4 PA bins x 4 sub-bands, "
                                                     f"{len(cf.mueller())} Mueller elements)" if args.full_pol else "")
                   + (" (two-field mosaic: per-row phase centres)" if args.mosaic else ""),
                   "cf_terms": max(cf.rank, 1), "cf_storage":
                   "separable factors" if cf.separable else "full tables", "cf_build_s": t_cf,
                   "kernel_config_per_support": tuned, "autotune_s": t_tune,
                   "autotune_ms_per_config": tune_ms,
                   "visibilities_per_step": vis_per_step, "kept_samples": kept, "dropped_samples": dropped,
                   "mean_taps": sum_taps / max(kept, 1), "l2": "inputs larger than L2 (2.7 GB per step)",
                   "parallelism": f"dp{world}" if world > 1 else "single GPU"},
        "cf_gmac_per_s": 2 * P * sum_taps * world / (ms / 1e3) / 1e9,
        "ops_ms": {k: statistics.mean(v) for k, v in op_ms.items()},
        "cuda_graph": None if graph_ms is None else {"ms_per_step": graph_ms,
                                                     "value": vis_per_step / (graph_ms / 1e3)},
        "ops": ops,
        "roofline": {"bound": "alu", "kernel": f"{dom}_visibilities (all supports)", "achieved": achieved,
                     "peak": peak_tf, "unit": "TFLOP/s", "frac": achieved / peak_tf,
                     "traffic": measured_traffic(dom, args.mosaic or args.full_pol),
                     "peak_basis": "measured: sustained FP32 FMA rate of awg_fp32_fma_probe "
                                   f"({fma['launches']} launches of {fma['launch_ms']:.0f} ms)",
                     "peak_burst": fma["burst_tflops"],
                     "peak_nominal": nominal_tf,
                     "peak_nominal_basis": f"{sms} SMs x 128 FP32 lanes x 2 FLOP x {max_mhz:.0f} MHz (max SM clock)",
                     "note": "achieved = the method's FLOP (8 P sum S^2 per operator) over the operator's time, against "
                             "the FP32 FMA pipe; supports on configuration 3 run the product on the tensor cores "
                             "(3xTF32 splits of padded windows: several times the method's FLOP on the tensor pipe)",
                     "kernel_config_per_support": tuned},
        "clocks": {k: cs[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "gpu_launches": int(launches),
        "e2e": e2e,
    }
    if cf.separable and cf.rank > 1:
        # fused kernels form each tap's CF value from its terms (4 FMA per term) and apply it to the
        # P pols (4 FMA per pol): (terms + P) / P x the method's arithmetic, and a full-polarisation
        # set runs 3 such 4-pol passes for its n_elem elements: 3 (terms + 4) / n_elem x; otherwise
        # one rank-1 record runs per (sample, term): terms x
        n_el = len(cf.mueller())
        if cf.fused_terms:
            mult = 3 * (cf.fused_terms + 4) / n_el if n_el else (cf.fused_terms + P) / P
        else:
            mult = cf.rank
        line["executed_tflops"] = {k: mult * ops[k]["tflops"] for k in ops}
    if not args.no_cpu_baseline and CONFIG == "wproj" and not args.mosaic:
        host_wl = dataclasses.replace(wl, vis=vis.cpu().numpy(), weight=wt.cpu().numpy())
        cb = run_cpu_baseline(host_wl, args.cpu_sample_every or 40, single_thread=True)
        line["accuracy"] = sample_accuracy(cf, wl, vis, wt, cb, dev)
        line["plain_fp64_gpu"] = plain_fp64_on_sample(wl, vis, wt, cb, dev)
        for k in ("seconds", "rows", "grid", "sumwt", "degrid", "support"):
            cb.pop(k)
        line["cpu_baseline"] = cb
    if CONFIG == "wproj" and world == 1 and not (args.no_aw or args.mosaic or args.n_int or args.kernel_config):
        line["awproj"] = aw_side_measure(args, dev, peak_tf)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
