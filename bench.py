"""Benchmark of the 7DGS render path on GB300: Mpix/s and FPS of the 800x800 / 300k-Gaussian
forward render, plus fwd+bwd it/s, through libsdgs's C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one full forward render of one camera view (conditional slicing + projection + SH,
tile binning with the depth/tile radix sort, compositing) of the 300k-Gaussian object-scale scene
at 800x800; the camera cycles over the scene's 100 orbit cameras, each at its own time t.  Rank 0
prints one JSON line.  With N > 1 (torchrun), every rank renders its own cameras (replicas: the
render path needs no collective) and the value is the images of all ranks over the slowest rank's
time.  `--impl reference` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import synth  # noqa: E402

METRIC = "Mpix/s & FPS at 800×800/300k Gaussians; fwd+bwd it/s; p50/p99 serving latency"
WORKLOAD = ("config 1: 300k 7D Gaussians, 800x800, 100 orbit cameras (random frame each), white background, "
            "lambda_t = lambda_d = 0.05")
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


class L2Flush:
    """Empties the 129 MB L2 between timed steps: writes a 256 MiB buffer, then reads a second one.

    The write alone would leave L2 full of dirty lines of the flush buffer, and the next step's
    first reads would pay for writing them back to DRAM (about 129 MB, which a render loop never
    has to write); reading a second buffer afterwards moves those write-backs into the flush, so
    every step starts with an L2 that holds none of its inputs and nothing dirty."""

    def __init__(self, dev):
        self.w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        self.r = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.out = torch.empty((), dtype=torch.float32, device=dev)

    def __call__(self):
        self.w.zero_()
        torch.sum(self.r, dim=0, out=self.out)

    DESCRIPTION = "flushed (256 MiB written, then 256 MiB of another buffer read) between steps, outside the per-step CUDA events"
# FP32 work of compositing: 15 FLOP per evaluated (pixel, Gaussian) pair
# (offsets, exponent, opacity clamp and tests, transmittance) plus one ex2, and 3 FMA = 6 FLOP per
# blended pair (the colour update).  The counting variant of render_fwd counts both kinds of pair.
FLOP_PER_EVAL = 15
FLOP_PER_CONTRIB = 6
# DRAM bytes (read + write) per launch of the dominant kernel on this workload, from one
# `ncu --set full` capture of render_fwd_kernel.  Set to None whenever render_fwd_kernel changes
# until it is captured again.
RENDER_FWD_TRAFFIC_BYTES = 12.84736e6


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return dict(hbm_gbs=float(p["hbm_gbs"]), sm_max_mhz=float(p.get("sm_max_mhz", 2070.0)),
                    source="measured")
    except (OSError, KeyError, ValueError):
        return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


def measure_alu_peaks(dev, iters: int = 4096) -> dict:
    """FP32 and MUFU ex2 peaks of this GPU, measured: one launch of each throughput probe of
    libsdgs (scalar FFMA, paired FFMA2, ex2.approx; 64 warps per SM, independent chains), timed
    with CUDA events after a warm-up launch.  FP32 TFLOP/s is the faster of the two FMA forms."""
    from paper_2503_07946_gb300 import sdgs
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(sms * 8 * 256, dtype=torch.float32, device=dev)
    out = {}
    for kind, name in ((0, "ffma_tflops"), (1, "ffma2_tflops"), (2, "ex2_tera_per_s")):
        sdgs.alu_peak_probe(kind, 64, sink)
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ops = sdgs.alu_peak_probe(kind, iters, sink)
            e1.record()
            torch.cuda.synchronize()
            rate = ops / (e0.elapsed_time(e1) * 1e-3) / 1e12
            best = rate if best is None else max(best, rate)
        out[name] = best
    out["fp32_tflops"] = max(out["ffma_tflops"], out["ffma2_tflops"])
    out["sms"] = sms
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# Reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------------------------

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


ORACLE_KEYS = ("mean2d", "conic", "alpha_cond", "rgb", "depth", "rect")
_WORKER = {}


def _oracle_worker_init(shm_name: str, n: int, cfg: int):
    """Pool worker: one torch thread; maps the per-Gaussian records from shared memory."""
    from multiprocessing import shared_memory
    torch.set_num_threads(1)
    shm = shared_memory.SharedMemory(name=shm_name)
    _WORKER.update(shm=shm, n=n, cams=synth.config_cameras(cfg))


def _oracle_records(buf, n: int) -> dict:
    cols = {"mean2d": 2, "conic": 3, "alpha_cond": 1, "rgb": 3, "depth": 1, "rect": 4}
    out, off = {}, 0
    for k in ORACLE_KEYS:
        dt = np.int64 if k == "rect" else np.float64
        a = np.ndarray((n, cols[k]) if cols[k] > 1 else (n,), dtype=dt, buffer=buf, offset=off)
        out[k] = a
        off += a.nbytes
    return out


def _oracle_tiles(job) -> int:
    """Composites whole tiles of camera cam_index from the shared records (the oracle as it stands:
    render_pixels over the rectangle lists); returns the pixels done."""
    from oracle import render as orender
    cam_index, tiles = job
    cam = _WORKER["cams"][cam_index]
    g = {k: torch.as_tensor(v) for k, v in _oracle_records(_WORKER["shm"].buf, _WORKER["n"]).items()}
    pix = []
    for t in tiles:
        tx, ty = t % cam.tiles_x, t // cam.tiles_x
        ys, xs = np.meshgrid(np.arange(ty * 16, min(ty * 16 + 16, cam.height)),
                             np.arange(tx * 16, min(tx * 16 + 16, cam.width)), indexing="ij")
        pix.append(np.stack([ys.reshape(-1), xs.reshape(-1)], 1))
    pix = np.concatenate(pix)
    orender.render_pixels(g, cam, pix)
    return int(len(pix))


class OracleFrames:
    """The FP64 oracle on the host cores: its per-Gaussian stage (slicing, projection, SH, tile
    rectangles) in this process with torch's threads, then the compositing of whole 16x16 tiles
    spread over a spawn pool of one process per core, the records shared through shared memory."""

    def __init__(self, cfg: int, procs: int | None = None):
        from multiprocessing import get_context, shared_memory
        self.cfg = cfg
        self.scene = synth.config_scene(cfg)
        self.cams = synth.config_cameras(cfg)
        self.procs = procs or os.cpu_count() or 1
        n = self.scene.n
        nbytes = n * 8 * (2 + 3 + 1 + 3 + 1 + 4)
        self.shm = shared_memory.SharedMemory(create=True, size=nbytes)
        self.pool = get_context("spawn").Pool(self.procs, initializer=_oracle_worker_init,
                                              initargs=(self.shm.name, n, cfg))
        self.pool.map(int, range(self.procs))  # wait for the workers to start

    def stage(self, cam_index: int) -> float:
        from oracle import render as orender
        t0 = time.perf_counter()
        cam = self.cams[cam_index]
        g = orender.gaussians(orender.params_from_scene(self.scene), cam, self.scene.lambda_t, self.scene.lambda_d)
        recs = _oracle_records(self.shm.buf, self.scene.n)
        for k in ORACLE_KEYS:
            v = g[k].detach().numpy()
            recs[k][...] = v.reshape(recs[k].shape)
        return time.perf_counter() - t0

    def tiles(self, cam_index: int, tiles) -> tuple[int, float]:
        t0 = time.perf_counter()
        tiles = list(tiles)
        jobs = [(cam_index, tiles[i::self.procs * 2]) for i in range(self.procs * 2)]
        pixels = sum(self.pool.map(_oracle_tiles, [j for j in jobs if j[1]]))
        return pixels, time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()
        self.shm.close()
        self.shm.unlink()


def oracle_sample(frames: OracleFrames, cam_index: int, n_tiles: int, seed: int) -> dict:
    """One bounded sample: the per-Gaussian stage for every Gaussian plus n_tiles random whole tiles,
    both measured; `frame_s_estimate` scales the tiles' time to the whole frame."""
    cam = frames.cams[cam_index]
    ntiles = cam.tiles_x * cam.tiles_y
    t_stage = frames.stage(cam_index)
    tiles = np.random.default_rng(seed).choice(ntiles, size=min(n_tiles, ntiles), replace=False)
    pixels, t_tiles = frames.tiles(cam_index, tiles)
    return dict(stage_s=t_stage, tiles_s=t_tiles, pixels=pixels, tiles=len(tiles), step_s=t_stage + t_tiles,
                frame_s_estimate=t_stage + t_tiles * ntiles / len(tiles))


def run_reference(args, rank: int, world: int):
    """The reference arm: the oracle on the host cores, on our arm's workload.  Each step is one
    measured bounded sample of a config-1 frame (the next orbit camera): the per-Gaussian stage of
    all 300k Gaussians plus 4 whole tiles per host core; the value is the pixels composited per
    second of step time (the per-Gaussian stage included), so ms_per_step is the measured step."""
    if rank != 0:
        return
    frames = OracleFrames(1)
    cores = frames.procs
    try:
        steps = []
        for i in range(args.warmup + args.steps):
            r = oracle_sample(frames, i % len(frames.cams), 4 * cores, seed=i)
            if i >= args.warmup:
                steps.append(r)
    finally:
        frames.close()
    step_s = float(np.mean([r["step_s"] for r in steps]))
    mpix = float(np.mean([r["pixels"] for r in steps])) / step_s / 1e6
    est = float(np.mean([r["frame_s_estimate"] for r in steps]))
    sample = ("per step, measured: the oracle's per-Gaussian stage for all 300k Gaussians (%.2f s) plus "
              "compositing of %d random whole 16x16 tiles of one 800x800 view over %d processes (%.2f s)"
              % (np.mean([r["stage_s"] for r in steps]), steps[0]["tiles"], cores,
                 np.mean([r["tiles_s"] for r in steps])))
    line = {"impl": "reference", "metric": METRIC, "value": mpix, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_gaussians": 300000, "width": 800, "height": 800},
            "cpu_baseline": {"value": mpix, "unit": "Mpix/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model(), "frame_s_estimate": est,
                             "frame_mpix_s_estimate": 800 * 800 / est / 1e6},
            "e2e": {"value": mpix, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def oracle_frames_report() -> dict:
    """Whole frames of the oracle as the measurement plan lists them: config 0 (every tile), the
    first camera of config 1 (every tile), the FD gradient case (N = 64, 32 x 32), with the host's
    core count and CPU model.  Long (minutes): run on its own with --oracle-frames."""
    from oracle import render as orender
    out = {"nproc": os.cpu_count(), "cpu_model": cpu_model(), "torch_threads": torch.get_num_threads()}
    for cfg in (0, 1):
        frames = OracleFrames(cfg)
        try:
            cam = frames.cams[0]
            t0 = time.perf_counter()
            t_stage = frames.stage(0)
            pixels, t_tiles = frames.tiles(0, range(cam.tiles_x * cam.tiles_y))
            t = time.perf_counter() - t0
        finally:
            frames.close()
        out[f"config{cfg}_frame"] = {"seconds": t, "stage_s": t_stage, "composite_s": t_tiles, "pixels": pixels,
                                     "mpix_s": pixels / t / 1e6, "processes": frames.procs,
                                     "n_gaussians": frames.scene.n, "width": cam.width, "height": cam.height}
    scene = synth.make_scene(64, seed=16, box=0.6)
    cam = synth.make_camera((0.0, 0.0, -3.0), 32, 32, 60.0, 0.5, bg=(0.3, 0.3, 0.3))
    dL = np.random.default_rng(17).normal(size=(32, 32, 3))
    t0 = time.perf_counter()
    orender.vjp(scene, cam, dL)
    t_vjp = time.perf_counter() - t0
    t0 = time.perf_counter()
    h = 1e-6
    for k in range(8):  # central differences of 8 parameters (two renders each)
        for sgn in (1, -1):
            s2 = synth.Scene(scene.mean7.astype(np.float64), scene.L28.astype(np.float64), scene.opacity.copy(),
                             scene.sh, scene.lambda_t, scene.lambda_d, scene.bg)
            s2.mean7.reshape(-1)[k] += sgn * h
            orender.render(s2, cam)
    t_fd = (time.perf_counter() - t0) / 16
    out["fd_case"] = {"vjp_s": t_vjp, "render_s": t_fd, "n_gaussians": 64, "width": 32, "height": 32}
    return out


# ---------------------------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------------------------

def launches_per_frame(n: int, capacity: int, width: int, height: int) -> int:
    """Kernels libsdgs launches for one render: slice_project; the binning clear kernel; the
    depth keys (with the depth digit histograms); 4 depth radix passes; then, for images of at
    most 256 tiles per side, the single-pass span walk (row spans in depth order, K, the row
    histogram), ceil(row bits / 8) row radix passes, the per-chunk column counts and the
    expansion into the tile lists; else the kept-tile count per warp of 32 Gaussians, its scan
    (one kernel up to 11264 warps, else three), the instance emit (with the tile digit
    histograms), ceil(tile bits / 8) tile radix passes and the tile ranges; the rasteriser."""
    tx, ty = (width + 15) // 16, (height + 15) // 16
    head = 1 + 1 + 1 + 4
    if tx <= 256 and ty <= 256:
        row_passes = (max(0, (ty - 1).bit_length()) + 7) // 8
        return head + 1 + row_passes + 2 + 1
    scan = 1 if (n + 31) // 32 <= 11 * 1024 else 3
    tile_passes = (max(0, (tx * ty - 1).bit_length()) + 7) // 8
    return head + 1 + scan + 1 + tile_passes + 1 + 1


def binning_bytes(n: int, k: int, spans: int, visible: int) -> dict:
    """Algorithmic DRAM bytes of one span-binning call: each kernel's reads and writes once.
    depth keys 20 B per Gaussian (depth 4 + rect 8 in, key + value 8 out); 4 depth passes 16 B per
    Gaussian each (key + value in and out); the span walk 36 B per visible Gaussian (order 4,
    rect 8, mean2d 8, conic 16) and 8 B written per span; the row pass 16 B per span; the column
    count reads 4 B per span; the expansion reads 8 B per span and writes 4 B per instance (the
    point list).  The per-chunk tables and block statuses are a few hundred kB."""
    per_kernel = {"depth_keys": 20 * n, "depth_passes": 64 * n, "span_walk": 36 * visible + 8 * spans,
                  "row_pass": 16 * spans, "span_count": 4 * spans, "span_expand": 8 * spans + 4 * k}
    return {"total": sum(per_kernel.values()), "per_kernel": per_kernel}


def count_spans(bins, k: int, tiles_x: int) -> int:
    """Row spans behind the tile lists: one per (Gaussian, tile row) pair that has instances (the
    lists lie in tile order)."""
    pl = bins.point_list[:k].to(torch.int64)
    rng = bins.ranges.to(torch.int64)
    cnt = rng[:, 1] - rng[:, 0]
    tile = torch.repeat_interleave(torch.arange(rng.shape[0], device=pl.device), cnt)
    return int(torch.unique(pl * 65536 + tile // tiles_x).numel())


def cpu_baseline(cam_index: int) -> dict:
    """The oracle on the host cores, timed on one whole frame of the headline workload (config 1,
    800x800, 300k Gaussians): its per-Gaussian stage, then all 2500 tiles composited over one
    process per core (about 25 s on 16 cores)."""
    frames = OracleFrames(1)
    try:
        cam = frames.cams[cam_index]
        t_stage = frames.stage(cam_index)
        pixels, t_tiles = frames.tiles(cam_index, range(cam.tiles_x * cam.tiles_y))
    finally:
        frames.close()
    t = t_stage + t_tiles
    return {"value": pixels / t / 1e6, "unit": "Mpix/s", "cores": frames.procs, "kind": "oracle",
            "cpu_model": cpu_model(), "measured_s": t,
            "sample": ("one whole 800x800 frame of config 1 (orbit camera %d), measured: the oracle's per-Gaussian "
                       "stage for all 300k Gaussians (%.2f s) plus compositing of all 2500 tiles over %d processes "
                       "(%.2f s)" % (cam_index, t_stage, frames.procs, t_tiles))}


def replica_order(rank: int, n_cams: int, count: int) -> list[int]:
    """Cameras of a rank's frames: each rank starts at its own offset of the orbit and renders the
    same number of frames at every N (replicas: per-rank work fixed, no data exchanged)."""
    return [(rank * 37 + i) % n_cams for i in range(count)]


def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's value: the job's throughput is every rank's work over the slowest rank's
    time.  A collective over the default process group when world > 1."""
    if world <= 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_mpix_s(world: int, pixels_per_step: int, ms_per_step: float) -> float:
    """Whole-job Mpix/s: every rank renders pixels_per_step per step in ms_per_step (its slowest)."""
    return world * pixels_per_step / (ms_per_step * 1e-3) / 1e6


def run_ours(args, rank: int, world: int):
    from paper_2503_07946_gb300 import render as prender
    from paper_2503_07946_gb300 import sdgs

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    sdgs.lib()  # fails loudly if the CUDA library is missing
    peaks = load_peaks()
    scene = synth.config_scene(1)
    cams = synth.config_cameras(1)
    W, H = 800, 800
    t_scene = prender.scene_to_device(scene)
    st = sdgs.scene_struct(t_scene, scene.lambda_t, scene.lambda_d)
    steps, warm = args.steps, args.warmup
    order = replica_order(rank, len(cams), steps + warm)
    views = [sdgs.view_struct(cams[i]) for i in order]

    # size the instance lists once from the frames this run renders
    sizing = prender.Renderer(scene.n, W, H, capacity=4096)
    kmax = 0
    for v in views[: min(len(views), 100)]:
        sdgs.slice_project(st, v, sizing.proj)
        kmax = max(kmax, sizing.bin(v))
    del sizing
    r = prender.Renderer(scene.n, W, H, capacity=int(kmax * 1.02) + 4096)
    flush = L2Flush(dev)
    n_eval = torch.zeros(2, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()

    def step(v, ev=None):
        if ev is not None:
            ev[0].record(stream)
        sdgs.slice_project(st, v, r.proj, stream)
        if ev is not None:
            ev[1].record(stream)
        sdgs.bin_sort(r.proj, v, r.bins, sync=False, stream=stream)
        if ev is not None:
            ev[2].record(stream)
        sdgs.render_fwd(r.proj, r.bins, v, r.image, r.final_T, r.n_contrib, None, stream)
        if ev is not None:
            ev[3].record(stream)

    # settle (untimed): frames of the run's views for at least 0.5 s, so that the GPU leaves the
    # idle state of the host-bound sizing pass and every buffer has been touched; then the W
    # warm-up steps
    t_settle, i = time.perf_counter(), 0
    while i < 100 or time.perf_counter() - t_settle < 0.5:
        step(views[i % len(views)])
        flush()
        i += 1
        if i % 50 == 0:
            torch.cuda.synchronize()
    for i in range(warm):
        step(views[i])
        flush()
    torch.cuda.synchronize()
    n_eval.zero_()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    def roll(seconds):
        """Untimed frames of the same workload for `seconds`, so that the clock sampler (50 ms
        period) has samples on both sides of a short timed region."""
        t, k = time.perf_counter(), 0
        while time.perf_counter() - t < seconds:
            step(views[k % len(views)])
            flush()
            k += 1
            if k % 20 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()

    with ClockSampler(dev.index) as clk:
        roll(0.25)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for i in range(steps):
            step(views[warm + i], evs[i])
            flush()  # outside the step's events: every step starts with a cold L2
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        roll(0.25)
    if world > 1:
        torch.distributed.barrier()
    phase = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])] for e in evs])
    # compositing work of the timed frames, counted in a separate untimed pass per frame
    n_eval.zero_()
    for i in range(steps):
        v = views[warm + i]
        sdgs.slice_project(st, v, r.proj, stream)
        sdgs.bin_sort(r.proj, v, r.bins, sync=False, stream=stream)
        sdgs.render_fwd(r.proj, r.bins, v, r.image, r.final_T, r.n_contrib, n_eval, stream)
    torch.cuda.synchronize()
    step_ms = phase.sum(1)
    ms = max_over_ranks(float(step_ms.mean()), world, dev)
    evals, contribs = (int(x) for x in n_eval.tolist())
    k_inst = int(r.bins.num_instances.item())
    visible = int(((r.proj.rect[:, 2] > r.proj.rect[:, 0]) & (r.proj.rect[:, 3] > r.proj.rect[:, 1])).sum())

    if args.frames_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": job_mpix_s(world, W * H, ms), "unit": "Mpix/s",
                              "ms_per_step": ms, "frames_only": True, "clocks": clk.summary(),
                              "phases_ms": {"slice_project": float(phase[:, 0].mean()),
                                            "bin_sort": float(phase[:, 1].mean()),
                                            "render_fwd": float(phase[:, 2].mean())}}), flush=True)
        return

    # ---- end to end: the public API with the image read back to pinned host memory ----
    # (a streaming renderer: the instance count is checked one frame later instead of
    # synchronising after binning; no timed frame may have overflowed)
    re_ = prender.Renderer(scene.n, W, H, capacity=r.bins.capacity, deferred_check=True)
    host_img = torch.empty(H, W, 3, dtype=torch.float32, pin_memory=True)
    view_bytes = ctypes_sizeof_view()
    for i in range(warm):
        re_.forward(st, views[i])
        host_img.copy_(re_.image, non_blocking=True)
    torch.cuda.synchronize()
    re_.check_deferred()
    overflowed = re_.overflowed_frames
    t0 = time.perf_counter()
    for i in range(steps):
        re_.forward(st, views[warm + i])
        host_img.copy_(re_.image, non_blocking=True)
        torch.cuda.synchronize()
    e2e_one_s = max_over_ranks((time.perf_counter() - t0) / steps, world, dev)
    re_.check_deferred()
    assert re_.overflowed_frames == overflowed, "a timed end-to-end frame exceeded the bins' capacity"
    del re_
    # the same with K frames in flight, as a streaming client runs: K renderers on K streams;
    # every frame's image is copied to pinned host memory and waited for (by the host) before its
    # renderer takes the frame K later.  The line reports K = 4; K = 2 and 3 are timed beside it.
    kmax_fif = 4
    rs = [prender.Renderer(scene.n, W, H, capacity=r.bins.capacity, deferred_check=True) for _ in range(kmax_fif)]
    sts = [torch.cuda.Stream(dev) for _ in range(kmax_fif)]
    hosts = [torch.empty(H, W, 3, dtype=torch.float32, pin_memory=True) for _ in range(kmax_fif)]

    def stream_frames(count, first, k):
        done = [None] * k
        for i in range(count):
            j = i % k
            if done[j] is not None:
                done[j].synchronize()  # frame i - k's image is on the host
            with torch.cuda.stream(sts[j]):
                rs[j].forward(st, views[first + i], sts[j])
                hosts[j].copy_(rs[j].image, non_blocking=True)
                done[j] = torch.cuda.Event()
                done[j].record(sts[j])
        for ev in done:
            if ev is not None:
                ev.synchronize()

    e2e_by_k = {}
    for k in range(2, kmax_fif + 1):
        stream_frames(warm, 0, k)
        for q in rs:
            q.check_deferred()
        overflowed = [q.overflowed_frames for q in rs]
        t0 = time.perf_counter()
        stream_frames(steps, warm, k)
        e2e_by_k[k] = max_over_ranks((time.perf_counter() - t0) / steps, world, dev)
        for q, o in zip(rs, overflowed):
            q.check_deferred()
            assert q.overflowed_frames == o, "a timed end-to-end frame exceeded the bins' capacity"
    fif = kmax_fif
    e2e_s = e2e_by_k[fif]
    del rs

    # ---- fwd + bwd (L2 loss against a target from perturbed parameters, camera 0) ----
    big_scene = synth.config_scene(2)
    large = frames_on(big_scene, synth.config_cameras(2), min(steps, 200), warm, dev, flush)
    large["workload"] = ("config 2: 1.5M 7D Gaussians in 64 clusters, 1352x1014, forward-facing arc cameras, "
                         "black background, lambda_t = lambda_d = 0.1")
    del big_scene
    pipe = {str(k): pipelined_frames(scene, t_scene, views, min(steps, 1000), warm, dev, k) for k in (2, 3, 4)}
    # (the training iterations are timed over at least 200 of them: 20 take 17 ms, short enough
    # for the host's launch queue to show)
    fb = fwd_bwd_its(scene, cams[0], max(steps, 200), warm, dev)
    fb_agr = fwd_bwd_its(scene, cams[0], max(min(steps, 200), 100), warm, dev, agr=True)
    agr = agr_frames(scene, t_scene, views, flush, min(steps, 300), warm, dev)
    dens = densify_ms(t_scene, scene, views[0], flush, 20, dev)
    serving = None if args.no_serving else serving_bench(dev, count=args.serve_requests)

    pix = W * H
    value = job_mpix_s(world, pix, ms)
    raster_ms = float(phase[:, 2].mean())
    achieved_tflops = ((evals * FLOP_PER_EVAL + contribs * FLOP_PER_CONTRIB) / steps) / (raster_ms * 1e-3) / 1e12
    clocks = clk.summary()
    clocks["window"] = "the timed steps and 0.25 s of the same frames right before and after them"
    with ClockSampler(dev.index) as clk_alu:
        alu = measure_alu_peaks(dev)
    alu["clocks"] = clk_alu.summary()
    peak_tflops = alu["fp32_tflops"]
    ex2_rate = (evals / steps) / (raster_ms * 1e-3) / 1e12
    slice_gbs = (scene.n * 148 + visible * (192 + 60)) / (float(phase[:, 0].mean()) * 1e-3) / 1e9
    spans = count_spans(r.bins, k_inst, (W + 15) // 16)
    bin_bytes = binning_bytes(scene.n, k_inst, spans, visible)
    bin_gbs = bin_bytes["total"] / (float(phase[:, 1].mean()) * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": steps, "warmup": warm,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "fps": world * 1000.0 / ms,
        "config": {"workload": WORKLOAD, "n_gaussians": scene.n, "width": W, "height": H, "parallelism": f"replicas x{world}",
                   "l2": L2Flush.DESCRIPTION},
        "phases_ms": {"slice_project": float(phase[:, 0].mean()), "bin_sort": float(phase[:, 1].mean()),
                      "render_fwd": raster_ms},
        "workload_stats": {"instances": k_inst, "visible": visible, "evaluations_per_frame": evals // steps,
                           "contributions_per_frame": contribs // steps},
        "large_scene_frames": large,
        "pipelined_frames": pipe,
        "fwd_bwd_it_s": fb,
        "fwd_bwd_agr_it_s": fb_agr,
        "agr_frames": agr,
        "densify_stats": dens,
        "serving": serving,
        "e2e": {"value": job_mpix_s(world, pix, e2e_s * 1e3), "unit": "Mpix/s", "h2d_bytes_per_step": view_bytes,
                "d2h_bytes_per_step": pix * 3 * 4 + 8, "frames_in_flight": fif,
                "by_frames_in_flight": {str(k): job_mpix_s(world, pix, v * 1e3) for k, v in e2e_by_k.items()},
                "one_frame_in_flight": job_mpix_s(world, pix, e2e_one_s * 1e3)},
        "gpu_launches": steps * launches_per_frame(scene.n, r.bins.capacity, W, H),
        "roofline": {"kernel": "render_fwd_kernel", "bound": "alu", "achieved": achieved_tflops,
                     "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved_tflops / peak_tflops,
                     "traffic": RENDER_FWD_TRAFFIC_BYTES,
                     "peak_source": "measured (FP32 FMA probe, faster of scalar and paired forms)",
                     "note": "%d FLOP per evaluated and %d per blended (pixel, Gaussian) pair, counted by the "
                             "kernel's counting variant over the timed frames" % (FLOP_PER_EVAL, FLOP_PER_CONTRIB),
                     "mufu": {"achieved": ex2_rate, "peak": alu["ex2_tera_per_s"], "unit": "T ex2/s",
                              "frac": ex2_rate / alu["ex2_tera_per_s"]}},
        "alu_peaks": alu,
        "slice_project_hbm": {"achieved": slice_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                              "frac": slice_gbs / peaks["hbm_gbs"], "peak_source": peaks["source"]},
        "binning_hbm": {"achieved": bin_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": bin_gbs / peaks["hbm_gbs"], "peak_source": peaks["source"],
                        "bytes_per_frame": bin_bytes["total"], "bytes_per_kernel": bin_bytes["per_kernel"],
                        "spans": spans, "note": "algorithmic bytes of the last timed frame's binning (each kernel's "
                                                "reads and writes once) over the mean binning phase time"},
        "clocks": clocks,
        "wall_s_timed_region": t_wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(order[0])
    if rank == 0:
        print(json.dumps(line), flush=True)


def ctypes_sizeof_view() -> int:
    import ctypes

    from paper_2503_07946_gb300 import sdgs
    return ctypes.sizeof(sdgs.View)


SERVE_SIZES = [(400, 400), (800, 800), (1352, 1014), (1920, 1080)]


def serving_trace(rate: float, count: int, seed: int, radii) -> list:
    """Poisson arrivals at `rate` req/s; each request picks a scene, a resolution, a camera on
    that scene's orbit and a time t, all uniformly."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for i in range(count):
        sid = int(rng.integers(0, len(radii)))
        w, h = SERVE_SIZES[int(rng.integers(0, len(SERVE_SIZES)))]
        d = rng.normal(size=3)
        eye = radii[sid] * d / np.linalg.norm(d)
        out.append((float(t[i]), sid, synth.make_camera(eye, w, h, 60.0, float(rng.uniform()))))
    return out


def serving_bench(dev, rates=(100.0, 200.0, 500.0, 1000.0, 2000.0), count: int = 4000, slots: int = 8,
                  budget: int = 8 << 30) -> dict:
    """p50/p99 latency and Mpix/s of the render server on Poisson traces (the serving stream
    workload: 4 resident scenes, 4000 requests per rate, an 8 GiB budget for per-request memory),
    against serving the same trace one request at a time through the plain path: each request's
    plain-path service time is measured, then replayed through a FIFO queue against the arrival
    times (exact for a single FIFO server whose service times do not depend on arrivals)."""
    from paper_2503_07946_gb300 import render as prender
    from paper_2503_07946_gb300 import sdgs
    scenes = synth.serving_scenes()
    radii = [4.0, 4.0, 8.0, 8.0]
    tens = [prender.scene_to_device(s) for s in scenes]
    ring = 48
    bufs = {wh: [torch.empty(wh[1], wh[0], 3, dtype=torch.float32, device=dev) for _ in range(ring)]
            for wh in SERVE_SIZES}
    result = {"scenes": [s.n for s in scenes], "resolutions": SERVE_SIZES, "requests_per_rate": count,
              "slots": slots, "budget_bytes": budget, "output": "device buffers",
              "one_at_a_time_method": "measured plain-path service time of every request, replayed through a "
                                      "FIFO queue against the same arrival times"}
    renderers = {}

    def plain(sid, cam):
        key = (sid, cam.width, cam.height)
        if key not in renderers:
            renderers[key] = prender.Renderer(scenes[sid].n, cam.width, cam.height)
        r = renderers[key]
        st = sdgs.scene_struct(tens[sid], scenes[sid].lambda_t, scenes[sid].lambda_d)
        img = r.forward(st, sdgs.view_struct(cam))
        bufs[(cam.width, cam.height)][0].copy_(img)
        torch.cuda.synchronize()

    def live(srv, ids, trace):
        """Submits the trace at its arrival times; returns latencies (s) and completion times."""
        rids, subs = [], []
        t0 = time.perf_counter()
        for i, (ta, sid, cam) in enumerate(trace):
            while time.perf_counter() - t0 < ta:
                pass
            if i >= ring:
                srv.wait(rids[i - ring], 60_000)  # its output buffer is reused now
            rids.append(srv.submit(ids[sid], sdgs.view_struct(cam), bufs[(cam.width, cam.height)][i % ring]))
            subs.append(time.perf_counter() - t0)
        lat = np.array([srv.wait(r, 60_000) for r in rids]) * 1e-3
        srv.release()
        return lat, np.array(subs) + lat

    def one_at_a_time(trace):
        service = []
        for _, sid, cam in trace:
            a = time.perf_counter()
            plain(sid, cam)
            service.append(time.perf_counter() - a)
        finish, lat1 = 0.0, []
        for (ta, _, _), sv in zip(trace, service):
            finish = max(finish, ta) + sv
            lat1.append(finish - ta)
        return np.array(lat1), finish

    def stats_line(lat, span, pix):
        return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mpix_s": pix / span / 1e6}

    plain_at = {}
    with sdgs.Server(budget_bytes=budget, slots=slots) as srv:
        ids = [srv.add_scene(t, s.lambda_t, s.lambda_d) for t, s in zip(tens, scenes)]
        warm = serving_trace(100.0, 16, 99, radii)
        for _, sid, cam in warm:  # allocate slot buffers and learn instance counts
            srv.wait(srv.submit(ids[sid], sdgs.view_struct(cam), bufs[(cam.width, cam.height)][1]), 60_000)
            plain(sid, cam)
        for rate in rates:
            trace = serving_trace(rate, count, int(rate), radii)
            lat, done = live(srv, ids, trace)
            pix = sum(c.width * c.height for _, _, c in trace)
            lat1, finish = one_at_a_time(trace)
            plain_at[rate] = (lat1, finish)
            result[f"rate_{int(rate)}"] = dict(stats_line(lat, done.max() - trace[0][0], pix),
                                               one_at_a_time=stats_line(lat1, finish - trace[0][0], pix),
                                               server_stats_so_far=srv.stats())
        result["server_stats"] = srv.stats()
    # the two highest rates again with a batching window: the server waits up to 300 us for more
    # requests while slots are free, trading latency for larger batches
    with sdgs.Server(budget_bytes=budget, slots=slots, batch_window_us=300) as srv:
        ids = [srv.add_scene(t, s.lambda_t, s.lambda_d) for t, s in zip(tens, scenes)]
        for _, sid, cam in serving_trace(100.0, 16, 99, radii):
            srv.wait(srv.submit(ids[sid], sdgs.view_struct(cam), bufs[(cam.width, cam.height)][1]), 60_000)
        for rate in rates[-2:]:
            trace = serving_trace(rate, count, int(rate), radii)
            lat, done = live(srv, ids, trace)
            pix = sum(c.width * c.height for _, _, c in trace)
            lat1, finish = plain_at[rate]
            result[f"window300us_rate_{int(rate)}"] = dict(stats_line(lat, done.max() - trace[0][0], pix),
                                                           one_at_a_time=stats_line(lat1, finish - trace[0][0], pix),
                                                           server_stats_so_far=srv.stats())
        # bursts: 8 requests (one per slot) submitted at once, 50 times, against the same 8 one at a time
        rng = np.random.default_rng(7)
        burst_lat, burst_plain = [], []
        for b in range(50):
            reqs = []
            for k in range(slots):
                sid = int(rng.integers(0, len(scenes)))
                w, h = SERVE_SIZES[int(rng.integers(0, len(SERVE_SIZES)))]
                d = rng.normal(size=3)
                reqs.append((sid, synth.make_camera(radii[sid] * d / np.linalg.norm(d), w, h, 60.0,
                                                    float(rng.uniform()))))
            t0 = time.perf_counter()
            rids = [srv.submit(ids[sid], sdgs.view_struct(cam), bufs[(cam.width, cam.height)][2 + k])
                    for k, (sid, cam) in enumerate(reqs)]
            for r in rids:
                srv.wait(r, 60_000)
            burst_lat.append(time.perf_counter() - t0)
            srv.release()
            t0 = time.perf_counter()
            for sid, cam in reqs:
                plain(sid, cam)
            burst_plain.append(time.perf_counter() - t0)
        result["bursts_of_8"] = {"server_ms_per_burst": float(np.median(burst_lat) * 1e3),
                                 "one_at_a_time_ms_per_burst": float(np.median(burst_plain) * 1e3),
                                 "bursts": 50, "server_stats": srv.stats()}
    return result


def frames_on(scene, cams, steps: int, warm: int, dev, flush) -> dict:
    """Forward frames of another scene (slice -> bin -> render), timed per frame with L2 flushes
    between frames, like the headline measurement."""
    from paper_2503_07946_gb300 import render as prender
    from paper_2503_07946_gb300 import sdgs
    t_scene = prender.scene_to_device(scene)
    st = sdgs.scene_struct(t_scene, scene.lambda_t, scene.lambda_d)
    views = [sdgs.view_struct(cams[i % len(cams)]) for i in range(steps + warm)]
    W, H = views[0].width, views[0].height
    sizing = prender.Renderer(scene.n, W, H, capacity=4096)
    kmax = 0
    for v in views[: min(len(views), 60)]:
        sdgs.slice_project(st, v, sizing.proj)
        kmax = max(kmax, sizing.bin(v))
    del sizing
    r = prender.Renderer(scene.n, W, H, capacity=int(kmax * 1.02) + 4096)
    stream = torch.cuda.current_stream()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for i in range(warm + steps):
        ev = evs[i - warm] if i >= warm else None
        if ev:
            ev[0].record(stream)
        sdgs.slice_project(st, views[i], r.proj, stream)
        if ev:
            ev[1].record(stream)
        sdgs.bin_sort(r.proj, views[i], r.bins, sync=False, stream=stream)
        if ev:
            ev[2].record(stream)
        sdgs.render_fwd(r.proj, r.bins, views[i], r.image, r.final_T, r.n_contrib, None, stream)
        if ev:
            ev[3].record(stream)
        flush()
    torch.cuda.synchronize()
    ph = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])] for e in evs])
    ms = float(ph.sum(1).mean())
    return {"value": W * H / (ms * 1e-3) / 1e6, "unit": "Mpix/s", "ms_per_frame": ms, "fps": 1000.0 / ms,
            "phases_ms": {"slice_project": float(ph[:, 0].mean()), "bin_sort": float(ph[:, 1].mean()),
                          "render_fwd": float(ph[:, 2].mean())},
            "instances": int(r.bins.num_instances.item()), "steps": steps}


def pipelined_frames(scene, t_scene, views, steps: int, warm: int, dev, k: int = 2) -> dict:
    """Throughput with k frames in flight: independent views rotate over k streams with their own
    buffers, so one frame's latency-bound binning overlaps another's compositing.  No L2 flush
    between frames (scene, records and lists together exceed the 129 MB L2)."""
    from paper_2503_07946_gb300 import render as prender
    from paper_2503_07946_gb300 import sdgs
    st = sdgs.scene_struct(t_scene, scene.lambda_t, scene.lambda_d)
    W, H = views[0].width, views[0].height
    sizing = prender.Renderer(scene.n, W, H, capacity=4096)
    kmax = 0
    for v in views[: min(len(views), 100)]:
        sdgs.slice_project(st, v, sizing.proj)
        kmax = max(kmax, sizing.bin(v))
    del sizing
    rs = [prender.Renderer(scene.n, W, H, capacity=int(kmax * 1.02) + 4096) for _ in range(k)]
    streams = [torch.cuda.Stream(device=dev) for _ in range(k)]

    def run(lo, hi):
        for i in range(lo, hi):
            r, s = rs[i % k], streams[i % k]
            sdgs.slice_project(st, views[i], r.proj, s)
            sdgs.bin_sort(r.proj, views[i], r.bins, sync=False, stream=s)
            sdgs.render_fwd(r.proj, r.bins, views[i], r.image, r.final_T, r.n_contrib, None, s)

    run(0, warm)
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for s in streams:
        s.wait_event(e0)
    run(warm, warm + steps)
    for s in streams:
        ev = torch.cuda.Event()
        ev.record(s)
        cur.wait_event(ev)
    e1.record(cur)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"value": W * H / (ms * 1e-3) / 1e6, "unit": "Mpix/s", "ms_per_frame": ms, "fps": 1000.0 / ms,
            "frames_in_flight": k, "steps": steps}


def agr_weights_dev(dev) -> dict:
    return {k: torch.as_tensor(v, device=dev).contiguous() for k, v in synth.make_agr_weights(scale=0.1).items()}


def agr_frames(scene, t_scene, views, flush, steps: int, warm: int, dev) -> dict:
    """Forward frames with adaptive refinement: refine (at each view's t) -> slice -> bin -> render."""
    from paper_2503_07946_gb300 import render as prender
    from paper_2503_07946_gb300 import sdgs
    w = agr_weights_dev(dev)
    m_out, l_out = torch.empty_like(t_scene["mean7"]), torch.empty_like(t_scene["L28"])
    st_raw = sdgs.scene_struct(t_scene, scene.lambda_t, scene.lambda_d)
    st_ref = sdgs.scene_struct(dict(t_scene, mean7=m_out, L28=l_out), scene.lambda_t, scene.lambda_d)
    W, H = views[0].width, views[0].height
    sizing = prender.Renderer(scene.n, W, H, capacity=4096)
    kmax = 0
    for v in views[: min(len(views), 100)]:
        sdgs.agr_refine(st_raw, w, v.t, m_out, l_out)
        sdgs.slice_project(st_ref, v, sizing.proj)
        kmax = max(kmax, sizing.bin(v))
    del sizing
    r = prender.Renderer(scene.n, W, H, capacity=int(kmax * 1.02) + 4096)
    stream = torch.cuda.current_stream()

    def step(v, ev=None):
        if ev is not None:
            ev[0].record(stream)
        sdgs.agr_refine(st_raw, w, v.t, m_out, l_out, stream)
        if ev is not None:
            ev[1].record(stream)
        sdgs.slice_project(st_ref, v, r.proj, stream)
        sdgs.bin_sort(r.proj, v, r.bins, sync=False, stream=stream)
        sdgs.render_fwd(r.proj, r.bins, v, r.image, r.final_T, r.n_contrib, None, stream)
        if ev is not None:
            ev[2].record(stream)

    for i in range(warm):
        step(views[i])
        flush()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        step(views[warm + i], evs[i])
        flush()
    torch.cuda.synchronize()
    ph = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])] for e in evs])
    ms = float(ph.sum(1).mean())
    return {"value": W * H / (ms * 1e-3) / 1e6, "unit": "Mpix/s", "ms_per_frame": ms,
            "agr_refine_ms": float(ph[:, 0].mean()), "steps": steps,
            "workload": "config 1 frames with adaptive refinement (random weights, scale 0.1) before slicing"}


def densify_ms(t_scene, scene, view, flush, steps: int, dev) -> dict:
    from paper_2503_07946_gb300 import sdgs
    st = sdgs.scene_struct(t_scene, scene.lambda_t, scene.lambda_d)
    for _ in range(3):
        sdgs.densify_stats(st, view, scene.n, 3.0)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    outs = []
    for e in evs:
        flush()
        e[0].record()
        outs.append(sdgs.densify_stats(st, view, scene.n, 3.0))
        e[1].record()
        outs.clear()
    torch.cuda.synchronize()
    return {"ms": float(np.mean([a.elapsed_time(b) for a, b in evs])), "n": scene.n,
            "note": "scale/rotation (Jacobi), |Sigma_pt|, sqrt(Sigma_t), split and prune flags; includes the "
                    "output allocations from the caching allocator"}


def fwd_bwd_its(scene, cam, steps: int, warm: int, dev, agr: bool = False) -> dict:
    from paper_2503_07946_gb300 import render as prender
    from paper_2503_07946_gb300 import sdgs
    target_scene = synth.perturb_scene(scene)
    view = sdgs.view_struct(cam)
    # the training-loop renderer: no host synchronisation per frame (the instance count is
    # checked one frame later; no timed frame may have overflowed)
    r = prender.Renderer(scene.n, cam.width, cam.height, deferred_check=True)
    tt = prender.scene_to_device(target_scene)
    with torch.no_grad():  # the target through the synchronising renderer (capacity checked)
        target = prender.Renderer(scene.n, cam.width, cam.height).forward(
            sdgs.scene_struct(tt, scene.lambda_t, scene.lambda_d), view).clone()
    params = {k: v.clone().requires_grad_(True) for k, v in prender.scene_to_device(scene).items()}
    weights = {k: v.clone().requires_grad_(True) for k, v in agr_weights_dev(dev).items()} if agr else None

    def it():
        m7, l28 = params["mean7"], params["L28"]
        if weights is not None:
            m7, l28 = prender.agr_refine(m7, l28, weights, cam.t)
        img = prender.render_image(m7, l28, params["opacity"], params["sh"], view,
                                   scene.lambda_t, scene.lambda_d, r)
        loss = ((img - target) ** 2).mean()
        loss.backward()
        for p in list(params.values()) + (list(weights.values()) if weights else []):
            p.grad = None
        return loss

    for _ in range(max(warm, 1)):
        it()
    r.check_deferred()
    torch.cuda.synchronize()
    overflowed = r.overflowed_frames
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        it()
    e1.record()
    torch.cuda.synchronize()
    r.check_deferred()
    assert r.overflowed_frames == overflowed, "a timed frame exceeded the bins' capacity"
    ms = e0.elapsed_time(e1) / steps
    return {"value": 1000.0 / ms, "unit": "it/s", "ms_per_it": ms,
            "workload": "config 3: 300k Gaussians, 800x800, camera 0, L2 loss vs a perturbed-parameter target"
                        + (", with adaptive refinement (weights trained too)" if agr else "")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving latency benchmark")
    ap.add_argument("--serve-requests", type=int, default=4000, help="requests per arrival rate (serving)")
    ap.add_argument("--frames-only", action="store_true",
                    help="time the forward frames only (no e2e, fwd+bwd or CPU baseline); for profiling")
    ap.add_argument("--oracle-frames", action="store_true",
                    help="time whole oracle frames on the host (config 0, config 1 camera 0, the FD case); minutes")
    ap.add_argument("--fwd-bwd-only", action="store_true",
                    help="time the fwd+bwd iterations only (config 3 workload); for profiling the backward")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.oracle_frames:
        print(json.dumps({"oracle_frames": oracle_frames_report()}), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.fwd_bwd_only:
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
        torch.cuda.set_device(dev)
        fb = fwd_bwd_its(synth.config_scene(1), synth.config_cameras(1)[0], args.steps, args.warmup, dev)
        if rank == 0:
            print(json.dumps({"metric": "fwd+bwd it/s", "fwd_bwd_it_s": fb}), flush=True)
    else:
        run_ours(args, rank, world)
    if world > 1 and args.impl == "ours":
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
