"""Benchmark of the LFDPR per-frame path on GB300.

A step is one whole frame of the paper-shaped workload (10^6 triangles, 48
views of 420x560, 2560x1600 panel): set-up and point generation, fetch,
splat, resolve and interleave, with the scene rotating 3 degrees per frame.
Inputs are resident in HBM; L2 is flushed (a 512 MiB write) between timed
steps and each step is timed with CUDA events on the rendering stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--config learned times the learned quarter-view path (12 views rendered, the
U-Net's tensor-core kernels predict the 48 reconstructed views, interleave)
against the plain full render (96 views at 2x angular rate, tent, crosstalk,
interleave) on the paper-shaped scene, with PSNR and SSIM of the prediction
against the full render's reconstruction per frame.

--config batch times batched multi-scene frames instead: 32 paper-shaped
scenes of 50k-2M triangles, each on its own display (24, 48 or 96 views at
420x560 or 640x360, 2560x1600 panel), one texture set, rendered and
interleaved by one replayed CUDA graph per batch after the library's
autotuner has picked its configuration; it reports frames/s over all scenes,
p50/p99 batch latency and the same scenes rendered one after another.

Under torchrun (N > 1) every rank renders its own frames of the same scene
(weak scaling, no data-path collective); the timed total is the max over ranks.
--impl reference times the CPU oracle (the only reference this paper has: it
publishes no code) on complete frames of the same workload, rank 0 only: its
set-up on one core and its per-view splat and resolve spread over pinned
worker processes, one per host core.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "48-view display frames/s and splatted points/s; learned vs plain at PSNR>=38 dB"
WORKLOAD = ("paper-shaped LFDPR frame: 1,000,000 triangles (200 displaced meshes, log-uniform "
            "areas over 3 decades), 64 RGBA8 textures 64^2-4096^2, 48 views over 40 deg at "
            "420x560, 2560x1600 panel, slant 0.2")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--config", choices=["paper", "angular", "gauss", "gauss2x", "tiny", "pbr", "batch", "learned"],
                   default="paper")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--view-band", type=int, default=None,
                   help="views per band of key clear, splat and resolve (0: all at once; default: the library's)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-secondary", action="store_true",
                   help="skip the 96-view and learned-path measurements after the main timed region")
    p.add_argument("--batch-scenes", type=int, default=32, help="--config batch: scenes per batch")
    p.add_argument("--batch-tris", type=str, default="50000,2000000",
                   help="--config batch: triangle-count range per scene (log-uniform)")
    p.add_argument("--scene-instances", type=int, default=200,
                   help="meshes of the paper-shaped scene (200: 10^6 triangles); fewer make the small "
                        "case of the same kernels for ncu captures, never a bench line")
    return p.parse_args()


def workload(cfg, instances=200):
    from dataclasses import replace
    from paper_2601_19901_gb300 import scenes as S
    if instances != 200:
        # the same display and scene recipe with fewer meshes (profiling only)
        wl = WORKLOAD.replace("1,000,000 triangles (200 displaced meshes",
                              "%d triangles (%d displaced meshes: a reduced case for profiling, not the workload"
                              % (5000 * instances, instances))
        if cfg == "angular":
            return S.display_angular_ss(), S.scene_paper(n_instances=instances), wl
        if cfg == "paper":
            return S.display_paper(), S.scene_paper(n_instances=instances), wl
        raise SystemExit("--scene-instances applies to --config paper and angular")
    if cfg == "tiny":
        return S.display_tiny(), S.scene_tiny(), "tiny: 2,048 triangles, 8 views 128x128, 512x512 panel"
    if cfg == "angular":
        return (S.display_angular_ss(), S.scene_paper(),
                WORKLOAD.replace("48 views", "96 views tent-reconstructed to 48 (+crosstalk 0.15)"))
    if cfg == "gauss2x":
        d = S.display_angular_ss()
        return (replace(d, recon=2, view_w=2 * d.view_w, view_h=2 * d.view_h, ss_level=1), S.scene_paper(),
                WORKLOAD.replace("48 views over 40 deg at 420x560", "96 views at 840x1120 (2x spatial and 2x "
                                 "angular supersampling, random angles), a mip level of each view at 420x560, "
                                 "Gaussian reconstruction (8 samples) to 48 views over 40 deg at 420x560 "
                                 "(+crosstalk 0.15)"))
    if cfg == "gauss":
        return (replace(S.display_angular_ss(), recon=2), S.scene_paper(),
                WORKLOAD.replace("48 views", "96 views at random angles in their intervals, Gaussian "
                                             "reconstruction (8 samples, spatial diameter 2.25 px, angular "
                                             "support 2 views) to 48 (+crosstalk 0.15)"))
    if cfg == "pbr":
        return (S.display_paper(), S.scene_pbr_paper(),
                WORKLOAD.replace("64 RGBA8 textures 64^2-4096^2",
                                 "16 materials of four RGBA8 textures (albedo, normal, roughness, metallic) "
                                 "64^2-4096^2 each, physically based shading (one directional light + ambient)"))
    return S.display_paper(), S.scene_paper(), WORKLOAD


def shading_of(cfg):
    from paper_2601_19901_gb300 import scenes as S
    return S.Shading() if cfg == "pbr" else None


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline object and the reference arm)
# ---------------------------------------------------------------------------

def cpu_info():
    """Host cores and CPU model of the machine the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "usable_cores": len(os.sched_getaffinity(0)), "cpu_model": model or "unknown"}


def oracle_frame_single_core(d, sc, model, textures=None, shading=None, core=None):
    """One complete oracle frame (set-up, emission, fetch, splat and resolve
    of every rendered view, interleave), single-threaded, with the process
    pinned to one host core (as taskset -c would). Returns seconds."""
    import oracle as O
    old = os.sched_getaffinity(0)
    core = min(old) if core is None else core
    os.sched_setaffinity(0, {core})
    try:
        t0 = time.perf_counter()
        O.render(d, sc, model, textures=textures, shading=shading)
        return time.perf_counter() - t0
    finally:
        os.sched_setaffinity(0, old)


# Worker processes of the reference arm: each pinned to its own core, they
# splat and resolve their share of a frame's views from the frame's records
# and points in shared memory, and write their RGBA views back there.
_W = {}


def _worker_init(cores, counter, names, d, shading):
    import oracle as O
    from multiprocessing import shared_memory
    with counter.get_lock():
        k = counter.value
        counter.value += 1
    os.sched_setaffinity(0, {cores[k % len(cores)]})
    _W["shm"] = {n: shared_memory.SharedMemory(name=v) for n, v in names.items()}
    _W["d"] = d
    _W["shading"] = shading
    O.lib()


def _worker_views(views, n_points, n_tris):
    import oracle as O
    d = _W["d"]
    shm = _W["shm"]
    tri = np.ndarray((n_tris, O.TRI_FLOATS), np.float32, buffer=shm["tri"].buf)
    pts = np.ndarray((n_points, 4), np.uint32, buffer=shm["points"].buf)
    tvx = np.ndarray((n_points, 6), np.uint32, buffer=shm["tvx"].buf) if _W["shading"] is not None else None
    out = np.ndarray((d.n_render_views, d.view_h, d.view_w, 4), np.uint8, buffer=shm["rgba"].buf)
    _, rgba = O.splat_resolve(d, tri, pts, views, tvx=tvx, shading=_W["shading"])
    out[list(views)] = rgba
    return len(views)


class OracleFrames:
    """Complete oracle frames on the host cores: set-up, emission and fetch
    in this process, the splat and resolve of every rendered view spread over
    one pinned worker process per core, then the interleave here."""

    def __init__(self, cfg, d, sc, n_workers):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        import oracle as O
        self.d, self.sc, self.cfg = d, sc, cfg
        self.O = O
        cores = sorted(os.sched_getaffinity(0))
        self.n_workers = max(1, min(n_workers, len(cores), d.n_render_views))
        nr, T = d.n_render_views, sc.n_tris
        self.cap = 0
        self.shm = {"tri": shared_memory.SharedMemory(create=True, size=T * O.TRI_FLOATS * 4),
                    "rgba": shared_memory.SharedMemory(create=True, size=nr * d.view_h * d.view_w * 4)}
        self._points(1 << 22)
        ctx = mp.get_context("spawn")
        counter = ctx.Value("i", 0)
        self.pool = ctx.Pool(self.n_workers, initializer=_worker_init,
                             initargs=(cores, counter, {k: v.name for k, v in self.shm.items()}, d,
                                       shading_of(cfg)))
        self.groups = [list(g) for g in np.array_split(np.arange(nr), self.n_workers) if len(g)]

    def _points(self, cap):
        from multiprocessing import shared_memory
        if cap <= self.cap:
            return False
        for k in ("points", "tvx"):
            if k in self.shm:
                self.shm[k].close()
                self.shm[k].unlink()
        self.shm["points"] = shared_memory.SharedMemory(create=True, size=cap * 16)
        self.shm["tvx"] = shared_memory.SharedMemory(create=True, size=cap * 24)
        self.cap = cap
        return True

    def frame(self, model, textures=None, shading=None):
        O, d = self.O, self.d
        fr = O.render(d, self.sc, model, splat=False, textures=textures)
        P = len(fr.points)
        if self._points(max(P, 1)):
            # workers attach to buffers by name when they start: restart them
            raise RuntimeError("oracle frame needs %d points, more than the shared buffers hold" % P)
        np.ndarray((self.sc.n_tris, O.TRI_FLOATS), np.float32, buffer=self.shm["tri"].buf)[:] = fr.tri
        np.ndarray((P, 4), np.uint32, buffer=self.shm["points"].buf)[:] = fr.points
        if fr.tvx is not None:
            np.ndarray((P, 6), np.uint32, buffer=self.shm["tvx"].buf)[:] = fr.tvx
        done = self.pool.starmap(_worker_views, [(g, P, self.sc.n_tris) for g in self.groups])
        assert sum(done) == d.n_render_views
        rgba = np.ndarray((d.n_render_views, d.view_h, d.view_w, 4), np.uint8, buffer=self.shm["rgba"].buf)
        return O.interleave(d, rgba), P

    def close(self):
        self.pool.close()
        self.pool.join()
        for v in self.shm.values():
            v.close()
            v.unlink()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.config in ("batch", "learned"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single frames "
                          "(--config paper)"}), flush=True)
        return
    import oracle as O
    from paper_2601_19901_gb300 import scenes as S
    O.build()
    d, sc, wl = workload(args.config, args.scene_instances)
    tx = O.Textures(sc.textures)
    info = cpu_info()
    frames = OracleFrames(args.config, d, sc, info["usable_cores"])
    try:
        times, pts = [], []
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            _, P = frames.frame(S.model_matrix(k), textures=tx, shading=shading_of(args.config))
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                times.append(dt)
                pts.append(P)
    finally:
        frames.close()
    ms = 1000.0 * statistics.mean(times)
    v = 1000.0 / ms
    sample = ("complete frames, nothing extrapolated: the C oracle's set-up, emission and fetch on one core, "
              "its splat and resolve of all %d rendered views spread over %d worker processes pinned one per "
              "core, its interleave of the full panel; %d host cores usable (nproc %s), CPU %s"
              % (d.n_render_views, frames.n_workers, info["usable_cores"], info["nproc"], info["cpu_model"]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl, "l2": "n/a (CPU)", "points_per_frame": statistics.mean(pts)},
            "cpu_baseline": {"value": v, "unit": "frames/s", "cores": frames.n_workers, "kind": "oracle",
                             "sample": sample, "host": info},
            "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def atomic_peak(n_words, sm_stream):
    """Measured throughput (ops/s) of uncontended 64-bit atomicMin on a buffer
    of n_words, resolved in L2: at random indices ("global") and with every
    warp instruction on 32 consecutive words at a random base ("coherent");
    and in shared memory ("shared")."""
    import torch
    from paper_2601_19901_gb300 import lfdpr
    g = torch.Generator(device="cuda").manual_seed(7)
    n_ops = 1 << 26
    words = torch.full((n_words,), -1, dtype=torch.int64, device="cuda")
    idx = torch.randint(0, n_words, (n_ops,), dtype=torch.int32, device="cuda", generator=g)
    val = torch.randint(0, 1 << 62, (n_ops,), dtype=torch.int64, device="cuda", generator=g)
    out = {}
    for name, mode, nw in (("global", lfdpr.PROBE_RANDOM, n_words), ("coherent", lfdpr.PROBE_COHERENT, n_words),
                           ("shared", lfdpr.PROBE_SHARED, 4096)):
        for _ in range(2):
            lfdpr.lfdpr_probe_atomic_min(words.data_ptr(), nw, idx.data_ptr(), val.data_ptr(), n_ops, mode,
                                         sm_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = math.inf
        for _ in range(3):
            e0.record(sm_stream)
            lfdpr.lfdpr_probe_atomic_min(words.data_ptr(), nw, idx.data_ptr(), val.data_ptr(), n_ops, mode,
                                         sm_stream)
            e1.record(sm_stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1000.0)
        out[name] = n_ops / best
    del words, idx, val
    return out


def source_digest(sources) -> str:
    """sha256 of kernel sources with their comments and blank space removed,
    so that a comment edit does not orphan an ncu summary of the same code."""
    import hashlib
    import re
    hsh = hashlib.sha256()
    for f in sources:
        text = open(os.path.join(ROOT, "paper_2601_19901_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        hsh.update(" ".join(text.split()).encode())
    return hsh.hexdigest()


def profiled_traffic(profile: str, sources):
    """DRAM bytes (read + write) per launch from a committed ncu summary, if
    the kernel's sources still hash to what was captured; else None."""
    import re
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"sha256: ([0-9a-f]{64})", text)
    if not m or m.group(1) != source_digest(sources):
        return None
    rd = re.search(r"dram__bytes_read\.sum`\) \| ([0-9.]+) Mbyte", text)
    wr = re.search(r"dram__bytes_write\.sum`\) \| ([0-9.]+) Mbyte", text)
    if not rd or not wr:
        return None
    return (float(rd.group(1)) + float(wr.group(1))) * 1e6


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2601_19901_gb300 import build as B, lfdpr, multigpu, scenes as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        dist.barrier()
    lfdpr.lib()
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    d, sc, wl = workload(args.config, args.scene_instances)
    stream = torch.cuda.Stream()
    R = lfdpr.Renderer(d, sc, max_points=(1 << 24) if args.config == "gauss2x" else 0, stream=stream,
                       shading=shading_of(args.config))
    R.set_stage_timing(True)
    if args.view_band is not None:
        lfdpr.lfdpr_set_view_band(R.disp, args.view_band)
    if d.recon in (2, 3):
        # Sec. 4's random angles and Gaussian samples (seeded; sigma = diameter / 4, in output
        # pixels: with spatial supersampling the reconstruction reads the views' mip level
        # whose texels are output pixels)
        rng = np.random.default_rng(2024)
        R.set_view_jitter(rng.random(d.n_render_views).astype(np.float32))
        R.set_recon_samples((rng.normal(0.0, 1.0, (8, 3)) * [2.25 / 4, 2.25 / 4, 0.5]).astype(np.float32))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    panel = torch.empty((d.panel_h, d.panel_w, 4), dtype=torch.uint8, device="cuda")
    frames = multigpu.rank_frames(rank, world, args.warmup + args.steps)
    e2e_frames = multigpu.rank_frames(rank, world, max(3, args.steps // 2), start=50000)

    def frame_model(k):
        return S.model_matrix(frames[k])

    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            R.render(frame_model(k), stream)
            R.interleave(panel.data_ptr(), stream)
            R.stats(stream)

    peaks_atomic = atomic_peak(d.n_render_views * d.view_w * d.view_h, stream)

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    step_ms, stage = [], {n: [] for n in lfdpr.STAGES}
    n_points = []
    n_writes = []
    # the timed frames carry no per-stage events (about 20 us a frame on the
    # device); the stages are timed in as many instrumented frames right after
    R.set_stage_timing(False)
    launches0 = R.stats(stream).kernel_launches
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 255)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R.render(frame_model(args.warmup + k), stream)
        R.interleave(panel.data_ptr(), stream)
        e1.record(stream)
        st = R.stats(stream)
        step_ms.append(e0.elapsed_time(e1))
        n_points.append(st.n_points)
        n_writes.append(getattr(st, "n_splat_writes", 0))
    torch.cuda.synchronize()
    launches = R.stats(stream).kernel_launches - launches0
    clk = clocks.stop()
    R.set_stage_timing(True)
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 255)
        R.render(frame_model(args.warmup + k), stream)
        R.interleave(panel.data_ptr(), stream)
        st = R.stats(stream)
        for i, n in enumerate(lfdpr.STAGES):
            stage[n].append(st.stage_ms[i])
    R.set_stage_timing(False)
    total_ms = multigpu.max_over_ranks(sum(step_ms), device="cuda")
    if world > 1:
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = multigpu.job_rate(world, args.steps, total_ms / 1000.0)
    P = statistics.mean(n_points)

    # e2e: the public API with host buffers (model matrix in, panel out to pinned memory)
    e2e = None
    if not args.no_e2e:
        host_panel = torch.empty((d.panel_h, d.panel_w, 4), dtype=torch.uint8).pin_memory()
        model_host = torch.empty((4, 4), dtype=torch.float32).pin_memory()
        e2e_s = 0.0
        n_e2e = len(e2e_frames)
        for k in range(n_e2e):
            with torch.cuda.stream(stream):
                flush.fill_(k & 255)
            torch.cuda.synchronize()
            model_host.copy_(torch.from_numpy(S.model_matrix(e2e_frames[k])))
            t0 = time.perf_counter()
            R.render(model_host.numpy(), stream)
            R.interleave(host_panel.data_ptr(), stream)   # copies to host and waits
            e2e_s += time.perf_counter() - t0
        e2e_s = multigpu.max_over_ranks(e2e_s, device="cuda")
        e2e = {"value": multigpu.job_rate(world, n_e2e, e2e_s), "unit": "frames/s", "h2d_bytes_per_step": 64,
               "d2h_bytes_per_step": 4 * d.panel_w * d.panel_h}
        # what the host link allows: the panel's bytes copied device -> pinned host
        # by the copy engine (the interleave's own stores into pinned memory cross
        # the same link)
        link = []
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with torch.cuda.stream(stream):
                host_panel.copy_(panel, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            link.append(e0.elapsed_time(e1))
        link_ms = statistics.median(link)
        e2e["host_link"] = {"d2h_gbs": 4 * d.panel_w * d.panel_h / (link_ms / 1000.0) / 1e9,
                            "panel_copy_ms": link_ms,
                            "what": "the panel copied device -> pinned host by the copy engine, median of 10"}

    if rank != 0:
        R.close()
        if world > 1:
            dist.destroy_process_group()
        return

    st_mean = {n: statistics.mean(v) for n, v in stage.items()}
    splat_ms = st_mean["splat"]
    npix = d.n_render_views * d.view_w * d.view_h
    b = R.buffers()
    n_live = R.stats(stream).n_live_tris
    # the splat's algorithmic bytes: each point's 16 B and its triangle's 80 B
    # read once, each view pixel's 8-B key written once
    splat_bytes = 16 * P + 80 * n_live + 8 * npix
    achieved = splat_bytes / (splat_ms / 1000.0) / 1e9
    traffic = profiled_traffic("k_splat_paper_frame.md", ["splat.cu", "lfdpr_internal.cuh"]) \
        if args.config == "paper" and args.scene_instances == 200 else None
    roof_hbm = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic, "kernel": "k_splat",
                "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": splat_bytes}
    writes = statistics.mean(n_writes)
    a_rate = writes / (splat_ms / 1000.0) / 1e9
    # against the faster of the two global patterns (the splat's atomics are
    # neither fully random nor fully coherent)
    a_which = "coherent" if peaks_atomic["coherent"] >= peaks_atomic["global"] else "global"
    a_peak = peaks_atomic[a_which] / 1e9
    roof_atomic = {"bound": "atomic", "achieved": a_rate, "peak": a_peak, "unit": "Gop/s",
                   "frac": a_rate / a_peak, "traffic": traffic, "kernel": "k_splat",
                   "peak_source": "measured in this run: uncontended 64-bit atomicMin over a buffer the size of "
                                  "the view keys, the faster of random indices (%.1f Gop/s) and warp-coherent "
                                  "runs of 32 consecutive words (%.1f Gop/s): %s"
                                  % (peaks_atomic["global"] / 1e9, peaks_atomic["coherent"] / 1e9, a_which),
                   "frac_of_random_peak": a_rate / (peaks_atomic["global"] / 1e9),
                   "frac_of_coherent_peak": a_rate / (peaks_atomic["coherent"] / 1e9),
                   "algorithmic_ops_per_launch": writes}
    roofline, roofline_other = (roof_atomic, roof_hbm) if roof_atomic["frac"] >= roof_hbm["frac"] \
        else (roof_hbm, roof_atomic)
    line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl, "l2": "flushed (512 MiB write) between timed steps",
                       "points_per_frame": P, "rendered_views": d.n_render_views,
                       "view_band": args.view_band},
            "points_per_s": value * P,
            "point_view_splats_per_s": P * d.n_render_views / (splat_ms / 1000.0),
            "stage_ms": st_mean,
            "stage_ms_note": "CUDA events between the stages of %d instrumented frames run right after the timed "
                             "ones (the same frames, L2 flushed); the events add about 20 us a frame, so the "
                             "timed frames carry none" % args.steps,
            "roofline": roofline,
            "roofline_other": roofline_other,
            "splat_writes_per_frame": writes,
            "atomic_peak_ops_per_s": peaks_atomic,
            "gpu_launches": int(launches),
            "clocks": clk}
    if e2e:
        line["e2e"] = e2e
    if world == 1 and not args.no_cpu_baseline and d.recon in (0, 1):
        import oracle as O
        O.build()
        info = cpu_info()
        core = min(os.sched_getaffinity(0))
        t_full = oracle_frame_single_core(d, sc, frame_model(0), shading=shading_of(args.config), core=core)
        t_tiny = oracle_frame_single_core(S.display_tiny(), S.scene_tiny(), S.model_matrix(0), core=core)
        line["cpu_baseline"] = {"value": 1.0 / t_full, "unit": "frames/s", "cores": 1, "kind": "oracle",
                                "sample": "one complete frame of this workload (all %d rendered views, nothing "
                                          "extrapolated) by the single-threaded C oracle pinned to host core %d; "
                                          "%d cores usable (nproc %s), CPU %s"
                                          % (d.n_render_views, core, info["usable_cores"], info["nproc"],
                                             info["cpu_model"]),
                                "seconds_per_frame": t_full,
                                "tiny_frame_seconds": t_tiny,
                                "tiny_frame": "2,048 triangles, 8 views of 128x128, 512x512 panel",
                                "host": info}
    if world == 1 and args.config == "paper" and not args.no_secondary:
        line["secondary"] = secondary_measurements(args, sc, stream)
    print(json.dumps(line), flush=True)
    R.close()
    if world > 1:
        dist.destroy_process_group()


def batch_measure(n_scenes, tris_range, steps, warmup, stream, world=1, rank=0, clocks=None):
    """Batched multi-scene frames (one CUDA graph per batch, autotuned): the
    batch's frames/s with L2 flushed between batches, per-scene latency, and
    the same frames one scene after another for comparison."""
    import torch
    from paper_2601_19901_gb300 import lfdpr, multigpu, scenes as S
    ds, scs = S.batch_paper(n_scenes=n_scenes, tris_range=tris_range)
    n = len(ds)
    ts = lfdpr.TextureSet(S.textures_paper(), stream)
    B = lfdpr.Batch(ds, scs, ts, [max(1 << 20, 6 * sc.n_tris) for sc in scs], stream)
    try:
        flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        base = multigpu.rank_frames(rank, world, 1)[0]

        def models(f):
            return np.stack([S.model_matrix(base + f + 7 * k) for k in range(n)]).astype(np.float32)

        cfg, tuned_ms = B.autotune(models(0), reps=2, stream=stream)
        table = B.autotune_table()
        for w in range(warmup):
            B.render(models(1 + w), stream)
        for i in range(n):
            st = B.stats(i, stream)
            if st.overflow or st.cell_overflow:
                raise RuntimeError("scene %d overflowed its point buffer" % i)
        torch.cuda.synchronize()
        if clocks is not None:
            clocks.start()
            time.sleep(0.3)
        ms, scene_ms = [], []
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.render(models(1 + warmup + k), stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            scene_ms.append(B.scene_ms())
        clk = clocks.stop() if clocks is not None else None
        points = sum(B.stats(i, stream).n_points for i in range(n))
        # the same frames one scene after another through lfdpr_render_frame + lfdpr_interleave
        seq = []
        for k in range(max(2, min(steps, 5))):
            m = models(1 + warmup + k)
            with torch.cuda.stream(stream):
                flush.fill_(k & 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(n):
                lfdpr.lfdpr_render_frame(B.disps[i], B.meshes[i], m[i], stream)
                lfdpr.lfdpr_interleave(B.disps[i], B.panel(i), stream)
            e1.record(stream)
            e1.synchronize()
            seq.append(e0.elapsed_time(e1))
        ms_sorted = sorted(ms)
        pct = lambda q: ms_sorted[min(len(ms_sorted) - 1, int(math.ceil(q * len(ms_sorted))) - 1)]
        seq_rate = n / (statistics.mean(seq) / 1000.0)
        return {"ms": ms, "n": n, "clk": clk, "points": points,
                "workload": "%d paper-shaped scenes, %d triangles in all (%d-%d per scene), 24/48/96 views at "
                            "420x560 or 640x360, 2560x1600 panels, 64 shared textures 64^2-4096^2"
                            % (n, sum(s.n_tris for s in scs), min(s.n_tris for s in scs), max(s.n_tris for s in scs)),
                "rendered_views": sum(d.n_render_views for d in ds),
                "batch_ms_p50": pct(0.50), "batch_ms_p99": pct(0.99),
                "scene_latency_ms": {
                    "p50": float(np.percentile(np.concatenate(scene_ms), 50)),
                    "p99": float(np.percentile(np.concatenate(scene_ms), 99)),
                    "per_scene_p50": [round(float(x), 3) for x in np.percentile(np.stack(scene_ms), 50, axis=0)],
                    "per_scene_p99": [round(float(x), 3) for x in np.percentile(np.stack(scene_ms), 99, axis=0)],
                    "what": "device time from the start of the batch's graph to the end of each scene's "
                            "interleave (events inside the graph), over every scene and timed batch"},
                "sequential_frames_per_s": seq_rate,
                "autotuned": {"branches": cfg.branches, "splat_blocks_per_sm": cfg.splat_blocks_per_sm,
                              "splat_slots": cfg.splat_slots, "ms_per_batch_while_tuning": tuned_ms,
                              "candidates_ms": {"%d/%d/%d" % t[:3]: round(t[3], 3) for t in table}}}
    finally:
        B.close()
        ts.close()


def run_batch(args):
    import torch
    import torch.distributed as dist
    from paper_2601_19901_gb300 import build as B_, lfdpr, multigpu

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        B_.build()
    if world > 1:
        dist.barrier()
    lfdpr.lib()
    lo, hi = (float(x) for x in args.batch_tris.split(","))
    stream = torch.cuda.Stream()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    if world > 1:
        dist.barrier()
    r = batch_measure(args.batch_scenes, (lo, hi), args.steps, args.warmup, stream, world, rank, ClockSampler(uuid))
    n, ms = r["n"], r["ms"]
    total_ms = multigpu.max_over_ranks(sum(ms), device="cuda")
    value = multigpu.job_rate(world, n * args.steps, total_ms / 1000.0)
    if world > 1:
        dist.barrier()
    if rank == 0:
        line = {"metric": "batched multi-scene display frames/s (every scene of the batch rendered and "
                          "interleaved)",
                "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": r["workload"], "l2": "flushed (512 MiB write) between timed batches",
                           "rendered_views": r["rendered_views"]},
                "batch_ms_p50": r["batch_ms_p50"], "batch_ms_p99": r["batch_ms_p99"],
                "scene_latency_ms": r["scene_latency_ms"],
                "points_per_batch": r["points"], "points_per_s": r["points"] * args.steps * world / (total_ms / 1000.0),
                "sequential_frames_per_s": r["sequential_frames_per_s"],
                "speedup_vs_sequential": value / world / r["sequential_frames_per_s"],
                "autotuned": r["autotuned"],
                "gpu_launches": int(args.steps * (7 * n + 1)),
                "clocks": r["clk"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def pbr_measure(stream, steps=10, warmup=3):
    """Meshes of materials with physically based shading on the paper-shaped
    geometry: frames/s with L2 flushed between frames, then the stages of as
    many instrumented frames."""
    import torch
    from paper_2601_19901_gb300 import lfdpr, scenes as S
    d, sc = S.display_paper(), S.scene_pbr_paper()
    R = lfdpr.Renderer(d, sc, stream=stream, shading=S.Shading())
    try:
        flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        panel = torch.empty((d.panel_h, d.panel_w, 4), dtype=torch.uint8, device="cuda")
        for k in range(warmup):
            R.render(S.model_matrix(k), stream)
            R.interleave(panel.data_ptr(), stream)
        ms, stage = [], {n: [] for n in lfdpr.STAGES}
        for timing in (False, True):
            R.set_stage_timing(timing)
            for k in range(steps):
                with torch.cuda.stream(stream):
                    flush.fill_(k & 255)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                R.render(S.model_matrix(warmup + k), stream)
                R.interleave(panel.data_ptr(), stream)
                e1.record(stream)
                st = R.stats(stream)
                if timing:
                    for i, n in enumerate(lfdpr.STAGES):
                        stage[n].append(st.stage_ms[i])
                else:
                    ms.append(e0.elapsed_time(e1))
        return {"what": "the paper-shaped geometry with 16 materials of four textures (albedo, normal, roughness, "
                        "metallic) 64^2-4096^2, physically based shading, 48 views, interleaved; %d frames, L2 "
                        "flushed" % steps,
                "frames_per_s": 1000.0 / statistics.mean(ms),
                "stage_ms": {n: statistics.mean(v) for n, v in stage.items()}}
    finally:
        R.close()


def learned_measure(sc, steps, warmup, quality_frames, stream=None):
    """The learned quarter-view path (12 views rendered, the U-Net's
    tensor-core kernels predict the 48 reconstructed views, interleave) and
    the plain renders it stands in for, on scene `sc`: frames/s of each with
    L2 flushed between frames, the network alone, and per-frame PSNR / SSIM
    of the prediction against both readings of its ground truth (the full render's
    96-view tent reconstruction, and the plain 48-view render)."""
    import torch
    from dataclasses import replace
    from paper_2601_19901_gb300 import lfdpr, recon_net as RN, scenes as S
    w, b, nin = RN.load_weights()
    d_in = replace(S.display_paper(), n_views=nin)
    d_full = S.display_angular_ss()
    d_out = replace(S.display_paper(), n_views=4 * nin, crosstalk=d_full.crosstalk)
    d_plain = S.display_paper()
    H, W = d_in.view_h, d_in.view_w
    stream = stream or torch.cuda.Stream()
    ts = lfdpr.TextureSet(sc.textures, stream)
    # input, full (2x angular), learned output, and the plain 4n-view render
    dis = [lfdpr.lfdpr_create_display(lfdpr.desc_of(d)) for d in (d_in, d_full, d_out, d_plain)]
    me = [lfdpr.lfdpr_upload_mesh_textured(dis[k], sc.xyz, sc.uv, sc.idx, sc.tri_tex, ts.handle, stream)
          for k in (0, 1, 3)]
    R = lfdpr.Recon(W, H, nin, w, b)
    in_eyes = torch.from_numpy(lfdpr.lfdpr_view_eyes(dis[0], nin)).cuda()
    out_eyes = torch.from_numpy(lfdpr.lfdpr_view_eyes(dis[2], 4 * nin)).cuda()
    panel = torch.empty((d_out.panel_h, d_out.panel_w, 4), dtype=torch.uint8, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    try:
        def learned(f):
            lfdpr.lfdpr_render_frame(dis[0], me[0], S.model_matrix(f), stream)
            R.run(dis[0], dis[2], stream)
            lfdpr.lfdpr_interleave(dis[2], panel.data_ptr(), stream)

        def full(f):
            lfdpr.lfdpr_render_frame(dis[1], me[1], S.model_matrix(f), stream)
            lfdpr.lfdpr_interleave(dis[1], panel.data_ptr(), stream)

        def plain(f):
            lfdpr.lfdpr_render_frame(dis[3], me[2], S.model_matrix(f), stream)
            lfdpr.lfdpr_interleave(dis[3], panel.data_ptr(), stream)

        def timed(fn, first):
            for k in range(warmup):
                fn(first + k)
            ms = []
            for k in range(steps):
                with torch.cuda.stream(stream):
                    flush.fill_(k & 255)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn(first + warmup + k)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            return statistics.mean(ms)

        # the network alone
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        learned(0)
        e0.record(stream)
        for _ in range(10):
            R.run(dis[0], dis[2], stream)
        e1.record(stream)
        e1.synchronize()
        net_ms = e0.elapsed_time(e1) / 10
        ms_learned = timed(learned, 0)
        ms_full = timed(full, 0)
        ms_plain = timed(plain, 0)
        q = []
        for f in quality_frames:
            learned(f)
            full(f)
            plain(f)
            torch.cuda.synchronize()
            bf = lfdpr.lfdpr_get_buffers(dis[1], me[1])
            truth = RN.tent_views(lfdpr.device_view(bf.views, (2 * d_full.n_views, H, W, 4), np.uint8))
            bo = lfdpr.lfdpr_get_buffers(dis[2], me[0])
            pred = lfdpr.device_view(bo.views, (4 * nin, H, W, 4), np.uint8)[..., :3]
            b4 = lfdpr.lfdpr_get_buffers(dis[3], me[2])
            plain48 = lfdpr.device_view(b4.views, (4 * nin, H, W, 4), np.uint8)[..., :3]
            bi = lfdpr.lfdpr_get_buffers(dis[0], me[0])
            warp = RN.warped_base(lfdpr.device_view(bi.views, (nin, H, W, 4), np.uint8),
                                  lfdpr.device_view(bi.keys, (nin, H, W), np.uint64), in_eyes, out_eyes,
                                  RN.pixels_per_unit(d_in))[..., :3]
            q.append((RN.psnr(pred, truth), RN.ssim(pred, truth), RN.psnr(plain48, truth),
                      RN.psnr(pred, plain48), RN.ssim(pred, plain48), RN.psnr(warp, truth), RN.psnr(warp, plain48)))
        # algorithmic FLOPs of one forward pass: the 3x3 layers over the padded
        # views plus the 1x1 output layer (32 x 3 * 4n); the warp is not counted
        flops = 0
        hp, wp = RN.padded(H, W)
        for ci, co, lev in RN.LAYERS:
            flops += 2 * 9 * ci * co * (hp >> lev) * (wp >> lev)
        flops += 2 * 32 * 3 * 4 * nin * hp * wp
    finally:
        R.close()
        for m_ in me:
            lfdpr.lfdpr_destroy_mesh(m_)
        for d_ in dis:
            lfdpr.lfdpr_destroy_display(d_)
        ts.close()
    return {"views_rendered": nin, "views_predicted": 4 * nin,
            "frames_per_s": 1000.0 / ms_learned, "ms_per_frame": ms_learned,
            "full_render_frames_per_s": 1000.0 / ms_full, "plain_48_view_frames_per_s": 1000.0 / ms_plain,
            "network_ms": net_ms, "network_flops": flops, "network_tflops": flops / (net_ms / 1000.0) / 1e12,
            "vs_full_render": {"what": "ground truth = the 96-view render's tent reconstruction (the display's "
                                       "angularly supersampled views)",
                               "psnr_db_mean": statistics.mean(x[0] for x in q),
                               "psnr_db_min": min(x[0] for x in q),
                               "ssim_mean": statistics.mean(x[1] for x in q),
                               "speedup": ms_full / ms_learned},
            "vs_plain_48_views": {"what": "ground truth = the plain 48-view render",
                                  "psnr_db_mean": statistics.mean(x[3] for x in q),
                                  "psnr_db_min": min(x[3] for x in q),
                                  "ssim_mean": statistics.mean(x[4] for x in q),
                                  "speedup": ms_plain / ms_learned},
            "plain_48_views_vs_full_render_psnr_db": statistics.mean(x[2] for x in q),
            "warped_base_alone_psnr_db": {"vs_full_render": statistics.mean(x[5] for x in q),
                                          "vs_plain_48_views": statistics.mean(x[6] for x in q)},
            "quality_frames": list(quality_frames)}


def run_learned(args):
    from paper_2601_19901_gb300 import build as B_, lfdpr, scenes as S
    B_.build()
    lfdpr.lib()
    m = learned_measure(S.scene_paper(), args.steps, args.warmup, range(0, 120, 8))
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak_tf = peaks.get("bf16_tflops", 1900.0)
    line = {"metric": "learned quarter-view path frames/s at PSNR vs the plain full render",
            "value": m["frames_per_s"], "unit": "frames/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_per_frame"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 (network), f32 (render)", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("48 views", "%d views rendered, 48 predicted"
                                                    % m["views_rendered"]),
                       "l2": "flushed (512 MiB write) between timed steps"},
            "learned": m,
            "roofline": {"bound": "tensor", "achieved": m["network_tflops"], "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": m["network_tflops"] / peak_tf, "traffic": None,
                         "kernel": "the network (k_conv_tc, tcgen05)",
                         "peak_source": "measured bf16 dense GEMM, burst (MEASURED_PEAKS.json)"
                         if "bf16_tflops" in peaks else "fallback 1.9 PFLOP/s bf16"}}
    print(json.dumps(line), flush=True)


def secondary_measurements(args, sc, stream):
    """Frames/s of the 96-view (2x angular, tent, crosstalk) frame on the same
    scene, the learned quarter-view path with its quality against both
    readings of its ground truth, a batch of 32 paper-shaped scenes, and the
    meshes of materials with physically based shading: measured after the
    main timed region, reported beside it (not part of `value`)."""
    import torch
    from paper_2601_19901_gb300 import lfdpr, scenes as S
    out = {}
    d = S.display_angular_ss()
    R = lfdpr.Renderer(d, sc, stream=stream)
    try:
        flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        panel = torch.empty((d.panel_h, d.panel_w, 4), dtype=torch.uint8, device="cuda")
        for k in range(3):
            R.render(S.model_matrix(k), stream)
            R.interleave(panel.data_ptr(), stream)
        ms, splat = [], []
        for timing in (False, True):   # whole frames uninstrumented, then the splat's stage time
            R.set_stage_timing(timing)
            for k in range(10):
                with torch.cuda.stream(stream):
                    flush.fill_(k & 255)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                R.render(S.model_matrix(3 + k), stream)
                R.interleave(panel.data_ptr(), stream)
                e1.record(stream)
                st = R.stats(stream)
                if timing:
                    splat.append(st.stage_ms[lfdpr.STAGES.index("splat")])
                else:
                    ms.append(e0.elapsed_time(e1))
        out["angular_96_views"] = {"what": "the same scene rendered at 2x angular rate (96 views of 420x560), "
                                           "tent to 48, crosstalk 0.15, interleaved; 10 frames, L2 flushed",
                                   "frames_per_s": 1000.0 / statistics.mean(ms),
                                   "splat_ms": statistics.mean(splat)}
    finally:
        R.close()
    try:
        out["learned"] = learned_measure(sc, 10, 3, range(0, 120, 15), stream)
    except Exception as e:   # the weights ship with the package; report rather than hide a failure
        out["learned"] = {"error": repr(e)}
    try:
        r = batch_measure(32, (5.0e4, 2.0e6), 5, 2, stream)
        out["batch_32_scenes"] = {
            "what": r["workload"] + "; one CUDA graph per batch, autotuned; 5 batches, L2 flushed",
            "frames_per_s": r["n"] * len(r["ms"]) / (sum(r["ms"]) / 1000.0),
            "batch_ms_p50": r["batch_ms_p50"], "scene_latency_ms_p50": r["scene_latency_ms"]["p50"],
            "scene_latency_ms_p99": r["scene_latency_ms"]["p99"],
            "sequential_frames_per_s": r["sequential_frames_per_s"], "autotuned": {
                k: r["autotuned"][k] for k in ("branches", "splat_blocks_per_sm", "splat_slots")}}
    except Exception as e:
        out["batch_32_scenes"] = {"error": repr(e)}
    try:
        out["pbr_materials"] = pbr_measure(stream)
    except Exception as e:
        out["pbr_materials"] = {"error": repr(e)}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "batch":
        run_batch(args)
    elif args.config == "learned":
        run_learned(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
