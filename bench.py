"""Benchmark: 1080p stabilised frames/s on one GB300 (batched vs plain) and
per-step latency percentiles.

Workload (one step): every stream of a batch of 16 independent 1920x1080 RGB
videos advances by one frame through the whole path -- luma + 5-level
pyramid with FP16 I/Ix/Iy planes, corner detection when due (every 5th
frame), pyramidal LK forward + backward on 1000 corners, robust similarity
fit (100 hypotheses), streaming 30-frame smoothing, RGB compensating warp --
as one CUDA-graph launch.  `value` = stabilised frames/s of the batch with
the frames already in HBM (an input ring larger than L2); `plain` = the same
path for one stream through the single-stream calls with FP32 planes;
`e2e` = the batch through stab_batch_step_host with pinned host frames in and
stabilised frames out.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun the job is N x 16 independent videos dealt round-robin to the
ranks (16 per GPU; no exchange between them), each rank runs its share as one
batch on its own GPU, and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes as C
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "1080p stabilized frames/s on 1 GB300 (batched vs plain); p99 frame latency ms"
W, H, CH = 1920, 1080, 3
STREAMS = 16
PARAMS = dict(max_corners=1000, levels=5, hypotheses=100, smooth_window=30, model=1)
PERIOD = 5      # re-detection period (Sec. 3.2: detect on one frame, track through the next five)
RING = 2 * (PARAMS["smooth_window"] // 2 + 2)   # >= W/2 + 5 frames, even for the retracing clip
FP32_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz max SM clock"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# LK algorithmic work per window sample: template pass = bilinear I, Ix, Iy
# (3 x 7 flop) + G accumulation (3 FMA = 6 flop) = 27; iteration = bilinear J
# (7) + residual (1) + b accumulation (2 FMA = 4) = 12.
LK_FLOP_TEMPLATE, LK_FLOP_ITER = 27, 12
# A coarser count of the same work (6.6 k and 3.1 k flop per 441-sample window,
# about 15 and 7 per sample: one sampled plane in the template pass), reported
# beside ours.
LK_FLOP_COARSE = (15, 7)
# DRAM traffic per launch of the dominant kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch on this workload,
# 16 streams); used only while the kernel source is unchanged.
TRAFFIC = {"lk": {"file": "k_lk.cu", "sha": "3a780bf14d08eb32", "bytes_per_launch": 198758912 + 6637056}}


def phase_of(g: int, staggered: bool) -> int:
    """Place of video g in its detection cycle: staggered videos enter the cycle
    at g mod period, so that a fifth of the streams detect at each step, as
    independently started videos would; lockstep videos all detect together."""
    return g % PERIOD if staggered else 0


def config_dict(streams, staggered=False):
    return {"workload": f"{streams} streams x 1920x1080 RGB, config-2 shape (K=1000 corners, 5 levels, "
                        "similarity, 100 hypotheses, 30-frame window), batched CUDA-graph step, FP16 plane storage",
            "streams": streams, "resolution": "1920x1080", "channels": 3, "corners": 1000, "levels": 5,
            "hypotheses": 100, "smooth_window": 30,
            "detection": (f"every {PERIOD}th frame; streams staggered (video g detects on frames t with "
                          f"(t + g) % {PERIOD} == 0)" if staggered else
                          f"every {PERIOD}th frame, all streams on the same steps"),
            "l2": "inputs larger than L2: each step reads new frames from a device ring of "
                  f"{streams} x {RING} RGB 1080p frames ({streams * RING * W * H * CH / 1e9:.1f} GB)"}


# ------------------------------------------------------------ distributed --
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def partition_streams(total: int, world: int, rank: int) -> list:
    """Stream indices of `rank` (round-robin): independent videos, no exchange."""
    return list(range(rank, total, world))


def partition_by_area(sizes: list, world: int, rank: int) -> list:
    """Indices of `rank`'s streams when streams of unequal size are spread over
    `world` GPUs: streams sorted by pixel area (largest first, ties by index)
    and dealt round-robin, so every rank gets a like mix of sizes."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i][0] * sizes[i][1], i))
    return sorted(order[k] for k in range(rank, len(order), world))


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu: int):
        self.gpu, self.proc, self.path = gpu, None, None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                rows.append((float(f[0]), float(f[1]), f[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


class NvmlClockSampler:
    """SM clock and clock-event reasons sampled through NVML every few ms by a
    separate process (this file run with --clock-sampler), so that even a timed
    region of a few ms holds several samples; only reads the GPU's state."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, device_index: int, uuid: str | None, period_ms: float = 2.0):
        self.index, self.uuid, self.period = device_index, uuid, period_ms
        self.proc, self.path = None, None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = [sys.executable, os.path.abspath(__file__), "--clock-sampler", self.path, "--clock-index",
                   str(self.index), "--clock-period-ms", str(self.period)]
            if self.uuid:
                cmd += ["--clock-uuid", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            deadline = time.time() + 10
            while time.time() < deadline and os.path.getsize(self.path) == 0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def stop(self, t0: float, t1: float):
        """Stats of the samples taken in [t0, t1] (time.time() seconds)."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = line.strip().split(",")
            if len(f) == 4:
                try:
                    rows.append((float(f[0]), float(f[1]), float(f[2]), int(f[3])))
                except ValueError:
                    pass
        os.unlink(self.path)
        inside = [r for r in rows if t0 <= r[0] <= t1]
        if not inside:
            return None
        reasons = sorted({name for r in inside for bit, name in self.REASONS.items() if r[3] & bit})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "sm_mhz_min": min(r[1] for r in inside), "reasons": reasons, "samples": len(inside),
                "period_ms": self.period, "source": "NVML, samples inside the timed region"}


def clock_sampler_main(path: str, index: int, uuid: str | None, period_ms: float):
    import signal
    L = C.CDLL("libnvidia-ml.so.1")
    if L.nvmlInit_v2() != 0:
        return
    h = C.c_void_p()
    ok = False
    if uuid:
        u = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        ok = L.nvmlDeviceGetHandleByUUID(u.encode(), C.byref(h)) == 0
    if not ok and L.nvmlDeviceGetHandleByIndex_v2(index, C.byref(h)) != 0:
        return
    try:
        reasons_fn = L.nvmlDeviceGetCurrentClocksEventReasons
    except AttributeError:
        reasons_fn = L.nvmlDeviceGetCurrentClocksThrottleReasons
    stop = []
    signal.signal(signal.SIGTERM, lambda *a: stop.append(1))
    clk, mx, rs = C.c_uint(), C.c_uint(), C.c_ulonglong()
    L.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx))          # 1 = NVML_CLOCK_SM
    with open(path, "w") as f:
        while not stop:
            t = time.time()
            if L.nvmlDeviceGetClockInfo(h, 1, C.byref(clk)) == 0 and reasons_fn(h, C.byref(rs)) == 0:
                f.write(f"{t:.6f},{clk.value},{mx.value},{rs.value}\n")
                f.flush()
            time.sleep(period_ms / 1e3)
    L.nvmlShutdown()


def device_uuid(dev) -> str | None:
    try:
        import torch
        u = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
        return str(u) if u is not None else None
    except Exception:
        return None


# ------------------------------------------------------------------ frames --
def make_frames(n_clips: int, ring: int, device: str):
    """n_clips seeded 1080p RGB clips of `ring` frames that retrace their path
    (frame ring == frame 0), so cycling the ring is a continuous video."""
    import dataclasses

    import torch
    from paper_1701_03572_gb300.synth import CONFIG_SPECS, make_clip
    spec = dataclasses.replace(CONFIG_SPECS[2], frames=ring, pingpong=True)
    return [make_clip(spec, 2000 + c, device=device, dtype=torch.float32)["frames"] for c in range(n_clips)]


# ----------------------------------------------------------- our arm (GPU) --
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = f"cuda:{local}" if ws > 1 else "cuda:0"
    torch.cuda.set_device(dev)
    from paper_1701_03572_gb300 import build as build_lib
    build_lib()
    from paper_1701_03572_gb300 import stab as S

    B = args.streams
    A = PARAMS["smooth_window"] // 2
    ring = RING
    # the job: ws x B independent videos dealt round-robin to the ranks; video g
    # shows seeded clip g % n_clips starting 3 (g // n_clips) frames in
    mine = partition_streams(ws * B, ws, rank)
    n_clips = min(args.clips, B)
    clips = make_frames(n_clips, ring, dev)
    staggered = args.detect_phases == "staggered"
    src_clip = [g % n_clips for g in mine]
    offs = [(g // n_clips) * 3 % ring for g in mine]

    def make_batch(stag):
        b = S.Batch([(W, H, CH, S.default_params(**PARAMS, precision=S.STAB_FP16_STORAGE,
                                                 redetect_phase=phase_of(g, stag))) for g in mine], ring=ring)
        for i in range(len(mine)):
            for s in range(ring):
                b.input_slot(i, s).copy_(clips[src_clip[i]][(s + offs[i]) % ring])
        return b

    batch = make_batch(staggered)
    stream = torch.cuda.current_stream()
    # prime the smoother's lookahead (no composed frame before step A + 3: the
    # step tracks one frame behind the frame it ingests and composes one step
    # after the fit),
    # pick the tracker variant for this GPU and batch shape, then warm up
    for _ in range(A + 2 + S.BATCH_OUT_LAG):
        batch.step(True)
    tuned = None
    if args.lk_variant >= 0:
        batch.set_lk_variant(args.lk_variant)
        tuned = {"lk_variant": args.lk_variant, "lk_variant_ms": None}
    elif not args.no_autotune:
        v, ms = batch.autotune(None)
        tuned = {"lk_variant": v, "lk_variant_ms": {str(k): round(x, 4) for k, x in ms.items()}}
    for _ in range(args.warmup):
        batch.step(True)
    torch.cuda.synchronize()
    # kernels per step: begin, level 0, REDUCE level 1, the fused launch of levels 2-4,
    # response, filter, select, tracker, compaction, fit (with the smoothing step), warp, advance
    n_k = 12
    # ---- timed region: K graph steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = ClockSampler(local)
    nvml = NvmlClockSampler(local, device_uuid(dev))
    clocks.start()
    nvml.start()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tw0 = time.time()
    ev[0].record(stream)
    for k in range(args.steps):
        batch.step(True)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    tw1 = time.time()
    wall = time.perf_counter() - t0
    barrier()
    clk_smi = clocks.stop()
    clk = nvml.stop(tw0, tw1) or clk_smi
    assert batch.sync() == 0
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms = max_over_ranks(total_ms, dev)
    value = ws * B * args.steps / (total_ms / 1e3)

    # ---- per-step latency: each step launched alone on an idle GPU, events
    # around it, over a fixed count of steps independent of --steps
    lat = latency_loop(batch, stream, args.lat_steps, args.lat_warmup) if args.lat_steps > 0 else None
    lat_other = None
    if lat:
        # the same videos with the other detection schedule: latency and mean
        # step time (a trade: staggered detection runs the latency-bound
        # detection kernels on a fifth of the streams at every step)
        lb = make_batch(not staggered)
        for _ in range(A + 2 + S.BATCH_OUT_LAG):
            lb.step(True)
        if tuned:
            lb.set_lk_variant(tuned["lk_variant"])
        lat_other = latency_loop(lb, stream, args.lat_steps, args.lat_warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            lb.step(True)
        e1.record(stream)
        torch.cuda.synchronize()
        lat_other["ms_per_step"] = round(e0.elapsed_time(e1) / args.steps, 4)
        lat_other["detection"] = config_dict(B, not staggered)["detection"]
        assert lb.sync() == 0
        del lb
        torch.cuda.synchronize()
    gaps = sorted(step_ms)

    # ---- per-kernel times (event-bracketed steps without a graph)
    kt, lkw = {}, []
    for _ in range(args.prof_steps):
        for name, ms in batch.step_profiled().items():
            kt.setdefault(name, []).append(ms)
        lkw.append(batch.lk_work())
    kavg = {k: sum(v) / len(v) for k, v in kt.items()}
    if kt:
        n_k = len(kt)   # the graph-free step launches the same kernels, one per entry
    roof = roofline(kavg, lkw, B) if kavg else None

    # ---- plain single-stream path, FP32 planes
    plain = run_plain(S, clips[0], ring, args.plain_steps, dev) if args.plain_steps > 0 else None

    # ---- end to end through host buffers
    e2e = run_e2e(S, batch, clips, src_clip, offs, ring, args.e2e_steps, ws, dev) if args.e2e_steps > 0 else None

    mixed = run_mixed(S, dev, args.mixed_steps, args.warmup, ws, rank) if args.mixed_steps > 0 else None
    gn = run_gn(S, dev, args.gn_pairs) if args.gn_pairs > 0 else None
    fits = run_fits(S, dev, args.fit_reps) if args.fit_reps > 0 else None

    out = {"metric": METRIC, "value": round(value, 1), "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "storage": "u8 frames, f16 I/Ix/Iy planes",
           "data": "synthetic", "config": config_dict(B, staggered),
           "latency_ms": dict(lat or {}, per="batch step (16 frames)",
                              # not in the step latency: the step that ingests frame t emits frame
                              # t - (BATCH_OUT_LAG + 1 + W/2), of which W/2 is the smoother's lookahead
                              output_delay_frames=S.BATCH_OUT_LAG + 1 + A, smoothing_lookahead_frames=A),
           ("latency_lockstep_ms" if staggered else "latency_staggered_ms"): lat_other,
           "step_interval_ms": {"p50": round(gaps[len(gaps) // 2], 4), "max": round(gaps[-1], 4),
                                "of": f"event gaps between the {args.steps} back-to-back timed steps"},
           "plain": plain, "e2e": e2e, "roofline": roof,
           "kernels_ms": {k: round(v, 4) for k, v in kavg.items()},
           "gpu_launches": n_k * args.steps, "clocks": clk, "clocks_nvidia_smi": clk_smi, "wall_s": round(wall, 3),
           "autotune": tuned, "streams_per_rank": len(mine),
           "mixed_64_streams": mixed, "photometric_gn": gn, "fits": fits}
    if ws == 1 and rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(clips[0].cpu().numpy(), args.cpu_frames, args.cpu_frames_single)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def latency_loop(batch, stream, steps: int, warm: int) -> dict:
    """p50 / p99 / max of the device time of one batched step launched with the
    GPU idle (CUDA events around the graph launch, a synchronisation after
    each), over `steps` steps after `warm` untimed ones.  A stream detects
    corners on one step in five: with the streams' detection steps staggered
    every step detects on a fifth of them, in lockstep one step in five detects
    on all (its p99 is that step)."""
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    ms = []
    for k in range(warm + steps):
        a.record(stream)
        batch.step(True)
        b.record(stream)
        b.synchronize()
        if k >= warm:
            ms.append(a.elapsed_time(b))
    ms.sort()
    q = lambda f: ms[min(len(ms) - 1, int(math.ceil(f * len(ms))) - 1)]
    return {"p50": round(q(0.5), 4), "p99": round(q(0.99), 4), "max": round(ms[-1], 4), "steps": steps,
            "warmup": warm, "how": "each step alone on an idle GPU, CUDA events around the graph launch"}


def kernel_source_sha(name: str) -> str:
    path = os.path.join(ROOT, "paper_1701_03572_gb300", "csrc", name)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def roofline(kavg: dict, lkw: list, B: int) -> dict:
    import json as _json
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = _json.load(open(pk))
    hbm = peaks.get("hbm_gbs")
    hbm_src = "of measured" if hbm else "of fallback"
    hbm = hbm or 6800.0
    dom = max(kavg, key=kavg.get)
    # algorithmic bytes per launch of the HBM-bound kernels (16 streams)
    L = PARAMS["levels"]
    sizes = [(W, H)]
    for _ in range(1, L):
        sizes.append(((sizes[-1][0] + 1) // 2, (sizes[-1][1] + 1) // 2))
    alg_bytes = {
        # RGB in (3 B/px), luma level 0 out (1 B/px), I + (Ix, Iy) FP16 out (6 B/px)
        "level0": B * W * H * (3 + 1 + 6),
        # warp: RGB frame in, RGB frame out
        "warp": B * W * H * CH * 2,
    }
    for l in range(1, L):
        pw, ph = sizes[l - 1]
        w_, h_ = sizes[l]
        alg_bytes[f"pyr_down_{l}"] = B * (pw * ph + w_ * h_ * (1 + 6))
    # the fused launch of levels l0 .. l0+2: level l0-1 read once, each level written once
    for l0 in range(2, L, 3):
        pw, ph = sizes[l0 - 1]
        alg_bytes[f"pyr_tail_{l0}"] = B * (pw * ph + sum(w_ * h_ * (1 + 6) for w_, h_ in sizes[l0:l0 + 3]))
    kernels = {}
    for k, ms in kavg.items():
        if k in alg_bytes and ms > 0:
            gbs = alg_bytes[k] / (ms / 1e3) / 1e9
            kernels[k] = {"bound": "hbm", "achieved": round(gbs, 1), "unit": "GB/s", "frac": round(gbs / hbm, 3),
                          "ms": round(ms, 4)}
    it = sum(x[0] for x in lkw) / max(len(lkw), 1)
    tp = sum(x[1] for x in lkw) / max(len(lkw), 1)
    n_win = (2 * 10 + 1) ** 2
    lk_flop = tp * n_win * LK_FLOP_TEMPLATE + it * n_win * LK_FLOP_ITER
    if kavg.get("lk", 0) > 0:
        tf = lk_flop / (kavg["lk"] / 1e3) / 1e12
        tf_s = (tp * n_win * LK_FLOP_COARSE[0] + it * n_win * LK_FLOP_COARSE[1]) / (kavg["lk"] / 1e3) / 1e12
        kernels["lk"] = {"bound": "alu", "achieved": round(tf, 3), "unit": "TFLOP/s",
                         "frac": round(tf / FP32_PEAK_TFLOPS, 4), "ms": round(kavg["lk"], 4),
                         "iterations": int(it), "template_passes": int(tp),
                         "flop_per_sample": {"template": LK_FLOP_TEMPLATE, "iteration": LK_FLOP_ITER},
                         "frac_at_coarse_count": {"flop_per_sample": list(LK_FLOP_COARSE),
                                                     "frac": round(tf_s / FP32_PEAK_TFLOPS, 4)}}
    if dom in kernels:
        d = kernels[dom]
        traffic = None
        tr = TRAFFIC.get(dom)
        if tr and tr.get("sha") == kernel_source_sha(tr["file"]):
            traffic = tr["bytes_per_launch"]
        peak = FP32_PEAK_TFLOPS if d["bound"] == "alu" else hbm
        res = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": round(peak, 1),
               "unit": d["unit"], "frac": d["frac"], "traffic": traffic,
               "peak_source": FP32_PEAK_NOTE if d["bound"] == "alu" else f"MEASURED_PEAKS.json hbm_gbs ({hbm_src})",
               "per_kernel": kernels}
        if d["bound"] == "alu":
            res["algorithmic_flop_per_launch"] = round(lk_flop)
        else:
            res["algorithmic_bytes_per_launch"] = alg_bytes[dom]
        return res
    return {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": None, "per_kernel": kernels}


def run_plain(S, clip, ring, steps, dev):
    """One 1080p stream through stab_track / stab_fit / stab_smooth_push /
    stab_warp with FP32 planes, buffers allocated once."""
    import torch
    p = S.default_params(**PARAMS, precision=S.STAB_FP32)
    ctx = S.Context(W, H, p)
    L = S.lib()
    K = p.max_corners
    src = torch.zeros((K, 2), device=dev)
    dst = torch.zeros((K, 2), device=dev)
    status = torch.zeros(K, dtype=torch.uint8, device=dev)
    n = torch.zeros(1, dtype=torch.int32, device=dev)
    mot = torch.zeros(S.MOTION_WORDS, device=dev)
    Minv = torch.zeros(6, device=dev)
    ready = torch.zeros(1, dtype=torch.int32, device=dev)
    out = torch.zeros((H, W, CH), dtype=torch.uint8, device=dev)
    fr = clip.contiguous()
    A = p.smooth_window // 2
    s = S._s()
    pitch = W * CH
    vp = C.c_void_p

    def frame_step(t):
        prev, nxt = fr[(t - 1) % ring], fr[t % ring]
        L.stab_track(ctx._h, vp(prev.data_ptr()), vp(nxt.data_ptr()), pitch, CH, 1 if t > 1 else 0,
                     vp(src.data_ptr()), vp(dst.data_ptr()), vp(status.data_ptr()), vp(n.data_ptr()), s)
        L.stab_fit(ctx._h, vp(src.data_ptr()), vp(dst.data_ptr()), vp(n.data_ptr()), p.model, t,
                   vp(mot.data_ptr()), s)
        L.stab_smooth_push(ctx._h, vp(mot.data_ptr()), vp(Minv.data_ptr()), vp(ready.data_ptr()), s)
        u = t - 1 - A
        if u >= 0:
            L.stab_warp(ctx._h, vp(fr[u % ring].data_ptr()), pitch, vp(out.data_ptr()), pitch, CH,
                        vp(Minv.data_ptr()), s)

    t = 1
    for _ in range(A + 4):
        frame_step(t)
        t += 1
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    # pick the tracker variant for a single stream (few features per SM favour two
    # warps per feature), timing a few frames of each
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tune = {}
    for v in range(S.LK_VARIANTS):
        ctx.set_lk_variant(v)
        frame_step(t)
        t += 1
        e0.record(stream)
        for _ in range(6):
            frame_step(t)
            t += 1
        e1.record(stream)
        torch.cuda.synchronize()
        tune[v] = e0.elapsed_time(e1) / 6
    best = min(tune, key=tune.get)
    ctx.set_lk_variant(best)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for k in range(steps):
        frame_step(t)
        t += 1
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    assert ctx.sync() == 0
    ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    tot = ev[0].elapsed_time(ev[-1])
    lat = sorted(ms)
    return {"value": round(steps / (tot / 1e3), 1), "unit": "frames/s", "p50_ms": round(lat[len(lat) // 2], 4),
            "p99_ms": round(lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)], 4),
            "config": "1 stream 1920x1080 RGB, FP32 planes, single-stream calls (no graph)", "frames": steps,
            "lk_variant": best, "lk_variant_frame_ms": {str(k): round(v, 4) for k, v in tune.items()}}


def run_e2e(S, batch, clips, src_clip, offs, ring, steps, ws, dev):
    import torch
    B = batch.n
    host = [c.cpu().pin_memory() for c in clips]
    outs = [torch.empty((H, W, CH), dtype=torch.uint8).pin_memory() for _ in range(B)]
    stream = torch.cuda.current_stream()
    t0 = batch.frame

    def one(t):
        frames = [host[src_clip[i]][(t + offs[i]) % ring] for i in range(B)]
        batch.step_host(frames, outs)

    for k in range(3):
        one(t0 + k)
    torch.cuda.synchronize()
    t0 = batch.frame
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for k in range(steps):
        one(t0 + k)
    e1.record(stream)
    torch.cuda.synchronize()
    assert batch.sync() == 0
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    return {"value": round(ws * B * steps / (ms / 1e3), 1), "unit": "frames/s",
            "h2d_bytes_per_step": B * W * H * CH, "d2h_bytes_per_step": B * W * H * CH,
            "api": "stab_batch_step_host (pinned host frames in, stabilised frames out)", "steps": steps}


# ------------------------------------------- mixed-resolution batch (64) --
MIXED = [(320, 240, 200, 3), (640, 480, 292, 4), (1280, 720, 538, 5), (1920, 1080, 1000, 5)]


def run_mixed(S, dev, steps, warmup, ws=1, rank=0):
    """64 gray streams, 16 each of 320x240, 640x480, 1280x720, 1920x1080, with
    200-1000 corners in proportion to area; one graph launch per frame step.
    With several ranks the 64 streams are spread by pixel area (each rank a
    like mix of sizes) and the value counts every rank's frames."""
    import dataclasses

    import torch
    from paper_1701_03572_gb300.synth import ClipSpec, make_clip
    W15 = 15
    ring = 2 * (W15 // 2 + 2)
    clips = [make_clip(ClipSpec(w, h, ring, pingpong=True), 3000 + k, device=dev, dtype=torch.float32)["frames"]
             for k, (w, h, _, _) in enumerate(MIXED)]
    descs, src = [], []
    for k, (w, h, K, L) in enumerate(MIXED):
        p = S.default_params(max_corners=K, levels=L, hypotheses=100, smooth_window=W15,
                             precision=S.STAB_FP16_STORAGE)
        for i in range(16):
            descs.append((w, h, 1, p))
            src.append((k, (3 * i) % ring))
    mine = partition_by_area([(d[0], d[1]) for d in descs], ws, rank)
    descs = [descs[i] for i in mine]
    src = [src[i] for i in mine]
    b = S.Batch(descs, ring=ring)
    for i, (k, off) in enumerate(src):
        for sl in range(ring):
            b.input_slot(i, sl).copy_(clips[k][(sl + off) % ring])
    for _ in range(W15 // 2 + 2 + S.BATCH_OUT_LAG):
        b.step(True)
    v, _ = b.autotune(None)
    for _ in range(warmup):
        b.step(True)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    barrier()
    ev[0].record(stream)
    for k in range(steps):
        b.step(True)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    assert b.sync() == 0
    ms = sorted(ev[k].elapsed_time(ev[k + 1]) for k in range(steps))
    tot = max_over_ranks(ev[0].elapsed_time(ev[-1]), dev)
    area = sum(16 * w * h for w, h, _, _ in MIXED)
    return {"streams": 64, "resolutions": "16 x each of 320x240, 640x480, 1280x720, 1920x1080 (gray)",
            "corners": [k for _, _, k, _ in MIXED], "value": round(64 * steps / (tot / 1e3), 1), "unit": "frames/s",
            "equiv_1080p_frames_per_s": round(steps * area / (W * H) / (tot / 1e3), 1),
            "step_ms_p50": round(ms[len(ms) // 2], 4),
            "step_ms_p99": round(ms[min(len(ms) - 1, int(math.ceil(0.99 * len(ms))) - 1)], 4),
            "lk_variant": v, "steps": steps, "streams_per_rank": len(mine),
            "scaling": "strong (the 64 streams spread over the ranks by area)" if ws > 1 else None}


# ----------------------------------------------- photometric Gauss-Newton --
def run_gn(S, dev, pairs, steps_gn=10):
    """Refine the tracker's estimate of `pairs` 640x480 FP32 frame pairs with
    10 Gauss-Newton steps on the Charbonnier photometric loss."""
    import numpy as np
    import torch
    from paper_1701_03572_gb300.synth import make_pair_f32
    w, h, M, EPS = 640, 480, 48, 1e-3
    ps = [make_pair_f32(w, h, 5000 + k, device=dev) for k in range(pairs)]
    It = torch.stack([p["cur"] for p in ps]).contiguous()
    Ip = torch.stack([p["prev"] for p in ps]).contiguous()
    truth = np.stack([p["theta"] for p in ps])
    p = S.default_params(max_corners=500, levels=4, hypotheses=256)
    ctx = S.Context(w, h, p)
    est = torch.zeros((pairs, 4), dtype=torch.float32, device=dev)
    out = torch.zeros((pairs, S.MOTION_WORDS), dtype=torch.float32, device=dev)
    q8 = lambda x: torch.clamp(torch.floor(x + 0.5), 0, 255).to(torch.uint8)
    for k in range(pairs):
        src, dst, st, n = ctx.track(q8(Ip[k]), q8(It[k]))
        ctx.fit(src, dst, n, S.STAB_SIMILARITY, 1, out=out[k])
    est.copy_(out[:, :4])
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    S.charb_gauss_newton(It, Ip, est, steps_gn, M, EPS)      # warm-up
    torch.cuda.synchronize()
    e0.record()
    th = S.charb_gauss_newton(It, Ip, est, steps_gn, M, EPS)
    e1.record()
    torch.cuda.synchronize()
    gn_ms = e0.elapsed_time(e1)
    e0.record()
    loss, dth, _ = S.charb_forward(It, Ip, th, M, EPS)
    dIt, dIp = S.charb_backward_image(It, Ip, th, M, EPS)
    e1.record()
    torch.cuda.synchronize()
    fb_ms = e0.elapsed_time(e1)
    r = math.hypot(w, h) / 2
    err = lambda t: np.abs(t - truth)[:, :2].max(1) + r * np.abs(t - truth)[:, 2:].max(1)
    before, after = err(est.cpu().numpy().astype(np.float64)), err(th.cpu().numpy().astype(np.float64))
    omega = (w - 2 * M) * (h - 2 * M)
    return {"pairs": pairs, "gn_steps": steps_gn, "gn_ms": round(gn_ms, 3),
            "forward_backward_ms": round(fb_ms, 3),
            "gn_step_GBps": round(pairs * omega * 8 * steps_gn / (gn_ms / 1e3) / 1e9, 1),
            "err_px_before": {"median": round(float(np.median(before)), 4), "max": round(float(before.max()), 4)},
            "err_px_after": {"median": round(float(np.median(after)), 5), "max": round(float(after.max()), 5)},
            "improved_frac": round(float((after <= before).mean()), 4),
            "err_unit": "px at the image corner (translation + radius x angle / log-scale error)"}


def run_fits(S, dev, reps):
    """Latency of one robust fit call on 1000 pairs of a 1920x1080 frame (0.3 px
    jitter, 5 % outliers, 100 hypotheses): similarity, a hybrid decision
    transition (both models fitted and compared), and the 6-DOF affine fit."""
    import numpy as np
    import torch
    w, h, n = 1920, 1080, 1000
    rng = np.random.default_rng(77)
    c = np.array([(w - 1) / 2, (h - 1) / 2])
    th, sc = 0.004, 1.002
    R = sc * np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    src = rng.uniform([40, 40], [w - 40, h - 40], (n, 2))
    dst = (src - c) @ R.T + np.array([1.7, -0.9]) + c + rng.normal(0, 0.3, (n, 2))
    bad = rng.choice(n, n // 20, replace=False)
    dst[bad] += rng.uniform(5, 30, (len(bad), 2))
    srcd = torch.as_tensor(src.astype(np.float32), device=dev)
    dstd = torch.as_tensor(dst.astype(np.float32), device=dev)
    nd = torch.tensor([n], dtype=torch.int32, device=dev)
    ctx = S.Context(w, h, S.default_params(max_corners=n, hypotheses=100, model=S.STAB_HYBRID))
    out = torch.zeros(max(S.MOTION_WORDS, S.AFFINE_WORDS), dtype=torch.float32, device=dev)
    calls = {"similarity_us": lambda: ctx.fit(srcd, dstd, nd, S.STAB_SIMILARITY, 1, out=out),
             "hybrid_decision_us": lambda: ctx.fit(srcd, dstd, nd, S.STAB_HYBRID, 1, out=out),
             "affine_us": lambda: ctx.fit_affine(srcd, dstd, nd, 1, out=out)}
    res = {"pairs": n, "hypotheses": 100, "outliers": len(bad), "calls": reps}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for name, fn in calls.items():
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        res[name] = round(e0.elapsed_time(e1) * 1e3 / reps, 2)
    assert ctx.sync() == 0
    return res


# ---------------------------------------------------- oracle (CPU) timing --
def oracle_stream(frames, n_frames, warm=0):
    """Time the oracle frame by frame on one 1080p RGB stream (the same per-
    frame path, FP64 C, one thread).  Returns (frames timed, seconds)."""
    from oracle import oracle as O
    p = O.Params(max_corners=PARAMS["max_corners"], levels=PARAMS["levels"], hypotheses=PARAMS["hypotheses"],
                 smooth_window=PARAMS["smooth_window"], rigid=False)
    ring = frames.shape[0]
    roi = O.roi_of(W, H)
    A = p.smooth_window // 2
    incs = [[0.0, 0.0, 0.0, 0.0]]
    gray_prev = O.luma(frames[0])
    pyr_prev = O.pyramid(gray_prev, p.levels)
    feats = None
    t_start, counted = None, 0
    for t in range(1, warm + n_frames + 1):
        if t == warm + 1:
            t_start = time.perf_counter()
        rgb = frames[t % ring]
        gray = O.luma(rgb)
        pyr = O.pyramid(gray, p.levels)
        if feats is None or (t - 1) % p.redetect_period == 0 or len(feats) < p.min_tracks:
            feats, _, _ = O.detect(gray_prev, roi, p.max_corners, p.quality)
        tr = O.track(pyr_prev, pyr, feats, p.win_r, p.max_iters, p.eps, p.min_eig, p.fb_thresh)
        keep = tr["status"] == 1
        dst = tr["fwd"][keep].astype("float32")
        f = O.fit(feats[keep], dst, W, H, p.rigid, p.hypotheses, p.seed, t, p.inlier_thresh, p.min_fit)
        incs.append(list(f["m"]))
        feats = dst
        u = t - 1 - A
        if u >= 0:
            import numpy as np
            _, _, mp = O.smooth(np.array(incs), p.smooth_window)
            O.warp(frames[u % ring], O.warp_inverse(mp[u + 1], W, H))
        gray_prev, pyr_prev = gray, pyr
        if t > warm:
            counted += 1
    return counted, time.perf_counter() - t_start


def cpu_info() -> dict:
    """Host CPU: model name and the cores this process may run on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"cpu_model": model, "nproc": usable, "cpu_count": os.cpu_count()}


def oracle_all_cores():
    """Point the oracle at its OpenMP build with one thread per usable core;
    returns (restore handle, threads) or (None, 1) if that build fails."""
    from oracle import oracle as O
    try:
        path = O.build_omp()
    except Exception:
        return None, 1
    prev = O.use_library(path)
    n = cpu_info()["nproc"] or 1
    try:
        O.lib().omp_set_num_threads(n)
        threads = int(O.lib().omp_get_max_threads())
    except AttributeError:
        threads = n
    return prev, threads


def cpu_baseline(frames, n, n1):
    """The oracle timed on one 1080p RGB stream: single-threaded (the build the
    tests use) and on all usable host cores (its OpenMP build over rows and
    features).  `value` / `cores` are the all-core run's."""
    from oracle import oracle as O
    info = cpu_info()
    cnt1, sec1 = oracle_stream(frames, n1)
    single = {"value": round(cnt1 / sec1, 4), "unit": "frames/s", "cores": 1, "frames": cnt1,
              "seconds": round(sec1, 2)}
    prev, threads = oracle_all_cores()
    if prev is None:
        return dict(single, kind="oracle", single_thread=single, **info,
                    sample=f"{cnt1} consecutive frames of one 1920x1080 RGB stream, single thread (the OpenMP "
                           f"build failed)")
    try:
        cnt, sec = oracle_stream(frames, n)
    finally:
        O.restore_library(prev)
    return {"value": round(cnt / sec, 4), "unit": "frames/s", "cores": threads, "kind": "oracle",
            "sample": f"{cnt} consecutive frames of one 1920x1080 RGB stream (luma, pyramid, detection when due, "
                      f"LK fwd+bwd, fit, streaming smoothing, RGB warp) on {threads} threads, {sec:.1f} s; "
                      f"single thread: {cnt1} frames, {sec1:.1f} s",
            "single_thread": single, **info}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import torch
    from paper_1701_03572_gb300.synth import CONFIG_SPECS, make_clip
    import dataclasses
    ring = RING
    spec = dataclasses.replace(CONFIG_SPECS[2], frames=ring, pingpong=True)
    frames = make_clip(spec, 2000, device="cpu", dtype=torch.float32,
                       frames=range(min(ring, args.warmup + args.steps + 1)))["frames"].numpy()
    from oracle import oracle as O
    prev, threads = oracle_all_cores()
    try:
        cnt, sec = oracle_stream(frames, args.steps, warm=args.warmup)
    finally:
        if prev is not None:
            O.restore_library(prev)
    v = cnt / sec
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "frames/s",
                      "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": round(1e3 * sec / cnt, 2), "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(STREAMS),
                      "cpu_baseline": {"value": round(v, 4), "unit": "frames/s", "cores": threads, "kind": "oracle",
                                       "sample": f"one step = one 1920x1080 RGB frame of one stream through the "
                                                 f"FP64 C oracle on {threads} threads; {cnt} steps",
                                       **cpu_info()},
                      "e2e": {"value": round(v, 4), "unit": "frames/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--streams", type=int, default=STREAMS)
    ap.add_argument("--prof-steps", type=int, default=10)
    ap.add_argument("--plain-steps", type=int, default=60)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-frames", type=int, default=640,
                    help="frames of the oracle's all-core timing (about 10 s on 16 cores)")
    ap.add_argument("--cpu-frames-single", type=int, default=40,
                    help="frames of the oracle's single-thread timing (about 10 s)")
    ap.add_argument("--lat-steps", type=int, default=300, help="steps of the latency loop (0 = skip)")
    ap.add_argument("--lat-warmup", type=int, default=20)
    ap.add_argument("--clock-sampler", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--clock-index", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--clock-uuid", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--clock-period-ms", type=float, default=2.0, help=argparse.SUPPRESS)
    ap.add_argument("--mixed-steps", type=int, default=30, help="steps of the 64-stream mixed batch (0 = skip)")
    ap.add_argument("--gn-pairs", type=int, default=256, help="frame pairs of the photometric refinement (0 = skip)")
    ap.add_argument("--fit-reps", type=int, default=200, help="timed calls per fit model (0 = skip)")
    ap.add_argument("--clips", type=int, default=4, help="distinct seeded clips shared round-robin by the streams")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--lk-variant", type=int, default=-1, help="force a tracker variant instead of autotuning")
    ap.add_argument("--detect-phases", default="lockstep", choices=["staggered", "lockstep"],
                    help="spread the streams' detection steps over the cycle, or detect on all streams together")
    args = ap.parse_args()
    if args.clock_sampler:
        clock_sampler_main(args.clock_sampler, args.clock_index, args.clock_uuid, args.clock_period_ms)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
