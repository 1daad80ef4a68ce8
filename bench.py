"""Benchmark of the voxel-cone-tracing hot path on GB300.

One step = one frame of the 256^3 room workload: Morton packing + mip build
of the resident level-0 grid (vct_build_mips) followed by the trace of a
1920x1080 G-buffer with 9 diffuse + 1 specular + 1 occlusion cone per pixel
(vct_trace).  The metric is cone samples per second (Gcone-samples/s); the
1080p trace time is reported beside it.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference this project
has: the thesis ships no runnable code here) on the host cores.
Under torchrun each rank traces its own replica of the frame (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

TEXEL_BYTES = {"f32": 16, "f16": 8}
PIXEL_IO_BYTES = 12 + 12 + 4 + 1 + 16 + 16 + 4  # pos, normal, roughness, mask; D, S, Vis
TRACE_SOURCES = ["paper_2104_00618_gb300/csrc/trace.cu",
                 "paper_2104_00618_gb300/csrc/trace_common.cuh",
                 "paper_2104_00618_gb300/csrc/vct_internal.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--dtype", choices=["f32", "f16"], default="f32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 4-scene batched extra")
    ap.add_argument("--profile", action="store_true",
                    help="only warm-up + timed frames (for ncu captures); no e2e/extras/baseline")
    ap.add_argument("--profile-bwd", action="store_true",
                    help="only fwd+bwd steps of a reduced learnable-grid case (for ncu captures)")
    ap.add_argument("--only-extra", default=None,
                    help="run one secondary measurement alone and print it (for ncu captures)")
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _code_only(text: str) -> str:
    """C/C++ source without comments and blank space (string literals kept),
    so that edits of comments do not change the hash of a kernel."""
    out, i, n = [], 0, len(text)
    while i < n:
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif text[i] == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(text[i])
            i += 1
    return " ".join("".join(out).split())


def percentiles(xs):
    """p10 / median / p90 of per-step event times (nearest rank)."""
    v = sorted(xs)
    if not v:
        return None
    pick = lambda q: v[min(len(v) - 1, max(0, int(round(q * (len(v) - 1)))))]
    return {"p10": pick(0.1), "p50": pick(0.5), "p90": pick(0.9), "n": len(v)}


def sources_hash(files) -> str:
    """sha1[:16] of the code (comments and spacing removed) of the files."""
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def ncu_counters(kernel: str, workload: str):
    """Per-launch ncu counters (DRAM bytes, warp instructions) from the
    committed summary, if it was taken on the current kernel sources (else
    an empty dict)."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return {}
    d = json.load(open(p))
    e = d.get(f"{kernel}|{workload}")
    if not e or e.get("sources") != sources_hash(TRACE_SOURCES):
        return {}
    return e


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, or None."""
    e = ncu_counters(kernel, workload)
    return float(e["dram_bytes_per_launch"]) if "dram_bytes_per_launch" in e else None


# Instruction issue: every SM has 4 sub-partitions, each issuing at most one
# warp instruction per clock.
ISSUE_PER_SM_PER_CLOCK = 4


def issue_roofline(kernel: str, workload: str, launch_ms: float, clocks: dict, sms: int,
                   gather_bytes: float, hbm_peak: float, hbm_kind: str):
    """The trace kernel against the limiter that binds it: warp instructions
    per launch (ncu smsp__inst_executed.sum of one full-size launch) over the
    event-timed launch, against the issue peak of the device's SMs at the
    median SM clock sampled during the timed region.  Secondary keys: L1
    throughput (ncu), DRAM traffic against the HBM peak, and the algorithmic
    gather bytes per launch (16 texels per sample), which are delivered
    mostly by L1 and so exceed the HBM peak."""
    e = ncu_counters(kernel, workload)
    inst = e.get("warp_inst_per_launch")
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = sms * ISSUE_PER_SM_PER_CLOCK * mhz * 1e6 / 1e9  # G warp instructions / s
    t = launch_ms / 1e3
    out = {"bound": "alu", "limiter": "instruction issue", "achieved": None, "peak": peak,
           "unit": "Gwarp-inst/s", "frac": None, "traffic": None, "kernel": kernel,
           "peak_source": f"{sms} SMs x {ISSUE_PER_SM_PER_CLOCK} issue slots/clock x "
                          f"{mhz:.0f} MHz (median SM clock sampled in the timed region)"}
    gather = {"achieved_gbs": gather_bytes / t / 1e9,
              "bytes_per_launch": gather_bytes,
              "of_hbm_peak": gather_bytes / t / 1e9 / hbm_peak,
              "note": "algorithmic texel bytes (16 texels x texel size per sample + pixel I/O) "
                      "per event-timed launch; served mostly by L1, so not an HBM figure"}
    out["gather_delivery"] = gather
    if inst is None:
        return out
    out.update({"achieved": inst / t / 1e9, "frac": inst / t / 1e9 / peak,
                "warp_inst_per_launch": inst,
                "warp_inst_per_sample": e.get("warp_inst_per_sample")})
    dram = e.get("dram_bytes_per_launch")
    if dram is not None:
        out["traffic"] = dram
        out["dram"] = {"bytes_per_launch": dram, "achieved_gbs": dram / t / 1e9,
                       "peak_gbs": hbm_peak, "frac": dram / t / 1e9 / hbm_peak,
                       "peak_source": hbm_kind}
    if e.get("l1tex_bytes_per_launch") is not None:
        l1 = e["l1tex_bytes_per_launch"]
        out["l1"] = {"bytes_per_launch": l1, "achieved_gbs": l1 / t / 1e9,
                     "ncu_throughput_pct": e.get("l1tex_throughput_pct")}
    return out


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self, t0=None, t1=None):
        """Median SM clock and throttle reasons of the samples taken between
        host times t0 and t1 (the timed region), or of all samples if none
        fall there."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = [ln for t, ln in self.lines
                 if t0 is not None and t1 is not None and t0 <= t <= t1]
        if not lines:
            lines = [ln for _, ln in self.lines]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_workload(width=1920, height=1080):
    import vct_synth as vs
    return vs.config_room_1080p(width=width, height=height)


def oracle_frame(oracle, scene, view, prm, idx=None):
    """One step of the workload on the FP64 oracle: mip build of the level-0
    grid, then the trace of the view's pixels (all, or the listed subset).
    Returns (seconds, cone samples)."""
    t0 = time.perf_counter()
    O = oracle.build_mips(scene["grid"])
    r = oracle.trace(O, view, prm, idx=idx)
    return time.perf_counter() - t0, int(np.sum(r["steps"]))


def cpu_baseline(cfg, frames=3):
    """The FP64 oracle as it stands, on this host's cores: whole frames (mip
    build of the 256^3 grid + trace of all 1920x1080 pixels), median of
    `frames` runs."""
    import oracle
    scene, view, prm = cfg["scenes"][0], cfg["views"][0], cfg["params"]
    runs = [oracle_frame(oracle, scene, view, prm) for _ in range(frames)]
    secs = sorted(t for t, _ in runs)
    frame_s = secs[len(secs) // 2]
    samples = runs[0][1]
    return {"value": samples / frame_s / 1e9, "unit": "Gcone-samples/s",
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{frames} whole frames (FP64 mip build of the 256^3 grid + trace of all "
                      f"{view['width']}x{view['height']} pixels, {samples} samples), median "
                      f"frame {frame_s:.2f} s",
            "frame_s": frame_s, "frames_s": secs}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2104_00618_gb300 as vct

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    cfg = make_workload(args.width, args.height)
    scene, hv, prm = cfg["scenes"][0], cfg["views"][0], cfg["params"]
    n = scene["n"]
    level0 = torch.from_numpy(scene["grid"]).to(dev)
    view = vct.View.from_host(hv, device=dev)
    P = vct.Pyramid(n, None, args.dtype, device=dev)
    params = vct.make_params(prm)
    tws = torch.zeros(256, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        if ev is not None:
            ev[2].record(stream)
        vct.build_mips(level0, out=P)
        if ev is not None:
            ev[0].record(stream)
        vct.trace([P], [view], params, workspace=tws)
        if ev is not None:
            ev[1].record(stream)

    clocks = None
    if not args.profile:
        # the clock sampler starts before the warm-up, so that the GPU does
        # not idle between the warm-up and the timed steps
        clocks = ClockSampler(dev.index)
        clocks.start()
        time.sleep(0.3)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    stats = vct.read_stats(tws)
    samples = int(sum(stats["samples"]))
    if args.profile:
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize()
        return {"profile": True, "samples_per_frame": samples, "width": args.width,
                "height": args.height, "steps": args.steps, "warmup": max(3, args.warmup)}

    tev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3))
           for _ in range(args.steps)]
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_host0 = time.monotonic()
    e_start.record(stream)
    for i in range(args.steps):
        step(tev[i])
    e_end.record(stream)
    torch.cuda.synchronize()
    t_host1 = time.monotonic()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop(t_host0, t_host1)
    total_ms = e_start.elapsed_time(e_end)
    trace_ms = [a.elapsed_time(b) for a, b, _ in tev]
    build_ms = [c.elapsed_time(a) for a, _, c in tev]
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / args.steps
    trace_avg = sum(trace_ms) / len(trace_ms)
    build_avg = sum(build_ms) / len(build_ms)
    value = samples * ws * args.steps / (total_ms / 1e3) / 1e9

    # e2e: host buffers, copies inside the timed region
    e2e = run_e2e(torch, vct, dev, scene, hv, params, args, stream)

    line = None
    if rank == 0:
        hbm, peak_kind = measured_peaks()
        algo_bytes = samples * 16 * TEXEL_BYTES[args.dtype] + hv["width"] * hv["height"] * PIXEL_IO_BYTES
        workload = f"room{n}_1080p_{args.dtype}"
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        roof = issue_roofline("trace_kernel", workload, trace_avg, clk, sms, algo_bytes, hbm,
                              peak_kind)
        # the mip build streams level 0 once and writes the pyramid once
        tb = TEXEL_BYTES[args.dtype]
        mip_bytes = n ** 3 * 16 + sum((n >> l) ** 3 for l in range(P.levels)) * tb
        build_pct = percentiles(build_ms)
        line = {
            "metric": "Gcone-samples/s (256^3 room, 1920x1080, 11 cones/px: mip build + trace)",
            "value": value, "unit": "Gcone-samples/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.dtype == "f32" else "f16-storage/f32-compute",
            "data": "synthetic (seeded box room, raycast G-buffer)",
            "config": {"workload": workload, "grid": n, "levels": P.levels, "width": hv["width"],
                       "height": hv["height"], "cones_per_px": 11,
                       "samples_per_frame": samples, "trace_ms": trace_avg,
                       "l2": "inputs larger than L2 (268 MB level-0 grid, 307 MB pyramid)",
                       "parallelism": f"replica x{ws}"},
            "trace_ms": trace_avg,
            "trace_ms_percentiles": percentiles(trace_ms),
            "roofline": roof,
            "mip_build": {"ms": build_avg, "ms_percentiles": build_pct, "bytes": mip_bytes,
                          "achieved_gbs": mip_bytes / (build_avg / 1e3) / 1e9,
                          "frac_of_hbm_peak": mip_bytes / (build_avg / 1e3) / 1e9 / hbm,
                          "frac_of_hbm_peak_median":
                              mip_bytes / (build_pct["p50"] / 1e3) / 1e9 / hbm,
                          "peak_source": peak_kind,
                          "note": "level 0 read once (16 B/texel) + the whole pyramid written "
                                  "once, over the event-timed vct_build_mips (mean and median "
                                  "of the timed steps)"},
            "clocks": clk,
            "e2e": e2e,
            # per step: vct_build_mips of the 256^3 grid (the streaming kernel
            # for levels 0..4 and the one-CTA tail, FP32 or FP16) and the
            # persistent trace kernel
            "gpu_launches": 3 * args.steps,
        }
        if not args.no_extras:
            line["extras"] = run_extras(torch, vct, dev, args)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(cfg)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return line


def run_e2e(torch, vct, dev, scene, hv, params, args, stream, steps=None):
    """The step through the library's host-buffer pipeline (vct_pipeline_*):
    every step copies its inputs from page-locked host memory, builds the
    mips, traces and copies its outputs back; the library overlaps the
    copies of one step with the kernels of its neighbours."""
    steps = steps or max(3, min(args.steps, 30))  # the timed steps of the device leg, up to 30
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_grid = pin(scene["grid"])
    h_pos, h_nrm = pin(hv["position"]), pin(hv["normal"])
    h_rough, h_mask = pin(hv["roughness"]), pin(hv["mask"])
    npx = hv["width"] * hv["height"]
    h_D = torch.empty((npx, 4)).pin_memory()
    h_S = torch.empty((npx, 4)).pin_memory()
    h_V = torch.empty((npx,)).pin_memory()
    pipe = vct.Pipeline(scene["n"], hv["width"], hv["height"], params, dtype=args.dtype)
    cam = [float(c) for c in hv["camera"]]

    def one():
        pipe.submit(h_grid, h_pos, h_nrm, cam, h_D, h_S, h_V, h_rough, h_mask, stream=stream)

    for _ in range(2):
        one()
    pipe.wait()
    samples = int(sum(pipe.stats(0)["samples"]))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        one()
    pipe.join(stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    pipe.wait()
    pipe.close()
    h2d = sum(t.numel() * t.element_size() for t in (h_grid, h_pos, h_nrm, h_rough, h_mask))
    d2h = sum(t.numel() * t.element_size() for t in (h_D, h_S, h_V))
    return {"value": samples / (ms / 1e3) / 1e9, "unit": "Gcone-samples/s", "ms_per_step": ms,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "path": "vct_pipeline_submit (host buffers; copies overlapped with kernels)"}


def _time(torch, fn, reps, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def extra_fp16_single(torch, vct, dev):
    """The same 1080p frame with the pyramid stored in binary16."""
    cfg = make_workload()
    scene, hv, prm = cfg["scenes"][0], cfg["views"][0], cfg["params"]
    level0 = torch.from_numpy(scene["grid"]).to(dev)
    view = vct.View.from_host(hv, device=dev)
    P = vct.Pyramid(scene["n"], None, "f16", device=dev)
    params = vct.make_params(prm)
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    vct.build_mips(level0, out=P)
    tr_ms = _time(torch, lambda: vct.trace([P], [view], params, workspace=ws), 10)
    step_ms = _time(torch, lambda: (vct.build_mips(level0, out=P),
                                    vct.trace([P], [view], params, workspace=ws)), 10)
    samples = int(sum(vct.read_stats(ws)["samples"]))
    return {"workload": "room256_1080p_f16", "trace_ms": tr_ms, "ms_per_step": step_ms,
            "gsamples_per_s": samples / (step_ms / 1e3) / 1e9, "samples_per_frame": samples}


def extra_small(torch, vct, dev):
    """The 64^3 box scene with 128x128 surface samples (6 x 60 degree diffuse
    cones + one 10 degree specular cone), pyramid stored FP32 and FP16 (the
    same scene), each at the accuracy its GPU test asserts against the FP64
    oracle."""
    import vct_synth as vs
    c = vs.config_small_fp32()
    scene, hv, prm = c["scenes"][0], c["views"][0], c["params"]
    level0 = torch.from_numpy(scene["grid"]).to(dev)
    view = vct.View.from_host(hv, device=dev)
    params = vct.make_params(prm)
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    out = {"workload": "small64_128x128", "grid": scene["n"],
           "pixels": hv["width"] * hv["height"]}
    acc = {"f32": "max floored relative error <= 1e-4 per channel vs the FP64 oracle, whole "
                  "frame (tests/test_gpu_parity.py::test_small_config_full_frame)",
           "f16": "every pixel and channel within the binary16-storage bound (2^-11 per texel "
                  "through lerps and compositing, + 1e-4 floored), mean floored relative error "
                  "<= 2^-11 (tests/test_gpu_parity.py::test_fp16_storage_error_report)"}
    for dt in ("f32", "f16"):
        P = vct.Pyramid(scene["n"], None, dt, device=dev)
        vct.build_mips(level0, out=P)
        # 16 K pixels fill few of the default 16x16 tiles: let the library's
        # tuner pick the tile and lanes per pixel for this shape (vct_trace
        # then uses its choice)
        tuned = vct.autotune([P], [view], params, workspace=ws)
        tr_ms = _time(torch, lambda: vct.trace([P], [view], params, workspace=ws), 50, warm=5)
        st_ms = _time(torch, lambda: (vct.build_mips(level0, out=P),
                                      vct.trace([P], [view], params, workspace=ws)), 50, warm=5)
        samples = int(sum(vct.read_stats(ws)["samples"]))
        out[dt] = {"trace_ms": tr_ms, "ms_per_step": st_ms, "samples_per_frame": samples,
                   "gsamples_per_s": samples / (st_ms / 1e3) / 1e9, "accuracy": acc[dt],
                   "tuned": {"tile": [tuned.tile_w, tuned.tile_h],
                             "lanes_per_pixel": tuned.lanes_per_pixel}}
    return out


def extra_variants(torch, vct, dev):
    """The same 1080p frame (FP32) with the thesis's modified cones (occlusion
    fade-in, angular-grace specular, first-hit diffuse) and L_vxct shading
    into a radiance buffer, beside the plain trace."""
    import vct_synth as vs
    cfg = make_workload()
    scene, hv, prm = cfg["scenes"][0], dict(cfg["views"][0]), cfg["params"]
    hv["albedo"] = vs.albedo(hv["width"], hv["height"], 11)
    flags = (vct.FLAG_OCC_SMOOTH | vct.FLAG_SPEC_GRACE | vct.FLAG_DIFFUSE_FIRST_HIT
             | vct.FLAG_SHADE)
    level0 = torch.from_numpy(scene["grid"]).to(dev)
    view = vct.View.from_host(hv, device=dev, outputs=False)
    view.alloc_outputs(radiance=True)
    P = vct.build_mips(level0)
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    out = {"workload": "room256_1080p_f32_variants_shaded", "flags": flags}
    for name, p in (("plain", vct.make_params(prm)),
                    ("variants", vct.make_params(vs.variant_params(prm, flags)))):
        if name == "plain":
            view.out_radiance = None
        else:
            view.alloc_outputs(radiance=True)
        ms = _time(torch, lambda: vct.trace([P], [view], p, workspace=ws), 10)
        samples = int(sum(vct.read_stats(ws)["samples"]))
        out[name] = {"trace_ms": ms, "samples_per_frame": samples,
                     "gsamples_per_s": samples / (ms / 1e3) / 1e9}
    return out


def extra_revoxelize(torch, vct, dev):
    """The 1080p room frame with the scene revoxelized every frame (the
    thesis's continuous-revoxelization measurement, Ch. 6.3.2): the room as a
    mesh of about 244K triangles -> vct_voxelize -> vct_build_mips ->
    vct_trace, FP32."""
    import vct_synth as vs
    c = vs.config_room_mesh()
    mesh = vct.Mesh.from_host(c["mesh"], device=dev)
    n, light = c["scenes"][0]["n"], c["light"]
    view = vct.View.from_host(c["views"][0], device=dev)
    params = vct.make_params(c["params"])
    vws = vct.voxelize_workspace(n, mesh.indices.shape[0], dev)
    grid = torch.empty((n, n, n, 4), dtype=torch.float32, device=dev)
    P = vct.Pyramid(n, None, "f32", device=dev)
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)

    def vox():
        vct.voxelize(mesh, n, light=light, out=grid, workspace=vws)

    def vox_mips():
        vox()
        vct.build_mips(grid, out=P)

    def frame():
        vox_mips()
        vct.trace([P], [view], params, workspace=ws)

    v_ms = _time(torch, vox, 10)
    vm_ms = _time(torch, vox_mips, 10)
    f_ms = _time(torch, frame, 10)
    st = vct.read_voxelize_stats(vws)
    samples = int(sum(vct.read_stats(ws)["samples"]))
    out = {"workload": f"room{n}_1080p_f32_revoxelized", "triangles": int(mesh.indices.shape[0]),
           "fragments": st["fragments"], "voxelize_ms": v_ms, "voxelize_mips_ms": vm_ms,
           "frame_ms": f_ms, "mtriangles_per_s": mesh.indices.shape[0] / (v_ms / 1e3) / 1e6,
           "gsamples_per_s": samples / (f_ms / 1e3) / 1e9}
    # the whole frame from triangles on the GPU: the G-buffer is drawn from
    # the same mesh (vct_gbuffer) instead of being uploaded
    hv = c["views"][0]
    cam = vs.camera(hv["camera"], hv["target"], hv["width"], hv["height"])
    g = vct.gbuffer(mesh, cam)  # sizes the workspace (checked once)
    gws = g["workspace"]
    gview = vct.gbuffer_view(g, cam)

    def gbuf():
        vct.gbuffer(mesh, cam, out=g, workspace=gws, verify=False)

    def gpu_frame():
        vox_mips()
        gbuf()
        vct.trace([P], [gview], params, workspace=ws)

    # the G-buffer does not depend on the voxel grid: draw it on a second
    # stream while the grid is voxelized and filtered, join before the trace
    side = torch.cuda.Stream(device=dev)

    def gpu_frame_overlapped():
        main = torch.cuda.current_stream(dev)
        side.wait_stream(main)  # the previous frame's trace has read the G-buffer
        with torch.cuda.stream(side):
            gbuf()
        vox_mips()
        main.wait_stream(side)
        vct.trace([P], [gview], params, workspace=ws)

    gb_ms = _time(torch, gbuf, 10)
    gf_ms = _time(torch, gpu_frame, 10)
    gfo_ms = _time(torch, gpu_frame_overlapped, 10)
    gst = vct.read_gbuffer_stats(gws)
    gsamples = int(sum(vct.read_stats(ws)["samples"]))
    out["gbuffer"] = {"gbuffer_ms": gb_ms, "tile_pairs": gst["pairs"],
                      "triangles_in_view": int(mesh.indices.shape[0]) - gst["culled"]
                      - gst["degenerate"] - gst["skipped"],
                      "frame_ms": gf_ms, "gsamples_per_s": gsamples / (gf_ms / 1e3) / 1e9,
                      "frame": "vct_voxelize + vct_build_mips + vct_gbuffer + vct_trace",
                      "frame_overlapped_ms": gfo_ms,
                      "overlap": "vct_gbuffer on a second stream beside voxelize + mips"}
    return out


def extra_bricks(torch, vct, dev, n=512):
    """Brick storage at 512^3: the room voxelized from its mesh (surface
    shells), pyramid bytes dense vs bricks, mip build and 1080p trace time in
    both layouts (same frame, identical outputs)."""
    import vct_synth as vs
    scene = vs.box_scene(n, 32, 2, room=True)
    mesh = vct.Mesh.from_host(vs.scene_mesh(scene, tess=24, n_spheres=4, seed=102), device=dev)
    rng = np.random.default_rng(2)
    hv = vs.interior_view(scene, 1920, 1080, rng)
    params = vct.make_params(vs.params_room9(scene["light"]))
    del scene
    level0 = vct.voxelize(mesh, n, light={"light_dir": (0.36, 0.8, 0.48)})
    view = vct.View.from_host(hv, device=dev)
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    out = {"workload": f"room{n}_mesh_1080p_f32", "triangles": int(mesh.indices.shape[0])}
    t0 = time.perf_counter()
    occ, _ = vct.plan_bricks(level0)
    out["plan_ms"] = (time.perf_counter() - t0) * 1e3
    for name in ("dense", "bricks"):
        P = (vct.Pyramid(n, None, "f32", device=dev) if name == "dense" else
             vct.Pyramid(n, None, "f32", device=dev, layout="bricks", occupied=occ))
        build_ms = _time(torch, lambda: vct.build_mips(level0, out=P), 5)
        trace_ms = _time(torch, lambda: vct.trace([P], [view], params, workspace=ws), 5)
        samples = int(sum(vct.read_stats(ws)["samples"]))
        out[name] = {"pyramid_bytes": int(P.storage.numel()), "build_ms": build_ms,
                     "trace_ms": trace_ms, "gsamples_per_s": samples / (trace_ms / 1e3) / 1e9}
        del P
        torch.cuda.empty_cache()
    out["occupied_bricks"] = occ
    out["bytes_ratio"] = out["bricks"]["pyramid_bytes"] / out["dense"]["pyramid_bytes"]
    return out


def extra_aniso(torch, vct, dev):
    """The 1080p room frame (FP32) on an anisotropic pyramid (six directional
    volumes per coarse level, Ch. 5.1) beside the isotropic one: pyramid
    bytes, mip build and trace time."""
    cfg = make_workload()
    scene, hv, prm = cfg["scenes"][0], cfg["views"][0], cfg["params"]
    level0 = torch.from_numpy(scene["grid"]).to(dev)
    view = vct.View.from_host(hv, device=dev)
    params = vct.make_params(prm)
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    out = {"workload": "room256_1080p_f32_aniso"}
    for name in ("dense", "aniso"):
        P = vct.Pyramid(scene["n"], None, "f32", device=dev, layout=name)
        build_ms = _time(torch, lambda: vct.build_mips(level0, out=P), 10)
        trace_ms = _time(torch, lambda: vct.trace([P], [view], params, workspace=ws), 10)
        samples = int(sum(vct.read_stats(ws)["samples"]))
        out[name] = {"pyramid_bytes": int(P.storage.numel()), "build_ms": build_ms,
                     "trace_ms": trace_ms, "gsamples_per_s": samples / (trace_ms / 1e3) / 1e9}
        del P
    out["bytes_ratio"] = out["aniso"]["pyramid_bytes"] / out["dense"]["pyramid_bytes"]
    return out


def extra_fwd_bwd(torch, vct, dev, n=128, n_views=32, res=512):
    """Learnable 128^3 grid at 0.1, 32 views of 512x512 of a ground-truth box
    scene, L2 loss: forward (mips + trace) and forward + adjoint (trace
    adjoint + mip adjoint) against the plain forward."""
    import vct_synth as vs
    cfg = vs.config_learnable(n=n, n_views=n_views, width=res, height=res)
    gt = torch.from_numpy(cfg["scenes"][0]["grid"]).to(dev)
    learn = torch.from_numpy(cfg["learnable"]).to(dev)
    params = vct.make_params(cfg["params"])
    views = [vct.View.from_host(v, device=dev) for v in cfg["views"]]
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    Pgt = vct.build_mips(gt)
    vct.trace([Pgt], views, params, workspace=ws)
    targets = [(v.out_diffuse.clone(), v.out_specular.clone(), v.out_visibility.clone())
               for v in views]
    # the training forward also records each cone's length for the adjoint
    states = [v.alloc_cone_state(params).cone_state for v in views]
    P = vct.Pyramid(n, None, "f32", device=dev)
    bws = vct.backward_workspace(P)
    grad = torch.zeros_like(learn)

    def use_state(on):
        for v, st in zip(views, states):
            v.cone_state = st if on else None

    def fwd():
        vct.build_mips(learn, out=P)
        vct.trace([P], views, params, workspace=ws)

    def fwd_bwd():
        fwd()
        grads = [(v.out_diffuse - t[0], v.out_specular - t[1], v.out_visibility - t[2])
                 for v, t in zip(views, targets)]
        grad.zero_()
        vct.trace_backward(P, views, grads, params, grad_level0=grad, workspace=bws)

    dws = vct.backward_workspace(P, deterministic=True)

    def fwd_bwd_det():
        fwd()
        grads = [(v.out_diffuse - t[0], v.out_specular - t[1], v.out_visibility - t[2])
                 for v, t in zip(views, targets)]
        grad.zero_()
        vct.trace_backward(P, views, grads, params, grad_level0=grad, workspace=dws,
                           deterministic=True)

    use_state(False)
    f_ms = _time(torch, fwd, 5)         # the plain forward
    fbr_ms = _time(torch, fwd_bwd, 5)   # the adjoint re-marches every cone to find its length
    use_state(True)
    fb_ms = _time(torch, fwd_bwd, 5)    # forward records each cone's length for the adjoint
    fbd_ms = _time(torch, fwd_bwd_det, 3)  # the same with the reproducible adjoint
    samples = int(sum(vct.read_stats(ws)["samples"]))
    return {"workload": f"learnable{n}_{n_views}x{res}^2_f32", "fwd_ms": f_ms, "fwd_bwd_ms": fb_ms,
            "fwd_bwd_over_fwd": fb_ms / f_ms,
            "fwd_bwd_mode": "forward stores per cone its sample count and transmittance before "
                            "the last sample (8 B per cone); the adjoint recomputes every "
                            "sample from the pyramid (no per-sample state)",
            "fwd_bwd_recompute_ms": fbr_ms, "fwd_bwd_recompute_over_fwd": fbr_ms / f_ms,
            "fwd_bwd_recompute_mode": "no state at all: the adjoint marches each cone forwards "
                                      "to find its length, then walks it back recomputing",
            "samples_per_fwd": samples,
            "fwd_gsamples_per_s": samples / (f_ms / 1e3) / 1e9,
            "fwd_bwd_deterministic_ms": fbd_ms}


def extra_batched(torch, vct, dev, grids=(128, 256, 256, 512), views_per_scene=64):
    """4 scenes x 64 interior views of uneven resolution, FP16 pyramids, one
    persistent launch captured in a CUDA graph, launch shape autotuned."""
    import vct_synth as vs
    t0 = time.perf_counter()
    cfg = vs.config_batched(grids=grids, views_per_scene=views_per_scene)
    gen_s = time.perf_counter() - t0
    params = vct.make_params(cfg["params"])
    pyrs = []
    for sc in cfg["scenes"]:
        g = torch.from_numpy(sc["grid"]).to(dev)
        pyrs.append(vct.build_mips(g, dtype="f16"))
        del g
    views = [vct.View.from_host(v, device=dev) for v in cfg["views"]]
    npx = sum(v.width * v.height for v in views)
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    # autotune on a probe: one reduced view per scene
    probe_host = []
    rng = np.random.default_rng(7)
    for si, sc in enumerate(cfg["scenes"]):
        pv = vs.interior_view(sc, 480, 270, rng)
        pv["pyramid"] = si
        probe_host.append(pv)
    probe = [vct.View.from_host(v, device=dev) for v in probe_host]
    best = vct.autotune(pyrs, probe, params, workspace=ws)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(stream):
        vct.trace(pyrs, views, params, workspace=ws)  # warm (tuned shape)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        vct.trace(pyrs, views, params, workspace=ws)
    ms = _time(torch, graph.replay, 3, warm=1)
    samples = int(sum(vct.read_stats(ws)["samples"]))
    return {"workload": f"batched_{len(grids)}scenes{list(grids)}_{len(views)}views_f16",
            "pixels": npx, "trace_ms": ms, "samples": samples,
            "gsamples_per_s": samples / (ms / 1e3) / 1e9,
            "tuned": {"tile": [best.tile_w, best.tile_h], "lanes_per_pixel": best.lanes_per_pixel},
            "launches_per_replay": 1, "graph": True, "gen_s": gen_s}


EXTRAS = {}


def run_extras(torch, vct, dev, args):
    """Secondary measurements reported beside the main metric."""
    out = {}
    for name, fn in EXTRAS.items():
        if name == "batched_fp16" and args.no_batched:
            continue
        try:
            out[name] = fn(torch, vct, dev)
        except Exception as e:  # report, keep the main line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        finally:
            try:  # release what the measurement cached, even after a failure
                torch.cuda.empty_cache()
            except Exception as e:
                out.setdefault("cache_release_errors", []).append(f"{name}: {e}")
    return out


def run_only_extra(args):
    import torch
    import paper_2104_00618_gb300 as vct
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    vct.lib()
    return {"only_extra": args.only_extra,
            args.only_extra: EXTRAS[args.only_extra](torch, vct, dev)}


def _register_extras():
    for name, fn in (("small_64", extra_small),
                     ("fp16_single_view", extra_fp16_single), ("variants", extra_variants),
                     ("revoxelize", extra_revoxelize), ("bricks_512", extra_bricks),
                     ("aniso", extra_aniso),
                     ("fwd_bwd", extra_fwd_bwd),
                     ("batched_fp16", extra_batched)):
        EXTRAS[name] = fn


_register_extras()


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
# Wall-clock budget of the reference arm's warm-up + timed steps, and the
# FP64 oracle's frame time for this workload on 16 host cores (about 3.1 s):
# each step is a whole frame while that fits the budget, else a seeded
# pixel subset of the frame (with the whole mip build) sized to fit it.
REFERENCE_BUDGET_S = 150.0
REFERENCE_FRAME_S_EST = 3.2


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    cfg = make_workload()
    scene, view, prm = cfg["scenes"][0], cfg["views"][0], cfg["params"]
    npx = view["width"] * view["height"]
    steps, warm = args.steps, max(0, args.warmup)
    frac = min(1.0, REFERENCE_BUDGET_S / ((steps + warm) * REFERENCE_FRAME_S_EST))
    idx = None
    if frac < 1.0:
        rng = np.random.default_rng(1)
        idx = np.sort(rng.choice(npx, max(1, int(npx * frac)), replace=False))
    for _ in range(warm):
        oracle_frame(oracle, scene, view, prm, idx)
    total_s, samples = 0.0, 0
    for _ in range(steps):
        t, k = oracle_frame(oracle, scene, view, prm, idx)
        total_s += t
        samples += k
    value = samples / total_s / 1e9
    what = ("a whole frame" if idx is None else
            f"the FP64 mip build + {len(idx)} seeded pixels ({len(idx) / npx:.4f} of the frame)")
    base = {"kind": "oracle", "cores": oracle.num_threads(), "value": value,
            "unit": "Gcone-samples/s",
            "sample": f"each step is {what}: FP64 mip build of the 256^3 grid + trace; "
                      f"{samples // steps} cone samples per step"}
    return {"metric": "Gcone-samples/s (256^3 room, 1920x1080, 11 cones/px: mip build + trace)",
            "value": value, "unit": "Gcone-samples/s", "n_gpus": ws, "steps": steps,
            "warmup": args.warmup, "ms_per_step": total_s / steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded box room, raycast G-buffer)",
            "config": {"workload": "room256_1080p_f32", "samples_per_step": samples // steps,
                       "pixels_per_step": npx if idx is None else len(idx)},
            "impl": "reference", "cpu_baseline": base,
            "e2e": {"value": value, "unit": "Gcone-samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_profile_bwd(args):
    import torch

    import paper_2104_00618_gb300 as vct
    import vct_synth as vs
    dev = torch.device("cuda", 0)
    cfg = vs.config_learnable(n=128, n_views=4, width=256, height=256)
    learn = torch.from_numpy(cfg["learnable"]).to(dev)
    gt = torch.from_numpy(cfg["scenes"][0]["grid"]).to(dev)
    params = vct.make_params(cfg["params"])
    views = [vct.View.from_host(v, device=dev) for v in cfg["views"]]
    vct.trace([vct.build_mips(gt)], views, params)
    targets = [(v.out_diffuse.clone(), v.out_specular.clone(), v.out_visibility.clone())
               for v in views]
    P = vct.Pyramid(128, None, "f32", device=dev)
    bws = vct.backward_workspace(P)
    grad = torch.zeros_like(learn)
    for _ in range(args.warmup + args.steps):
        vct.build_mips(learn, out=P)
        vct.trace([P], views, params)
        grads = [(v.out_diffuse - t[0], v.out_specular - t[1], v.out_visibility - t[2])
                 for v, t in zip(views, targets)]
        vct.trace_backward(P, views, grads, params, grad_level0=grad, workspace=bws)
    torch.cuda.synchronize()
    return {"profile_bwd": True, "steps": args.steps, "warmup": args.warmup}


def main():
    args = parse()
    if args.profile_bwd:
        print(json.dumps(run_profile_bwd(args)))
        return
    if args.only_extra:
        print(json.dumps(run_only_extra(args)))
        return
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
