"""Throughput benchmark of the HO-DMAS hot path (one JSON line on rank 0).

Default workload (cfg2 geometry): 128-element linear array, 0.3 mm pitch,
2048 samples at 40 MHz, 512 x 512 grid over 38.4 x 40 mm; DAS, DMAS and
DMAS-3 (k = 3) in the same pass, then band-pass + Hilbert envelope + log
compression; FP32 RF.  A step beamforms ``--frames`` seeded synthetic frames
(each rank its own frames) into their displayed log images.

Metric: Gpixel.ch/s = nx * nz * N * frames / time.  ``value`` is device
time (CUDA events around each step on the launching stream, inputs resident
in HBM, L2 flushed by a 256 MiB write between steps, outside the events).
The steps run through the default CUDA-graph launch; the roofline's fused
kernel time comes from event-record nodes around that kernel inside the
same graphs.
``e2e`` is the same metric through ``pa_beamform_host`` (pinned host RF in,
log images out, copies inside the timed region).

``--impl reference`` times the FP64 CPU oracle on the host cores instead.

``--case WORKLOAD`` (for profiling one configuration under ncu, or with
CUDA-event timing alone) runs that workload's launch sequence ``--launches``
times after ``--warmup`` launches on seeded random RF of its shape (the
arithmetic does not depend on the values), each launch after a 256 MiB L2
flush, and prints its kernel times, e.g. ``python bench.py --case cfg5
--frames 4``.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HO-DMAS k=3 Gpixel·ch/s vs plain FP32 form; serving p50/p99 frame latency ms"
UNIT = "Gpixel·ch/s"
CSRC = os.path.join(ROOT, "paper_2203_14906_gb300", "csrc")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=None,
                    help="frames per step (default 32; with --case, the workload's)")
    ap.add_argument("--order", type=int, default=None,
                    help="order k (default 3; with --case, the workload's)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip precision form and cpu baseline")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--serve-requests", type=int, default=6000)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--form", default="fp32", choices=["fp32", "precision"],
                    help="arithmetic form of the headline leg: FP32 RF and plain sums, or BF16 "
                         "RF with Kahan-compensated sums")
    ap.add_argument("--case", default=None, choices=["cfg1", "cfg2", "cfg3", "cfg5"],
                    help="profile one workload's launch sequence instead of the benchmark")
    ap.add_argument("--rf", default=None, choices=["f32", "bf16", "f16"],
                    help="--case: RF storage type (default: the workload's)")
    ap.add_argument("--compensated", type=int, default=None, choices=[0, 1],
                    help="--case: Kahan-compensated sums (default: the workload's)")
    ap.add_argument("--nx", type=int, default=None, help="--case: lateral pixels")
    ap.add_argument("--nz", type=int, default=None, help="--case: depth pixels")
    ap.add_argument("--launches", type=int, default=3, help="--case: timed launches")
    ap.add_argument("--table", default="auto", choices=["auto", "lattice", "full"],
                    help="--case: delay-table form")
    ap.add_argument("--interp", default="linear", choices=["linear", "nearest"],
                    help="--case: sampling of the delayed signal")
    ap.add_argument("--lanes", type=int, default=0, choices=[0, 4, 8, 32],
                    help="--case: time the channels-on-lanes mapping (pa_lanes_raw) with this "
                         "many lanes per pixel instead of the launch sequence")
    args = ap.parse_args()
    if args.case is None:
        args.frames = 32 if args.frames is None else args.frames
        args.order = 3 if args.order is None else args.order
    return args


def form_dtype(args):
    """(RF storage type, compensated) of the headline leg."""
    return ("bf16", 1) if args.form == "precision" else ("f32", 0)


def workload():
    import synth

    return synth.workload("cfg2")


def config_dict(args, wl, extra=None):
    d = {
        "workload": (
            f"cfg2 geometry: {wl['n_elem']} el x {wl['n_samples']} samples @ {wl['fs_hz']/1e6:g} MHz, "
            f"{wl['nx']}x{wl['nz']} grid; DAS+DMAS+DMAS-{args.order} in one pass; band-pass, "
            "Hilbert envelope, log; "
            + ("BF16 RF, Kahan-compensated sums" if args.form == "precision" else "FP32 RF")
        ),
        "frames_per_step": args.frames,
        "order_k": args.order,
        "n_elem": wl["n_elem"],
        "n_samples": wl["n_samples"],
        "grid": [wl["nx"], wl["nz"]],
        "stages": "log (raw and envelope computed in place)",
        "l2": "flushed between steps by a 256 MiB write (outside the timed events)",
        "parallelism": f"replicas x{args.gpus} (frames sharded, no collective)",
    }
    if extra:
        d.update(extra)
    return d


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch

            torch.cuda.set_device(local)  # each rank's collectives on its own GPU
        dist.init_process_group(backend=backend)
        pg = dist
    return ws, rank, local, pg


# ------------------------------------------------------------- multi-rank
def rank_frames(rank: int, frames_per_rank: int):
    """Frame indices of one rank: replicas over frames, no overlap."""
    return list(range(rank * frames_per_rank, (rank + 1) * frames_per_rank))


def max_over_ranks(t: float, pg, device=None) -> float:
    """Slowest rank's time (the job's time)."""
    if pg is None:
        return t
    import torch

    x = torch.tensor([t], dtype=torch.float64, device=device)
    pg.all_reduce(x, op=pg.ReduceOp.MAX)
    return float(x.item())


def job_value(pairs_per_rank_step: float, world: int, steps: int, t_max: float) -> float:
    """Whole-job Gpixel.ch/s: every rank's pairs over the slowest rank's time."""
    return pairs_per_rank_step * world * steps / t_max / 1e9


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons (200 ms period)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
         "clocks.mem,temperature.gpu")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, mem, temp = [], 0.0, set(), [], []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
            try:
                mem.append(float(f[9]))
                temp.append(float(f[10]))
            except (IndexError, ValueError):
                pass
        if not sm:
            return None
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
               "samples": len(sm)}
        if mem:
            out["mem_mhz_median"] = statistics.median(mem)
        if temp:
            out["temp_c_max"] = max(temp)
        return out


# ------------------------------------------------------------------ helpers
def sm_max_mhz():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return float(json.load(open(p))["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
        except Exception:
            pass
    return 2070.0, "nominal maximum SM clock (recipe fallback)"


def kernel_source_hash():
    """Hash of the fused kernel's sources, with comments and blank space
    removed, so that a change of wording does not void a measurement.  The
    launch configuration the plan picks is checked separately
    (LAUNCH_FIELDS)."""
    import re

    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        if f.startswith("pa_bf") or f == "pa_internal.cuh":
            src = open(os.path.join(CSRC, f)).read()
            src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
            src = re.sub(r"//[^\n]*", " ", src)
            h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


# Plan facts that fix the fused kernel's launch (grid, block, shared memory).
LAUNCH_FIELDS = ("threads", "blocks_per_sm", "window", "chunk_steps", "tile_x", "tile_z",
                 "tma_staging", "lane_rows")


def measured_traffic(kind, info=None):
    """DRAM bytes per launch of the fused kernel from the committed ncu
    summary, only if it was taken on the current kernel source and the plan
    launches it the same way."""
    p = os.path.join(ROOT, "profiles", "bf_fused_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        if d.get("kernel_hash") != kernel_source_hash():
            return None
        launch = d.get("launch", {})
        if info is not None and any(launch.get(f) != info.get(f) for f in LAUNCH_FIELDS):
            return None
        return d.get(kind)
    except Exception:
        return None


def ops_per_pair(k):
    """Algorithmic FP32-pipe ops per (pixel, channel) pair for the combined
    DAS + DMAS + DMAS-k pass (FMA = 1): floor/frac 2, lerp 2, root scale 1,
    powers k-1, power sums k, plus DAS and the two DMAS sums (3)."""
    if k == 1:
        return 5 + 2  # DAS + the two DMAS sums
    if k == 2:
        return 2 * k + 4 + 1
    return 2 * k + 7


# ------------------------------------------------------------------ oracle
def oracle_run(wl, rf64_frames, k, budget_s):
    """FP64 oracle over whole frames until ``budget_s`` is spent (>= 1 frame)."""
    import oracle

    pairs = wl["nx"] * wl["nz"] * wl["n_elem"]
    t0 = time.perf_counter()
    done = 0
    nf = rf64_frames.shape[0]
    while True:  # cycle through the step's frames until the budget is spent
        oracle.frame(wl, rf64_frames[done % nf], order_k=k, stages=("raw", "env", "log"))
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return done, pairs * done / dt / 1e9, dt, oracle.get_threads()


def oracle_timing():
    """FP64 oracle pairs/s per workload: cfg1 and cfg2 frames on all host
    cores and on one core, one cfg5 frame on all cores; median of the runs
    after one warm-up (5 runs; 3 for the slow one-core cfg2 frame)."""
    import oracle
    import synth

    oracle.build()
    n_all = oracle.get_threads()
    out = {}
    for name, seed, cores_list in (("cfg1", 1, (n_all, 1)), ("cfg2", 11, (n_all, 1)),
                                   ("cfg5", 41, (n_all,))):
        wl = synth.workload(name)
        rf = synth.quantize(synth.make_frame(wl, seed, 0), "f32")[1]
        pairs = wl["nx"] * wl["nz"] * wl["n_elem"]
        for cores in cores_list:
            oracle.set_threads(cores)
            runs = 3 if (cores == 1 and name != "cfg1") else 5
            oracle.frame(wl, rf, order_k=wl["order_k"])
            ts = []
            for _ in range(runs):
                t0 = time.perf_counter()
                oracle.frame(wl, rf, order_k=wl["order_k"])
                ts.append(time.perf_counter() - t0)
            out[f"{name}_{cores}core{'s' if cores > 1 else ''}"] = {
                "gpixel_ch_per_s": pairs / float(np.median(ts)) / 1e9,
                "ms_per_frame": float(np.median(ts)) * 1e3, "runs": runs, "k": wl["order_k"]}
    oracle.set_threads(n_all)
    return out


def run_reference(args):
    ws, rank, local, pg = dist_setup(args)
    if rank != 0:
        return 0
    import synth

    wl = workload()
    frames = np.stack([synth.quantize(synth.make_frame(wl, 11, f), "f32")[1] for f in range(2)])
    import oracle

    oracle.build()
    pairs = wl["nx"] * wl["nz"] * wl["n_elem"]
    for _ in range(args.warmup):
        oracle.frame(wl, frames[0], order_k=args.order)
    ts = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        oracle.frame(wl, frames[s % 2], order_k=args.order)
        ts.append(time.perf_counter() - t0)
    tot = sum(ts)
    value = pairs * args.steps / tot / 1e9
    sample = (f"1 frame per step of the workload ({wl['nx']}x{wl['nz']} x {wl['n_elem']} ch, "
              f"k={args.order}, raw+env+log), FP64")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded cfg2 recipe)",
        "config": config_dict(args, wl, {"frames_per_step": 1,
                                         "l2": "not applicable (FP64 oracle on the host cores)"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ours
def _errors(out, ref):
    """Per output: error of one GPU frame [stage][output] against an oracle frame."""
    import oracle

    rep = {}
    for oi, o in enumerate(oracle.OUTPUT_ORDER):
        r, e, lg = ref["raw"][o], ref["env"][o], ref["log"][o]
        sel = lg >= -6.0
        rep[o] = {
            "raw_max_err_of_peak": float(np.max(np.abs(out[0, oi] - r)) / np.max(np.abs(r))),
            "env_max_err_of_peak": float(np.max(np.abs(out[1, oi] - e)) / np.max(np.abs(e))),
            "log_max_abs_db_top6db": float(np.max(np.abs(out[2, oi][sel] - lg[sel]))),
            "log_mean_abs_db": float(np.mean(np.abs(out[2, oi] - lg))),
        }
    return rep


def precision_report(pa, wl, k, frames64, rf_dtype, comp, tol):
    """Errors of every GPU image of the given frames against the FP64 oracle:
    on the unquantised RF (end to end) and, for 16-bit RF, on the dequantised
    RF (the arithmetic alone).  Per output the worst frame is reported, and
    whether every image is within its tolerance (tol of the image peak before
    the log, 0.05 dB on the pixels within 6 dB of the peak after it; the
    arithmetic alone of a 16-bit form at the FP32 tolerance, 1e-4)."""
    import torch

    import oracle
    import synth

    F = frames64.shape[0]
    store, deq = synth.quantize(frames64, rf_dtype)
    desc = pa.make_desc(wl, order_k=k, outputs=7, rf_dtype=rf_dtype, compensated=comp,
                        max_batch=F)
    with pa.Plan(desc) as plan:
        if rf_dtype == "bf16":
            t = torch.from_numpy(store.view(np.int16)).cuda().view(torch.bfloat16)
        else:
            t = torch.from_numpy(store).cuda()
        out = pa.beamform(plan, t, 7).cpu().numpy()
    legs = {"vs_unquantised_rf": frames64}
    if rf_dtype != "f32":
        legs["vs_dequantised_rf"] = deq
    rep = {"frames": F}
    ok = True
    for leg, rf in legs.items():
        worst = {}
        for f in range(F):
            e = _errors(out[f], oracle.frame(wl, rf[f], order_k=k))
            for o, d in e.items():
                w = worst.setdefault(o, {kk: 0.0 for kk in d})
                for kk, v in d.items():
                    w[kk] = max(w[kk], v) if kk != "log_mean_abs_db" else w[kk] + v / F
        t_leg = 1e-4 if leg == "vs_dequantised_rf" else tol
        for o, d in worst.items():
            ok &= d["raw_max_err_of_peak"] <= t_leg and d["env_max_err_of_peak"] <= t_leg
            ok &= d["log_max_abs_db_top6db"] <= 0.05
        rep[leg] = worst
    rep["within_tolerance"] = bool(ok)
    rep["tolerance_of_peak"] = tol
    return rep


def time_form(pa, torch, wl, args, rf_dtype, comp, frames64, stream, flush, order=None,
              steps=None):
    """Device-timed steps of one arithmetic form; returns (times_s, profile, plan_info)."""
    import synth

    order = args.order if order is None else order
    steps = args.steps if steps is None else steps
    F = frames64.shape[0]
    store, _ = synth.quantize(frames64, rf_dtype)
    if rf_dtype == "bf16":
        rf = torch.from_numpy(store.view(np.int16)).cuda().view(torch.bfloat16)
    else:
        rf = torch.from_numpy(store).cuda()
    desc = pa.make_desc(wl, order_k=order, outputs=7, rf_dtype=rf_dtype, max_batch=F,
                        compensated=comp)
    plan = pa.Plan(desc, stream=stream)
    stages = pa.PA_STAGE_LOG
    out = torch.empty(plan.out_shape(F, stages), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush()
            pa.beamform(plan, rf, stages, out=out, stream=stream)
        stream.synchronize()
        plan.profile_read()
        plan.profile(True, fused_only=True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for s in range(steps):
            flush()
            evs[s][0].record(stream)
            pa.beamform(plan, rf, stages, out=out, stream=stream)
            evs[s][1].record(stream)
        stream.synchronize()
    prof = plan.profile_read()
    plan.profile(False)
    times = [a.elapsed_time(b) / 1e3 for a, b in evs]

    def again():
        with torch.cuda.stream(stream):
            for s in range(steps):
                flush()
                evs[s][0].record(stream)
                pa.beamform(plan, rf, stages, out=out, stream=stream)
                evs[s][1].record(stream)
            stream.synchronize()
        return [a.elapsed_time(b) / 1e3 for a, b in evs]

    # the same steps without the event nodes, then kernel by kernel with
    # events recorded on the stream around every launch (the post-filter and
    # log kernels' times come from there)
    time_form.graph_times = again()
    plan.use_graph(False)
    plan.profile(True)
    time_form.direct_times = again()
    time_form.direct_prof = plan.profile_read()
    plan.profile(False)
    plan.use_graph(True)
    prof = dict(time_form.direct_prof, bf_fused=prof["bf_fused"])
    info = plan.info()
    plan.close()
    return times, prof, info


def fused_roofline(prof, info, frames, k, peak):
    """Fused-kernel time per launch and its fraction of the FP32-issue
    roofline (active pairs x ops per pair / time / peak)."""
    ms, n = prof["bf_fused"]
    t = ms / 1e3 / max(n, 1)
    achieved = info["active_pairs"] * frames * ops_per_pair(k) / t / 1e12
    return {"kernel_ms_per_launch": t * 1e3, "achieved_top_s": achieved, "frac": achieved / peak,
            "ops_per_pair": ops_per_pair(k)}


def post_roofline(prof, wl, n_images, hbm_gbs, fp32_tflops):
    """Post filter (band-pass + Hilbert envelope) per launch against both
    roofs.  Algorithmic work per column pair: three complex M-point FFTs
    (one forward transform of the packed pair, one inverse per column),
    5 M log2 M flops each; bytes: the raw column read and the envelope
    written, 8 B per pixel."""
    ms, n = prof["post"]
    t = ms / 1e3 / max(n, 1)
    m = 1
    while m < wl["nz"]:
        m *= 2
    log2m = m.bit_length() - 1
    pairs = n_images * ((wl["nx"] + 1) // 2)
    flops = pairs * 3 * 5 * m * log2m
    nbytes = n_images * wl["nx"] * wl["nz"] * 8
    f, b = flops / t / 1e12, nbytes / t / 1e9
    return {"kernel_ms_per_launch": t * 1e3, "fft_points": m, "images": n_images,
            "flops_per_launch": flops, "achieved_tflops": f, "frac_fp32": f / fp32_tflops,
            "bytes_per_launch": nbytes, "achieved_gbs": b, "frac_hbm": b / hbm_gbs,
            "fp32_peak_tflops": fp32_tflops, "hbm_peak_gbs": hbm_gbs,
            "bound": "latency (both fractions low: shared-memory round trips and team barriers)"}


def off_lattice_bench(pa, torch, args, stream, flush, peak, lattice_value):
    """The headline workload on a grid off the lattice: cfg2 geometry (128 el
    x 2048 samples, 38.4 x 40 mm) on 400 x 512 pixels, pitch / dx = 3.125,
    so the plan takes the full per-pixel delay table; FP32 RF, k as the
    headline, 32 frames per step."""
    import synth

    wl = synth.workload("cfg2", nx=400)
    F = args.frames
    frames = np.stack([synth.make_frame(wl, 11, f) for f in range(F)])
    steps = max(3, min(args.steps, 50))
    t, prof, info = time_form(pa, torch, wl, args, "f32", 0, frames, stream, flush, steps=steps)
    value = wl["nx"] * wl["nz"] * wl["n_elem"] * F * steps / sum(t) / 1e9
    out = {
        "workload": (f"cfg2 geometry on a {wl['nx']}x{wl['nz']} grid (pitch / dx = 3.125, off the "
                     f"lattice): full per-pixel delay table, FP32 RF, k={args.order}, {F} frames"),
        "value": value, "unit": UNIT, "vs_lattice_headline": value / lattice_value,
        "delay_table": "full" if info["delay_table"] == 2 else "lattice",
        "table_bytes": info["table_bytes"], "steps": steps,
        "roofline": fused_roofline(prof, info, F, args.order, peak),
    }
    return out


def cfg3_bench(pa, torch, args, stream, flush, peak):
    """cfg3, the reduced-precision workload: 256 el x 4096 samples at 50 MHz,
    1024 x 1024 grid over 76.8 x 60 mm, 8 frames per step.  Rates of the
    BF16 + Kahan form and the plain FP32 form at k = 3 and k = 5 (device
    time, L2 flushed between steps), and the errors of every image of two
    frames against the FP64 oracle for BF16 and FP16 storage."""
    import synth

    wl = synth.workload("cfg3")
    F = 8
    frames = np.stack([synth.make_frame(wl, wl["seeds"][0], f) for f in range(F)])
    steps = max(3, min(args.steps, 20))
    pairs = wl["nx"] * wl["nz"] * wl["n_elem"] * F
    out = {"workload": ("cfg3: 256 el x 4096 samples @ 50 MHz, 1024x1024 grid, 20 points over "
                        "40 dB, unit-RMS RF; DAS+DMAS+DMAS-k, log images, 8 frames per step"),
           "frames_per_step": F, "steps": steps, "unit": UNIT}
    for k in (3, 5):
        leg = {}
        for name, dt, comp in (("bf16_kahan", "bf16", 1), ("fp32", "f32", 0)):
            t, prof, info = time_form(pa, torch, wl, args, dt, comp, frames, stream, flush,
                                      order=k, steps=steps)
            leg[name] = {"value": pairs * steps / sum(t) / 1e9,
                         "roofline": fused_roofline(prof, info, F, k, peak)}
        leg["bf16_kahan_vs_fp32"] = leg["bf16_kahan"]["value"] / leg["fp32"]["value"]
        out[f"k{k}"] = leg
    rep_frames = frames[:2]
    out["precision_report"] = {
        "bf16_kahan_k3": precision_report(pa, wl, 3, rep_frames, "bf16", 1, 5e-3),
        "f16_kahan_k3": precision_report(pa, wl, 3, rep_frames, "f16", 1, 5e-3),
        "bf16_kahan_k5": precision_report(pa, wl, 5, rep_frames, "bf16", 1, 5e-3),
        "against": "FP64 oracle, every image of 2 frames (worst frame per output)",
    }
    return out


def metrics_rois(wl):
    """Ten target discs (r = 0.5 mm) in five depth pairs, the layout of the
    paper's simulated phantom (Section 3), each with a 1-2 mm annulus as
    background."""
    w = wl["x1_m"] - wl["x0_m"]
    h = wl["z1_m"] - wl["z0_m"]
    rois = []
    for fz in (0.2, 0.35, 0.5, 0.65, 0.8):
        for fx in (-0.15, 0.15):
            xc, zc = wl["x0_m"] + (0.5 + fx) * w, wl["z0_m"] + fz * h
            rois.append((dict(shape="disc", xc_m=xc, zc_m=zc, a_m=0.5e-3),
                         dict(shape="annulus", xc_m=xc, zc_m=zc, a_m=1.0e-3, b_m=2.0e-3)))
    return rois


def metrics_bench(pa, torch, wl, args, frames64, stream, flush):
    """pa_image_metrics on the envelope images of one step (frames x 3
    outputs), device-timed with an L2 flush before each call."""
    import ctypes

    import synth
    from paper_2203_14906_gb300._native import Metrics

    F = frames64.shape[0]
    store, _ = synth.quantize(frames64, "f32")
    rf = torch.from_numpy(store).cuda()
    desc = pa.make_desc(wl, order_k=args.order, outputs=7, rf_dtype="f32", max_batch=F)
    rois = metrics_rois(wl)
    reps = max(3, min(args.steps, 50))
    with pa.Plan(desc, stream=stream) as plan, torch.cuda.stream(stream):
        env = pa.beamform(plan, rf, pa.PA_STAGE_ENV, stream=stream)[:, 0].contiguous()
        n_img = env.shape[0] * env.shape[1]
        rec = torch.empty(n_img * len(rois) * ctypes.sizeof(Metrics), dtype=torch.uint8,
                          device=env.device)
        for _ in range(args.warmup):
            pa.image_metrics(env, wl, rois, stream=stream, out=rec)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(reps)]
        for a, b in evs:
            flush()
            a.record(stream)
            pa.image_metrics(env, wl, rois, stream=stream, out=rec)
            b.record(stream)
        stream.synchronize()
        m = pa.image_metrics(env, wl, rois, stream=stream)
    t = float(np.mean([a.elapsed_time(b) for a, b in evs])) / 1e3
    # algorithmic bytes: both passes read every member pixel once (4 B each)
    members = float(np.sum(m["n_in"]) + np.sum(m["n_out"]))
    nbytes = 2 * 4 * members
    return {
        "images_per_s": n_img / t, "ms_per_call": t * 1e3, "images_per_call": n_img,
        "roi_pairs_per_image": len(rois), "launches_per_call": 5,
        "member_pixels_per_call": members, "algorithmic_bytes_per_call": nbytes,
        "achieved_gbs": nbytes / t / 1e9,
        "note": ("launch- and latency-bound, not HBM-bound: the regions cover "
                 f"{members / n_img / (wl['nx'] * wl['nz']):.1%} of each image"),
        "sample_hodmas_frame0": {kk: float(np.nanmean(m[kk][2])) for kk in
                                 ("snr_db", "cr_db", "gcnr", "fwhm_m")},
    }


def throughput_batch(pa, torch, args, stream, flush):
    """The throughput-batch workload: 64 frames of 128 channels x 2048 BF16
    samples per launch, 1024 x 1024 grid, DAS + DMAS + DMAS-4, F-number 1.5
    dynamic aperture with Hann apodisation, Kahan sums, CUDA-graph launch;
    device-timed with an L2 flush before each step."""
    import synth

    wl = synth.workload("cfg5")
    F = int(wl.get("n_frames", 64))
    frames = np.stack([synth.make_frame(wl, wl["seeds"][0], f) for f in range(F)])
    store, _ = synth.quantize(frames, "bf16")
    rf = torch.from_numpy(store.view(np.int16)).cuda().view(torch.bfloat16)
    desc = pa.make_desc(wl, order_k=wl["order_k"], outputs=7, rf_dtype="bf16", max_batch=F,
                        compensated=1)
    steps = max(3, min(args.steps, 20))
    with pa.Plan(desc, stream=stream) as plan, torch.cuda.stream(stream):
        out = torch.empty(plan.out_shape(F, pa.PA_STAGE_LOG), dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            flush()
            pa.beamform(plan, rf, pa.PA_STAGE_LOG, out=out, stream=stream)
        stream.synchronize()
        plan.profile_read()
        plan.profile(True, fused_only=True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for a, b in evs:
            flush()
            a.record(stream)
            pa.beamform(plan, rf, pa.PA_STAGE_LOG, out=out, stream=stream)
            b.record(stream)
        stream.synchronize()
        prof = plan.profile_read()
        # the post and log kernels: the same steps again with every kernel timed
        plan.profile(True)
        for _ in range(steps):
            flush()
            pa.beamform(plan, rf, pa.PA_STAGE_LOG, out=out, stream=stream)
        stream.synchronize()
        prof = dict(plan.profile_read(), bf_fused=prof["bf_fused"])
        plan.profile(False)
        info = plan.info()
    t = float(np.mean([a.elapsed_time(b) for a, b in evs])) / 1e3
    nominal = info["nominal_pairs"] * F
    active = info["active_pairs"] * F
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    peak = n_sm * 128 * sm_max_mhz()[0] * 1e6 / 1e12
    hbm_gbs = 6687.1
    try:
        hbm_gbs = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        pass
    fused = fused_roofline(prof, info, F, wl["order_k"], peak)
    # the apodisation multiply is one more operation per active pair
    fused["ops_per_pair_with_apodisation"] = fused["ops_per_pair"] + 1
    fused["frac_with_apodisation"] = fused["frac"] * (fused["ops_per_pair"] + 1) / fused["ops_per_pair"]
    return {
        "roofline": fused,
        "post_filter": post_roofline(prof, wl, F * 3, hbm_gbs, 2 * peak),
        "workload": ("cfg5: 64 frames x 128 el x 2048 samples BF16 @ 40 MHz, 1024x1024 grid, "
                     "DAS+DMAS+DMAS-4, F# 1.5 Hann dynamic aperture, Kahan sums, log images"),
        "frames_per_s": F / t, "ms_per_step": t * 1e3, "steps": steps,
        "value_nominal": nominal / t / 1e9, "value_active": active / t / 1e9, "unit": UNIT,
        "active_fraction": active / nominal,
        "kernels_ms_per_launch": {kk: v[0] / max(v[1], 1) for kk, v in prof.items()},
    }


class _ServeSet:
    """Requests of cfg4 traces for one arithmetic form: pinned RF frames per
    (channels, samples) class, one descriptor per plan class, a ring of
    pinned output buffers (results are not read; timing only)."""

    RING = 64

    def __init__(self, pa, rf_dtype, comp):
        import torch

        import synth

        self.pa, self.rf_dtype, self.comp = pa, rf_dtype, comp
        self.pool, self.descs = {}, {}
        self.ring = torch.empty((self.RING, 3 * 1024 * 1024), dtype=torch.float32).pin_memory()
        self._synth = synth

    def requests(self, n, seed, rate_hz):
        """[(arrival_s, desc, rf, pairs)] of a seeded Poisson trace."""
        import torch

        synth = self._synth
        out = []
        for i, (t_arr, wl) in enumerate(synth.serving_mix(n, seed=seed, rate_hz=rate_hz)):
            key = (wl["n_elem"], wl["n_samples"])
            if key not in self.pool:
                fr = []
                for j in range(2):
                    store, _ = synth.quantize(synth.make_frame(wl, 31, 1000 + j), self.rf_dtype)
                    t = torch.from_numpy(store.view(np.int16) if self.rf_dtype == "bf16" else store)
                    fr.append(t.pin_memory())
                self.pool[key] = fr
            dk = (wl["n_elem"], wl["n_samples"], wl["nx"], wl["order_k"])
            if dk not in self.descs:
                self.descs[dk] = self.pa.make_desc(wl, order_k=wl["order_k"], outputs=7,
                                                   rf_dtype=self.rf_dtype, compensated=self.comp)
            out.append((t_arr, self.descs[dk], self.pool[key][i % 2],
                        wl["nx"] * wl["nz"] * wl["n_elem"]))
        return out

    def warm(self, srv):
        """One request per plan class, so every plan is resident."""
        for i, d in enumerate(self.descs.values()):
            rf = self.pool[(d.n_elem, d.n_samples)][0]
            srv.wait(srv.submit(d, rf.data_ptr(), self.ring[i % self.RING].data_ptr()))

    def replay(self, srv, reqs, timed_arrivals=True, local=0):
        """Submit a trace (arrival times replayed, or every request at once)
        and wait for all of it; served rate, latency percentiles, clocks."""
        from paper_2203_14906_gb300.serving import percentiles

        clk = ClockSampler(local)
        clk.start()
        st0 = srv.stats()
        t0 = srv.now() + 0.2
        tickets = [srv.submit(d, rf.data_ptr(), self.ring[i % self.RING].data_ptr(),
                              t0 + (t_arr if timed_arrivals else 0.0))
                   for i, (t_arr, d, rf, _) in enumerate(reqs)]
        res = [srv.wait(t) for t in tickets]
        st1 = srv.stats()
        clocks = clk.stop()
        lat = [r["latency_ms"] for r in res if r["status"] == 0]
        span = max(r["done_s"] for r in res) - (t0 if timed_arrivals else
                                                 min(r["start_s"] for r in res))
        # the requests above the 99th percentile: queue wait (arrival to
        # issue) against service (issue to completion seen), and their classes
        tail = {}
        if lat:
            cut = float(np.percentile(lat, 99))
            slow = [(r, rq) for r, rq in zip(res, reqs) if r["status"] == 0 and r["latency_ms"] >= cut]
            cls = {}
            for r, (_, d, _, _) in slow:
                k = f"N{d.n_elem} Ns{d.n_samples} {d.nx}^2 k{d.order_k}"
                cls[k] = cls.get(k, 0) + 1
            tail = {"wait_ms_median": float(np.median([(r["start_s"] - r["arrival_s"]) * 1e3
                                                       for r, _ in slow])),
                    "service_ms_median": float(np.median([(r["done_s"] - r["start_s"]) * 1e3
                                                          for r, _ in slow])),
                    "device_ms_median": float(np.median([r["device_ms"] for r, _ in slow])),
                    "arrival_s_span": [float(min(r["arrival_s"] for r, _ in slow) - t0),
                                       float(max(r["arrival_s"] for r, _ in slow) - t0)],
                    "classes": sorted(cls.items(), key=lambda kv: -kv[1])[:3]}
        out = {"frames": len(res), "failed": sum(r["status"] != 0 for r in res),
               "served_frames_per_s": len(res) / span,
               "gpixel_ch_per_s": sum(p for *_, p in reqs) / span / 1e9,
               "mean_batch_frames": float(np.mean([r["batch_frames"] for r in res])),
               "batches": st1["batches"] - st0["batches"],
               "plans_resident": st1["plans_resident"], "device_bytes_peak": st1["bytes_peak"],
               "latency_ms_mean": float(np.mean(lat)) if lat else None,
               "device_ms_mean": float(np.mean([r["device_ms"] for r in res])),
               "sm_mhz_median": clocks["sm_mhz"] if clocks else None,
               "clock_reasons": clocks["reasons"] if clocks else None,
               "mem_mhz_median": clocks.get("mem_mhz_median") if clocks else None,
               "temp_c_max": clocks.get("temp_c_max") if clocks else None,
               "p99_tail": tail}
        out.update({f"latency_ms_{q}": v for q, v in percentiles(lat).items()})
        return out


def _spread(runs, key):
    v = [r[key] for r in runs if r.get(key) is not None]
    if not v:
        return None
    m = float(np.median(v))
    return {"median": m, "min": float(min(v)), "max": float(max(v)),
            "spread_of_median": (max(v) - min(v)) / m if m else None}


SERVER_CFG = dict(budget_bytes=16 << 30, slots=4, max_batch=8)


def serving_legs(pa, args, local):
    """cfg4 serving, per arithmetic form (BF16 + Kahan and plain FP32):
    * offered: the stated trace (Poisson, --serve-rate frames/s, plans
      resident), three repeats with their own seeds;
    * saturation: every request queued at once (closed queue), three repeats:
      the maximum sustained frames/s and Gpixel.ch/s;
    * load points: Poisson traces at 30 / 60 / 90 % of the measured
      saturation rate, three repeats each: p50 / p99 latency;
    * cold: the stated trace on a fresh server with no plan resident (plans
      are built on the server's builder thread as their first request comes).
    Every run records the median SM clock sampled while it ran."""
    from paper_2203_14906_gb300.serving import Server

    n_sat = 4000
    out = {"workload": (f"cfg4 mix: N in {{64,128,256}}, Ns in {{1024,2048,4096}} @ 40 MHz, grid "
                        "{256,512,1024}^2, k uniform in 2..5; DAS+DMAS+DMAS-k log images "
                        "returned to pinned host memory; server: 4 slots, batches up to 8 "
                        "frames of one descriptor, 16 GiB budget"),
           "offered_frames_per_s": args.serve_rate}
    for form, (dt, comp) in (("bf16_kahan", ("bf16", 1)), ("fp32", ("f32", 0))):
        ss = _ServeSet(pa, dt, comp)
        offered_reqs = [ss.requests(args.serve_requests, 31 + r, args.serve_rate) for r in range(3)]
        sat_reqs = [ss.requests(n_sat, 131 + r, 1e6) for r in range(3)]
        leg = {}
        with Server(**SERVER_CFG, stages=pa.PA_STAGE_LOG) as srv:
            ss.warm(srv)
            offered = [ss.replay(srv, rq, True, local) for rq in offered_reqs]
            sat = [ss.replay(srv, rq, False, local) for rq in sat_reqs]
            cap = float(np.median([r["served_frames_per_s"] for r in sat]))
            loads = {}
            for frac in (0.3, 0.6, 0.9):
                rate = frac * cap
                n = int(min(20000, max(1000, rate * 1.5)))
                traces = [ss.requests(n, 231 + r, rate) for r in range(3)]
                ss.warm(srv)  # any plan class these traces add is resident too
                runs = [ss.replay(srv, rq, True, local) for rq in traces]
                loads[f"{int(frac * 100)}pct"] = {
                    "offered_frames_per_s": rate, "frames_per_run": n,
                    "p99_tail": [r["p99_tail"] for r in runs],
                    "served_frames_per_s": _spread(runs, "served_frames_per_s"),
                    "latency_ms_p50": _spread(runs, "latency_ms_p50"),
                    "latency_ms_p99": _spread(runs, "latency_ms_p99"),
                    "mean_batch_frames": _spread(runs, "mean_batch_frames"),
                    "sm_mhz_median": [r["sm_mhz_median"] for r in runs]}
        leg["offered"] = {
            "runs": offered,
            "latency_ms_p50": _spread(offered, "latency_ms_p50"),
            "latency_ms_p99": _spread(offered, "latency_ms_p99"),
            "served_frames_per_s": _spread(offered, "served_frames_per_s")}
        leg["saturation"] = {
            "frames_per_run": n_sat, "runs": sat,
            "served_frames_per_s": _spread(sat, "served_frames_per_s"),
            "gpixel_ch_per_s": _spread(sat, "gpixel_ch_per_s"),
            "mean_batch_frames": _spread(sat, "mean_batch_frames")}
        leg["load_points"] = loads
        with Server(**SERVER_CFG, stages=pa.PA_STAGE_LOG) as srv:
            leg["cold"] = ss.replay(srv, offered_reqs[0], True, local)
        out[form] = leg
    b, f = out["bf16_kahan"]["saturation"], out["fp32"]["saturation"]
    ratio = b["gpixel_ch_per_s"]["median"] / f["gpixel_ch_per_s"]["median"]
    noise = max(b["gpixel_ch_per_s"]["spread_of_median"], f["gpixel_ch_per_s"]["spread_of_median"])
    out["saturation_bf16_kahan_vs_fp32"] = {
        "ratio": ratio, "run_to_run_spread": noise,
        "difference_exceeds_spread": abs(ratio - 1.0) > noise,
        "note": "the forms' legs ran one after the other; see paired_forms"}
    out["paired_forms"] = paired_forms(pa, args, local)
    return out


def paired_forms(pa, args, local, pairs=5, n_sat=4000, offered_pairs=4):
    """The two forms measured in pairs on one server that holds both forms'
    plans (warm): runs alternate BF16 + Kahan / FP32 in ABBA order, each on
    its own request set, so that a drift of the box over the process weighs
    on both forms alike.  Saturation (every request queued at once): each
    pair's throughput ratio.  The stated trace (--serve-rate Poisson): each
    pair's p50 / p99.  A difference holds when every pair lies on the same
    side."""
    from paper_2203_14906_gb300.serving import Server

    sets = {"bf16_kahan": _ServeSet(pa, "bf16", 1), "fp32": _ServeSet(pa, "f32", 0)}
    sat_reqs = {k: [ss.requests(n_sat, 331 + r, 1e6) for r in range(pairs)]
                for k, ss in sets.items()}
    off_reqs = {k: [ss.requests(args.serve_requests, 431 + r, args.serve_rate)
                    for r in range(offered_pairs)] for k, ss in sets.items()}
    sat = {k: [] for k in sets}
    off = {k: [] for k in sets}

    def order(r):
        return ("bf16_kahan", "fp32") if r % 2 == 0 else ("fp32", "bf16_kahan")

    with Server(**SERVER_CFG, stages=pa.PA_STAGE_LOG) as srv:
        for ss in sets.values():
            ss.warm(srv)
        for r in range(pairs):
            for k in order(r):
                sat[k].append(sets[k].replay(srv, sat_reqs[k][r], False, local))
        for r in range(offered_pairs):
            for k in order(r):
                off[k].append(sets[k].replay(srv, off_reqs[k][r], True, local))
    ratios = [a["gpixel_ch_per_s"] / b["gpixel_ch_per_s"]
              for a, b in zip(sat["bf16_kahan"], sat["fp32"])]
    p99 = {k: [r["latency_ms_p99"] for r in off[k]] for k in off}
    p99_ratio = [a / b for a, b in zip(p99["bf16_kahan"], p99["fp32"])]

    def same_side(v):
        return all(x > 1.0 for x in v) or all(x < 1.0 for x in v)

    return {
        "server": "one server, both forms' plans resident", "order": "ABBA...",
        "saturation": {
            "pairs": pairs, "frames_per_run": n_sat,
            "bf16_kahan_gpixel_ch_per_s": [r["gpixel_ch_per_s"] for r in sat["bf16_kahan"]],
            "fp32_gpixel_ch_per_s": [r["gpixel_ch_per_s"] for r in sat["fp32"]],
            "bf16_kahan_frames_per_s": [r["served_frames_per_s"] for r in sat["bf16_kahan"]],
            "fp32_frames_per_s": [r["served_frames_per_s"] for r in sat["fp32"]],
            "ratio_per_pair": ratios, "ratio_median": float(np.median(ratios)),
            "every_pair_same_side": same_side(ratios)},
        "offered": {
            "pairs": offered_pairs, "frames_per_run": args.serve_requests,
            "offered_frames_per_s": args.serve_rate,
            "bf16_kahan_p50_ms": [r["latency_ms_p50"] for r in off["bf16_kahan"]],
            "fp32_p50_ms": [r["latency_ms_p50"] for r in off["fp32"]],
            "bf16_kahan_p99_ms": p99["bf16_kahan"], "fp32_p99_ms": p99["fp32"],
            "p99_ratio_per_pair": p99_ratio, "p99_ratio_median": float(np.median(p99_ratio)),
            "every_pair_same_side": same_side(p99_ratio)},
        "plans_resident": sorted({r["plans_resident"] for d in (sat, off) for k in d for r in d[k]}),
        "sm_mhz_median": sorted({r["sm_mhz_median"] for d in (sat, off) for k in d for r in d[k]})}


def run_ours(args):
    ws, rank, local, pg = dist_setup(args)
    import torch

    import synth
    import paper_2203_14906_gb300 as pa

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = workload()
    F, k = args.frames, args.order
    pairs_step = wl["nx"] * wl["nz"] * wl["n_elem"] * F
    frames64 = np.stack([synth.make_frame(wl, 11, f) for f in rank_frames(rank, F)])
    stream = torch.cuda.Stream(dev)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def flush():
        flush_buf.zero_()

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    # ---- FP32 form (the headline)
    barrier()
    clk = ClockSampler(local)
    clk.start()
    rf_dtype, comp = form_dtype(args)
    times, prof, info = time_form(pa, torch, wl, args, rf_dtype, comp, frames64, stream, flush)
    clocks = clk.stop()
    barrier()
    graph_times = time_form.graph_times
    t_tot = max_over_ranks(sum(times), pg, dev)
    value = job_value(pairs_step, ws, args.steps, t_tot)
    step_median_ms = float(np.median(times)) * 1e3
    t_graph = max_over_ranks(sum(graph_times), pg, dev)
    t_direct = max_over_ranks(sum(time_form.direct_times), pg, dev)
    dp = time_form.direct_prof["bf_fused"]
    graph_path = {
        "value": job_value(pairs_step, ws, args.steps, t_graph), "unit": UNIT,
        "ms_per_step": t_graph / args.steps * 1e3,
        "note": ("the same steps through the same CUDA graphs without the two event-record "
                 "nodes that time the fused kernel in the headline steps"),
        "kernel_by_kernel": {
            "value": job_value(pairs_step, ws, args.steps, t_direct), "unit": UNIT,
            "ms_per_step": t_direct / args.steps * 1e3,
            "fused_kernel_ms_per_launch": dp[0] / max(dp[1], 1),
            "note": "graphs off: each kernel launched on the stream between two CUDA events"}}

    # roofline of the dominant kernel (the fused beamformer)
    bf_ms, bf_n = prof["bf_fused"]
    bf_s = bf_ms / 1e3 / max(bf_n, 1)
    opp = ops_per_pair(k)
    achieved = info["active_pairs"] * F * opp / bf_s / 1e12
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz, mhz_src = sm_max_mhz()
    peak = n_sm * 128 * mhz * 1e6 / 1e12
    roofline = {
        "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Top/s (FP32 pipe, FMA=1)",
        "frac": achieved / peak, "traffic": measured_traffic("dram_bytes_per_launch", info),
        "kernel": "k_bf_fused", "ops_per_pair": opp,
        "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x {mhz:g} MHz ({mhz_src})",
        "kernel_ms_per_launch": bf_s * 1e3,
        "share_of_step": bf_s / (t_tot / args.steps),
        "kernels_ms_per_launch": {kk: (v[0] / max(v[1], 1)) for kk, v in prof.items()},
        "kernel_timing": ("fused kernel: event-record nodes around it in the timed steps' "
                          "graphs; post and log: the kernel-by-kernel pass of the same steps"),
    }
    hbm_gbs = 6687.1
    try:
        hbm_gbs = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        pass
    roofline["post_filter"] = post_roofline(prof, wl, F * 3, hbm_gbs, 2 * peak)
    # the three kernels profiled per launch sequence, plus its clearing kernel
    launches = int(sum(v[1] for v in prof.values()) + prof["bf_fused"][1])

    # ---- end to end through the host-buffer ABI call
    desc = pa.make_desc(wl, order_k=k, outputs=7, rf_dtype=rf_dtype, max_batch=F, compensated=comp)
    store, _ = synth.quantize(frames64, rf_dtype)
    if rf_dtype == "bf16":
        rf_h = torch.from_numpy(store.view(np.int16)).view(torch.bfloat16).pin_memory()
    else:
        rf_h = torch.from_numpy(store).pin_memory()
    with pa.Plan(desc) as plan:
        out_h = torch.empty(plan.out_shape(F, pa.PA_STAGE_LOG), dtype=torch.float32).pin_memory()
        for _ in range(max(1, args.warmup)):
            pa.beamform_host(plan, rf_h, pa.PA_STAGE_LOG, out=out_h)
        # the plan times candidate chunk schedules on its first calls of a shape
        for _ in range(200):
            chunks, state = plan.host_schedule(F, pa.PA_STAGE_LOG)
            if state != 1:
                break
            pa.beamform_host(plan, rf_h, pa.PA_STAGE_LOG, out=out_h)
        barrier()
        e2e_steps = max(1, min(args.steps, 50))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            pa.beamform_host(plan, rf_h, pa.PA_STAGE_LOG, out=out_h)
        te = time.perf_counter() - t0
    te = max_over_ranks(te, pg, dev)
    e2e = {"value": job_value(pairs_step, ws, e2e_steps, te), "unit": UNIT,
           "h2d_bytes_per_step": int(rf_h.numel() * rf_h.element_size()),
           "d2h_bytes_per_step": int(out_h.numel() * out_h.element_size()),
           "call": "pa_beamform_host (pinned host buffers)", "steps": e2e_steps,
           "chunks": chunks}

    extras = {}
    # serving first: the CPU-heavy oracle legs below would compete with the
    # server's scheduler thread for host cores
    if not args.no_serving and rank == 0:
        extras["serving"] = serving_legs(pa, args, local)

    if not args.no_extras:
        # reduced-precision form on the same workload: BF16 RF + Kahan sums
        t_bf, prof_bf, _ = time_form(pa, torch, wl, args, "bf16", 1, frames64, stream, flush)
        v_bf = pairs_step * args.steps / sum(t_bf) / 1e9
        extras["precision_form"] = {
            "value": v_bf * ws, "unit": UNIT, "rf_dtype": "bf16", "compensated": True,
            "vs_fp32_form": v_bf * ws / value,
            "kernel_ms_per_launch": prof_bf["bf_fused"][0] / max(prof_bf["bf_fused"][1], 1),
        }
        # nearest-sample delays (Eq. 1's integer index), FP32, same workload
        wl_n = dict(wl, interp="nearest")
        t_nn, prof_nn, _ = time_form(pa, torch, wl_n, args, "f32", 0, frames64, stream, flush)
        v_nn = pairs_step * args.steps / sum(t_nn) / 1e9
        extras["nearest_form"] = {
            "value": v_nn * ws, "unit": UNIT, "interp": "nearest (Eq. 1 integer delay)",
            "vs_fp32_form": v_nn * ws / value,
            "kernel_ms_per_launch": prof_nn["bf_fused"][0] / max(prof_nn["bf_fused"][1], 1),
        }
        extras["off_lattice_form"] = off_lattice_bench(pa, torch, args, stream, flush, peak,
                                                       value / ws)
        if args.order == 3 and rank == 0:
            extras["mapping_comparison"] = mapping_bench(pa, torch, args, wl, frames64, stream,
                                                         flush, bf_s * 1e3, peak)
        if rank == 0:
            nrep = min(8, frames64.shape[0])
            extras["precision_report"] = {
                "fp32": precision_report(pa, wl, k, frames64[:nrep], "f32", 0, 1e-4),
                "bf16_kahan": precision_report(pa, wl, k, frames64[:nrep], "bf16", 1, 5e-3),
                "against": (f"FP64 oracle, every image of the first {nrep} frames (worst frame "
                            "per output)"),
            }
            extras["metrics_form"] = metrics_bench(pa, torch, wl, args, frames64, stream, flush)
            extras["precision_cfg3"] = cfg3_bench(pa, torch, args, stream, flush, peak)
            extras["oracle_timing"] = oracle_timing()
            extras["throughput_batch"] = throughput_batch(pa, torch, args, stream, flush)
            done, v_cpu, dt, cores = oracle_run(wl, frames64, k, args.cpu_seconds)
            extras["cpu_baseline"] = {
                "value": v_cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": (f"{done} whole frame(s) of the workload (raw+env+log, k={k}), "
                           f"{dt:.1f} s, FP64, OpenMP over image columns"),
            }
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_tot / args.steps * 1e3,
            "ms_per_step_median": step_median_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded point + line absorbers, 3% noise; cfg2 recipe)",
            "config": config_dict(args, wl), "clocks": clocks, "e2e": e2e,
            "gpu_launches": launches, "roofline": roofline, "graph_path": graph_path,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def lanes_times(pa, torch, plan, rf, F, lanes, warmup, launches, stream, flush):
    """CUDA-event times (s) of pa_lanes_raw launches, an L2 flush before each."""
    from paper_2203_14906_gb300 import _native

    L = _native.load()
    out = torch.empty(plan.out_shape(F, pa.PA_STAGE_RAW), dtype=torch.float32, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(launches)]
    with torch.cuda.stream(stream):
        for i in range(warmup + launches):
            flush()
            if i >= warmup:
                evs[i - warmup][0].record(stream)
            st = L.pa_lanes_raw(plan.handle, rf.data_ptr(), F, out.data_ptr(), lanes,
                                stream.cuda_stream)
            if st != 0:
                raise RuntimeError(L.pa_last_error().decode())
            if i >= warmup:
                evs[i - warmup][1].record(stream)
        stream.synchronize()
    return [a.elapsed_time(b) / 1e3 for a, b in evs]


def run_case_lanes(args, pa, torch, wl, F, k, rf, desc, stream, flush):
    with pa.Plan(desc, stream=stream) as plan:
        t = lanes_times(pa, torch, plan, rf, F, args.lanes, args.warmup, args.launches, stream,
                        lambda: flush.zero_())
    print(json.dumps({"case": args.case, "grid": [wl["nx"], wl["nz"]], "frames": F,
                      "order_k": k, "lanes_per_pixel": args.lanes,
                      "k_lanes_ms_per_launch": float(np.mean(t)) * 1e3}), flush=True)
    return 0


def mapping_bench(pa, torch, args, wl, frames64, stream, flush, fused_ms, peak):
    """The channels-on-lanes mapping (pa_lanes_raw, 4 / 8 / 32 lanes per
    pixel, partial sums added by warp shuffles) against the fused kernel's
    pixels-on-lanes mapping, on the headline workload's frames (FP32, k = 3,
    RAW planes), device-timed with an L2 flush before each launch."""
    import synth

    F = frames64.shape[0]
    store, _ = synth.quantize(frames64, "f32")
    rf = torch.from_numpy(store).cuda()
    out = {"workload": "headline frames, FP32, k = 3, raw sums only",
           "fused_kernel_ms": fused_ms}
    desc = pa.make_desc(wl, order_k=3, outputs=7, rf_dtype="f32", max_batch=F)
    pairs = wl["nx"] * wl["nz"] * wl["n_elem"] * F
    with pa.Plan(desc, stream=stream) as plan:
        for lanes in (4, 8, 32):
            t = float(np.mean(lanes_times(pa, torch, plan, rf, F, lanes, 3, 10, stream, flush)))
            out[f"lanes_{lanes}"] = {
                "kernel_ms": t * 1e3, "vs_fused": fused_ms / (t * 1e3),
                "frac": pairs * ops_per_pair(3) / t / 1e12 / peak}
    return out


def run_case(args):
    """One workload's launch sequence, timed per kernel (see the module
    docstring); no oracle, no extras."""
    import torch

    import synth
    import paper_2203_14906_gb300 as pa

    over = {kk: v for kk, v in (("nx", args.nx), ("nz", args.nz)) if v is not None}
    wl = synth.workload(args.case, delay_table=args.table, interp=args.interp, **over)
    F = args.frames or int(wl.get("n_frames", 1))
    k = args.order or int(wl.get("order_k", 3))
    rf_dtype = args.rf or wl.get("rf_dtype", "f32")
    comp = args.compensated if args.compensated is not None else int(wl.get("compensated", 0))
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    x = torch.randn(F, wl["n_elem"], wl["n_samples"], device=dev, generator=g)
    rf = x.to({"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[rf_dtype])
    desc = pa.make_desc(wl, order_k=k, outputs=7, rf_dtype=rf_dtype, max_batch=F, compensated=comp)
    if args.lanes:
        return run_case_lanes(args, pa, torch, wl, F, k, rf, desc, stream, flush)
    with pa.Plan(desc, stream=stream) as plan, torch.cuda.stream(stream):
        out = torch.empty(plan.out_shape(F, pa.PA_STAGE_LOG), dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            flush.zero_()
            pa.beamform(plan, rf, pa.PA_STAGE_LOG, out=out, stream=stream)
        stream.synchronize()
        plan.profile_read()
        plan.profile(True)
        for _ in range(args.launches):
            flush.zero_()
            pa.beamform(plan, rf, pa.PA_STAGE_LOG, out=out, stream=stream)
        stream.synchronize()
        prof = plan.profile_read()
        plan.profile(False)
        info = plan.info()
    print(json.dumps({
        "case": args.case, "grid": [wl["nx"], wl["nz"]], "frames": F, "order_k": k,
        "rf": rf_dtype, "compensated": comp, "interp": args.interp,
        "kernels_ms_per_launch": {kk: v[0] / max(v[1], 1) for kk, v in prof.items()},
        "plan": {f: info[f] for f in LAUNCH_FIELDS + ("lattice_m", "tmem_columns", "delay_table",
                                                      "table_bytes")},
        "nominal_pairs": info["nominal_pairs"] * F, "active_pairs": info["active_pairs"] * F,
        "device_error_flags": info["device_error_flags"],
    }), flush=True)
    return 0 if info["device_error_flags"] == 0 else 1


def main():
    args = parse()
    if args.case is not None:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
