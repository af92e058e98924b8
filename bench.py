"""Benchmark of the Hadamard-spectral-code shading path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hsc|reference]

Workload (one step = one frame): a 1920x1080 G-buffer with a secondary
G-buffer for one indirect bounce, n = 81 samples (380-780 nm at 5 nm), k = 6,
64 point lights (32 blackbody, 32 narrow-band), 288 materials; seeded
synthetic inputs.  The latent frame is: encode materials and lights, fused
k-channel shading writing the latent image, its XYZ and its 8-bit sRGB (the
decode of Fig. 2b in the shading kernel's epilogue).
``value`` is pixel-light evaluations per second of that frame (2 x 64 per
pixel).  The other parts of the metric are measured in the same run on the
same frame: n-sample spectral shading (the comparison), the k/3-pass form,
k = 9, the FP32 and tensor-core spectral decodes (GB/s) and the frame-time
percentiles.  L2 is flushed before every timed iteration (256 MB write, then
a 256 MB read of another buffer so that the write's dirty lines are written
back before, not inside, the timed region).

``--impl reference`` times the FP64 CPU oracle on a band of rows of the same
frame (the only reference implementation this project has).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import hsc_inputs as hi  # noqa: E402

METRIC = "pixel-light evals/s latent vs n-sample spectral; decode GB/s; p50/p99 frame ms"
UNIT = "pixel-light evals/s"
WORKLOAD = "1920x1080 G-buffer + secondary bounce, n=81, k=6, 64 lights, 288 materials: latent frame (encode, fused shade + XYZ + sRGB8)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hsc", choices=["hsc", "reference"])
    ap.add_argument("--k", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true", help="skip the secondary rows (spectral, passes, decodes)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--tune-file", default="",
                    help="load tuned launch configurations from this file if it exists, save them there after the run")
    ap.add_argument("--serve-seconds", type=float, default=8.0,
                    help="length of the Poisson request stream served (0 = skip); the first quarter is warm-up")
    ap.add_argument("--serve-idle-us", type=float, default=-1.0,
                    help="host sleep of an idle scheduler pass in microseconds (default: the server's own)")
    ap.add_argument("--rows-only", default="",
                    help="comma list of secondary row groups to run: core, precision, small, batch, chains, "
                         "upsample, pathtrace, sweep, serve (default: all)")
    ap.add_argument("--step-launch", choices=("graph", "stream"), default="graph",
                    help="the timed frame step as a CUDA graph of its API calls (default) or as stream launches")
    ap.add_argument("--sweep-epochs", type=int, default=150,
                    help="epoch cap of the 700-variant codec sweep (0 = skip the sweep row)")
    return ap.parse_args()


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- oracle leg

def host_cpu_info():
    """Host CPUs seen by the bench: count, the affinity mask's size and the
    BLAS/OpenMP thread setting the oracle leg overrides (it runs one thread)."""
    try:
        aff = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        aff = None
    return {"cpu_count": os.cpu_count(), "affinity_cpus": aff, "machine": platform.machine(),
            "omp_num_threads_env": os.environ.get("OMP_NUM_THREADS"), "oracle_threads": 1}


def oracle_rate(seconds: float, k: int, threads: int = 1, max_rows: int = 1080):
    """Run the FP64 oracle's latent frame (encode, shading, decode to XYZ) on
    consecutive 32-row bands of the 1920x1080 frame (the last one clamped to
    the frame) in a child process with ``threads`` BLAS/OpenMP threads until
    ``seconds`` elapse or ``max_rows`` rows are done (at least one band);
    returns (evals per second, rows done, seconds)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    code = (
        "import sys, time, json, numpy as np\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import hsc_inputs as hi\n"
        "from oracle import cmf, shade\n"
        "f = hi.frame_config2()\n"
        f"E, D = hi.load_codec({k}, 81)\n"
        "T = cmf.cmf_weights(*f.grid)\n"
        "W = f.width\n"
        f"top = min({max_rows}, f.height)\n"
        "rows = 0; evals = 0\n"
        "t0 = time.perf_counter()\n"
        f"while rows < top and (rows == 0 or time.perf_counter() - t0 < {seconds}):\n"
        "    band = min(32, top - rows)\n"
        "    idx = np.arange(rows * W, (rows + band) * W)\n"
        "    g1 = hi.GBuffer(f.g1.normal[idx], f.g1.pos[idx], f.g1.mat[idx])\n"
        "    g2 = hi.GBuffer(f.g2.normal[idx], f.g2.pos[idx], f.g2.mat[idx])\n"
        "    sf = hi.Frame(len(idx), 1, f.grid, f.mat_spectra, f.light_spd, f.light_pos, f.light_intensity, g1, g2)\n"
        "    z = shade.shade_latent(sf, E.astype(np.float64))\n"
        "    xyz = shade.decode_xyz(z, D.astype(np.float64), T)\n"
        "    rows += band; evals += sf.evals\n"
        "dt = time.perf_counter() - t0\n"
        "print(json.dumps({'rows': rows, 'evals': evals, 'seconds': dt}))\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle leg failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["evals"] / d["seconds"], d["rows"], d["seconds"]


# --------------------------------------------------------------------------- GPU leg

def run_hsc(args, rank: int, world: int):
    import torch
    import torch.distributed as dist
    import paper_2602_18741_gb300 as hsc

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    ctx = hsc.Context(dev.index)
    hsc.hsc_set_autotune(ctx, True)   # tile shape / pixels per thread picked on the first (warm-up) call
    if args.tune_file and os.path.exists(args.tune_file):
        with open(args.tune_file) as fh:
            hsc.hsc_tune_load(ctx, fh.read())
    stream = torch.cuda.current_stream()
    k = args.k

    f = hi.frame_config2(seed=hi.MASTER_SEED + 2 + rank)
    E, D = hi.load_codec(k, 81)

    def t(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    g1 = hsc.GBuffer(t(f.g1.normal), t(f.g1.pos), t(f.g1.mat))
    g2 = hsc.GBuffer(t(f.g2.normal), t(f.g2.pos), t(f.g2.mat))
    lights = hsc.Lights(t(f.light_pos), t(f.light_intensity))
    mats, spd = t(f.mat_spectra), t(f.light_spd)
    Ed, Dd = t(E), t(D)
    P = f.pixels
    T = torch.empty(3, 81, device=dev)
    hsc.hsc_cmf_weights(ctx, 81, f.grid[0], f.grid[1], T)
    M = torch.empty(3, k, device=dev)
    hsc.hsc_fold_xyz(ctx, T, Dd, M)
    zm = torch.empty(mats.shape[0], k, device=dev)
    zl = torch.empty(spd.shape[0], k, device=dev)
    lat = torch.empty(P, k, device=dev)
    xyz = torch.empty(P, 3, device=dev)
    rgb = torch.empty(P, 3, device=dev, dtype=torch.uint8)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    flush_read = torch.ones(256 * 1024 * 1024 // 4, device=dev)
    flush_sink = torch.empty((), device=dev)

    def l2_flush():
        # write 256 MB (evicts everything a kernel could reuse), then read
        # another 256 MB, so that the write's dirty lines are written back
        # here and not inside the next timed region
        flush.zero_()
        torch.sum(flush_read, dim=0, out=flush_sink)
    evals = f.evals
    gpu_launches_per_step = 2

    def frame(ev=None):
        hsc.hsc_encode_assets(ctx, Ed, mats, zm, spd, zl)
        if ev is not None:
            ev[0].record(stream)
        hsc.hsc_shade_latent(ctx, g1, g2, zm, lights, zl, hsc.HSC_FUSED, lat, xyz_out=xyz, M_xyz=M, srgb8_out=rgb)
        if ev is not None:
            ev[1].record(stream)

    def frame_on_current_stream(ev):
        # the same calls on the capturing stream (the binding launches on torch's current stream)
        cur = torch.cuda.current_stream()
        hsc.hsc_encode_assets(ctx, Ed, mats, zm, spd, zl)
        ev[0].record(cur)
        hsc.hsc_shade_latent(ctx, g1, g2, zm, lights, zl, hsc.HSC_FUSED, lat, xyz_out=xyz, M_xyz=M, srgb8_out=rgb)
        ev[1].record(cur)

    def timed(fn, steps, warmup, inner_events=False):
        """Per-iteration device times (ms) with an L2 flush before each."""
        for _ in range(warmup):
            l2_flush()
            fn(None) if inner_events else fn()
        torch.cuda.synchronize()
        outer, inner = [], []
        evs = []
        for _ in range(steps):
            l2_flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ie = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) if inner_events else None
            a.record(stream)
            fn(ie) if inner_events else fn()
            b.record(stream)
            evs.append((a, b, ie))
        torch.cuda.synchronize()
        for a, b, ie in evs:
            outer.append(a.elapsed_time(b))
            if ie is not None:
                inner.append(ie[0].elapsed_time(ie[1]))
        return outer, inner

    # ---------------- main timed region
    for _ in range(args.warmup):
        l2_flush()
        frame()
    torch.cuda.synchronize()
    hsc.hsc_sync(ctx)
    # The frame's two API calls (tuned by the eager warm-up) are captured once
    # in a CUDA graph and replayed every step: the same two kernels without
    # the stream-launch gaps.  The shading launch is bracketed by timing
    # events recorded inside the graph; the L2 flush and the step's own events
    # stay outside it.
    graph = make_frame_graph(torch, frame_on_current_stream, dev) if args.step_launch == "graph" else None
    step_launch = "CUDA graph of the frame's API calls, replayed per step" if graph else "stream launches"
    if graph is not None:
        for _ in range(args.warmup):
            l2_flush()
            graph[0].replay()
        torch.cuda.synchronize()
    clocks = ClockSampler(dev.index) if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    wall0 = time.perf_counter()
    if graph is not None:
        per_step, shade_ms = timed_graph(graph, args.steps, l2_flush, stream)
    else:
        per_step, shade_ms = timed(frame, args.steps, 0, inner_events=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    hsc.hsc_sync(ctx)
    if graph is not None:
        # the step's graph is freed before the secondary rows
        graph[0].reset()
        graph = None
        torch.cuda.synchronize()
    total_ms = max_over_ranks(sum(per_step), world, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(evals * args.steps, world, total_ms)

    result = None
    if rank == 0:
        rows = {}
        clk_box = {}

        def stop_clocks():
            # the nvidia-smi sampler queries the driver every 100 ms; it is
            # stopped before the serving rows, whose latencies it would disturb
            if clocks is not None and "clk" not in clk_box:
                clk_box["clk"] = clocks.stop()

        if not args.no_rows:
            rows = secondary_rows(args, hsc, ctx, f, dev, stream, g1, g2, lights, mats, spd, T, Dd, zm, zl, lat,
                                  timed, flush, before_serve=stop_clocks)
        stop_clocks()
        clk = clk_box.get("clk")
        # roofline of the dominant kernel: the fused shading launch
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_mhz = _peak_sm_mhz()
        ops_per_eval = 13 + k          # 12 FP32 geometry ops + 1 MUFU rsqrt + k FMAs
        ops = evals * ops_per_eval
        shade_avg_s = statistics.mean(shade_ms) * 1e-3
        achieved = ops / shade_avg_s / 1e12
        peak = sm_count * 128 * peak_mhz * 1e6 / 1e12
        roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "Tops/s",
                    "frac": round(achieved / peak, 4), "traffic": _traffic_from_profile(),
                    "kernel": "shade_codes_kernel<6,PPT,true,...,RGB> (fused latent shade + XYZ + sRGB8)",
                    "ops_per_eval": ops_per_eval, "peak_basis": f"{sm_count} SMs x 128 FP32 lanes x {peak_mhz:.0f} MHz"}
        probe = fp32_probe(hsc, ctx, dev, stream)
        probe["frac_of_burst"] = round(achieved / probe["burst"], 4)
        roofline["fp32_probe"] = probe
        e2e = e2e_leg(args, hsc, ctx, f, dev, stream, Ed, M, evals)
        tune = [ln for ln in hsc.hsc_tune_report(ctx).splitlines() if ln.strip()]
        if args.tune_file:
            with open(args.tune_file, "w") as fh:
                fh.write(hsc.hsc_tune_save(ctx))
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            rate, nrows, secs = oracle_rate(args.cpu_seconds, k, threads=1)
            cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"FP64 NumPy oracle latent frame (encode, shading, XYZ decode) on the first {nrows} rows "
                             f"of the same 1920x1080 frame ({secs:.1f} s, one thread)",
                   "host": host_cpu_info()}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded G-buffers, spectra, lights)",
            "config": {"workload": WORKLOAD, "pixels": f.pixels, "lights": f.lights, "k": k, "n": 81,
                       "evals_per_step": evals, "l2": "flushed before every timed step (256 MB write, then 256 MB read so its writebacks fall outside the timed region)",
                       "launch": step_launch, "parallelism": f"replicas x{world}"},
            "frame_ms": {"p50": _pct(per_step, 50), "p99": _pct(per_step, 99), "min": min(per_step)},
            "gpu_launches": gpu_launches_per_step * args.steps,
            "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk, "rows": rows, "autotune": tune,
            "wall_s_timed_region": round(wall, 4),
        }
    ctx.close()
    return result


def fp32_probe(hsc, ctx, dev, stream, iters: int = 2048, sustain_s: float = 1.0):
    """Measured FP32 FMA issue rate (T lane-ops/s) of the library's
    register-only FFMA probe: best of 10 single launches (burst) and the mean
    over back-to-back launches for about `sustain_s` seconds (sustained),
    CUDA events on the launching stream."""
    import torch
    sink = torch.empty(8 * torch.cuda.get_device_properties(dev).multi_processor_count * 256, device=dev)
    for _ in range(3):
        ops = hsc.hsc_fp32_peak_probe(ctx, sink, iters, stream=stream)
    torch.cuda.synchronize()
    best = math.inf
    for _ in range(10):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hsc.hsc_fp32_peak_probe(ctx, sink, iters, stream=stream)
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b) * 1e-3)
    reps = max(int(sustain_s / best), 1)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        hsc.hsc_fp32_peak_probe(ctx, sink, iters, stream=stream)
    b.record(stream)
    b.synchronize()
    hsc.hsc_sync(ctx)
    sustained = ops * reps / (a.elapsed_time(b) * 1e-3)
    return {"burst": round(ops / best / 1e12, 3), "sustained": round(sustained / 1e12, 3), "unit": "T lane-ops/s",
            "how": f"hsc_fp32_peak_probe: 8 CTAs x 256 threads per SM, 32 register-only FFMAs x {iters} per thread; "
                   f"best of 10 launches and {reps} launches back to back"}


def max_over_ranks(value: float, world: int, device) -> float:
    """The slowest rank's value (the job's time is set by its slowest GPU)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, total_ms_max: float) -> float:
    """Units all ranks processed per second of the slowest rank."""
    return world * units_per_rank / (total_ms_max * 1e-3)


def _pct(xs, q):
    v = sorted(xs)
    return v[max(int(math.ceil(q / 100.0 * len(v))) - 1, 0)]


def _peak_sm_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh).get("sm_max_mhz", 2070.0))
    except (OSError, ValueError):
        return 2070.0


# Sources whose compiled code the fused shading launch runs; the committed
# DRAM-traffic figure is used only while their hash matches the one recorded
# with it (any change to the kernel makes the figure stale).
TRAFFIC_SOURCES = ("paper_2602_18741_gb300/csrc/shade_latent_kernel.cuh",
                   "paper_2602_18741_gb300/csrc/shade_latent.cuh",
                   "paper_2602_18741_gb300/csrc/common.cuh",
                   "paper_2602_18741_gb300/csrc/shade_latent_k6.cu")


def make_frame_graph(torch, frame_fn, dev):
    """Captures frame_fn(events) once in a CUDA graph on a side stream.
    Returns (graph, (ev_before_shade, ev_after_shade)), the events recorded
    inside the graph as timing nodes, or None where this PyTorch cannot
    record timing events inside a graph (the step then launches on the
    stream)."""
    try:
        evs = (torch.cuda.Event(enable_timing=True, external=True),
               torch.cuda.Event(enable_timing=True, external=True))
    except TypeError:
        return None
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            frame_fn(evs)
    torch.cuda.synchronize(dev)
    return g, evs


def timed_graph(graph, steps, l2_flush, stream):
    """Per-step device times (ms) of graph replays with an L2 flush before
    each, and the shading launch's time from the events inside the graph
    (read after each replay, before the next one records them again)."""
    import torch
    g, (e0, e1) = graph
    outer, inner = [], []
    for _ in range(steps):
        l2_flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.replay()
        b.record(stream)
        b.synchronize()
        outer.append(a.elapsed_time(b))
        inner.append(e0.elapsed_time(e1))
    return outer, inner


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(rel.encode() + b"\0" + fh.read())
    return h.hexdigest()


def _traffic_from_profile():
    """DRAM bytes (read + write) per launch of the fused shading kernel from
    the committed ncu summary profiles/shade_codes_fused_1080p.json, or None
    when the kernel sources changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "shade_codes_fused_1080p.json")
    try:
        with open(p) as fh:
            rec = json.load(fh)
        if rec.get("source_sha256") != kernel_source_hash():
            return None
        return rec.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        return None


def secondary_rows(args, hsc, ctx, f, dev, stream, g1, g2, lights, mats, spd, T, Dd, zm, zl, lat, timed, flush,
                   before_serve=None):
    import torch
    if "core" not in wanted_rows(args):
        return group_rows(args, hsc, ctx, dev, timed, before_serve)
    P = f.pixels
    evals = f.evals
    K, W = args.steps, args.warmup
    rows = {}
    xyz_s = torch.empty(P, 3, device=dev)
    xyz_l = torch.empty(P, 3, device=dev)

    def spectral():
        hsc.hsc_shade_spectral(ctx, g1, g2, mats, lights, spd, T, xyz_s)

    ms, _ = timed(spectral, K, W)
    spec_ms = statistics.mean(ms)
    rows["spectral_n81"] = {"ms": spec_ms, "evals_per_s": evals / (spec_ms * 1e-3),
                            "ops_per_eval": 13 + 81}

    Mk = _M(hsc, ctx, T, Dd)

    def fused():
        hsc.hsc_shade_latent(ctx, g1, g2, zm, lights, zl, hsc.HSC_FUSED, lat, xyz_out=xyz_l, M_xyz=Mk)

    ms, _ = timed(fused, K, W)
    fused_ms = statistics.mean(ms)
    rows[f"latent_fused_k{args.k}_xyz"] = {"ms": fused_ms, "evals_per_s": evals / (fused_ms * 1e-3),
                                            "ops_per_eval": 13 + args.k}
    rows["speedup_latent_fused_vs_spectral"] = spec_ms / fused_ms

    lat_p = torch.empty_like(lat)
    xyz_p = torch.empty(P, 3, device=dev)
    hsc.hsc_reserve(ctx, hsc.hsc_shade_latent_scratch_bytes(P, args.k, hsc.HSC_PASSES, hsc.HSC_F32))

    def passes():
        hsc.hsc_shade_latent(ctx, g1, g2, zm, lights, zl, hsc.HSC_PASSES, lat_p, xyz_out=xyz_p, M_xyz=Mk)

    ms, _ = timed(passes, K, W)
    pms = statistics.mean(ms)
    rows[f"latent_passes_k{args.k}_xyz"] = {"ms": pms, "evals_per_s": evals / (pms * 1e-3),
                                             "bit_identical_to_fused": bool(torch.equal(lat_p, lat))}
    rows["speedup_latent_passes_vs_spectral"] = spec_ms / pms

    # k = 9
    E9, D9 = hi.load_codec(9, 81)
    E9d, D9d = torch.from_numpy(E9).to(dev), torch.from_numpy(D9).to(dev)
    zm9 = torch.empty(mats.shape[0], 9, device=dev)
    zl9 = torch.empty(spd.shape[0], 9, device=dev)
    hsc.hsc_encode(ctx, E9d, mats, zm9)
    hsc.hsc_encode(ctx, E9d, spd, zl9)
    M9 = torch.empty(3, 9, device=dev)
    hsc.hsc_fold_xyz(ctx, T, D9d, M9)
    lat9 = torch.empty(P, 9, device=dev)

    def fused9():
        hsc.hsc_shade_latent(ctx, g1, g2, zm9, lights, zl9, hsc.HSC_FUSED, lat9, xyz_out=xyz_l, M_xyz=M9)

    ms, _ = timed(fused9, K, W)
    f9 = statistics.mean(ms)
    rows["latent_fused_k9_xyz"] = {"ms": f9, "evals_per_s": evals / (f9 * 1e-3), "ops_per_eval": 22}
    rows["speedup_latent_fused_k9_vs_spectral"] = spec_ms / f9

    # k = 9 as three RGB passes and their reassembly (Fig. 2b)
    lat9p = torch.empty(P, 9, device=dev)
    xyz9p = torch.empty(P, 3, device=dev)
    hsc.hsc_reserve(ctx, hsc.hsc_shade_latent_scratch_bytes(P, 9, hsc.HSC_PASSES, hsc.HSC_F32))

    def passes9():
        hsc.hsc_shade_latent(ctx, g1, g2, zm9, lights, zl9, hsc.HSC_PASSES, lat9p, xyz_out=xyz9p, M_xyz=M9)

    ms, _ = timed(passes9, K, W)
    p9 = statistics.mean(ms)
    rows["latent_passes_k9_xyz"] = {"ms": p9, "evals_per_s": evals / (p9 * 1e-3),
                                    "bit_identical_to_fused": bool(torch.equal(lat9p, lat9))}
    rows["speedup_latent_passes_k9_vs_spectral"] = spec_ms / p9
    del lat9p, xyz9p

    # decode of the k = 9 FP32 latent to spectra (tensor cores, three-part split)
    spec9 = torch.empty(P, 81, device=dev)

    def dec9():
        hsc.hsc_decode_spectra(ctx, lat9, D9d, spec9)

    ms, _ = timed(dec9, K, W)
    m9 = statistics.mean(ms)
    b9 = P * (9 * 4 + 81 * 4)
    rows["decode_spectra_f32_k9"] = {"ms": m9, "GB_per_s": b9 / (m9 * 1e-3) / 1e9, "Mpx_per_s": P / (m9 * 1e-3) / 1e6,
                                     "bytes": b9}
    del spec9

    # decode to spectra (FP32 CUDA cores): P x 81 float32 out
    spec_out = torch.empty(P, 81, device=dev)

    def dec():
        hsc.hsc_decode_spectra(ctx, lat, Dd, spec_out)

    ms, _ = timed(dec, K, W)
    dms = statistics.mean(ms)
    dbytes = P * (args.k * 4 + 81 * 4)
    rows["decode_spectra_f32"] = {"ms": dms, "GB_per_s": dbytes / (dms * 1e-3) / 1e9,
                                  "Mpx_per_s": P / (dms * 1e-3) / 1e6, "bytes": dbytes}

    # tensor-core decode (tcgen05, BF16 operands, FP32 accumulation) from a
    # bf16 latent and from an fp8 latent with per-channel scales, at 1920x1080
    # and at 3840x2160 (four copies of the frame's latent image)
    lat_bf = lat.to(torch.bfloat16)
    codes = torch.empty(P, args.k, device=dev, dtype=torch.uint8)
    scales = torch.empty(args.k, device=dev)
    hsc.hsc_quantize_fp8(ctx, lat, codes, scales)
    for tag, src, sc, esz in (("bf16", lat_bf, None, 2), ("fp8", codes, scales, 1)):
        def dtc(src=src, sc=sc):
            hsc.hsc_decode_spectra(ctx, src, Dd, spec_out, scales=sc)
        ms, _ = timed(dtc, K, W)
        m_ = statistics.mean(ms)
        b_ = P * (args.k * esz + 81 * 4)
        rows[f"decode_spectra_tc_{tag}_1080p"] = {"ms": m_, "GB_per_s": b_ / (m_ * 1e-3) / 1e9,
                                                  "Mpx_per_s": P / (m_ * 1e-3) / 1e6, "bytes": b_}
    del spec_out
    P4 = 4 * P
    out4 = torch.empty(P4, 81, device=dev)
    for tag, src, sc, esz in (("bf16", lat_bf.repeat(4, 1), None, 2), ("fp8", codes.repeat(4, 1), scales, 1)):
        def dtc4(src=src, sc=sc):
            hsc.hsc_decode_spectra(ctx, src, Dd, out4, scales=sc)
        ms, _ = timed(dtc4, K, W)
        m_ = statistics.mean(ms)
        b_ = P4 * (args.k * esz + 81 * 4)
        rows[f"decode_spectra_tc_{tag}_4k"] = {"ms": m_, "GB_per_s": b_ / (m_ * 1e-3) / 1e9,
                                               "Mpx_per_s": P4 / (m_ * 1e-3) / 1e6, "bytes": b_}
    # context for the decode rows (write-dominated streams): a write-only
    # fill (torch) of the same output sizes
    fill = {}
    for tag, buf in (("1080p", out4[:P]), ("4k", out4)):
        ms, _ = timed(lambda buf=buf: buf.fill_(0.0), K, W)
        m_ = statistics.mean(ms)
        fill[f"GB_per_s_{tag}"] = buf.numel() * 4 / (m_ * 1e-3) / 1e9
    fill["note"] = "torch fill_ of a P x 81 float32 buffer: write-only bandwidth, context for the decode rows"
    rows["hbm_write_only_fill"] = fill
    del out4

    xyz_only = torch.empty(P, 3, device=dev)

    def decx():
        hsc.hsc_decode_xyz(ctx, lat, Mk, xyz_only)

    ms, _ = timed(decx, K, W)
    xms = statistics.mean(ms)
    xbytes = P * (args.k * 4 + 12)
    rows["decode_xyz_f32"] = {"ms": xms, "GB_per_s": xbytes / (xms * 1e-3) / 1e9, "bytes": xbytes}

    # Delta E 2000 of the latent render against the spectral one
    st = torch.zeros(8, device=dev, dtype=torch.float64)
    fused()
    spectral()

    def de():
        hsc.hsc_delta_e(ctx, xyz_l, xyz_s, T, st)

    fused()
    ms, _ = timed(de, K, W)
    hsc.hsc_sync(ctx)
    s = st.cpu().numpy()
    rows["delta_e_latent_vs_spectral"] = {"ms": statistics.mean(ms), "de2000_mean": float(s[0]),
                                          "de2000_p95": float(s[1]), "de94_mean": float(s[2]),
                                          "de76_mean": float(s[3])}
    hsc.hsc_sync(ctx)
    rows.update(group_rows(args, hsc, ctx, dev, timed, before_serve))
    return rows


def precision_rows(args, hsc, ctx, dev, timed):
    """The 3840x2160 frame (n = 81, 64 lights, primary + secondary, k = 6
    and 9) shaded with the codes stored in FP32, BF16 and FP16 (fused launch
    with the XYZ epilogue), and with BF16 codes into an FP8 E4M3 latent image
    with per-channel scales (fused launch writing FP32 to scratch with the
    channel maxima, then the quantisation pass), followed by the XYZ decode of
    the FP8 image.  Accuracy beside each row: relative XYZ error and Delta E
    2000 (mean, p95) against the FP32 render of the same frame, which matches
    the FP64 oracle to ~1e-6 (the oracle itself is compared in the precision
    tests)."""
    import torch
    f = hi.frame_config3()
    P = f.pixels
    evals = f.evals

    def t(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    g1 = hsc.GBuffer(t(f.g1.normal), t(f.g1.pos), t(f.g1.mat))
    g2 = hsc.GBuffer(t(f.g2.normal), t(f.g2.pos), t(f.g2.mat))
    lights = hsc.Lights(t(f.light_pos), t(f.light_intensity))
    mats, spd = t(f.mat_spectra), t(f.light_spd)
    T = torch.empty(3, 81, device=dev)
    hsc.hsc_cmf_weights(ctx, 81, f.grid[0], f.grid[1], T)
    out = {"frame": "3840x2160, n = 81, 64 lights, primary + secondary", "evals": evals}
    st = torch.zeros(8, device=dev, dtype=torch.float64)
    for k in (6, 9):
        E, D = hi.load_codec(k, 81)
        Ed, Dd = t(E), t(D)
        M = _M(hsc, ctx, T, Dd)
        hsc.hsc_reserve(ctx, hsc.hsc_shade_latent_scratch_bytes(P, k, hsc.HSC_FUSED, hsc.HSC_FP8_E4M3))
        xyz_ref = torch.empty(P, 3, device=dev)
        xyz = torch.empty(P, 3, device=dev)
        lat = torch.empty(P, k, device=dev)
        codes = torch.empty(P, k, device=dev, dtype=torch.uint8)
        scales = torch.empty(k, device=dev)
        rows_k = {}
        for name, dt in (("f32_codes", torch.float32), ("bf16_codes", torch.bfloat16), ("f16_codes", torch.float16),
                         ("bf16_codes_fp8_latent", torch.bfloat16)):
            zm = torch.empty(mats.shape[0], k, device=dev, dtype=dt)
            zl = torch.empty(spd.shape[0], k, device=dev, dtype=dt)
            hsc.hsc_encode(ctx, Ed, mats, zm)
            hsc.hsc_encode(ctx, Ed, spd, zl)
            if name.endswith("fp8_latent"):
                def shade():
                    hsc.hsc_shade_latent(ctx, g1, g2, zm, lights, zl, hsc.HSC_FUSED, codes, latent_scales=scales)

                def dec():
                    hsc.hsc_decode_xyz(ctx, codes, M, xyz, scales=scales)
            else:
                def shade():
                    hsc.hsc_shade_latent(ctx, g1, g2, zm, lights, zl, hsc.HSC_FUSED, lat,
                                         xyz_out=(xyz_ref if name == "f32_codes" else xyz), M_xyz=M)
                dec = None
            ms, _ = timed(shade, args.steps, args.warmup)
            m_ = statistics.mean(ms)
            row = {"ms": m_, "evals_per_s": evals / (m_ * 1e-3), "frac_alu": evals * (13 + k) / (m_ * 1e-3) /
                   (torch.cuda.get_device_properties(dev).multi_processor_count * 128 * _peak_sm_mhz() * 1e6)}
            if dec is not None:
                ms, _ = timed(dec, args.steps, args.warmup)
                row["xyz_decode_ms"] = statistics.mean(ms)
                row["ms_with_decode"] = m_ + row["xyz_decode_ms"]
            if name != "f32_codes":
                hsc.hsc_delta_e(ctx, xyz, xyz_ref, T, st)
                hsc.hsc_sync(ctx)
                s_ = st.cpu().numpy()
                ref = xyz_ref.abs().amax(dim=1)
                den = torch.clamp(ref, min=1e-3 * float(ref.max()))
                row["rel_xyz_vs_f32"] = float(((xyz - xyz_ref).abs().amax(dim=1) / den).max())
                row["de2000_vs_f32_mean"] = float(s_[0])
                row["de2000_vs_f32_p95"] = float(s_[1])
            rows_k[name] = row
        out[f"k{k}"] = rows_k
        del xyz_ref, xyz, lat, codes
    return {"precision_3840x2160": out}


def wanted_rows(args):
    """The secondary row groups to run (all unless --rows-only names some)."""
    groups = ("core", "precision", "small", "batch", "chains", "upsample", "pathtrace", "sweep", "serve")
    if not args.rows_only:
        return set(groups)
    want = {g.strip() for g in args.rows_only.split(",") if g.strip()}
    unknown = want - set(groups)
    if unknown:
        raise SystemExit(f"--rows-only: unknown groups {sorted(unknown)}; known: {', '.join(groups)}")
    return want


def group_rows(args, hsc, ctx, dev, timed, before_serve=None):
    want = wanted_rows(args)
    rows = {}
    if "precision" in want:
        rows.update(precision_rows(args, hsc, ctx, dev, timed))
    if "small" in want:
        rows.update(small_frame_rows(args, hsc, ctx, dev))
    if "batch" in want:
        rows.update(batch_rows(args, hsc, ctx, dev, timed))
    if "chains" in want:
        rows.update(chain_rows(args, hsc, ctx, dev, timed))
    if "upsample" in want:
        rows.update(upsample_rows(args, hsc, ctx, dev, timed))
    if "pathtrace" in want:
        rows.update(pathtrace_rows(args, hsc, ctx, dev, timed))
    if "sweep" in want and args.sweep_epochs > 0:
        rows.update(codec_sweep_rows(args, hsc, ctx, dev))
    if "serve" in want and args.serve_seconds > 0:
        if before_serve is not None:
            before_serve()
        rows.update(serve_rows(args, hsc, ctx, dev))
    return rows


def small_frame_rows(args, hsc, ctx, dev, replays: int = 20, frames_per_graph: int = 10):
    """The 256x256 frame (n = 31, k = 6, 4 lights, direct only): launch
    bound, so the latent frame (one encode launch for materials and lights
    + fused shade with XYZ), the
    latent shade alone (assets already encoded), the latent frame with the
    encode inside the shading launch (hsc_shade_latent_assets) and the
    spectral frame are each captured in a CUDA graph of `frames_per_graph`
    frames, replayed back to back (the host's cost per replay is spread over
    the frames, so the device's time per frame is what is measured);
    microseconds per frame (inputs of ~4 MB stay in L2)."""
    import torch
    f = hi.frame_config1()
    E, D = hi.load_codec(6, 31)

    def t(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    g1 = hsc.GBuffer(t(f.g1.normal), t(f.g1.pos), t(f.g1.mat))
    lights = hsc.Lights(t(f.light_pos), t(f.light_intensity))
    mats, spd, Ed, Dd = t(f.mat_spectra), t(f.light_spd), t(E), t(D)
    T = torch.empty(3, 31, device=dev)
    hsc.hsc_cmf_weights(ctx, 31, f.grid[0], f.grid[1], T)
    M = torch.empty(3, 6, device=dev)
    hsc.hsc_fold_xyz(ctx, T, Dd, M)
    zm = torch.empty(mats.shape[0], 6, device=dev)
    zl = torch.empty(spd.shape[0], 6, device=dev)
    lat = torch.empty(f.pixels, 6, device=dev)
    xyz_l = torch.empty(f.pixels, 3, device=dev)
    xyz_s = torch.empty(f.pixels, 3, device=dev)

    def latent():
        hsc.hsc_encode_assets(ctx, Ed, mats, zm, spd, zl)
        hsc.hsc_shade_latent(ctx, g1, None, zm, lights, zl, hsc.HSC_FUSED, lat, xyz_out=xyz_l, M_xyz=M)

    def latent_shade():
        # assets are encoded once per scene (Fig. 2b): the frame is one launch
        hsc.hsc_shade_latent(ctx, g1, None, zm, lights, zl, hsc.HSC_FUSED, lat, xyz_out=xyz_l, M_xyz=M)

    def latent_assets():
        # the assets encoded again every frame, inside the shading launch
        hsc.hsc_shade_latent_assets(ctx, g1, None, Ed, mats, lights, spd, lat, xyz_out=xyz_l, M_xyz=M)

    def spectral():
        hsc.hsc_shade_spectral(ctx, g1, None, mats, lights, spd, T, xyz_s)

    out = {}
    side = torch.cuda.Stream(dev)
    for name, fn in (("latent_k6", latent), ("latent_k6_shade_only", latent_shade),
                     ("latent_k6_encode_in_shading_launch", latent_assets), ("spectral_n31", spectral)):
        for _ in range(3):          # eager warm-up (and the autotuner's first call)
            fn()
        torch.cuda.synchronize(dev)
        hsc.hsc_sync(ctx)
        g = torch.cuda.CUDAGraph()
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                for _ in range(frames_per_graph):
                    fn()
        torch.cuda.synchronize(dev)
        for _ in range(3):
            g.replay()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(replays):
            g.replay()
        b.record()
        b.synchronize()
        hsc.hsc_sync(ctx)
        us = a.elapsed_time(b) * 1e3 / (replays * frames_per_graph)
        out[name] = {"us_per_frame": us, "evals_per_s": f.evals / (us * 1e-6)}
    return {"small_frame_256x256_graph": {"frame": "256x256, n = 31, 4 lights, direct only", "replays": replays,
                                          "frames_per_graph": frames_per_graph,
                                          "evals": f.evals, **out,
                                          "speedup_latent_vs_spectral":
                                              out["spectral_n31"]["us_per_frame"] / out["latent_k6"]["us_per_frame"],
                                          "speedup_latent_shade_only_vs_spectral":
                                              out["spectral_n31"]["us_per_frame"]
                                              / out["latent_k6_shade_only"]["us_per_frame"],
                                          "speedup_latent_encode_in_shading_launch_vs_spectral":
                                              out["spectral_n31"]["us_per_frame"]
                                              / out["latent_k6_encode_in_shading_launch"]["us_per_frame"]}}


def upsample_rows(args, hsc, ctx, dev, timed):
    """RGB-to-latent upsampling network (3 -> 128 -> 128 -> 6, SiLU) over a
    3840x2160 texture of seeded uniform RGB values, fitted k = 6 weights."""
    import torch
    w = hi.load_upsampler(6, 81)
    W = [torch.from_numpy(w[n]).to(dev) for n in ("W1", "b1", "W2", "b2", "W3", "b3")]
    P = 3840 * 2160
    gen = torch.Generator(device=dev)
    gen.manual_seed(hi.MASTER_SEED + 7)
    rgb = torch.rand(P, 3, device=dev, generator=gen)
    z = torch.empty(P, 6, device=dev)

    def run():
        hsc.hsc_upsample_rgb(ctx, rgb, *W, z)

    ms, _ = timed(run, args.steps, args.warmup)
    m = statistics.mean(ms)
    flops = P * 2 * (3 * 128 + 128 * 128 + 128 * 6)          # algorithmic
    mma_flops = P * 2 * (16 * 128 + 144 * 128 + 144 * 16)    # as issued (K and N padded, bias K step)
    del rgb, z
    # the epilogue's bound: one hardware tanh per hidden value (2 x 128 per
    # pixel) at the MUFU rate of the library's FP32 tanh probe (best of 10);
    # the packed f16x2 form's rate per result beside it (the same rate: it
    # brings no speed-up, so the kernel keeps the FP32 form)
    sink = torch.empty(8 * torch.cuda.get_device_properties(dev).multi_processor_count * 256, device=dev)

    def probe_rate(packed):
        best = 0.0
        for _ in range(11):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ops = hsc.hsc_tanh_peak_probe(ctx, sink, 4096, packed=packed)
            b.record()
            b.synchronize()
            best = max(best, ops / (a.elapsed_time(b) * 1e-3))
        return best

    rate_f16x2, rate_f32 = probe_rate(True), probe_rate(False)
    hsc.hsc_sync(ctx)
    mufu_ms = 2 * 128 * P / rate_f32 * 1e3
    bf16_peak = _measured_peak("bf16_tflops", 1900.0)   # FP16 dense rate = BF16's
    return {"upsample_rgb_4k": {"ms": m, "Mpx_per_s": P / (m * 1e-3) / 1e6,
                                "operands": "f16, FP32 accumulation and SiLU",
                                "TFLOP_per_s": flops / (m * 1e-3) / 1e12,
                                "tensor_TFLOP_per_s_issued": mma_flops / (m * 1e-3) / 1e12,
                                "frac_of_f16_tensor_peak": flops / (m * 1e-3) / 1e12 / bf16_peak,
                                "tanh_f16x2_probe_G_results_per_s": rate_f16x2 / 1e9,
                                "tanh_f32_probe_G_per_s": rate_f32 / 1e9,
                                "mufu_bound_ms": mufu_ms,
                                "frac_of_mufu_bound": mufu_ms / m}}


def _measured_peak(key: str, fallback: float) -> float:
    """A peak from MEASURED_PEAKS.json (written on the GPU machine before the
    run), else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key])
    except (OSError, ValueError, KeyError):
        return fallback


def pathtrace_rows(args, hsc, ctx, dev, timed):
    """Path tracing of the Cornell-box stand-in at 1920x1080, 16 samples per
    pixel, up to 3 reflections: the same paths with n = 81 spectral channels
    and with the k = 6 codes; Delta E 2000 of the latent render against the
    spectral one."""
    import torch
    W, H, spp, depth = 1920, 1080, 16, 3
    sc = hi.cornell_scene(W, H)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    n = sc.grid[2]
    T = torch.empty(3, n, device=dev)
    hsc.hsc_cmf_weights(ctx, n, sc.grid[0], sc.grid[1], T)
    E, D = hi.load_codec(6, n)
    Ed, Dd = t(E), t(D)
    zr = torch.empty(sc.refl.shape[0], 6, device=dev)
    ze = torch.empty(1, 6, device=dev)
    hsc.hsc_encode(ctx, Ed, t(sc.refl), zr)
    hsc.hsc_encode(ctx, Ed, t(sc.emit[None, :]), ze)
    M = torch.empty(3, 6, device=dev)
    hsc.hsc_fold_xyz(ctx, T, Dd, M)
    geo = (t(sc.quads), t(sc.spheres), t(sc.cam))
    xs = torch.empty(W * H, 3, device=dev)
    xl = torch.empty(W * H, 3, device=dev)
    z = torch.empty(W * H, 6, device=dev)
    out = {}
    mats_s, emit_s, emit_z = t(sc.refl), t(sc.emit), ze[0].contiguous()
    runs = {"spectral_n81": lambda: hsc.hsc_path_trace(ctx, *geo, W, H, spp, depth, 7, mats_s, emit_s, T, xs),
            "latent_k6": lambda: hsc.hsc_path_trace(ctx, *geo, W, H, spp, depth, 7, zr, emit_z, M, xl, z)}
    paths = W * H * spp
    for name, fn in runs.items():
        ms, _ = timed(fn, max(3, args.steps // 2), args.warmup)
        m = statistics.mean(ms)
        out[f"pathtrace_{name}"] = {"ms": m, "Mpaths_per_s": paths / (m * 1e-3) / 1e6, "spp": spp, "depth": depth}
    out["speedup_pathtrace_latent_vs_spectral"] = out["pathtrace_spectral_n81"]["ms"] / out["pathtrace_latent_k6"]["ms"]
    st = torch.zeros(8, device=dev, dtype=torch.float64)
    hsc.hsc_delta_e(ctx, xl, xs, T, st)
    hsc.hsc_sync(ctx)
    s = st.cpu().numpy()
    out["pathtrace_delta_e_latent_vs_spectral"] = {"de2000_mean": float(s[0]), "de2000_p95": float(s[1])}
    return out


def codec_sweep_rows(args, hsc, ctx, dev):
    """The hyper-parameter sweep of the codec fit (Sec. 4.5) on the GPU: the
    700 loss-weight variants of the k = 6, n = 81 codec, softplus
    parameterisation, Adam (lr 1e-3), mini-batches of 128 of the 4096 training
    pairs (32 per epoch), at most 150 epochs with early stopping (patience 15)
    on a 256-pair validation batch; then every kept codec is scored by 500
    depth-3 chains (mean CIE94 over the depths) and the best is selected.  The
    projected-gradient codec used by the shading rows is scored on the same
    chains beside it."""
    import torch
    from paper_2602_18741_gb300 import sweep
    k, g, epochs, patience = 6, hi.GRID_81, args.sweep_epochs, 15
    ts = hi.training_set(g)
    n = g[2]
    sched = hi.sweep_schedule(ts, epochs=epochs, batch=128, val_pairs=256)
    t = lambda a, dt=np.float32: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)
    T = torch.empty(3, n, device=dev)
    hsc.hsc_cmf_weights(ctx, n, g[0], g[1], T)
    W = hi.sweep_weight_grid()
    V = W.shape[0]
    E0, D0 = sweep.band_init_raw(k, n)
    Et0 = t(np.broadcast_to(E0, (V, k, n)))
    Dt0 = t(np.broadcast_to(D0, (V, n, k)))
    R, L, Wd = t(ts.R), t(ts.L), t(W)
    train = (t(sched.train_r, np.int32), t(sched.train_l, np.int32), t(sched.train_s))
    val = (t(sched.val_r, np.int32), t(sched.val_l, np.int32), t(sched.val_s))
    res = sweep.fit_variants(hsc, ctx, R, L, T, Wd, train, val, Et0, Dt0, epochs=epochs, patience=patience, lr=1e-3)
    held = hi.training_set(g, seed=hi.MASTER_SEED + 200)
    rng = np.random.default_rng(hi.MASTER_SEED + 10)
    C = 500
    cl = t(rng.integers(0, held.L.shape[0], C), np.int32)
    cr = t(rng.integers(0, held.R.shape[0], (C, 3)), np.int32)
    Rh, Lh = t(held.R), t(held.L)
    res = sweep.score_variants(hsc, ctx, res, R, L, T, Wd, val, Rh, Lh, cl, cr)
    # the projected-gradient codec on the same chains
    Ep, Dp = hi.load_codec(k, n)
    d94 = torch.empty(3, C, device=dev)
    d00 = torch.empty(3, C, device=dev)
    stp = torch.zeros(12, dtype=torch.float64, device=dev)
    hsc.hsc_chain_eval(ctx, Rh, Lh, t(Ep), t(Dp), T, cl, cr, d94, d00, stp)
    hsc.hsc_sync(ctx)
    pg = stp.cpu().numpy().reshape(3, 4)
    ep = res.epochs.cpu().numpy()
    sel = res.selected
    return {"codec_sweep_700": {
        "variants": V, "max_epochs": epochs, "patience": patience, "batches_per_epoch": int(sched.train_r.shape[1]),
        "epochs_run": res.epochs_run, "epochs_mean": float(ep.mean()), "epochs_max": int(ep.max()),
        "stopped_early": int((ep < epochs).sum()), "step_launches": res.steps, "variant_steps": res.variant_steps,
        "train_s": res.seconds["train"], "score_s": res.seconds["score"],
        "variant_steps_per_s": res.variant_steps / res.seconds["train"],
        "selected_weights_e2e_rec_code_col": [float(x) for x in W[sel]] if sel >= 0 else None,
        "selected_de94_mean_per_depth": [float(x) for x in res.chain_stats[sel, :, 0]] if sel >= 0 else None,
        "median_score_de94": float(np.nanmedian(res.scores)),
        "projected_gradient_codec_de94_mean_per_depth": [float(x) for x in pg[:, 0]]}}


def serve_rows(args, hsc, ctx, dev):
    """Poisson arrivals (200 requests/s) of render-plus-decode requests over 8
    resident scenes (256 materials, 128-light pools), sizes from 512x512 to
    3840x2160, k in {6, 9}, n in {31, 81}, 16-128 lights, BF16 codes, 40 GB
    admission budget; served with continuous batching by the latent path and,
    on the same stream, by naive n-sample shading.  Latency: arrival to GPU
    completion; the first quarter of the stream is warm-up."""
    from paper_2602_18741_gb300 import serve
    scenes = serve.ResidentScenes(hsc, ctx, dev)
    reqs = hi.request_stream(duration_s=args.serve_seconds)
    warm = args.serve_seconds / 4.0
    arrivals = [r.arrival_s for r in sorted(reqs, key=lambda r: r.arrival_s)]
    out = {}
    idle = serve.IDLE_SLEEP_S if args.serve_idle_us < 0 else args.serve_idle_us * 1e-6
    for mode in ("latent", "spectral"):
        stats, _ = serve.serve(hsc, ctx, scenes, reqs, mode=mode, idle_sleep_s=idle)
        sm = stats.summary(warmup_s=warm, arrivals=arrivals)
        sm["offered_per_s"] = len(reqs) / args.serve_seconds
        sm["idle_sleep_us"] = idle * 1e6
        out[f"serve_{mode}"] = sm
    lat, spe = out["serve_latent"], out["serve_spectral"]
    if lat.get("p50_ms") and spe.get("p50_ms"):
        out["serve_latency_ratio_spectral_over_latent"] = {"p50": spe["p50_ms"] / lat["p50_ms"],
                                                           "p99": spe["p99_ms"] / lat["p99_ms"]}
    # the same kind of stream at 20x the rate for one second: the latent path
    # keeps up by batching requests into shared launches, the n-sample path
    # falls behind and its queue (and latency) grows
    rate_hi = 4000.0
    reqs_hi = hi.request_stream(seed=hi.MASTER_SEED + 7, rate_hz=rate_hi, duration_s=1.0)
    for mode in ("latent", "spectral"):
        stats, _ = serve.serve(hsc, ctx, scenes, reqs_hi, mode=mode, idle_sleep_s=idle, reserve_per_size=64)
        sm = stats.summary()
        sm["offered_per_s"] = float(len(reqs_hi))
        out[f"serve_{mode}_{int(rate_hi)}_per_s"] = sm
    del scenes
    return out


def chain_rows(args, hsc, ctx, dev, timed):
    """Multi-bounce chains (the codec-selection proxy of Sec. 4.5): 1,048,576
    chains of depth 3 over held-out synthetic reflectances and lights, k = 6,
    n = 81; CIE94 and CIEDE2000 of the latent chain against the spectral chain
    per depth (the paper reports mean CIE94 per depth on its own data)."""
    import torch
    ts = hi.training_set(hi.GRID_81, seed=hi.MASTER_SEED + 200)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    R, L = t(ts.R), t(ts.L)
    E, D = hi.load_codec(args.k, 81)
    T = torch.empty(3, 81, device=dev)
    hsc.hsc_cmf_weights(ctx, 81, 380.0, 5.0, T)
    C, depth = 1 << 20, 3
    gen = torch.Generator(device=dev)
    gen.manual_seed(hi.MASTER_SEED)
    cl = torch.randint(0, L.shape[0], (C,), generator=gen, device=dev, dtype=torch.int32)
    cr = torch.randint(0, R.shape[0], (C, depth), generator=gen, device=dev, dtype=torch.int32)
    d94 = torch.empty(depth, C, device=dev)
    d00 = torch.empty(depth, C, device=dev)
    st = torch.zeros(4 * depth, device=dev, dtype=torch.float64)
    Ed, Dd = t(E), t(D)

    def run():
        hsc.hsc_chain_eval(ctx, R, L, Ed, Dd, T, cl, cr, d94, d00, st)

    ms, _ = timed(run, args.steps, args.warmup)
    hsc.hsc_sync(ctx)
    s = st.cpu().numpy().reshape(depth, 4)
    m_ = statistics.mean(ms)
    return {"chains_depth3": {"ms": m_, "chains_per_s": C / (m_ * 1e-3), "chains": C,
                              "de94_mean": [float(v) for v in s[:, 0]], "de94_p95": [float(v) for v in s[:, 1]],
                              "de2000_mean": [float(v) for v in s[:, 2]], "de2000_p95": [float(v) for v in s[:, 3]]}}


def batch_rows(args, hsc, ctx, dev, timed):
    """64 frames of uneven size (W, H uniform in [256, 2048]), 4-256 lights,
    k in {6, 9}, n in {31, 81}, each with its own jittered codec, shaded and
    decoded to XYZ by one persistent launch replayed as a CUDA graph; codes in
    FP32 and in BF16.  G-buffers are drawn on the device with the same recipe
    as the host generator."""
    import torch
    specs = hi.batched_frame_specs()
    gen = torch.Generator(device=dev)
    keep = []
    frames = {torch.float32: [], torch.bfloat16: []}
    Ts = {}
    for s in specs:
        gen.manual_seed(s.seed)
        (n1, x1, m1), _ = hi.torch_gbuffers(gen, s.pixels, 64, False, dev)
        mats, spd, lpos, linten = hi.frame_assets(s)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        g1 = hsc.GBuffer(n1, x1, m1)
        lights = hsc.Lights(t(lpos), t(linten))
        if s.grid not in Ts:
            T = torch.empty(3, s.grid[2], device=dev)
            hsc.hsc_cmf_weights(ctx, s.grid[2], s.grid[0], s.grid[1], T)
            Ts[s.grid] = T
        Ed, Dd = t(s.E), t(s.D)
        M = torch.empty(3, s.k, device=dev)
        hsc.hsc_fold_xyz(ctx, Ts[s.grid], Dd, M)
        xyz = torch.empty(s.pixels, 3, device=dev)
        for dt in frames:
            zm = torch.empty(mats.shape[0], s.k, device=dev, dtype=dt)
            zl = torch.empty(s.lights, s.k, device=dev, dtype=dt)
            hsc.hsc_encode(ctx, Ed, t(mats), zm)
            hsc.hsc_encode(ctx, Ed, t(spd), zl)
            frames[dt].append(hsc.BatchFrame(g1, None, zm, lights, zl, M, xyz))
        keep.append((g1, lights, Ed, Dd, M, xyz))
    px = sum(s.pixels for s in specs)
    evals = sum(s.pixels * s.lights for s in specs)
    out = {}
    for dt, name in ((torch.float32, "f32"), (torch.bfloat16, "bf16")):
        batch = hsc.hsc_batch_create(ctx, frames[dt])

        def run(batch=batch):
            hsc.hsc_batch_shade(ctx, batch)

        ms, _ = timed(run, args.steps, args.warmup)
        m_ = statistics.mean(ms)
        out[f"batch64_{name}"] = {"ms": m_, "frames_per_s": len(specs) / (m_ * 1e-3), "Mpx_per_s": px / (m_ * 1e-3) / 1e6,
                                  "evals_per_s": evals / (m_ * 1e-3), "pixels": px, "evals": evals,
                                  "p50_ms": _pct(ms, 50), "p99_ms": _pct(ms, 99)}
        batch.close()
    hsc.hsc_sync(ctx)
    return out


def _M(hsc, ctx, T, Dd):
    import torch
    k = Dd.shape[1]
    M = torch.empty(3, k, device=Dd.device)
    hsc.hsc_fold_xyz(ctx, T, Dd, M)
    return M


def e2e_leg(args, hsc, ctx, f, dev, stream, Ed, M, evals):
    """Same latent frame through the public API with host buffers: pinned
    host G-buffers, lights and spectra copied in and the frame's displayed
    result, its 8-bit sRGB image, copied out, every step, all inside the
    timed region (the kernels still write the latent and XYZ images too, as
    in the device-timed step).  Frames stream through two
    buffer sets: the copy-in of frame i + 1 (one copy stream) and the copy-out
    of frame i - 1 (another) overlap the kernels of frame i (one compute
    stream, so the shading launches keep their one-at-a-time order); events
    order each buffer's reuse."""
    import torch
    K, W = max(3, args.steps // 2), 2
    h = {}
    for name, a in (("n1", f.g1.normal), ("x1", f.g1.pos), ("m1", f.g1.mat), ("n2", f.g2.normal),
                    ("x2", f.g2.pos), ("m2", f.g2.mat), ("lp", f.light_pos), ("li", f.light_intensity),
                    ("mats", f.mat_spectra), ("spd", f.light_spd)):
        h[name] = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    P = f.pixels
    k = args.k
    sets = []
    for _ in range(2):
        d = {name: torch.empty_like(t, device=dev) for name, t in h.items()}
        sets.append({
            "d": d,
            "zm": torch.empty(f.mat_spectra.shape[0], k, device=dev),
            "zl": torch.empty(f.lights, k, device=dev),
            "lat": torch.empty(P, k, device=dev),
            "xyz": torch.empty(P, 3, device=dev),
            "rgb": torch.empty(P, 3, device=dev, dtype=torch.uint8),
            "rgb_h": torch.empty(P, 3, dtype=torch.uint8).pin_memory(),
            "g1": hsc.GBuffer(d["n1"], d["x1"], d["m1"]),
            "g2": hsc.GBuffer(d["n2"], d["x2"], d["m2"]),
            "lights": hsc.Lights(d["lp"], d["li"]),
            "in_done": torch.cuda.Event(), "comp_done": torch.cuda.Event(), "out_done": torch.cuda.Event(),
        })
    h2d = sum(t.numel() * t.element_size() for t in h.values())
    d2h = sets[0]["rgb_h"].numel()
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    used = [False, False]

    def step(i):
        b = sets[i % 2]
        with torch.cuda.stream(s_in):
            if used[i % 2]:
                s_in.wait_event(b["comp_done"])          # the kernels of frame i - 2 have read these inputs
            for name in h:
                b["d"][name].copy_(h[name], non_blocking=True)
            b["in_done"].record(s_in)
        stream.wait_event(b["in_done"])
        if used[i % 2]:
            stream.wait_event(b["out_done"])             # frame i - 2's outputs have been copied out
        hsc.hsc_encode_assets(ctx, Ed, b["d"]["mats"], b["zm"], b["d"]["spd"], b["zl"], stream=stream)
        hsc.hsc_shade_latent(ctx, b["g1"], b["g2"], b["zm"], b["lights"], b["zl"], hsc.HSC_FUSED, b["lat"],
                             xyz_out=b["xyz"], M_xyz=M, srgb8_out=b["rgb"], stream=stream)
        b["comp_done"].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(b["comp_done"])
            b["rgb_h"].copy_(b["rgb"], non_blocking=True)
            b["out_done"].record(s_out)
        used[i % 2] = True

    for i in range(W):
        step(i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(W, W + K):
        step(i)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / K
    hsc.hsc_sync(ctx)
    return {"value": evals / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": dt * 1e3, "steps": K,
            "pipelined": "two buffer sets; copy-in, kernels, copy-out overlap"}


# --------------------------------------------------------------------------- reference arm

def run_reference(args, rank: int, world: int):
    if rank != 0:
        return None
    K, W = args.steps, args.warmup
    per = []
    ncores = 1
    # each step: one 32-row band (61,440 pixels x 128 evaluations) through the oracle
    for i in range(W + K):
        rate, nrows, secs = oracle_rate(0.0, args.k, threads=ncores, max_rows=32)
        if i >= W:
            per.append((nrows * 1920 * 128, secs))
    ev = sum(e for e, _ in per)
    tot = sum(s for _, s in per)
    value = ev / tot
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": tot / K * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded G-buffers, spectra, lights)", "impl": "reference",
            "config": {"workload": WORKLOAD, "pixels": 1920 * 1080, "lights": 64, "k": args.k, "n": 81,
                       "sample": "each step: one 32-row band of the frame (61,440 pixels)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                             "sample": "32-row band of the 1920x1080 frame per step, FP64 NumPy, one thread",
                             "host": host_cpu_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "hsc" else "gloo")
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_hsc(args, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
