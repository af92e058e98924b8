"""Continuous-batching render-plus-decode server over the C ABI.

Requests (hsc_inputs.request_stream) name a resident scene, an image size, a
code length k, a spectral grid n and a light count L.  Everything a request
reads stays on the device: per scene and size a G-buffer, per scene its 256
materials and a pool of 128 lights (SPDs on both grids), and for every
(scene, k, n) the material and light codes and the folded decode matrix.

The scheduler is continuous batching: on every turn of the loop it retires
finished launches (freeing their output memory), admits newly arrived
requests in arrival order while the HBM footprint of admitted requests stays
under the budget, and launches everything admitted so far as one batched
persistent launch (hsc_shade_frames) on the next of a few streams, so new
work overlaps the work already on the GPU.  Latency is measured from a
request's arrival to the GPU completion event of its launch.  The same stream
can be served by the naive n-sample shader (hsc_shade_spectral, one launch per
request) for comparison.

The scheduler core (Scheduler) is independent of the GPU and is tested on the
host with a fake backend.
"""
from __future__ import annotations

import collections
import gc
import math
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

import hsc_inputs as hi


# --------------------------------------------------------------------------- scheduler

# Longest host sleep of a scheduler pass that finds the GPU idle and no
# request waiting (seconds), and how long before the next arrival it wakes.
# Polling without a pause keeps one host core busy all the time, and a thread
# that never sleeps is the one the kernel preempts when the host is busy;
# while launches are in flight the loop still polls, so completions are seen
# at once.
IDLE_SLEEP_S = 1e-3
WAKE_MARGIN_S = 100e-6

@dataclass
class Inflight:
    handle: object          # backend completion handle
    requests: list
    nbytes: int


@dataclass
class ServeStats:
    latencies_ms: List[float] = field(default_factory=list)
    launches: int = 0
    max_inflight_bytes: int = 0
    max_batch: int = 0
    wall_s: float = 0.0
    first_arrival_s: float = 0.0
    last_done_ms: float = 0.0
    max_launch_call_ms: float = 0.0   # longest host time inside one backend.launch
    max_loop_gap_ms: float = 0.0      # longest host time between two scheduler passes
    launch_parts_ms: Dict[str, float] = field(default_factory=dict)  # longest time per part of a launch
    max_inflight_launches: int = 0    # most launches submitted and not yet complete, seen at a launch
    batch_hist: Dict[int, int] = field(default_factory=dict)  # requests per launch -> number of launches
    idle_sleeps: int = 0              # scheduler passes that found nothing to do and slept
    host: Dict[str, float] = field(default_factory=dict)      # host CPU accounting of the run (host_usage)

    def summary(self, warmup_s: float = 0.0, arrivals: Optional[Sequence[float]] = None) -> dict:
        lat = np.asarray(self.latencies_ms, dtype=np.float64)
        if arrivals is not None and warmup_s > 0:
            keep = np.asarray(arrivals) >= warmup_s
            lat = lat[keep[:len(lat)]]
        if lat.size == 0:
            return {"requests": 0}
        srt = np.sort(lat)

        def nr(q):
            return float(srt[max(int(math.ceil(q * srt.size)) - 1, 0)])

        return {"requests": int(lat.size), "p50_ms": nr(0.50), "p99_ms": nr(0.99), "mean_ms": float(lat.mean()),
                "max_ms": float(srt[-1]), "launches": self.launches, "max_batch": self.max_batch,
                "max_inflight_MB": self.max_inflight_bytes / 1e6,
                "frames_per_s": float(len(self.latencies_ms) / max(self.wall_s, 1e-9)),
                "max_launch_call_ms": self.max_launch_call_ms, "max_loop_gap_ms": self.max_loop_gap_ms,
                "max_launch_parts_ms": dict(self.launch_parts_ms),
                "max_inflight_launches": self.max_inflight_launches,
                "batch_hist": {str(b): c for b, c in sorted(self.batch_hist.items())},
                "idle_sleeps": self.idle_sleeps, "host": dict(self.host)}


class Scheduler:
    """Admission by footprint and continuous batching, independent of the GPU.

    backend.launch(requests) -> handle  (asynchronous)
    backend.done(handle) -> Optional[float]  (completion time in ms since start, or None)
    backend.footprint(request) -> bytes
    backend.now_s() -> seconds since start
    backend.sleep(seconds)  (optional; time.sleep when absent)
    """

    def __init__(self, backend, budget_bytes: int, max_inflight: int = 4, max_batch: int = 64):
        self.b = backend
        self.budget = int(budget_bytes)
        self.max_inflight = max_inflight
        self.max_batch = max_batch

    def run(self, requests: Sequence[hi.Request], idle_sleep_s: float = 0.0) -> ServeStats:
        """Serve ``requests`` (arrival times in seconds from the start).  A
        pass of the loop that finds the GPU idle and no request waiting sleeps
        for up to ``idle_sleep_s``, waking WAKE_MARGIN_S before the next
        arrival; with launches in flight it polls continuously.  0 never
        sleeps."""
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        for r in reqs:
            if self.b.footprint(r) > self.budget:
                raise ValueError(f"request {r.rid} alone exceeds the memory budget")
        st = ServeStats()
        st.latencies_ms = [float("nan")] * len(reqs)
        index = {r.rid: i for i, r in enumerate(reqs)}
        queue: collections.deque = collections.deque()
        inflight: List[Inflight] = []
        used = 0
        nxt = 0
        done = 0
        t_start = self.b.now_s()
        prev = t_start
        while done < len(reqs):
            now = self.b.now_s()
            st.max_loop_gap_ms = max(st.max_loop_gap_ms, 1e3 * (now - prev))
            prev = now
            while nxt < len(reqs) and reqs[nxt].arrival_s <= now:
                queue.append(reqs[nxt])
                nxt += 1
            # retire finished launches
            still = []
            for f in inflight:
                t_done = self.b.done(f.handle)
                if t_done is None:
                    still.append(f)
                    continue
                for r in f.requests:
                    st.latencies_ms[index[r.rid]] = t_done - 1e3 * r.arrival_s
                    done += 1
                st.last_done_ms = max(st.last_done_ms, t_done)
                used -= f.nbytes
            retired = len(inflight) != len(still)
            inflight = still
            # admit in arrival order while the footprint fits, launch as one batch
            if queue and len(inflight) < self.max_inflight:
                batch, nbytes = [], 0
                while queue and len(batch) < self.max_batch:
                    fp = self.b.footprint(queue[0])
                    if used + nbytes + fp > self.budget:
                        break
                    batch.append(queue.popleft())
                    nbytes += fp
                if batch:
                    t_l = self.b.now_s()
                    h = self.b.launch(batch)
                    st.max_launch_call_ms = max(st.max_launch_call_ms, 1e3 * (self.b.now_s() - t_l))
                    inflight.append(Inflight(h, batch, nbytes))
                    used += nbytes
                    st.launches += 1
                    st.max_batch = max(st.max_batch, len(batch))
                    st.batch_hist[len(batch)] = st.batch_hist.get(len(batch), 0) + 1
                    st.max_inflight_launches = max(st.max_inflight_launches, len(inflight))
                    st.max_inflight_bytes = max(st.max_inflight_bytes, used)
                    continue
            if idle_sleep_s > 0 and not retired and not inflight and not queue:
                # nothing on the GPU and nothing waiting: sleep, but wake a
                # little before the next arrival (sleeps overshoot by tens of
                # microseconds); with launches in flight the loop keeps polling
                # so that completions are seen at once
                wait = idle_sleep_s
                if nxt < len(reqs):
                    wait = min(wait, reqs[nxt].arrival_s - now - WAKE_MARGIN_S)
                if wait > 0:
                    st.idle_sleeps += 1
                    getattr(self.b, "sleep", time.sleep)(wait)
        st.wall_s = self.b.now_s() - t_start
        return st


def host_usage() -> Dict[str, float]:
    """Host CPU accounting of this process and its control group: CPU seconds
    used, voluntary and involuntary context switches, and the cgroup's CPU
    quota and throttling counters (cgroup v2 cpu.max / cpu.stat, where
    readable).  A scheduler pass that stalls for tens of milliseconds without
    doing work is either descheduled by the kernel (involuntary switches) or
    held by a CPU quota that the group has used up (nr_throttled)."""
    import resource
    ru = resource.getrusage(resource.RUSAGE_SELF)
    out = {"cpu_s": ru.ru_utime + ru.ru_stime, "nvcsw": float(ru.ru_nvcsw), "nivcsw": float(ru.ru_nivcsw)}
    try:
        with open("/sys/fs/cgroup/cpu.stat") as fh:
            for line in fh:
                key, _, val = line.partition(" ")
                if key in ("nr_periods", "nr_throttled", "throttled_usec", "usage_usec"):
                    out["cg_" + key] = float(val)
    except OSError:
        pass
    try:
        with open("/sys/fs/cgroup/cpu.max") as fh:
            quota, _, period = fh.read().strip().partition(" ")
            out["cg_quota_cpus"] = -1.0 if quota == "max" else float(quota) / float(period)
    except (OSError, ValueError):
        pass
    return out


def usage_delta(before: Dict[str, float], after: Dict[str, float]) -> Dict[str, float]:
    """Counters of host_usage() over an interval (the quota as it stands)."""
    d = {k: after[k] - before[k] for k in after if k in before and k != "cg_quota_cpus"}
    if "cg_quota_cpus" in after:
        d["cg_quota_cpus"] = after["cg_quota_cpus"]
    return d


# --------------------------------------------------------------------------- GPU state

class ResidentScenes:
    """Device-resident scenes: G-buffers per size, materials, light pools and
    codes/decode matrices per (k, n)."""

    def __init__(self, hsc, ctx, device, scenes: int = 8, sizes=hi.SERVE_SIZES, ks=(6, 9), grids=(hi.GRID_31, hi.GRID_81),
                 n_mat: int = 256, pool: int = 128, code_dtype=None, seed: int = hi.MASTER_SEED + 6):
        import torch
        self.hsc, self.ctx, self.dev = hsc, ctx, device
        code_dtype = code_dtype or torch.bfloat16
        self.code_dtype = code_dtype
        gen = torch.Generator(device=device)
        rngs = hi.streams(seed, scenes)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.gbuf: Dict[tuple, object] = {}
        self.lights: Dict[int, tuple] = {}
        self.mats: Dict[tuple, object] = {}
        self.spd: Dict[tuple, object] = {}
        self.codes: Dict[tuple, tuple] = {}
        self.M: Dict[tuple, object] = {}
        self.T: Dict[int, object] = {}
        for g in grids:
            T = torch.empty(3, g[2], device=device)
            hsc.hsc_cmf_weights(ctx, g[2], g[0], g[1], T)
            self.T[g[2]] = T
        for s in range(scenes):
            r = rngs[s]
            for (w, h) in sizes:
                gen.manual_seed(int(r.integers(0, 2**31 - 1)))
                (n1, x1, m1), _ = hi.torch_gbuffers(gen, w * h, n_mat, False, device)
                self.gbuf[(s, w, h)] = hsc.GBuffer(n1, x1, m1)
            lpos, linten = hi.light_positions(r, pool)
            self.lights[s] = (t(lpos), t(linten))
            temps = r.uniform(2000.0, 10000.0, size=pool // 2)
            mus = r.uniform(400.0, 700.0, size=pool - pool // 2)
            sig = r.uniform(5.0, 20.0, size=pool - pool // 2)
            mseed = int(r.integers(0, 2**31 - 1))
            for g in grids:
                lam = hi.grid(*g)
                mrng = np.random.default_rng([mseed, g[2]])
                mats = np.concatenate([hi.smooth_reflectances(mrng, lam, n_mat - n_mat // 8),
                                       hi.sawtooth_reflectances(mrng, lam, n_mat // 8)], axis=0).astype(np.float32)
                spd = np.concatenate([hi.blackbody(lam, temps), hi.narrowband(lam, mus, sig)], axis=0).astype(np.float32)
                self.mats[(s, g[2])] = t(mats)
                self.spd[(s, g[2])] = t(spd)
                for k in ks:
                    E, D = hi.load_codec(k, g[2])
                    Ed, Dd = t(E), t(D)
                    zm = torch.empty(n_mat, k, device=device, dtype=code_dtype)
                    zl = torch.empty(pool, k, device=device, dtype=code_dtype)
                    hsc.hsc_encode(ctx, Ed, self.mats[(s, g[2])], zm)
                    hsc.hsc_encode(ctx, Ed, self.spd[(s, g[2])], zl)
                    self.codes[(s, k, g[2])] = (zm, zl)
                    if (k, g[2]) not in self.M:
                        M = torch.empty(3, k, device=device)
                        hsc.hsc_fold_xyz(ctx, self.T[g[2]], Dd, M)
                        self.M[(k, g[2])] = M
        torch.cuda.synchronize(device)

    def frame_inputs(self, req: hi.Request):
        g1 = self.gbuf[(req.scene, req.width, req.height)]
        lpos, linten = self.lights[req.scene]
        lights = self.hsc.Lights(lpos[:req.lights], linten[:req.lights])
        zm, zl = self.codes[(req.scene, req.k, req.n)]
        return g1, lights, zm, zl[:req.lights], self.M[(req.k, req.n)]


def _ceil_log2(v: int) -> int:
    """The smallest b with 2^b >= v (the tuner's bucket of a count)."""
    return max(0, (int(v) - 1).bit_length())


def tuning_class(r) -> tuple:
    """The shape class a request's launch is tuned for: code length, sample
    count, and the light and pixel counts rounded up to powers of two."""
    return (r.k, r.n, _ceil_log2(r.lights), _ceil_log2(r.width * r.height))


def warmup_requests(requests) -> list:
    """The requests the warm-up runs before the first arrival, each once.
    The first launch of a kernel loads its code, which can wait for the
    device; kernels are specialised by light count too (all lights in one
    shared-memory stage or not), so each (k, n) runs with its fewest and its
    most lights.  The spectral launch is tuned on the first call of each
    shape class, which times every candidate and waits for the device, so
    one request of every class in the stream runs as well."""
    firsts = {}
    for r in requests:
        lo, hi = firsts.get((r.k, r.n), (r, r))
        firsts[(r.k, r.n)] = (r if r.lights < lo.lights else lo, r if r.lights > hi.lights else hi)
    warm = {id(x): x for pair in firsts.values() for x in pair}
    classes = {}
    for r in requests:
        classes.setdefault(tuning_class(r), r)
    for r in classes.values():
        warm[id(r)] = r
    return list(warm.values())


class GpuBackend:
    """Launches admitted requests on the GPU.  mode 'latent': one batched
    launch per admitted group (hsc_shade_frames); mode 'spectral': one
    hsc_shade_spectral launch per request.  Streams are used round-robin."""

    def __init__(self, hsc, ctx, scenes: ResidentScenes, mode: str = "latent", streams: int = 3,
                 keep_outputs: bool = False):
        import torch
        self.hsc, self.ctx, self.sc, self.mode = hsc, ctx, scenes, mode
        self.streams = [torch.cuda.Stream(device=scenes.dev) for _ in range(streams)]
        self.si = 0
        self.keep = keep_outputs
        self.outputs: Dict[int, object] = {}
        self.ref = torch.cuda.Event(enable_timing=True)
        self.t0 = None
        # output buffers by pixel count; a buffer returns to its list when the
        # launch that wrote it has completed (so any stream may reuse it)
        self.pool: Dict[int, list] = collections.defaultdict(list)
        self.parts: Dict[str, float] = {}

    def reserve(self, requests, per_size: int = 16):
        """Prepare before the first arrival: the descriptor ring, a few
        requests of every (k, n) through the real path so that their kernels
        are loaded, and `per_size` output buffers of every request size.  A
        device allocation or the first launch of a kernel inside the serving
        loop can wait for all queued work, which would stall every request
        behind it."""
        import torch
        if self.mode == "latent":
            self.hsc.hsc_shade_frames(self.ctx, [], stream=self.streams[0])   # allocates the descriptor ring
        handles = [self.launch([r]) for r in warmup_requests(requests)]
        torch.cuda.synchronize(self.sc.dev)
        for _, outs in handles:
            if self.keep:   # warm-up outputs are not the caller's
                for _, xyz in outs:
                    self.pool[xyz.shape[0]].append(xyz)
                outs.clear()
            else:
                self._release(outs)
        self.outputs.clear()
        sizes = collections.Counter(r.width * r.height for r in requests)
        for px in sorted(sizes):
            # outputs kept for the caller never return to the pool: one each
            want = max(per_size, sizes[px]) if self.keep else per_size
            while len(self.pool[px]) < want:
                self.pool[px].append(torch.empty(px, 3, device=self.sc.dev))

    def _buffer(self, px: int, stream=None):
        import torch
        free = self.pool[px]
        if free:
            return free.pop()
        # a pool that ran dry: allocate on the launch's stream, so that the
        # caching allocator orders the buffer's reuse after this launch
        with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream(self.sc.dev)):
            return torch.empty(px, 3, device=self.sc.dev)

    def start(self):
        import torch
        torch.cuda.synchronize(self.sc.dev)
        self.ref.record(torch.cuda.current_stream(self.sc.dev))
        torch.cuda.synchronize(self.sc.dev)
        self.t0 = time.perf_counter()

    def now_s(self) -> float:
        return time.perf_counter() - self.t0

    def sleep(self, seconds: float):
        time.sleep(seconds)

    def footprint(self, r: hi.Request) -> int:
        return r.width * r.height * 12 + 4096

    def _part(self, name, t0):
        t1 = time.perf_counter()
        self.parts[name] = max(self.parts.get(name, 0.0), 1e3 * (t1 - t0))
        return t1

    def launch(self, requests):
        """Every call below takes the stream explicitly, so the launch does not
        switch torch's current stream (a device guard and two stream switches
        per launch on the host's critical path)."""
        import torch
        t = time.perf_counter()
        stream = self.streams[self.si]
        self.si = (self.si + 1) % len(self.streams)
        outs = []
        if self.mode == "latent":
            frames = []
            for r in requests:
                g1, lights, zm, zl, M = self.sc.frame_inputs(r)
                xyz = self._buffer(r.width * r.height, stream)
                frames.append(self.hsc.BatchFrame(g1, None, zm, lights, zl, M, xyz))
                outs.append((r.rid, xyz))
            t = self._part("inputs", t)
            self.hsc.hsc_shade_frames(self.ctx, frames, stream=stream)
            t = self._part("shade_frames", t)
        else:
            for r in requests:
                g1 = self.sc.gbuf[(r.scene, r.width, r.height)]
                lpos, linten = self.sc.lights[r.scene]
                lights = self.hsc.Lights(lpos[:r.lights], linten[:r.lights])
                xyz = self._buffer(r.width * r.height, stream)
                self.hsc.hsc_shade_spectral(self.ctx, g1, None, self.sc.mats[(r.scene, r.n)], lights,
                                            self.sc.spd[(r.scene, r.n)][:r.lights], self.sc.T[r.n], xyz,
                                            stream=stream)
                outs.append((r.rid, xyz))
            t = self._part("shade_spectral", t)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        self._part("event", t)
        if self.keep:
            for rid, xyz in outs:
                self.outputs[rid] = xyz
        return (ev, outs)

    def _release(self, outs):
        if not self.keep:
            for _, xyz in outs:
                self.pool[xyz.shape[0]].append(xyz)
        outs.clear()

    def done(self, handle) -> Optional[float]:
        ev, outs = handle
        if not ev.query():
            return None
        self._release(outs)
        return float(self.ref.elapsed_time(ev))


def serve(hsc, ctx, scenes: ResidentScenes, requests, mode="latent", budget_bytes=40 * 10**9, max_batch=64,
          keep_outputs=False, max_inflight=4, idle_sleep_s=IDLE_SLEEP_S, reserve_per_size=16):
    """Serve `requests` in real time.  Launch-configuration tuning is switched
    off while serving: tuning a new shape class synchronises the stream, which
    would stall the requests behind it (a server tunes ahead of time and
    loads the result with hsc_tune_load).  Output buffers come from a pool
    filled before the first arrival (no device allocation inside the loop),
    and the garbage collector is paused for the loop.  A pass with nothing to
    do sleeps ``idle_sleep_s`` rather than polling again at once (see
    IDLE_SLEEP_S).  ``reserve_per_size`` output buffers of every request size
    are allocated before the first arrival; a stream that keeps more requests
    of one size in flight needs more."""
    backend = GpuBackend(hsc, ctx, scenes, mode=mode, keep_outputs=keep_outputs)
    sched = Scheduler(backend, budget_bytes, max_inflight=max_inflight, max_batch=max_batch)
    was = bool(ctx.autotune) if hasattr(ctx, "autotune") else False
    hsc.hsc_set_autotune(ctx, False)
    gc_was = gc.isenabled()
    gc.disable()                   # no collector pause inside the real-time loop
    try:
        backend.reserve(requests, per_size=reserve_per_size)
        backend.parts.clear()
        backend.start()
        u0 = host_usage()
        stats = sched.run(requests, idle_sleep_s=idle_sleep_s)
        stats.host = usage_delta(u0, host_usage())
        stats.launch_parts_ms = dict(backend.parts)
        hsc.hsc_sync(ctx)
    finally:
        if gc_was:
            gc.enable()
        hsc.hsc_set_autotune(ctx, was)
    return stats, backend
