"""Host-side tests of the continuous-batching scheduler with a fake backend
(simulated clock, launches that finish after a cost proportional to their
pixels): every request completes, in arrival order of admission, the admitted
footprint never exceeds the budget, and requests arriving while others run
join later launches (continuous batching, not one queue drain)."""
import importlib.util
import os
import sys

import pytest

import hsc_inputs as hi

# serve.py is pure Python at import time; load it by path so this host test
# does not need the CUDA library that the package import loads
_spec = importlib.util.spec_from_file_location(
    "_hsc_serve", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                               "paper_2602_18741_gb300", "serve.py"))
_serve = importlib.util.module_from_spec(_spec)
sys.modules["_hsc_serve"] = _serve
_spec.loader.exec_module(_serve)
Scheduler = _serve.Scheduler


class FakeBackend:
    def __init__(self, px_per_ms=2e6, tick_ms=0.05):
        self.t_ms = 0.0
        self.px_per_ms = px_per_ms
        self.tick = tick_ms
        self.gpu_free_ms = 0.0
        self.launched = []

    def now_s(self):
        self.t_ms += self.tick
        return self.t_ms / 1e3

    def footprint(self, r):
        return r.width * r.height * 12

    def launch(self, reqs):
        px = sum(r.width * r.height for r in reqs)
        start = max(self.t_ms, self.gpu_free_ms)
        end = start + px / self.px_per_ms
        self.gpu_free_ms = end
        self.launched.append([r.rid for r in reqs])
        return end

    def done(self, handle):
        return handle if self.t_ms >= handle else None

    def sleep(self, seconds):
        self.slept_ms = getattr(self, "slept_ms", 0.0) + 1e3 * seconds
        self.t_ms += 1e3 * seconds


def _requests(n=300, rate=400.0):
    reqs = hi.request_stream(seed=3, rate_hz=rate, duration_s=10.0)[:n]
    return reqs


def test_all_requests_complete_in_order_within_budget():
    reqs = _requests()
    fb = FakeBackend()
    budget = 300 * 10**6
    st = Scheduler(fb, budget, max_inflight=4, max_batch=16).run(reqs)
    assert all(lat == lat and lat >= 0 for lat in st.latencies_ms)   # no NaN, non-negative
    order = [rid for group in fb.launched for rid in group]
    assert order == sorted(order) and sorted(order) == sorted(r.rid for r in reqs)
    assert st.max_inflight_bytes <= budget
    assert st.max_batch <= 16
    assert st.launches < len(reqs)            # arrivals during busy periods were batched


def test_budget_limits_admission():
    reqs = _requests(n=120, rate=2000.0)
    fb = FakeBackend(px_per_ms=5e5)
    small = max(fb.footprint(r) for r in reqs)       # room for about one large request
    st = Scheduler(fb, small, max_inflight=8, max_batch=64).run(reqs)
    assert st.max_inflight_bytes <= small
    assert len(st.latencies_ms) == 120


def test_request_larger_than_budget_is_rejected():
    reqs = _requests(n=5)
    with pytest.raises(ValueError):
        Scheduler(FakeBackend(), 1000).run(reqs)


def test_summary_statistics():
    reqs = _requests(n=50)
    st = Scheduler(FakeBackend(), 10**12).run(reqs)
    s = st.summary()
    assert s["requests"] == 50 and s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]


def test_burst_is_batched_and_launches_overlap():
    # every request arrives at once: the first passes take max_batch requests
    # each, and while the (simulated) GPU works through one launch the next
    # ones are submitted, so several launches are in flight together
    reqs = [hi.Request(i, 0.0, 512, 512, 6, 31, 32, 0, i) for i in range(40)]
    fb = FakeBackend(px_per_ms=2e5)
    st = Scheduler(fb, 10**12, max_inflight=4, max_batch=8).run(reqs)
    s = st.summary()
    assert s["max_batch"] == 8 and s["launches"] == 5
    assert s["batch_hist"] == {"8": 5}
    assert s["max_inflight_launches"] == 4
    assert all(len(g) == 8 for g in fb.launched)


def test_idle_passes_sleep_until_the_next_arrival():
    # sparse arrivals: passes with nothing to do sleep (at most the time left
    # to the next arrival), so the loop does not poll continuously, and the
    # latencies stay those of the polling loop within a sleep
    reqs = _requests(n=60, rate=50.0)
    busy = Scheduler(FakeBackend(), 10**12).run(reqs)
    fb = FakeBackend()
    lazy = Scheduler(fb, 10**12).run(reqs, idle_sleep_s=1e-3)
    assert lazy.idle_sleeps > 0 and busy.idle_sleeps == 0
    assert fb.slept_ms > 0
    # the loop wakes before each arrival and polls while work is in flight,
    # so every request completes when it would with continuous polling
    for a, b in zip(busy.latencies_ms, lazy.latencies_ms):
        assert abs(b - a) <= 2 * fb.tick


def test_host_usage_counters():
    u0 = _serve.host_usage()
    sum(i * i for i in range(200000))
    d = _serve.usage_delta(u0, _serve.host_usage())
    assert d["cpu_s"] >= 0.0 and d["nivcsw"] >= 0.0 and d["nvcsw"] >= 0.0
    assert set(u0) >= {"cpu_s", "nvcsw", "nivcsw"}


def test_tuning_bucket_is_the_smallest_covering_power_of_two():
    for v in list(range(1, 5000)) + [2 ** 21 - 1, 2 ** 21, 2 ** 21 + 1, 3840 * 2160]:
        b = _serve._ceil_log2(v)
        assert 2 ** b >= v and (b == 0 or 2 ** (b - 1) < v), v


def test_warmup_covers_every_tuning_class_and_light_extreme():
    reqs = hi.request_stream(seed=11, rate_hz=400.0, duration_s=5.0)
    warm = _serve.warmup_requests(reqs)
    assert len({id(r) for r in warm}) == len(warm)          # each request once
    assert {_serve.tuning_class(r) for r in warm} == {_serve.tuning_class(r) for r in reqs}
    for kn in {(r.k, r.n) for r in reqs}:
        lights = [r.lights for r in reqs if (r.k, r.n) == kn]
        got = [r.lights for r in warm if (r.k, r.n) == kn]
        assert min(lights) in got and max(lights) in got
    # a class is warmed by one of its own requests
    assert all(r in reqs for r in warm)
