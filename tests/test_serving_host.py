"""Host tests of the serving scheduler (no GPU): admission by free memory, slot
limits, chunked stepping, retirement and latency bookkeeping, with a fake backend
and a simulated clock."""
import numpy as np
import pytest

from paper_2606_14073_gb300.serving import Request, Server, poisson_requests


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def now(self):
        return self.t

    def sleep(self, dt):
        self.t += max(0.0, dt)


class FakeBackend:
    """Device with `capacity` bytes; stepping costs atoms*steps/rate seconds of simulated time."""

    def __init__(self, clock, capacity=10_000, rate=1e6):
        self.clock, self.capacity, self.rate = clock, capacity, rate
        self.used = 0
        self.live = {}
        self.peak_active = 0
        self.steps_done = {}

    def bytes_needed(self, req):
        return 8 * req.cells ** 3

    def free_bytes(self):
        return self.capacity - self.used

    def create(self, req):
        self.used += self.bytes_needed(req)
        assert self.used <= self.capacity
        self.live[req.rid] = req
        self.steps_done[req.rid] = 0
        self.peak_active = max(self.peak_active, len(self.live))
        return req.rid

    def step(self, handles, n_steps, dts, Ts, Bs):
        work = sum(8 * self.live[h].cells ** 3 * n for h, n in zip(handles, n_steps))
        for h, n in zip(handles, n_steps):
            self.steps_done[h] += n
        self.clock.t += work / self.rate

    def atoms(self, h):
        return 8 * self.live[h].cells ** 3

    def result(self, h):
        return dict(steps=self.steps_done[h])

    def destroy(self, h):
        self.used -= self.bytes_needed(self.live.pop(h))


def test_every_request_gets_exactly_its_steps_and_memory_is_respected():
    clock = FakeClock()
    be = FakeBackend(clock, capacity=8 * 10 ** 3 * 2 + 100)   # room for two 10^3-cell replicas
    reqs = [Request(k, cells=10, T=300.0, B=(0, 0, 0), n_steps=120 + 17 * k, arrival=0.01 * k) for k in range(7)]
    out = Server(be, max_active=8, chunk=50, clock=clock).run(reqs)
    assert out["requests"] == 7
    for d in out["done"]:
        assert d.result["steps"] == d.n_steps
        assert d.finished >= d.admitted >= d.arrival
    assert be.peak_active == 2 and be.used == 0
    assert out["memory_waits"] > 0


def test_slot_limit_and_latency_percentiles():
    clock = FakeClock()
    be = FakeBackend(clock, capacity=10 ** 9)
    reqs = [Request(k, cells=8, T=100.0, B=(0, 0, 0), n_steps=100, arrival=0.0) for k in range(10)]
    out = Server(be, max_active=3, chunk=25, clock=clock).run(reqs)
    assert be.peak_active == 3
    lat = sorted(d.latency for d in out["done"])
    assert out["latency_p50_s"] == pytest.approx(np.percentile(lat, 50))
    assert lat[0] < lat[-1]


def test_idle_server_waits_for_arrivals():
    clock = FakeClock()
    be = FakeBackend(clock, capacity=10 ** 9, rate=1e9)
    reqs = [Request(0, cells=4, T=50.0, B=(0, 0, 0), n_steps=10, arrival=5.0)]
    out = Server(be, clock=clock).run(reqs)
    assert out["done"][0].admitted >= 5.0


def test_oversized_request_is_an_error():
    clock = FakeClock()
    be = FakeBackend(clock, capacity=100)
    with pytest.raises(RuntimeError):
        Server(be, clock=clock).run([Request(0, cells=10, T=1.0, B=(0, 0, 0), n_steps=1, arrival=0.0)])


def test_poisson_request_family():
    reqs = poisson_requests(50, rate=2.0, seed=1)
    gaps = np.diff([r.arrival for r in reqs])
    assert (gaps > 0).all() and abs(gaps.mean() - 0.5) < 0.25
    assert all(12 <= r.cells <= 40 and 200 <= r.n_steps <= 2000 for r in reqs)


class SlowCreateBackend(FakeBackend):
    """Creating a replica costs `create_s` seconds of host time."""

    def __init__(self, clock, create_s=0.5, **kw):
        super().__init__(clock, **kw)
        self.create_s = create_s

    def create(self, req):
        self.clock.t += self.create_s
        return super().create(req)


class AsyncBackend(SlowCreateBackend):
    """Chunks are submitted and run on simulated device time while the host goes on (creating
    replicas); wait() returns when the device is done."""

    def __init__(self, clock, **kw):
        super().__init__(clock, **kw)
        self.busy_until = 0.0
        self.flight = None

    def submit(self, handles, n_steps, dts, Ts, Bs):
        assert self.flight is None
        work = sum(8 * self.live[h].cells ** 3 * n for h, n in zip(handles, n_steps))
        self.busy_until = max(self.clock.t, self.busy_until) + work / self.rate
        self.flight = list(zip(handles, n_steps))

    def wait(self):
        for h, n in self.flight:
            self.steps_done[h] += n
        self.flight = None
        self.clock.t = max(self.clock.t, self.busy_until)

    def destroy(self, h):
        assert self.flight is None or all(h != f for f, _ in self.flight)   # never while in flight
        super().destroy(h)


def test_admission_overlaps_the_chunk_in_flight():
    """With submit/wait the server creates newly arrived replicas while a chunk runs, so host
    creation time hides behind device time; every request still gets exactly its steps."""
    reqs = [Request(k, cells=10, T=300.0, B=(0, 0, 0), n_steps=200 + 50 * k, arrival=0.3 * k) for k in range(8)]
    results = {}
    for name, cls in (("sync", SlowCreateBackend), ("overlap", AsyncBackend)):
        clock = FakeClock()
        be = cls(clock, capacity=10 ** 9, rate=2e6, create_s=0.4)
        out = Server(be, max_active=4, chunk=50, clock=clock).run([Request(**vars(r)) for r in reqs])
        assert out["requests"] == len(reqs) and be.used == 0
        for d in out["done"]:
            assert d.result["steps"] == d.n_steps
            assert d.finished >= d.admitted >= d.arrival
        results[name] = out["makespan_s"]
    assert results["overlap"] < results["sync"]
