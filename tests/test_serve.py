"""The serving loop's admission, memory accounting, failure handling and latency
bookkeeping, on a fake device and a fake clock (no GPU)."""
import pytest

from paper_2304_13746_b300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def now(self):
        return self.t

    def sleep_until(self, t):
        self.t = max(self.t, t)


class FakeBackend:
    """A device that runs a batch cycle in overhead + active_cells / rate seconds; a
    request needs `cycles_of(r)` cycles and `bytes_per_cell` bytes per cell."""

    def __init__(self, clock, rate=1e6, overhead=1e-3, bytes_per_cell=100, fail=()):
        self.clock, self.rate, self.overhead = clock, rate, overhead
        self.bpc = bytes_per_cell
        self.fail = set(fail)
        self.active = {}
        self.max_active = 0
        self.started = []

    @staticmethod
    def cycles_of(r):
        return 10 + r.n % 7

    def footprint(self, r):
        return r.n * r.n * self.bpc

    def start(self, r):
        if r.rid in self.fail:
            raise RuntimeError("non-physical initial state")
        self.active[r.rid] = [r, 0]
        self.started.append(r.rid)
        self.max_active = max(self.max_active, len(self.active))

    def step(self, k):
        for _ in range(k):
            live = [v for v in self.active.values() if v[1] < self.cycles_of(v[0])]
            if not live:
                return
            cells = sum(v[0].n * v[0].n for v in live)
            self.clock.t += self.overhead + cells / self.rate
            for v in live:
                v[1] += 1

    def poll(self):
        return [rid for rid, v in self.active.items() if v[1] >= self.cycles_of(v[0])]

    def finish(self, rid):
        r, c = self.active.pop(rid)
        return ["state"], c

    # one at a time
    def serve_one(self, r):
        if r.rid in self.fail:
            raise RuntimeError("non-physical initial state")
        for _ in range(self.cycles_of(r)):
            self.clock.t += self.overhead + r.n * r.n / self.rate
        return ["state"], self.cycles_of(r)


def stream(n=40, rate=50.0, seed=3):
    reqs = serve.poisson_stream(n, rate, seed=seed, sizes_2d=(16, 64), sizes_3d=(16, 64))
    for r in reqs:
        r.cells = r.n * r.n
    return reqs


def test_all_served_within_budget_oldest_first():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = stream()
    budget = 3 * 64 * 64 * 100
    st = serve.Server(be, budget, clock, cycles_per_poll=4).run(reqs)
    assert st["done"] == len(reqs) and st["failed"] == st["rejected"] == 0
    assert st["peak_bytes"] <= budget
    assert be.started == sorted(be.started)          # admitted oldest first
    assert all(r.admitted >= r.arrival and r.finished >= r.admitted for r in reqs)
    assert all(r.cycles == FakeBackend.cycles_of(r) for r in reqs)
    assert be.max_active > 1                          # requests overlapped on the device
    assert st["p99_s"] >= st["p50_s"] > 0


def test_oversized_request_is_rejected_without_blocking():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = stream(10)
    reqs[2].n = 1000                                  # far above the budget
    st = serve.Server(be, 2 * 64 * 64 * 100, clock).run(reqs)
    assert reqs[2].status == "rejected" and "budget" in reqs[2].error
    assert st["done"] == 9


def test_failed_start_is_reported_and_frees_nothing_twice():
    clock = FakeClock()
    be = FakeBackend(clock, fail={4, 7})
    reqs = stream(12)
    srv = serve.Server(be, 2 * 64 * 64 * 100, clock)
    st = srv.run(reqs)
    assert [r.rid for r in reqs if r.status == "failed"] == [4, 7]
    assert st["done"] == 10 and srv.used == 0


def test_latency_hand_computed():
    clock = FakeClock()
    be = FakeBackend(clock, rate=1e4, overhead=0.0)
    a = serve.Request(0, 0.0, "2d", 100, 0.1, 0)     # 10 + 100 % 7 = 12 cycles, 1 s each alone
    b = serve.Request(1, 0.5, "2d", 100, 0.1, 1)
    for r in (a, b):
        r.cells = r.n * r.n
    st = serve.Server(be, 10 ** 9, clock, cycles_per_poll=1).run([a, b])
    # pipelined loop: a runs alone for two 1 s cycles (b arrives during the first and joins
    # at the boundary t = 2); both then take 2 s per cycle, a's 12th cycle ends at t = 22
    # and its result is read while b's 11th... b runs its last cycle alone (t = 23, 24):
    # a is read back at t = 23, b finishes at t = 24
    assert a.finished == pytest.approx(23.0) and b.finished == pytest.approx(24.0)
    assert st["p50_s"] == pytest.approx(0.5 * ((23.0 - 0.0) + (24.0 - 0.5)))


def test_batching_beats_one_at_a_time_on_a_launch_bound_device():
    reqs1, reqs2 = stream(40, rate=200.0), stream(40, rate=200.0)
    c1, c2 = FakeClock(), FakeClock()
    st_b = serve.Server(FakeBackend(c1, overhead=5e-3), 10 ** 12, c1).run(reqs1)
    st_s = serve.serve_sequential(FakeBackend(c2, overhead=5e-3), reqs2, c2)
    assert st_b["cell_updates"] == st_s["cell_updates"]
    assert st_b["cell_updates_per_s"] > 2 * st_s["cell_updates_per_s"]
    assert st_b["p99_s"] < st_s["p99_s"]


def test_stream_is_seeded():
    a = serve.poisson_stream(20, 10.0, seed=7)
    b = serve.poisson_stream(20, 10.0, seed=7)
    assert [(r.arrival, r.kind, r.n, r.t_end) for r in a] == [(r.arrival, r.kind, r.n, r.t_end) for r in b]
    assert all(r.n % 8 == 0 for r in a)


def test_active_cell_cap_limits_concurrency():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = stream(40, rate=500.0)
    cap = 2 * 48 * 48
    seen = []
    orig_step = be.step

    def step(k):
        seen.append(sum(v[0].cells for v in be.active.values()
                        if v[1] < FakeBackend.cycles_of(v[0])))
        orig_step(k)
    be.step = step
    st = serve.Server(be, 10 ** 12, clock, max_active_cells=cap).run(reqs)
    assert st["done"] == len(reqs)
    biggest = max(r.cells for r in reqs)
    assert max(seen) <= max(cap, biggest)


def test_least_work_order_admits_small_requests_first():
    clock = FakeClock()
    be = FakeBackend(clock)
    reqs = stream(12)
    for r in reqs:
        r.arrival = 0.0                               # all arrive at once
    budget = 64 * 64 * 100                            # one large request's worth
    st = serve.Server(be, budget, clock, cycles_per_poll=2, order="least_work").run(reqs)
    assert st["done"] == len(reqs)
    work = {r.rid: serve.estimated_work(r) for r in reqs}
    started = [work[rid] for rid in be.started]
    # whenever the device frees up, the smallest waiting request goes next: the start
    # order is the work order
    assert started == sorted(started)
    with pytest.raises(ValueError):
        serve.Server(be, budget, clock, order="largest")
