"""Host-side logic of the serving scheduler (no GPU): FIFO admission under a
slot count and a device-memory budget, with a fake executor whose requests
finish after a fixed simulated duration."""
import pytest

from paper_2001_07124_gb300.serving import Request, Scheduler, latency_summary


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeExecutor:
    def __init__(self, clock, duration, sizes):
        self.clock, self.duration, self.sizes = clock, duration, sizes
        self.started, self.live, self.max_live, self.max_bytes, self.bytes = [], 0, 0, 0, 0

    def bytes_needed(self, req):
        return self.sizes[req.rid]

    def start(self, req, slot):
        self.started.append((req.rid, slot, self.clock()))
        self.live += 1
        self.bytes += self.sizes[req.rid]
        self.max_live = max(self.max_live, self.live)
        self.max_bytes = max(self.max_bytes, self.bytes)
        return (req, self.clock() + self.duration[req.rid])

    def done(self, h):
        return self.clock() >= h[1]

    def finish(self, h):
        self.live -= 1
        self.bytes -= self.sizes[h[0].rid]
        return None, None


def run(reqs, slots, budget, duration, sizes, step=0.001):
    clock = FakeClock()
    ex = FakeExecutor(clock, duration, sizes)

    def idle():
        clock.t += step

    res = Scheduler(ex, slots, budget, clock).run(reqs, idle=idle)
    return res, ex


def test_all_requests_complete_in_arrival_order():
    reqs = [Request(i, (8, 8, 8), (2, 2, 2), arrival=0.01 * i) for i in range(20)]
    res, ex = run(reqs, slots=3, budget=10 ** 9, duration={i: 0.05 for i in range(20)},
                  sizes={i: 100 for i in range(20)})
    assert sorted(r.rid for r in res) == list(range(20))
    assert [s[0] for s in ex.started] == list(range(20))            # FIFO admission
    assert ex.max_live <= 3
    for r in res:
        assert r.admitted >= r.arrival and r.finished >= r.admitted + 0.05 - 1e-9


def test_budget_limits_concurrency_and_blocks_the_head():
    sizes = {0: 60, 1: 60, 2: 10, 3: 10}
    reqs = [Request(i, (8, 8, 8), (2, 2, 2), arrival=0.0) for i in range(4)]
    res, ex = run(reqs, slots=4, budget=100, duration={i: 0.02 for i in range(4)}, sizes=sizes)
    assert ex.max_bytes <= 100
    # request 1 does not fit next to 0; 2 and 3 wait behind it (no overtaking)
    starts = {rid: t for rid, _, t in ex.started}
    assert starts[1] >= starts[0] + 0.02 - 1e-9
    assert starts[2] >= starts[1] and starts[3] >= starts[1]
    assert len(res) == 4


def test_request_larger_than_budget_is_rejected():
    reqs = [Request(0, (8, 8, 8), (2, 2, 2), arrival=0.0)]
    with pytest.raises(ValueError):
        run(reqs, slots=1, budget=10, duration={0: 0.01}, sizes={0: 11})


def test_latency_summary():
    reqs = [Request(i, (8, 8, 8), (2, 2, 2), arrival=0.0) for i in range(10)]
    res, _ = run(reqs, slots=1, budget=10 ** 9, duration={i: 0.01 for i in range(10)},
                 sizes={i: 1 for i in range(10)})
    s = latency_summary(res)
    assert s["requests"] == 10 and s["p99_ms"] >= s["p50_ms"] > 0
    assert s["decomps_per_s"] == pytest.approx(10 / max(r.finished for r in res), rel=1e-6)
