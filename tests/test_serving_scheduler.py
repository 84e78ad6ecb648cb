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
        self.released = []

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

    def release(self, slot):
        self.released.append(slot)


def run(reqs, slots, budget, duration, sizes, step=0.001):
    clock = FakeClock()
    ex = FakeExecutor(clock, duration, sizes)

    def idle():
        clock.t += step

    sched = Scheduler(ex, slots, budget, clock)
    res = sched.run(reqs, idle=idle)
    ex.sched = sched
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


class HoldingExecutor(FakeExecutor):
    """A fake executor whose slots keep their buffers after a request, as the GPU
    executor's arenas do: a slot holds the largest request it has run until it
    is released."""

    def __init__(self, clock, duration, sizes, slots):
        super().__init__(clock, duration, sizes)
        self.hold = [0] * slots
        self.max_hold = 0

    def start(self, req, slot):
        self.hold[slot] = max(self.hold[slot], self.sizes[req.rid])
        self.max_hold = max(self.max_hold, sum(self.hold))
        return super().start(req, slot)

    def release(self, slot):
        super().release(slot)
        self.hold[slot] = 0


def test_slot_holdings_never_exceed_the_budget():
    """Retained slot buffers count against the budget: a large request that
    ran on one slot keeps that slot's memory after it retires, so the next
    large request must reuse it or release it, never stack on top of it."""
    import random
    rnd = random.Random(5)
    n, slots, budget = 60, 4, 1000
    sizes = {i: rnd.choice([50, 120, 300, 700]) for i in range(n)}
    reqs = [Request(i, (8, 8, 8), (2, 2, 2), arrival=0.003 * i) for i in range(n)]
    clock = FakeClock()
    ex = HoldingExecutor(clock, {i: 0.01 + 0.02 * rnd.random() for i in range(n)}, sizes, slots)

    def idle():
        clock.t += 0.001

    sched = Scheduler(ex, slots, budget, clock)
    res = sched.run(reqs, idle=idle)
    assert sorted(r.rid for r in res) == list(range(n))
    assert ex.max_hold <= budget and sched.peak_held <= budget
    assert ex.released                                   # the 700s forced idle slots to give memory back
    assert sum(ex.hold) == sum(sched.held)               # both sides agree on what is held


def test_best_fit_reuses_a_covering_slot():
    sizes = {0: 500, 1: 100, 2: 450}
    reqs = [Request(0, (8, 8, 8), (2, 2, 2), arrival=0.0), Request(1, (8, 8, 8), (2, 2, 2), arrival=0.0),
            Request(2, (8, 8, 8), (2, 2, 2), arrival=0.05)]
    clock = FakeClock()
    ex = HoldingExecutor(clock, {0: 0.01, 1: 0.01, 2: 0.01}, sizes, 2)

    def idle():
        clock.t += 0.001

    sched = Scheduler(ex, 2, 700, clock)
    sched.run(reqs, idle=idle)
    slot_of = {rid: slot for rid, slot, _ in ex.started}
    assert slot_of[2] == slot_of[0]                      # 450 fits in the 500 the first slot holds
    assert not ex.released and sched.peak_held == 600
