"""Serving scheduler on a simulated device (no GPU): continuous batching
under an HBM budget, per-slot concurrency, rejection of requests that can
never fit, FIFO admission, latency accounting."""
import pytest

from paper_2410_13474_gb300.serving import Request, Scheduler, SimExecutor, percentile, poisson_arrivals


def _reqs(n, rate, sizes, seed=0):
    t = poisson_arrivals(n, rate, seed)
    return [Request(i, 0, None, float(t[i]), ws_bytes=sizes[i % len(sizes)]) for i in range(n)]


def test_all_complete_and_budget_respected():
    ex = SimExecutor(fixed=2e-3, per_byte=1e-11)
    sched = Scheduler(ex, budget_bytes=10 * 2**20, slots=2, max_batch=8, clock=ex.clock)
    reqs = _reqs(300, 500.0, [2**20, 3 * 2**20, 512 * 1024])
    st = sched.run(reqs)
    assert st.completed == 300 and st.rejected == 0
    assert st.max_inflight_bytes <= 10 * 2**20
    for r in reqs:
        assert r.t_admit >= r.t_arrival - 1e-12 and r.t_done > r.t_admit
    # at most `slots` batches overlap at any time
    ev = sorted([(t, +1) for _, _, t in ex.launched] + [(e, -1) for e in ex.ends])
    cur = peak = 0
    for _, d in ev:
        cur += d
        peak = max(peak, cur)
    assert peak <= 2


def test_continuous_batching_batches_arrivals_while_busy():
    ex = SimExecutor(fixed=20e-3, per_byte=0.0)  # slow device: arrivals queue up
    sched = Scheduler(ex, budget_bytes=64 * 2**20, slots=2, max_batch=16, clock=ex.clock)
    st = sched.run(_reqs(200, 1000.0, [2**20]))
    assert st.completed == 200
    assert st.mean_batch > 4          # requests that arrived during a batch were grouped
    assert st.batches < 200


def test_fifo_admission_and_rejection_of_oversized():
    ex = SimExecutor(fixed=1e-3)
    sched = Scheduler(ex, budget_bytes=4 * 2**20, slots=2, max_batch=4, clock=ex.clock)
    reqs = _reqs(50, 200.0, [2**20, 5 * 2**20, 3 * 2**20])  # 5 MiB exceeds the budget
    st = sched.run(reqs)
    assert st.rejected == 17 and st.completed == 33
    assert all(r.status == -2 for r in reqs if r.ws_bytes > 4 * 2**20)
    assert st.max_inflight_bytes <= 4 * 2**20
    order = [rid for _, rids, _ in ex.launched for rid in rids]
    assert order == sorted(order)     # admitted in arrival order


def test_latency_percentiles():
    assert percentile([1, 2, 3, 4, 5], 0.5) == 3
    assert abs(percentile(list(range(101)), 0.99) - 99.0) < 1e-9
    ex = SimExecutor(fixed=5e-3)
    sched = Scheduler(ex, budget_bytes=2**30, slots=1, max_batch=1, clock=ex.clock)
    reqs = [Request(i, 0, None, 0.1 * (i + 1), ws_bytes=1) for i in range(20)]
    st = sched.run(reqs)   # arrivals 100 ms apart on a 5 ms device: latency = service time
    assert abs(st.p50_ms - 5.0) < 1e-6 and abs(st.p99_ms - 5.0) < 1e-6
    # back-to-back arrivals on one slot queue behind each other
    ex = SimExecutor(fixed=5e-3)
    sched = Scheduler(ex, budget_bytes=2**30, slots=1, max_batch=1, clock=ex.clock)
    st = sched.run([Request(i, 0, None, 0.0, ws_bytes=1) for i in range(4)])
    assert abs(st.p99_ms - 19.85) < 0.2 and abs(st.wall_s - 0.02) < 1e-9


def test_overlap_guard_keeps_large_batches_apart():
    """With overlap_bytes set, two batches above it never run at once, and a
    small batch may start beside a large one."""
    big, small = 8 * 2**20, 2**20
    ex = SimExecutor(fixed=1e-3, per_byte=1e-9)
    sched = Scheduler(ex, budget_bytes=2**30, slots=2, max_batch=1, clock=ex.clock,
                      overlap_bytes=4 * 2**20)
    reqs = _reqs(200, 400.0, [big, small, big, small, small])
    st = sched.run(reqs)
    assert st.completed == 200
    size = {r.rid: r.ws_bytes for r in reqs}
    spans = [(t, e, sum(size[i] for i in rids)) for (_, rids, t), e in zip(ex.launched, ex.ends)]
    overlapped_small = 0
    for k, (t0, e0, b0) in enumerate(spans):
        for t1, e1, b1 in spans[k + 1:]:
            if t1 < e0 and t0 < e1:          # the two batches overlap in time
                assert not (b0 > 4 * 2**20 and b1 > 4 * 2**20)
                overlapped_small += 1
    assert overlapped_small > 0


def test_adaptive_batching_only_batches_a_backlog():
    """batch_queue = 4: batches of more than one request start only from a
    queue of at least four; under light load every request runs alone."""
    ex = SimExecutor(fixed=1e-3)
    sched = Scheduler(ex, budget_bytes=2**30, slots=1, max_batch=16, clock=ex.clock, batch_queue=4)
    st = sched.run(_reqs(200, 50.0, [2**20]))     # 50/s on a 1 ms device: no queue
    assert st.completed == 200 and st.mean_batch == 1.0
    ex = SimExecutor(fixed=20e-3)
    sched = Scheduler(ex, budget_bytes=2**30, slots=1, max_batch=16, clock=ex.clock, batch_queue=4)
    st = sched.run(_reqs(200, 1000.0, [2**20]))   # 1000/s on a 20 ms device: a backlog
    assert st.completed == 200 and st.mean_batch > 4
    assert all(len(rids) == 1 or len(rids) >= 4 for _, rids, _ in ex.launched)


def test_failed_requests_are_not_counted_as_served():
    """A request whose batch returns an error status counts as failed: it is
    left out of the completed count, the throughput and the latencies."""
    class Failing(SimExecutor):
        def launch(self, slot, batch):
            end, st = super().launch(slot, batch)
            return (end, [-2 if r.rid % 4 == 0 else 0 for r in batch])

    ex = Failing(fixed=1e-3)
    sched = Scheduler(ex, budget_bytes=2**30, slots=1, max_batch=1, clock=ex.clock)
    reqs = _reqs(100, 100.0, [2**20])
    st = sched.run(reqs)
    assert st.failed == 25 and st.completed == 75
    assert abs(st.throughput - 75 / st.wall_s) < 1e-9
