"""Host logic of the serving scheduler, with a fake backend (no GPU): FIFO admission by free
memory, head-of-line waiting, rejection of requests larger than the device, grouping, tick
sizes that never overshoot a request, harvesting that frees memory for waiting requests."""
import pytest

from paper_2010_11751_b300.serve import Request, Scheduler, summarize


class FakeBackend:
    def __init__(self, total):
        self.total = total
        self.used = 0
        self.steps = []  # (key, ids, n)
        self.live = {}

    def total_bytes(self):
        return self.total

    def free_bytes(self):
        return self.total - self.used

    def bytes_needed(self, req):
        return req.side ** 3

    def group_key(self, req):
        return (req.lattice, req.collision, req.precision)

    def start(self, req):
        self.used += self.bytes_needed(req)
        self.live[req.id] = req
        return req.id

    def step(self, key, handles, n):
        self.steps.append((key, tuple(handles), n))

    def sync(self):
        pass

    def finish(self, h):
        self.used -= self.bytes_needed(self.live.pop(h))
        return {"mass": 1.0, "energy": 0.0}


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


def req(i, side, steps, lattice=19, coll="BGK_W2", prec="f32", t=0.0):
    return Request(i, t, lattice, "cavity", coll, prec, side, steps)


def test_fifo_admission_by_free_memory():
    be = FakeBackend(total=1000)
    s = Scheduler(be, tick_steps=10, clock=Clock())
    s.t0 = 0.0
    for r in [req(0, 8, 30), req(1, 8, 30), req(2, 5, 30)]:  # 512, 512, 125 bytes
        s.offer(r)
    assert s.admit() == [0]  # request 1 does not fit; request 2 waits behind it (FIFO)
    assert [a.req.id for a in s.active] == [0]
    for _ in range(3):
        s.tick()
    assert [r.id for r in s.results] == [0]
    assert s.admit() == [1, 2]


def test_oversized_request_is_rejected_not_blocking():
    be = FakeBackend(total=100)
    s = Scheduler(be, tick_steps=4, clock=Clock())
    s.t0 = 0.0
    s.offer(req(0, 10, 5))  # 1000 bytes > device
    s.offer(req(1, 4, 5))
    assert s.admit() == [1]
    assert s.results[0].error == "request larger than the device"


def test_ticks_never_overshoot_and_group_by_kind():
    be = FakeBackend(total=10 ** 6)
    s = Scheduler(be, tick_steps=64, clock=Clock())
    s.t0 = 0.0
    s.offer(req(0, 4, 100))
    s.offer(req(1, 4, 30))
    s.offer(req(2, 4, 70, coll="K"))
    s.offer(req(3, 4, 64, lattice=27))
    s.admit()
    done = []
    while s.active:
        done += s.tick()
    assert sorted(done) == [0, 1, 2, 3]
    # per request, the steps taken sum exactly to its step count
    taken = {i: 0 for i in range(4)}
    for key, ids, n in be.steps:
        assert n >= 1
        kinds = {(r.lattice, r.collision, r.precision) for r in [req(i, 4, 1) for i in ids]}
        for i in ids:
            taken[i] += n
    assert taken == {0: 100, 1: 30, 2: 70, 3: 64}
    # groups: (19, BGK_W2) had members 0 and 1 together
    keys = {k for k, _, _ in be.steps}
    assert keys == {(19, "BGK_W2", "f32"), (19, "K", "f32"), (27, "BGK_W2", "f32")}
    first = [x for x in be.steps if x[0] == (19, "BGK_W2", "f32")][0]
    assert first[1] == (0, 1) and first[2] == 30  # min(tick, fewest remaining)


def test_continuous_admission_during_run():
    be = FakeBackend(total=2 * 512)
    clock = Clock()
    s = Scheduler(be, tick_steps=16, clock=clock)
    trace = [req(i, 8, 40 + 8 * i, t=0.002 * i) for i in range(6)]
    res = s.run(trace, time_scale=1.0, idle_sleep=0.0)
    assert [r.id for r in res] == list(range(6))
    assert all(r.error is None for r in res)
    assert s.max_active == 2  # memory admits two at a time; later ones join as others finish
    assert all(r.admitted_s >= r.arrival_s for r in res)
    summ = summarize(res, wall_s=1.0)
    assert summ["completed"] == 6 and summ["p99_latency_s"] >= summ["p50_latency_s"]


def test_memory_never_frees_is_reported():
    be = FakeBackend(total=100)
    s = Scheduler(be, clock=Clock())
    be.used = 90  # something else holds the device
    with pytest.raises(RuntimeError):
        s.run([req(0, 4, 10)], idle_sleep=0.0)


def test_queue_only_mode_runs_one_at_a_time():
    be = FakeBackend(total=10 ** 6)
    s = Scheduler(be, tick_steps=8, clock=Clock(), max_active=1)
    res = s.run([req(i, 4, 20, t=0.0) for i in range(4)], idle_sleep=0.0)
    assert s.max_active == 1 and [r.id for r in res] == [0, 1, 2, 3]
    assert all(len(ids) == 1 for _, ids, _ in be.steps)


def test_cell_budget_slots():
    be = FakeBackend(total=10 ** 9)
    s = Scheduler(be, tick_steps=8, clock=Clock(), max_active_cells=2 * 64 + 10)
    s.t0 = 0.0
    for i in range(4):
        s.offer(req(i, 4, 16))  # 64 cells each
    assert s.admit() == [0, 1]  # the third would exceed the budget
    while s.active:
        s.tick()
    assert s.admit() == [2, 3]
    s2 = Scheduler(be, clock=Clock(), max_active_cells=10)
    s2.t0 = 0.0
    s2.offer(req(9, 4, 8))  # larger than the budget alone: still admitted when nothing is active
    assert s2.admit() == [9]


def test_shortest_work_admits_small_request_past_a_blocked_large_one():
    be = FakeBackend(total=1000)
    s = Scheduler(be, tick_steps=10, clock=Clock(), policy="shortest", max_wait_s=100.0)
    s.t0 = 0.0
    s.offer(req(0, 9, 50))   # 729 cells: fits
    s.offer(req(1, 8, 50))   # 512: does not fit beside request 0
    s.offer(req(2, 4, 10))   # 64: fits
    # least work first: 2 (640 cell-steps), then 1 (25600) -- which does not fit once 2 is in?
    assert s.admit() == [2, 1]  # 64 + 512 = 576 <= 1000; request 0 (36450) no longer fits
    assert [r.id for r in s.pending] == [0]
    f = Scheduler(FakeBackend(total=1000), tick_steps=10, clock=Clock(), policy="fifo")
    f.t0 = 0.0
    for r in (req(0, 9, 50), req(1, 8, 50), req(2, 4, 10)):
        f.offer(r)
    assert f.admit() == [0]  # FIFO: request 1 blocks the head of the line, 2 waits behind it


def test_aged_request_goes_first_and_blocks_others_until_it_fits():
    be = FakeBackend(total=1000)
    clock = Clock()
    s = Scheduler(be, tick_steps=10, clock=clock, policy="shortest", max_wait_s=0.5)
    s.t0 = 0.0
    s.offer(req(0, 9, 40, t=0.0))
    assert s.admit() == [0]
    s.offer(req(1, 8, 400, t=0.0))  # 512 cells: waits for 0
    clock.t = 1.0                    # request 1 has now waited longer than max_wait_s
    s.offer(req(2, 2, 4, t=0.9))     # tiny and recent: would fit, but the aged request goes first
    assert s.admit() == []
    while s.active:
        s.tick()
    assert s.admit() == [1, 2]


def test_timed_ticks_use_the_backend_estimate():
    class Timed(FakeBackend):
        def step_seconds(self, key, cells):
            return None if key[1] == "K" else 1e-4 * cells / 64.0

    be = Timed(total=10 ** 6)
    s = Scheduler(be, tick_steps=7, clock=Clock(), tick_seconds=0.002)
    s.t0 = 0.0
    s.offer(req(0, 4, 100))                # 64 cells: 1e-4 s per step -> 20 steps per tick
    s.offer(req(1, 8, 100, lattice=27))    # other group, 512 cells: 8e-4 s per step -> 2 steps
    s.offer(req(2, 4, 100, coll="K"))      # no estimate: tick_steps
    s.admit()
    s.tick()
    got = {ids: n for _, ids, n in be.steps}
    assert got == {(0,): 20, (1,): 2, (2,): 7}
    s.offer(req(3, 4, 3))
    s.admit()
    be.steps.clear()
    s.tick()
    got = {ids: n for _, ids, n in be.steps}
    assert got[(0, 3)] == 3  # never past the member with the fewest remaining steps


def test_unknown_policy_is_refused():
    with pytest.raises(ValueError):
        Scheduler(FakeBackend(total=10), policy="lifo")
