"""Host logic of the continuous-batching server, on a fake slot pool (CPU)."""
import threading

import numpy as np

from paper_2512_24840_gb300.server import RUNNING, Server, latency_percentiles


class FakePool:
    """Each admitted request needs theta0[0] Adam steps; one step() runs at
    most `budget` of them per slot."""

    def __init__(self, n_slots):
        self.n_slots = n_slots
        self.need = np.zeros(n_slots, dtype=int)
        self.done = np.zeros(n_slots, dtype=int)
        self.status = np.zeros(n_slots, dtype=np.int32)
        self.theta = np.zeros((n_slots, 5), dtype=np.float32)
        self.admitted = []

    def admit(self, slots, reqs):
        for s, q in zip(slots, reqs):
            assert self.status[s] != RUNNING
            self.need[s] = int(q.theta0[0])
            self.done[s] = 0
            self.status[s] = RUNNING
            self.theta[s] = q.theta0
            self.admitted.append(q.rid)

    def step(self, budget, n_running=None):
        run = self.status == RUNNING
        # the scheduler sizes the launch by its count of running slots
        assert n_running is None or n_running == int(run.sum())
        self.done[run] += np.minimum(budget, self.need[run] - self.done[run])
        fin = run & (self.done >= self.need)
        self.status[fin] = 1

    def fetch(self):
        pass

    def wait(self):
        return self.status.copy(), self.theta.copy(), np.zeros(self.n_slots), self.done.copy()


def _req(steps):
    th = np.zeros(5, dtype=np.float32)
    th[0] = steps
    return np.zeros(4), np.zeros(4), np.ones(4, np.uint8), th


def test_admission_refill_and_retirement():
    pools = {"a": FakePool(3), "b": FakePool(2)}
    t = [0.0]
    srv = Server(pools, chunk=10, clock=lambda: t[0])
    steps = [5, 35, 10, 20, 15, 40, 5]
    ids = [srv.submit("a" if k % 2 == 0 else "b", *_req(s)) for k, s in enumerate(steps)]
    seen = {}
    ticks = 0
    while srv.pending():
        t[0] += 1.0
        for r in srv.tick():
            seen[r.rid] = r
        ticks += 1
        assert ticks < 100
        for name, p in pools.items():
            lane = srv.lanes[name]
            assert len(lane.busy) + len(lane.free) == p.n_slots
    assert sorted(seen) == ids
    for rid, r in seen.items():
        assert r.steps == steps[rid] and r.status == 1
        assert r.theta[0] == steps[rid]
        # a request needing s steps spends ceil(s / chunk) ticks on a slot
        assert r.latency >= np.ceil(steps[rid] / 10)
    # FIFO admission per lane
    assert pools["a"].admitted == [0, 2, 4, 6]
    assert pools["b"].admitted == [1, 3, 5]


def test_latency_percentiles_and_threaded_submit():
    pools = {"a": FakePool(4)}
    t = [0.0]
    srv = Server(pools, chunk=3, clock=lambda: t[0])
    ths = [threading.Thread(target=lambda k=k: [srv.submit("a", *_req(1 + (k + j) % 7))
                                                 for j in range(25)]) for k in range(4)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    assert srv.pending() == 100
    res = []
    while srv.pending():
        t[0] += 1.0
        res += srv.tick()
    assert len(res) == 100 and len({r.rid for r in res}) == 100
    pct = latency_percentiles(res)
    assert 0 < pct["p50_ms"] <= pct["p99_ms"]


def test_stalled_producer_does_not_block_ticks():
    """A producer thread that stops in mid-stream (here: waits on an event
    that the test sets later) leaves the scheduler usable: ticks return the
    fits already submitted, idle ticks return nothing at once, and the rest
    complete once the producer resumes.  A producer that dies with an
    exception leaves no half-submitted request behind."""
    pools = {"a": FakePool(2)}
    t = [0.0]
    srv = Server(pools, chunk=4, clock=lambda: t[0])
    go_on = threading.Event()
    first = threading.Event()

    def producer():
        for s in (3, 6, 2):
            srv.submit("a", *_req(s))
        first.set()
        go_on.wait(timeout=30)
        for s in (5, 1):
            srv.submit("a", *_req(s))
        raise RuntimeError("producer dies after its last request")

    errors = []
    th = threading.Thread(target=lambda: _catch(producer, errors))
    th.start()
    assert first.wait(timeout=30)
    done = []
    for _ in range(10):                      # the producer is stalled meanwhile
        t[0] += 1.0
        done += srv.tick()
    assert sorted(r.rid for r in done) == [0, 1, 2]
    assert srv.pending() == 0
    t[0] += 1.0
    assert srv.tick() == []                  # idle tick: nothing admitted, nothing retired
    go_on.set()
    th.join(timeout=30)
    assert not th.is_alive() and len(errors) == 1
    assert srv.pending() == 2
    while srv.pending():
        t[0] += 1.0
        done += srv.tick()
    assert sorted(r.rid for r in done) == [0, 1, 2, 3, 4]
    assert all(r.status == 1 for r in done)
    assert len(srv.lanes["a"].free) == 2 and not srv.lanes["a"].busy


def _catch(fn, errors):
    try:
        fn()
    except RuntimeError as e:
        errors.append(e)


class FlakyPool(FakePool):
    """Admission fails once (as a device copy might), before anything is admitted."""

    def __init__(self, n_slots, fail_at):
        super().__init__(n_slots)
        self.calls = 0
        self.fail_at = fail_at

    def admit(self, slots, reqs):
        self.calls += 1
        if self.calls == self.fail_at:
            raise RuntimeError("admission failed")
        super().admit(slots, reqs)


def test_failed_admission_is_rolled_back():
    """An admission that raises leaves its slots free and its requests
    waiting in submission order; the next tick admits them and every request
    completes once."""
    pool = FlakyPool(3, fail_at=2)
    t = [0.0]
    srv = Server({"a": pool}, chunk=5, clock=lambda: t[0])
    ids = [srv.submit("a", *_req(s)) for s in (4, 12, 3, 7, 9)]
    done = []
    t[0] += 1.0
    done += srv.tick()                      # admits 0, 1, 2; 0 and 2 finish
    assert sorted(r.rid for r in done) == [0, 2]
    t[0] += 1.0
    try:
        srv.tick()                          # the admission of 3 and 4 fails
        raise AssertionError("the failing admission did not raise")
    except RuntimeError:
        pass
    lane = srv.lanes["a"]
    assert [q.rid for q in lane.waiting] == [3, 4]
    assert sorted(lane.free) == [0, 2] and list(lane.busy) == [1]
    assert srv.pending() == 3
    while srv.pending():
        t[0] += 1.0
        done += srv.tick()
    assert sorted(r.rid for r in done) == ids
    assert pool.admitted == [0, 1, 2, 3, 4]
