"""Scheduling logic of the continuous-batching server, over a stand-in
backend on the CPU: admission by memory budget and slot count, first come
first served, removal of finished and failed jobs, latency bookkeeping."""
import numpy as np
import pytest

from paper_1503_05528_gb300.serve import Server, StreamBackend, poisson_arrivals, run_load


class FakeBackend:
    """Each job names its footprint and the number of rounds it needs; a job
    with fail=True ends in the failed state."""

    def __init__(self):
        self.live = {}
        self.order = []
        self.peak_used = 0
        self.used = 0
        self.next_id = 0
        self.steps = 0
        self.removed = []

    def footprint(self, req):
        return req.job["bytes"]

    def add(self, req):
        cid = self.next_id
        self.next_id += 1
        self.live[cid] = {"left": req.job["rounds"], "fail": req.job.get("fail", False),
                          "ticket": req.ticket}
        self.order.append(req.ticket)
        self.used += req.job["bytes"]
        self.peak_used = max(self.peak_used, self.used)
        self.bytes = getattr(self, "bytes", {})
        self.bytes[cid] = req.job["bytes"]
        return cid

    def step(self):
        self.steps += 1
        for st in self.live.values():
            st["left"] -= 1

    def poll(self, cid):
        st = self.live[cid]
        if st["left"] > 0:
            return 0
        return -1 if st["fail"] else 1

    def fetch(self, cid):
        return ("result", self.live[cid]["ticket"])

    def remove(self, cid):
        self.removed.append(cid)
        self.used -= self.bytes.pop(cid)
        del self.live[cid]


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1.0
        return self.t


def _mask():
    m = np.zeros((2, 4, 4), np.uint8)
    m[0, 1, 1] = 1
    return m


def _server(budget, slots=64):
    be = FakeBackend()
    return be, Server(be, budget, max_slots=slots, clock=FakeClock())


def test_budget_never_exceeded_and_fcfs():
    be, srv = _server(budget=100)
    sizes = [60, 30, 50, 20, 90, 10, 40]
    for i, b in enumerate(sizes):
        srv.submit(None, _mask(), bytes=b, rounds=1 + i % 3)
    while srv.step():
        assert srv.used <= 100
    assert be.peak_used <= 100
    assert be.order == list(range(len(sizes)))          # admitted in arrival order
    assert len(srv.done) == len(sizes) and srv.used == 0
    for t, r in srv.done.items():
        assert r.result == ("result", t)
        assert r.arrival <= r.admitted <= r.finished


def test_head_of_line_waits_for_memory():
    be, srv = _server(budget=100)
    srv.submit(None, _mask(), bytes=70, rounds=3)
    srv.submit(None, _mask(), bytes=50, rounds=1)       # does not fit beside the first
    srv.submit(None, _mask(), bytes=10, rounds=1)       # would fit, but FCFS keeps it behind
    srv.step()
    assert [r.ticket for r in srv.running.values()] == [0]
    assert [r.ticket for r in srv.queue] == [1, 2]
    while srv.step():
        pass
    assert be.order == [0, 1, 2]


def test_slot_limit():
    be, srv = _server(budget=10**9, slots=3)
    for i in range(10):
        srv.submit(None, _mask(), bytes=1, rounds=2)
    seen = 0
    while srv.step():
        seen = max(seen, len(srv.running))
        assert len(srv.running) <= 3
    assert srv.max_concurrent == 3 and seen <= 3
    assert len(srv.done) == 10


def test_oversize_rejected_at_submit():
    be, srv = _server(budget=100)
    with pytest.raises(ValueError):
        srv.submit(None, _mask(), bytes=101, rounds=1)
    assert srv.pending() == 0 and srv.next_ticket == 0


def test_failed_job_frees_its_memory():
    be, srv = _server(budget=100)
    srv.submit(None, _mask(), bytes=80, rounds=1, fail=True)
    srv.submit(None, _mask(), bytes=80, rounds=1)
    while srv.step():
        pass
    assert srv.done[0].info.get("failed") and srv.done[0].result is None
    assert srv.done[1].result == ("result", 1)
    assert srv.used == 0 and sorted(be.removed) == [0, 1]


def test_job_done_at_admission_is_collected_without_a_round():
    be, srv = _server(budget=100)
    srv.submit(None, _mask(), bytes=10, rounds=0)       # e.g. a clip with nothing to fill
    assert not srv.step()
    assert be.steps == 0 and srv.done[0].result == ("result", 0)


def test_hole_voxels_counted():
    be, srv = _server(budget=100)
    m = np.zeros((3, 5, 5), np.uint8)
    m[1, 2:4, 1:4] = 1
    srv.submit(None, m, bytes=1, rounds=1)
    assert srv.queue[0].hole_voxels == 6


def test_poisson_arrivals():
    a = poisson_arrivals(20000, 4.0, seed=7)
    assert np.all(np.diff(a) > 0)
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert abs(gaps.mean() - 0.25) < 0.01               # mean gap 1/rate
    assert abs(gaps.std() - 0.25) < 0.01                # exponential: std = mean
    assert np.array_equal(a, poisson_arrivals(20000, 4.0, seed=7))


def test_run_load_feeds_by_arrival_time():
    be, srv = _server(budget=100)
    clock = FakeClock()
    srv.clock = clock
    reqs = [(None, _mask(), {"bytes": 30, "rounds": 2}) for _ in range(6)]
    arrivals = np.array([0.5, 1.0, 40.0, 41.0, 42.0, 43.0])
    wall, srv = run_load(srv, reqs, arrivals, clock=clock)
    assert len(srv.done) == 6 and srv.pending() == 0
    lat = srv.latencies()
    assert lat.shape == (6,) and np.all(lat > 0)
    for r in srv.done.values():
        assert r.admitted >= r.arrival


def test_stream_priority_by_size():
    # smaller requests get higher priority (lower number); the largest get 0
    p = [StreamBackend.priority(v) for v in (1, 1_999_999, 2_000_000, 7_999_999, 8_000_000, 31_999_999,
                                             32_000_000, 10 ** 9)]
    assert p == [-3, -3, -2, -2, -1, -1, 0, 0]


class FakeNativeServer:
    """Stands in for vi.Server (the library's server): every request finishes
    after a number of polls; a request with fail=True ends in the failed
    state and its release raises."""

    def __init__(self, hbm_budget, max_slots=8, **defaults):
        self.jobs = {}
        self.next = 1
        self.closed = False

    def submit(self, rgb, mask, out=None, **job):
        t = self.next
        self.next += 1
        self.jobs[t] = {"left": job.get("polls", 1), "fail": job.get("fail", False), "rgb": rgb}
        return t

    def poll(self, t):
        j = self.jobs[t]
        if j["left"] > 0:
            j["left"] -= 1
            return 0
        return -1 if j["fail"] else 1

    def wait(self, t, timeout=-1.0):
        j = self.jobs[t]
        return 0 if j["left"] > 0 else (-1 if j["fail"] else 1)

    def release(self, t):
        j = self.jobs.pop(t)
        if j["fail"]:
            from paper_1503_05528_gb300 import vi
            raise vi.ViError(6, "request failed: planted")
        return ("result", j["rgb"])

    def info(self):
        return dict(queued=0, running=sum(1 for j in self.jobs.values() if j["left"] > 0), bytes_in_use=0)

    def close(self):
        self.closed = True


def test_native_front_bookkeeping(monkeypatch):
    # NativeServer (the submit/step front over vi_server_*): tickets numbered
    # from 0 in arrival order, results handed back with their latency,
    # failures recorded with the library's message, the server closed
    from paper_1503_05528_gb300 import serve, vi
    monkeypatch.setattr(vi, "Server", FakeNativeServer)

    class Clock:
        t = 0.0

        def __call__(self):
            return self.t

    clock = Clock()
    srv = serve.NativeServer(1 << 30, 4, clock=clock)
    t0 = srv.submit("a", None, arrival=0.0, polls=2)
    t1 = srv.submit("b", None, arrival=0.5, polls=0, fail=True)
    t2 = srv.submit("c", None, arrival=1.0, polls=1)
    assert (t0, t1, t2) == (0, 1, 2)
    clock.t = 2.0
    while srv.step():
        clock.t += 1.0
    assert srv.pending() == 0 and set(srv.done) == {0, 1, 2}
    assert srv.done[0].result == ("result", "a") and srv.done[2].result == ("result", "c")
    assert srv.done[1].info.get("failed") and "planted" in srv.done[1].info["error"]
    # finished at the step that saw them done: t = 2 (failed), 3, 4
    assert {t: r.latency for t, r in srv.done.items()} == {0: 4.0, 1: 1.5, 2: 2.0}
    srv.close()
    assert srv.srv.closed
