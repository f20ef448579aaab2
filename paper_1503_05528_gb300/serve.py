"""Inpainting server on one GPU: admission by an HBM budget, requests
running concurrently.

Requests (a clip and its occlusion mask) queue in arrival order. The server
admits queued requests while their device footprint (``vi_footprint_bytes``)
fits the HBM budget and a slot is free, and hands a finished request back at
once, which frees its memory and slot for the next one. Two backends run the
admitted requests:

- ``CudaBackend``: continuous batching (``vi_batch_*``). An admitted request
  joins the running batch, and every round runs one search/reconstruction
  iteration of every request in shared launches.
- ``StreamBackend``: every request runs alone (``vi_run``) in a worker thread
  on a stream of its own, smaller requests on higher-priority streams; the
  GPU interleaves the streams, so a small request is not held back to the pace
  of a large one.

``NativeServer`` offers the same front (submit / step / pending / done) over
the library's own server (``vi_server_*``), which does the admission and the
per-request streams in C++ worker threads.

Either way every job's result is bit-identical to running it alone. The
scheduling logic is plain Python over a small backend interface
(add / step / poll / fetch / remove / footprint), so it runs unchanged over
either backend or over a stand-in in tests.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    ticket: int
    rgb: object
    mask: object
    job: dict
    arrival: float                       # time.perf_counter() seconds
    footprint: int = 0
    admitted: float = None
    finished: float = None
    clip_id: int = None
    result: object = None
    hole_voxels: int = 0
    info: dict = field(default_factory=dict)

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


def _footprint(vi, defaults, req):
    import ctypes
    T, H, W = req.mask.shape[:3]
    cfg = vi.default_config(**{**defaults, **req.job})
    return int(vi.load().vi_footprint_bytes(ctypes.byref(cfg), W, H, T, int(req.hole_voxels)))


class CudaBackend:
    """The vi_batch of the CUDA library (continuous batching)."""

    def __init__(self, stream=None, **cfg):
        from . import vi
        self.vi = vi
        self.batch = vi.Batch(stream=stream, **cfg)
        self.cfg = vi.default_config(**cfg)

    def footprint(self, req):
        return _footprint(self.vi, self.batch.defaults, req)

    def add(self, req):
        return self.batch.add(req.rgb, req.mask, **req.job)

    def step(self):
        return self.batch.step()

    def poll(self, cid):
        return self.batch.poll(cid)[0]

    def fetch(self, cid):
        return self.batch.fetch(cid)

    def remove(self, cid):
        self.batch.remove(cid)

    def close(self):
        self.batch.close()


class StreamBackend:
    """Every admitted request runs alone through vi_run in a worker thread, on
    a stream the context creates with a priority by size: requests under
    2M / 8M / 32M voxels get the three highest priorities, larger ones the
    default. Stream-ordered device memory in the library keeps one request's
    allocation and release from stalling the others."""

    SIZE_CUTS = (2_000_000, 8_000_000, 32_000_000)

    def __init__(self, max_workers=8, device=None, **cfg):
        from concurrent.futures import ThreadPoolExecutor

        from . import vi
        self.vi = vi
        self.cfg = dict(cfg)
        init = None
        if device is not None:
            def init():
                import torch
                torch.cuda.set_device(device)
        self.pool = ThreadPoolExecutor(max_workers, initializer=init)
        self.jobs = {}
        self.next_id = 0

    def footprint(self, req):
        return _footprint(self.vi, self.cfg, req)

    @classmethod
    def priority(cls, voxels):
        import bisect
        return bisect.bisect_right(cls.SIZE_CUTS, voxels) - len(cls.SIZE_CUTS)

    def _run(self, rgb, mask, job):
        with self.vi.Context(**job) as ctx:
            ctx.upload(rgb, mask)
            ctx.run()
            return ctx.fetch_result()

    def add(self, req):
        voxels = int(np.prod(req.mask.shape[:3]))
        job = {**self.cfg, **req.job, "stream_priority": self.priority(voxels)}
        cid = self.next_id
        self.next_id += 1
        self.jobs[cid] = self.pool.submit(self._run, req.rgb, req.mask, job)
        return cid

    def step(self):
        from concurrent.futures import FIRST_COMPLETED, wait
        if self.jobs:
            wait(list(self.jobs.values()), timeout=0.002, return_when=FIRST_COMPLETED)

    def poll(self, cid):
        f = self.jobs[cid]
        if not f.done():
            return 0
        return -1 if f.exception() is not None else 1

    def fetch(self, cid):
        return self.jobs[cid].result()

    def remove(self, cid):
        self.jobs.pop(cid, None)

    def close(self):
        self.pool.shutdown(wait=True)


class Server:
    """Admission by footprint, continuous batching, per-request latency."""

    def __init__(self, backend, hbm_budget, max_slots=64, clock=time.perf_counter):
        self.backend = backend
        self.budget = int(hbm_budget)
        self.max_slots = int(max_slots)
        self.clock = clock
        self.queue = deque()
        self.running = {}            # clip id -> Request
        self.done = {}               # ticket -> Request
        self.used = 0
        self.next_ticket = 0
        self.max_concurrent = 0
        self.rounds = 0

    def submit(self, rgb, mask, arrival=None, **job):
        req = Request(self.next_ticket, rgb, mask, job, self.clock() if arrival is None else arrival)
        req.hole_voxels = int(np.count_nonzero(np.asarray(mask)))
        req.footprint = self.backend.footprint(req)
        if req.footprint > self.budget:
            raise ValueError(f"request needs {req.footprint} bytes, budget is {self.budget}")
        self.next_ticket += 1
        self.queue.append(req)
        return req.ticket

    def _admit(self):
        while self.queue and len(self.running) < self.max_slots:
            req = self.queue[0]
            if self.used + req.footprint > self.budget:
                break                            # first come, first served: wait for memory
            self.queue.popleft()
            req.admitted = self.clock()
            req.clip_id = self.backend.add(req)
            self.used += req.footprint
            self.running[req.clip_id] = req
        self.max_concurrent = max(self.max_concurrent, len(self.running))

    def _collect(self):
        for cid in list(self.running):
            state = self.backend.poll(cid)
            if state == 0:
                continue
            req = self.running.pop(cid)
            if state == 1:
                req.result = self.backend.fetch(cid)
            else:
                req.info["failed"] = True
            req.finished = self.clock()
            self.backend.remove(cid)
            self.used -= req.footprint
            self.done[req.ticket] = req

    def step(self):
        """Admit what fits, run one round, hand back what finished. Returns
        True while work is queued or running."""
        self._admit()
        self._collect()                          # jobs finished during preparation
        if self.running:
            self.backend.step()
            self.rounds += 1
            self._collect()
        return bool(self.queue or self.running)

    def pending(self):
        return len(self.queue) + len(self.running)

    def latencies(self):
        return np.array([r.latency for r in self.done.values() if r.latency is not None])


class NativeServer:
    """The library's server (vi_server_*: FCFS admission by footprint and a
    slot limit, one worker thread and one size-priority stream per running
    request) behind the front of ``Server``; step() hands back finished
    requests and waits briefly on the oldest running one."""

    def __init__(self, hbm_budget, max_slots=8, clock=time.perf_counter, **cfg):
        from . import vi
        self.srv = vi.Server(hbm_budget, max_slots, **cfg)
        self.clock = clock
        self.running = {}            # native ticket -> Request
        self.done = {}               # ticket -> Request
        self.next_ticket = 0
        self.max_concurrent = 0
        self.rounds = 0

    def submit(self, rgb, mask, arrival=None, **job):
        req = Request(self.next_ticket, rgb, mask, job, self.clock() if arrival is None else arrival)
        native = self.srv.submit(rgb, mask, **job)
        req.admitted = self.clock()
        self.next_ticket += 1
        self.running[native] = req
        return req.ticket

    def step(self):
        for native in list(self.running):
            state = self.srv.poll(native)
            if state == 0:
                continue
            req = self.running.pop(native)
            req.finished = self.clock()
            try:
                req.result = self.srv.release(native)
            except Exception as e:   # the request failed: keep the message
                req.info["failed"] = True
                req.info["error"] = str(e)
            self.done[req.ticket] = req
        self.max_concurrent = max(self.max_concurrent, self.srv.info()["running"])
        if self.running:
            self.rounds += 1
            self.srv.wait(next(iter(self.running)), 0.001)
        return bool(self.running)

    def pending(self):
        return len(self.running)

    def latencies(self):
        return np.array([r.latency for r in self.done.values() if r.latency is not None])

    def close(self):
        self.srv.close()


def poisson_arrivals(n, rate, seed):
    """n arrival times (seconds from 0) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def run_load(server, requests, arrivals, clock=time.perf_counter):
    """Feeds requests (rgb, mask, job) at the given arrival offsets, steps the
    server until everything finished; returns (wall seconds, server)."""
    t0 = clock()
    i = 0
    while i < len(requests) or server.pending():
        now = clock() - t0
        while i < len(requests) and arrivals[i] <= now:
            rgb, mask, job = requests[i]
            server.submit(rgb, mask, arrival=t0 + arrivals[i], **job)
            i += 1
        if not server.step() and i < len(requests):
            # idle until the next arrival
            wait = arrivals[i] - (clock() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.05))
    return clock() - t0, server
