"""Continuous-batching inpainting server on one GPU.

Requests (a clip and its occlusion mask) queue in arrival order. Between
batch rounds the server admits queued requests while their device footprint
(``vi_footprint_bytes``) fits the HBM budget and a slot is free; an admitted
request is prepared (pyramid, initialisation, onion peel) and joins the
running batch, so its iterations share launches with the requests already on
the GPU. A finished request is fetched and removed at once, which frees its
memory and slot for the next one. Every job's result is bit-identical to
running it alone (``vi_batch_*`` guarantees it).

The scheduling logic is plain Python over a small backend interface
(add / step / poll / fetch / remove / footprint), so it runs unchanged over
the CUDA batch or over a stand-in in tests.
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


class CudaBackend:
    """The vi_batch of the CUDA library."""

    def __init__(self, stream=None, **cfg):
        from . import vi
        self.vi = vi
        self.batch = vi.Batch(stream=stream, **cfg)
        self.cfg = vi.default_config(**cfg)

    def footprint(self, req):
        import ctypes
        T, H, W = req.mask.shape[:3]
        cfg = self.vi.default_config(**{**self.batch.defaults, **req.job})
        return int(self.vi.load().vi_footprint_bytes(ctypes.byref(cfg), W, H, T, int(req.hole_voxels)))

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
