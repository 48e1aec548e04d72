"""Serving many ideal-MHD simulations on one GPU with continuous batching.

Requests (an initial state, a grid, an end time) arrive over time.  The server admits
them (oldest first, or least estimated work first) as device memory frees up under a
fixed HBM budget; every admitted
request joins the running batch (idx_batch_*), where all of them advance together, each
with its own CFL dt, until its end time; a finished request's state is copied back to
the host and its memory released, which lets the next ones in.  Latency is arrival to
result-on-host.  The same stream can be served one request at a time for comparison.

The scheduler talks to a backend (the real one wraps libidx; tests use a fake device
and a fake clock), so its admission and accounting logic is tested without a GPU.
"""
from collections import deque
from dataclasses import dataclass, field
import math
import time
from typing import Optional

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the start of the stream
    kind: str                 # "2d" (Orszag-Tang) or "3d" (turbulent box)
    n: int
    t_end: float
    seed: int
    payload: Optional[object] = None   # inputs.IC, made before the stream starts
    # filled in by the server
    status: str = "pending"            # pending, running, done, failed, rejected
    admitted: Optional[float] = None
    finished: Optional[float] = None
    cycles: int = 0
    cells: int = 0
    state: Optional[list] = None
    error: Optional[str] = None


def poisson_stream(n_requests, rate, seed=7, sizes_2d=(64, 512), sizes_3d=(32, 128),
                   t_end=(0.01, 0.1), p2d=0.5):
    """Seeded request stream: exponential inter-arrival times of mean 1/rate; kind 2D with
    probability p2d; N log-uniform in the kind's range (a multiple of 8); t_end uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        kind = "2d" if rng.uniform() < p2d else "3d"
        lo, hi = sizes_2d if kind == "2d" else sizes_3d
        n = int(max(8, 8 * round(math.exp(rng.uniform(math.log(lo), math.log(hi))) / 8)))
        out.append(Request(i, t, kind, n, float(rng.uniform(*t_end)), seed=1000 + i))
    return out


def make_payloads(requests):
    from . import inputs
    for r in requests:
        r.payload = (inputs.orszag_tang_2d(r.n) if r.kind == "2d"
                     else inputs.turbulent_box(r.n, seed=r.seed))
        r.cells = r.payload.ncells
    return requests


class WallClock:
    def __init__(self):
        self.t0 = time.perf_counter()

    def now(self):
        return time.perf_counter() - self.t0

    def sleep_until(self, t):
        dt = t - self.now()
        if dt > 0:
            time.sleep(dt)


class IdxBackend:
    """libidx: one batch on its own stream; every request is a sim on a stream of its own,
    so its upload and its read-back overlap the batch's running chunk (a finished member
    is inert in the batch until it is retired at the next chunk boundary)."""

    def __init__(self, precision="fp64", cfl=0.4, stream=None):
        from . import idx
        self.idx = idx
        self.precision = precision
        self.cfl = cfl
        self.batch = idx.Batch(precision, stream=stream)
        self.sims = {}
        self.ready = []        # uploaded, joining at the next boundary

    def footprint(self, req):
        return self.idx.footprint(req.payload.shape, self.precision)

    def start(self, req):
        ic = req.payload
        s = self.idx.Sim(ic.shape, ic.lengths, ic.gamma, self.cfl, self.precision)
        try:
            s.set_primitive(ic.prim)
        except Exception:
            s.close()
            raise
        self.sims[req.rid] = s
        self.ready.append((req.rid, req.t_end))

    def commit(self):
        for rid, t_end in self.ready:
            self.batch.add(self.sims[rid], t_end)
        self.ready = []

    def step(self, ncycles):
        self.batch.step(ncycles)

    def poll(self):
        finished, _ = self.batch.poll()
        ids = {id(s): rid for rid, s in self.sims.items()}
        return [ids[id(s)] for s in finished]

    def finish(self, rid):
        """Read a finished member's result back (its own stream; the batch keeps running)."""
        s = self.sims[rid]
        return s.get_state(), s.step_count()

    def retire(self, rid):
        s = self.sims.pop(rid)
        try:
            self.batch.remove(s)
        finally:
            s.close()

    def close(self):
        for rid in list(self.sims):
            self.sims.pop(rid).close()
        self.batch.close()


class IdxSequential:
    """libidx one request at a time: the same sims advanced alone (idx_advance)."""

    def __init__(self, precision="fp64", cfl=0.4, stream=None):
        from . import idx
        self.idx = idx
        self.precision = precision
        self.cfl = cfl
        self.stream = stream

    def footprint(self, req):
        return self.idx.footprint(req.payload.shape, self.precision)

    def serve_one(self, req):
        ic = req.payload
        s = self.idx.Sim(ic.shape, ic.lengths, ic.gamma, self.cfl, self.precision,
                         stream=self.stream)
        try:
            s.set_primitive(ic.prim)
            s.advance(req.t_end)
            return s.get_state(), s.step_count()
        finally:
            s.close()


def _stats(requests, t_first, t_last):
    done = [r for r in requests if r.status == "done"]
    lat = np.array([r.finished - r.arrival for r in done]) if done else np.array([np.nan])
    wait = np.array([r.admitted - r.arrival for r in done]) if done else np.array([np.nan])
    work = float(sum(r.cells * r.cycles for r in done))
    span = max(t_last - t_first, 1e-12)
    return {"requests": len(requests), "done": len(done),
            "failed": sum(r.status == "failed" for r in requests),
            "rejected": sum(r.status == "rejected" for r in requests),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(np.mean(lat)), "wait_p50_s": float(np.percentile(wait, 50)),
            "cell_updates": work, "makespan_s": span, "cell_updates_per_s": work / span}


def estimated_work(r):
    """Cell-updates a request needs, up to a constant: cells x cycles, with cycles
    proportional to t_end / dt and dt to the cell size (CFL), i.e. to t_end * n."""
    return r.cells * r.n * r.t_end


class Server:
    """Continuous batching under an HBM budget."""

    ORDERS = ("oldest", "least_work")

    def __init__(self, backend, budget_bytes, clock=None, cycles_per_poll=8, chunk_s=None,
                 max_active_cells=None, order="oldest"):
        """cycles_per_poll: batched cycles between polls; with chunk_s set, that number
        adapts so that one chunk takes about chunk_s seconds (new arrivals and finished
        requests are handled at chunk boundaries).  max_active_cells: when set, a request
        waits while the running ones already hold that many cells (enough work to keep
        the device busy), so late arrivals do not slow down large running requests.
        order: which waiting request is admitted next -- the oldest, or the one with the
        least estimated work (shortest-job-first among those waiting)."""
        if order not in self.ORDERS:
            raise ValueError(order)
        self.backend = backend
        self.budget = int(budget_bytes)
        self.clock = clock or WallClock()
        self.k = int(cycles_per_poll)
        self.chunk_s = chunk_s
        self.max_cells = max_active_cells
        self.order = order
        self.used = 0
        self.peak = 0

    def run(self, requests):
        """Pipelined loop: launch the next chunk of batched cycles, then -- while it runs --
        read back the members that finished at the last boundary and upload new admissions;
        at the boundary, retire the read-back members and let the uploaded ones join."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        queue = deque()
        running = {}       # in the batch (or joining at the next boundary)
        bytes_of = {}
        to_read = []       # finished at the last boundary, results not read yet
        t_first = pending[0].arrival if pending else 0.0
        t_last = t_first
        phase = {"admit_s": 0.0, "step_s": 0.0, "poll_s": 0.0, "finish_s": 0.0, "idle_s": 0.0,
                 "chunks": 0}
        commit = getattr(self.backend, "commit", None)
        retire = getattr(self.backend, "retire", None)
        while pending or queue or running or to_read:
            now = self.clock.now()
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            if self.order == "least_work" and len(queue) > 1:
                queue = deque(sorted(queue, key=lambda q: (estimated_work(q), q.arrival)))
            in_batch = [rid for rid in running if rid not in to_read]
            t0 = self.clock.now()
            stepped = bool(in_batch)
            if stepped:
                self.backend.step(self.k)
            t1 = self.clock.now()
            phase["step_s"] += t1 - t0
            # overlapped with the chunk: results of the members finished last time
            for rid in to_read:
                r = running.pop(rid)
                tf = self.clock.now()
                try:
                    r.state, r.cycles = self.backend.finish(rid)
                    r.status = "done"
                except Exception as e:
                    r.status, r.error = "failed", str(e)
                r.finished = self.clock.now()
                phase["finish_s"] += r.finished - tf
                t_last = max(t_last, r.finished)
            # overlapped with the chunk: admissions in the server's order, while the budget allows
            while queue:
                r = queue[0]
                need = self.backend.footprint(r)
                if need > self.budget:
                    queue.popleft()
                    r.status, r.error = "rejected", f"needs {need} B > budget {self.budget} B"
                    continue
                if self.used + need > self.budget:
                    break
                if self.max_cells:
                    active = sum(q.cells for q in running.values())
                    if active > 0 and active + r.cells > self.max_cells:
                        break
                queue.popleft()
                ta = self.clock.now()
                try:
                    self.backend.start(r)
                except Exception as e:  # a request that fails to start is reported, not fatal
                    r.status, r.error = "failed", str(e)
                    r.finished = self.clock.now()
                    phase["admit_s"] += r.finished - ta
                    continue
                phase["admit_s"] += self.clock.now() - ta
                r.status, r.admitted = "running", self.clock.now()
                running[r.rid] = r
                bytes_of[r.rid] = need
                self.used += need
                self.peak = max(self.peak, self.used)
            # boundary
            t2 = self.clock.now()
            finished = self.backend.poll() if stepped else []
            t3 = self.clock.now()
            phase["poll_s"] += t3 - t2
            if stepped:
                phase["chunks"] += 1
                if self.chunk_s:
                    el = max(t3 - t0, 1e-6)
                    self.k = int(min(64, max(1, round(self.k * self.chunk_s / el))))
            for rid in to_read:
                if retire:
                    retire(rid)
                self.used -= bytes_of.pop(rid)
            to_read = [rid for rid in finished if rid in running]
            if commit:
                commit()
            if not stepped and not to_read and not running and pending and not queue:
                ti = self.clock.now()
                self.clock.sleep_until(pending[0].arrival)
                phase["idle_s"] += self.clock.now() - ti
        stats = _stats(requests, t_first, t_last)
        stats["peak_bytes"] = self.peak
        stats["budget_bytes"] = self.budget
        stats["phases"] = phase
        return stats


def serve_sequential(backend, requests, clock=None, budget_bytes=None):
    """The same stream, one request at a time, oldest first."""
    clock = clock or WallClock()
    reqs = sorted(requests, key=lambda r: r.arrival)
    t_first = reqs[0].arrival if reqs else 0.0
    t_last = t_first
    for r in reqs:
        clock.sleep_until(r.arrival)
        if budget_bytes is not None and backend.footprint(r) > budget_bytes:
            r.status, r.error = "rejected", "over budget"
            continue
        r.admitted = clock.now()
        try:
            r.state, r.cycles = backend.serve_one(r)
            r.status = "done"
        except Exception as e:
            r.status, r.error = "failed", str(e)
        r.finished = clock.now()
        t_last = max(t_last, r.finished)
    return _stats(requests, t_first, t_last)
