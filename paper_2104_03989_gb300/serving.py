"""Continuous batching of simplification jobs on one GPU.

Requests arrive at any time. A request is admitted as soon as the context's
HBM budget holds its resident state (candidate mesh, mip-mapped textures,
gradients, Adam moments and render scratch, plus its frozen reference); the
C ABI refuses with ADMS_ERR_BUDGET otherwise and the request waits, first in
first out. Every iteration takes one step of every live job at once: fresh
random views per job (keyed by the job's seed and its own iteration count,
so a job's result does not depend on who shares its batches), a reference
render per job, then forward + loss, backward and Adam for all live jobs in
one batched call per stage (one launch per pixel stage). Jobs that
reach their iteration count retire and free their memory for waiting
requests. A job whose loss or gradients turn non-finite (latched on the device,
where its optimizer steps are then skipped) is quarantined (retired with that
status) without disturbing the others; a cancelled request leaves the queue, or
retires between iterations, and frees its memory the same way.

All arithmetic runs in libadms.so; this module schedules.
"""

from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

import synth

from . import binding as B
from .engine import Context


@dataclass
class Request:
    rid: int
    cand: object              # scene to optimize (synth.Scene-like)
    ref: object               # reference scene (frozen)
    n_views: int = 8
    res: int = 256
    iterations: int = 200
    seed: int = 0
    loss: str = "logl1"
    lr0: float = 0.01
    arrival: float = 0.0      # seconds, relative to the server's start


@dataclass
class JobRecord:
    req: Request
    cand: int = -1
    ref: int = -1
    it: int = 0
    admitted: float = 0.0
    finished: float = 0.0
    status: str = "waiting"   # waiting, running, done, quarantined, rejected
    status_code: int = 0      # the latched device status of a quarantined job (e.g. ADMS_ERR_NONFINITE)
    losses: list = field(default_factory=list)
    ref_buf: torch.Tensor = None


class SimplificationServer:
    def __init__(self, hbm_budget_bytes=0, stream=None, loss_every=1, on_admit=None):
        """on_admit(server, record): called right after a job is admitted (tests inject faults here)."""
        self.stream = stream if stream is not None else torch.cuda.Stream()
        with torch.cuda.stream(self.stream):
            self.ctx = Context(hbm_budget_bytes, stream=self.stream)
        self.budget = hbm_budget_bytes
        self.blocked = False
        self.queue = deque()
        self.live = []
        self.done = []
        self.results = {}
        self.iter_ms = []
        self.pixels = 0
        self.max_live = 0
        self.loss_every = loss_every
        self.on_admit = on_admit
        self.t0 = None
        # references render on side streams (round robin over the live jobs), beside
        # each other and beside the candidates' forward; the loss waits for them
        self.sides = [torch.cuda.Stream() for _ in range(4)]
        self._fork, self._ready = torch.cuda.Event(), torch.cuda.Event()
        self._side_evs = [torch.cuda.Event() for _ in self.sides]

    # ------------------------------------------------------------------ admission
    def _headroom(self, recs):
        """Bytes kept free for the batched argument and work-item lists of one
        job set (lists of earlier sets are released on every admission and
        counted as in use until then):
        a 16-byte item per 64 pixels at the smallest tile width, arguments per
        job, allocation rounding."""
        px = sum(rec.req.n_views * rec.req.res * rec.req.res for rec in recs)
        return 2 * (px // 64 * 16 + len(recs) * 4096) + (64 << 10)

    def start(self):
        """Start the server's clock (run() does this; callers that drive
        admit/iterate themselves call it first)."""
        self.t0 = time.perf_counter()

    def submit(self, req: Request):
        self.queue.append(JobRecord(req))

    def cancel(self, rid):
        """Cancel request rid between iterations: a waiting request leaves the
        queue, a live job retires with its latents as of its last step. Returns
        False when rid is neither waiting nor live."""
        for rec in list(self.queue):
            if rec.req.rid == rid:
                self.queue.remove(rec)
                rec.status = "cancelled"
                rec.finished = self._now()
                self.done.append(rec)
                self.blocked = False      # the head of the queue may have changed
                return True
        for rec in list(self.live):
            if rec.req.rid == rid:
                with torch.cuda.stream(self.stream):
                    self.stream.synchronize()
                    self._retire(rec, "cancelled")
                return True
        return False

    def _now(self):
        return time.perf_counter() - self.t0

    def admit(self):
        """Admit waiting requests that have arrived, first in first out, while
        the budget holds them."""
        with torch.cuda.stream(self.stream):
            self._admit()

    def _admit(self):
        if self.blocked:
            return                    # the head request did not fit: wait for a retirement
        while self.queue and self.queue[0].req.arrival <= self._now():
            rec = self.queue[0]
            r = rec.req
            try:
                rec.ref = self.ctx.create_job(r.ref, frozen=True, seed=r.seed)
                rec.cand = self.ctx.create_job(r.cand, loss=r.loss, lr0=r.lr0, seed=r.seed)
                # all render scratch up front, plus headroom for the batched
                # work lists, so that no later call of this job allocates
                self.ctx.reserve(rec.ref, r.n_views, r.res, r.res)
                self.ctx.reserve(rec.cand, r.n_views, r.res, r.res)
                if self.budget and self.ctx.bytes_in_use() + self._headroom(self.live + [rec]) > self.budget:
                    raise B.AdmsError(B.ADMS_ERR_BUDGET, "no headroom for the batched work lists")
                B.adms_ctx_release_batches(self.ctx.ctx)   # the job set changes: drop the old lists
                rec.ref_buf = torch.empty((r.n_views, r.res, r.res, 3), dtype=torch.float32, device="cuda")
            except B.AdmsError as e:
                for h in (rec.cand, rec.ref):
                    if h >= 0:
                        self.ctx.destroy_job(h)
                rec.cand = rec.ref = -1
                if e.status == B.ADMS_ERR_BUDGET and self.live:
                    self.blocked = True
                    return
                rec.status = "rejected"
                self.queue.popleft()
                self.done.append(rec)
                continue
            rec.status = "running"
            rec.admitted = self._now()
            self.queue.popleft()
            self.live.append(rec)
            self.max_live = max(self.max_live, len(self.live))
            if self.on_admit is not None:
                self.on_admit(self, rec)

    def _retire(self, rec, status):
        rec.status = status
        rec.finished = self._now()
        p = self.ctx.params(rec.cand)
        self.results[rec.req.rid] = {k: p[k].clone() for k in ("pos", "kd", "orm", "nrm", "disp")
                                     if k in p and p[k] is not None}
        self.ctx.destroy_job(rec.cand)
        self.ctx.destroy_job(rec.ref)
        self.blocked = False
        rec.ref_buf = None
        self.live.remove(rec)
        self.done.append(rec)

    # ------------------------------------------------------------------ one iteration
    def iterate(self):
        """One step of every live job; returns the iteration's wall time in ms."""
        if not self.live:
            return 0.0
        with torch.cuda.stream(self.stream):
            return self._iterate()

    def _iterate(self):
        t = time.perf_counter()
        views = []
        self._fork.record(self.stream)
        for sd in self.sides:
            sd.wait_event(self._fork)
        try:
            for k, rec in enumerate(self.live):
                r = rec.req
                v = synth.sample_views(r.seed, rec.it, r.n_views, r.res, r.res)
                views.append(v)
                self.ctx.set_stream(self.sides[k % len(self.sides)])
                self.ctx.render_reference(rec.ref, v, r.res, r.res, out=rec.ref_buf)
        finally:
            for sd, ev in zip(self.sides[1:], self._side_evs[1:]):
                ev.record(sd)
                self.sides[0].wait_event(ev)
            self._ready.record(self.sides[0])
            self.ctx.set_stream(self.stream)
        self.ctx.set_ref_event(self._ready)
        jobs = [rec.cand for rec in self.live]
        try:
            loss = self.ctx.forward_loss(jobs, views, [rec.ref_buf for rec in self.live])
        finally:
            self.ctx.set_ref_event(None)
        self.ctx.backward(jobs)
        self.ctx.step(jobs)
        read = (self.live[0].it % self.loss_every) == 0
        # the latched device status of each job (a non-finite loss or gradient), read
        # back with the losses: such a job was not updated and is quarantined
        status = self.ctx.jobs_status(jobs).cpu().numpy() if read else None
        vals = loss.cpu().numpy() if read else None
        self.stream.synchronize()
        ms = (time.perf_counter() - t) * 1e3
        self.iter_ms.append(ms)
        for k, rec in enumerate(list(self.live)):
            rec.it += 1
            self.pixels += rec.req.n_views * rec.req.res * rec.req.res
            if vals is not None:
                rec.losses.append(float(vals[k]))
                if status[k] != 0 or not math.isfinite(float(vals[k])):
                    rec.status_code = int(status[k])
                    self._retire(rec, "quarantined")
                    continue
            if rec.it >= rec.req.iterations:
                self._retire(rec, "done")
        return ms

    def run(self, requests, idle_sleep=0.0005):
        """Serve requests (arrival times relative to the start) until all are done."""
        for r in sorted(requests, key=lambda r: r.arrival):
            self.submit(r)
        self.start()
        while self.queue or self.live:
            self.admit()
            if self.live:
                self.iterate()
            else:
                time.sleep(idle_sleep)
        return self.report()

    def report(self):
        ms = np.array(self.iter_ms) if self.iter_ms else np.zeros(1)
        wall = self._now()
        done = [r for r in self.done if r.status == "done"]
        return {
            "iterations": len(self.iter_ms),
            "p50_iteration_ms": float(np.percentile(ms, 50)),
            "p99_iteration_ms": float(np.percentile(ms, 99)),
            "job_completion_s": [r.finished - r.req.arrival for r in done],
            "aggregate_mpixels_per_s": self.pixels / max(wall, 1e-9) / 1e6,
            "done": len(done),
            "quarantined": sum(r.status == "quarantined" for r in self.done),
            "rejected": sum(r.status == "rejected" for r in self.done),
            "cancelled": sum(r.status == "cancelled" for r in self.done),
            "max_live": self.max_live,
            "wall_s": wall,
        }

    def close(self):
        self.ctx.close()


def poisson_arrivals(n, rate_per_s, seed=0):
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
