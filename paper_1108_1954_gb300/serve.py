"""Continuous-batching serving loop for independent PIC run requests.

Requests arrive over time (each a run: cells, particles, steps, beam and
thermal speeds, seed).  The loop keeps a pool of resident runs on the GPU
(`Pool`, one caller-owned arena with a memory budget):

  * arrived requests are admitted, in arrival order but letting smaller ones
    pass a head that does not fit, whenever a slot and arena space are free;
    the initial state is generated on the device (no host upload);
  * one `advance(k)` moves every resident run forward by up to k steps in a
    single cluster launch, so runs admitted while others are mid-flight share
    the launch with them;
  * runs that reached their step count are retired: their last diagnostics
    row is read back (the request's result), their memory is released, and
    (finish - arrival) is recorded as the request's latency;
  * a request cancelled before it finishes leaves the queue, or, if resident,
    has its slot and memory released at once;
  * if the worker that holds the pool is lost (`WorkerLost` from a pool call,
    or injected on the host with `crash_after`), the server builds a new pool
    and resubmits the requests that were resident, from their start: a
    request's initial state is generated from its seed, so the rerun gives
    the same result.

Each finished, rejected or cancelled request can be logged as one JSON line.
This module only sequences calls of the C ABI (admission, advance, result
read-back, release); every step of every run runs in the CUDA kernels.
"""
from __future__ import annotations

import collections
import json
import math
import time
from dataclasses import dataclass

import numpy as np

from . import PIC_EINVAL, Loading, Params, PicError, Pool, pool_run_bytes


class WorkerLost(RuntimeError):
    """The worker holding the pool is gone, and with it every resident run."""


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the start of the stream
    params: Params
    loading: Loading
    steps: int
    cancel_at: float = math.inf   # seconds after the start; cancelled then if not finished


@dataclass
class Record:
    rid: int
    arrival: float
    admitted: float = -1.0    # the last admission (after a restart, the rerun's)
    finished: float = -1.0
    npart: int = 0
    steps: int = 0
    result: object = None     # last diagnostics row, or (state, field) if kept
    rejected: bool = False    # invalid for the pool, or larger than all of it
    cancelled: float = -1.0   # when it was cancelled, if it was
    restarts: int = 0         # resubmissions after a lost worker

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def outcome(self) -> str:
        if self.rejected:
            return "rejected"
        if self.cancelled >= 0.0:
            return "cancelled"
        return "finished"

    def to_json(self) -> str:
        """One log line: the request's times, size and outcome."""
        d = dict(rid=self.rid, outcome=self.outcome, arrival=round(self.arrival, 6),
                 admitted=round(self.admitted, 6), npart=self.npart, steps=self.steps,
                 restarts=self.restarts)
        if self.outcome == "finished":
            d.update(finished=round(self.finished, 6), latency=round(self.latency, 6),
                     particle_steps=self.npart * self.steps)
        elif self.outcome == "cancelled":
            d.update(cancelled=round(self.cancelled, 6))
        return json.dumps(d)


def requests_from_stream(stream, modes_fn=None):
    """Request objects from workloads.request_stream dicts."""
    out = []
    for i, r in enumerate(stream):
        modes = modes_fn(r) if modes_fn else ()
        out.append(Request(i, r["arrival"],
                           Params(npart=r["npart"], ncell=r["ncell"], length=r["length"],
                                  dt=r["dt"]),
                           Loading(v0=r["v0"], vth=r["vth"], seed=r["seed"], modes=modes),
                           r["steps"]))
    return out


class Server:
    def __init__(self, arena_bytes: int, max_slots: int = 1024, ncell_max: int = 4096,
                 history: int = 8, advance_steps: int = 50, variant: int = 5,
                 cluster: int = 8, block: int = 512, device=None):
        if int(advance_steps) < 1:
            # advance(0) only initialises: no run would ever finish
            raise ValueError("advance_steps must be at least 1")

        def make_pool():
            return Pool(max_slots=max_slots, ncell_max=ncell_max, arena_bytes=arena_bytes,
                        history=history, variant=variant, cluster=cluster, block=block,
                        device=device)
        self.make_pool = make_pool
        self.pool = make_pool()
        self.k = int(advance_steps)
        self.history = history

    def close(self):
        self.pool.close()

    def _replace_pool(self):
        try:
            self.pool.close()
        except Exception:       # the lost worker's pool may not answer
            pass
        self.pool = self.make_pool()

    def serve(self, requests, keep=(), log=None, crash_after=()):
        """Serve the requests in real time (request.arrival is seconds after
        the call); returns (records, stats).
          keep         request ids whose final state, field and history are
                       read back before release;
          log          a writable text stream: one JSON line per request as
                       it finishes, is rejected or is cancelled;
          crash_after  advance counts after which the worker is taken as lost
                       (fault injection on the host): the pool is rebuilt and
                       its resident requests are resubmitted."""
        keep = set(keep)
        crash_after = set(int(c) for c in crash_after)
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        inflight = {}
        records = {}
        advances = 0
        active_sum = 0
        crashes = 0
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        def close_record(rec):
            if log is not None:
                log.write(rec.to_json() + "\n")

        def reject(req):
            rec = records.get(req.rid) or Record(req.rid, req.arrival)
            rec.npart, rec.steps, rec.rejected = req.params.npart, req.steps, True
            records[req.rid] = rec
            close_record(rec)

        while pending or waiting or inflight:
            t = now()
            while pending and pending[0].arrival <= t:
                waiting.append(pending.popleft())
            # cancellations: queued requests leave, resident ones are released
            for req in [r for r in waiting if r.cancel_at <= t]:
                waiting.remove(req)
                rec = records.get(req.rid) or Record(req.rid, req.arrival, npart=req.params.npart,
                                                     steps=req.steps)
                rec.cancelled = t
                records[req.rid] = rec
                close_record(rec)
            for slot in [s for s, r in inflight.items() if r.cancel_at <= t]:
                req = inflight.pop(slot)
                self.pool.release(slot)
                rec = records[req.rid]
                rec.cancelled = t
                close_record(rec)
            # admit what fits, oldest first; a head that does not fit does not
            # block smaller requests behind it
            for req in list(waiting):
                try:
                    slot = self.pool.admit_loaded(req.params, req.loading, req.steps)
                except PicError as e:
                    if e.code != PIC_EINVAL:
                        raise
                    # a request the pool cannot run (e.g. more cells than it
                    # was built for) is rejected, not served
                    waiting.remove(req)
                    reject(req)
                    continue
                if slot is None:
                    continue
                waiting.remove(req)
                inflight[slot] = req
                rec = records.get(req.rid) or Record(req.rid, req.arrival)
                rec.admitted, rec.npart, rec.steps = now(), req.params.npart, req.steps
                records[req.rid] = rec
            if not inflight:
                # what an empty pool cannot admit never fits: reject it
                while waiting:
                    reject(waiting.popleft())
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now(), 0.005)))
                continue
            try:
                active_sum += self.pool.advance(self.k)
                advances += 1
                if advances in crash_after:
                    raise WorkerLost("injected after advance %d" % advances)
                for slot in self.pool.finished():
                    req = inflight[slot]
                    rec = records[req.rid]
                    if req.rid in keep:
                        hist = (self.pool.diagnostics(slot, 0, req.steps + 1)
                                if req.steps + 1 <= self.history else None)
                        result = (self.pool.get_state(slot), self.pool.get_field(slot), hist)
                    else:
                        result = self.pool.diagnostics(slot, req.steps, 1)[0]
                    self.pool.release(slot)
                    # retired only once its result is read and its slot given back
                    del inflight[slot]
                    rec.result, rec.finished = result, now()
                    close_record(rec)
            except WorkerLost:
                # the resident runs are gone: a new pool, and the requests
                # that were resident (results not yet read included) go back
                # to the head of the queue
                crashes += 1
                self._replace_pool()
                lost = sorted(inflight.values(), key=lambda r: r.arrival)
                inflight.clear()
                for req in reversed(lost):
                    records[req.rid].restarts += 1
                    waiting.appendleft(req)
                continue
        wall = now()
        recs = [records[r.rid] for r in sorted(requests, key=lambda r: r.rid)]
        done = [r for r in recs if r.outcome == "finished"]
        lat = np.array([r.latency for r in done]) if done else np.zeros(1)
        work = float(sum(r.npart * r.steps for r in done))
        stats = dict(requests=len(recs), rejected=sum(r.rejected for r in recs),
                     cancelled=sum(r.outcome == "cancelled" for r in recs),
                     worker_crashes=crashes, restarts=sum(r.restarts for r in recs),
                     wall_s=wall, advances=advances,
                     advance_steps=self.k, mean_active=active_sum / max(1, advances),
                     p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                     mean_s=float(lat.mean()), particle_steps=work,
                     value=work / wall if wall > 0 else 0.0)
        return recs, stats


def arena_for(requests, history: int, concurrent: int, slack: float = 1.5) -> int:
    """A memory budget that holds `concurrent` of the largest requests."""
    sizes = sorted((pool_run_bytes(r.params, history) for r in requests), reverse=True)
    return int(sum(sizes[:concurrent]) * slack) + (64 << 20)
