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
    (finish - arrival) is recorded as the request's latency.

This module only sequences calls of the C ABI (admission, advance, result
read-back, release); every step of every run runs in the CUDA kernels.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass

import numpy as np

from . import PIC_EINVAL, Loading, Params, PicError, Pool, pool_run_bytes


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the start of the stream
    params: Params
    loading: Loading
    steps: int


@dataclass
class Record:
    rid: int
    arrival: float
    admitted: float = -1.0
    finished: float = -1.0
    npart: int = 0
    steps: int = 0
    result: object = None     # last diagnostics row, or (state, field) if kept
    rejected: bool = False    # invalid for the pool, or larger than all of it

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


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
        self.pool = Pool(max_slots=max_slots, ncell_max=ncell_max, arena_bytes=arena_bytes,
                         history=history, variant=variant, cluster=cluster, block=block,
                         device=device)
        self.k = int(advance_steps)
        self.history = history

    def close(self):
        self.pool.close()

    def serve(self, requests, keep=()):
        """Serve the requests in real time (request.arrival is seconds after
        the call); returns (records, stats).  `keep`: request ids whose final
        state, field and history are read back before release."""
        pool = self.pool
        keep = set(keep)
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        inflight = {}
        records = {}
        advances = 0
        active_sum = 0
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        while pending or waiting or inflight:
            t = now()
            while pending and pending[0].arrival <= t:
                waiting.append(pending.popleft())
            # admit what fits, oldest first; a head that does not fit does not
            # block smaller requests behind it
            for req in list(waiting):
                try:
                    slot = pool.admit_loaded(req.params, req.loading, req.steps)
                except PicError as e:
                    if e.code != PIC_EINVAL:
                        raise
                    # a request the pool cannot run (e.g. more cells than it
                    # was built for) is rejected, not served
                    waiting.remove(req)
                    records[req.rid] = Record(req.rid, req.arrival, npart=req.params.npart,
                                              steps=req.steps, rejected=True)
                    continue
                if slot is None:
                    continue
                waiting.remove(req)
                inflight[slot] = req
                records[req.rid] = Record(req.rid, req.arrival, admitted=now(),
                                          npart=req.params.npart, steps=req.steps)
            if not inflight:
                # what an empty pool cannot admit never fits: reject it
                while waiting:
                    req = waiting.popleft()
                    records[req.rid] = Record(req.rid, req.arrival, npart=req.params.npart,
                                              steps=req.steps, rejected=True)
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now(), 0.005)))
                continue
            active_sum += pool.advance(self.k)
            advances += 1
            for slot in pool.finished():
                req = inflight.pop(slot)
                rec = records[req.rid]
                if req.rid in keep:
                    hist = (pool.diagnostics(slot, 0, req.steps + 1)
                            if req.steps + 1 <= self.history else None)
                    rec.result = (pool.get_state(slot), pool.get_field(slot), hist)
                else:
                    rec.result = pool.diagnostics(slot, req.steps, 1)[0]
                rec.finished = now()
                pool.release(slot)
        wall = now()
        recs = [records[r.rid] for r in sorted(requests, key=lambda r: r.rid)]
        done = [r for r in recs if not r.rejected]
        lat = np.array([r.latency for r in done]) if done else np.zeros(1)
        work = float(sum(r.npart * r.steps for r in done))
        stats = dict(requests=len(recs), rejected=len(recs) - len(done), wall_s=wall,
                     advances=advances,
                     advance_steps=self.k, mean_active=active_sum / max(1, advances),
                     p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                     mean_s=float(lat.mean()), particle_steps=work,
                     value=work / wall if wall > 0 else 0.0)
        return recs, stats


def arena_for(requests, history: int, concurrent: int, slack: float = 1.5) -> int:
    """A memory budget that holds `concurrent` of the largest requests."""
    sizes = sorted((pool_run_bytes(r.params, history) for r in requests), reverse=True)
    return int(sum(sizes[:concurrent]) * slack) + (64 << 20)
