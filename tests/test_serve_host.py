"""The serving loop's host logic on the CPU, against a stand-in pool.

`serve.Server.serve` only sequences pool calls (admit, advance, finished,
diagnostics, release).  A stand-in pool with a byte budget and step counters
checks, without a GPU: every request finishes with its own step count; a head
request that does not fit does not block smaller ones behind it; requests that
arrive while others are resident join the same advances (continuous
batching); kept requests return their state, field and history; cancelled
requests leave the queue or give back their slot at once; a lost worker's
resident requests are resubmitted to a new pool and finish; each request is
logged as one JSON line.  The faults are made on the host: a stand-in pool
that raises `WorkerLost`, or the server's own injection after an advance.
"""
import io
import json
import math
import time

import numpy as np
import pytest

from paper_1108_1954_gb300 import PIC_EINVAL, Loading, Params, PicError, serve


class FakePool:
    def __init__(self, budget, max_slots=8, history=8, lose_on_advance=None, lose_on_read=None):
        self.budget, self.max_slots, self.history = budget, max_slots, history
        self.used = 0
        self.runs = {}          # slot -> [params, steps, done, bytes]
        self.next_slot = 0
        self.log = []           # (event, slot, resident count)
        self.released = {}      # slot -> steps done when released
        self.lose_on_advance = lose_on_advance
        self.lose_on_read = lose_on_read        # lost on this result read-back
        self.reads = 0
        self.advances = 0
        self.closed = False

    @staticmethod
    def bytes_of(p):
        return 16 * p.npart + 64 * p.ncell

    def admit_loaded(self, params, loading, steps):
        if params.ncell > 4096:                 # beyond the pool's grid limit
            raise PicError(PIC_EINVAL, "pic_pool_admit_loaded")
        b = self.bytes_of(params)
        if len(self.runs) >= self.max_slots or self.used + b > self.budget:
            return None
        slot = self.next_slot
        self.next_slot += 1
        self.runs[slot] = [params, steps, 0, b]
        self.used += b
        self.log.append(("admit", slot, len(self.runs)))
        return slot

    def advance(self, k):
        time.sleep(0.0005)      # an advance takes time, as on the device
        self.advances += 1
        if self.advances == self.lose_on_advance:
            raise serve.WorkerLost("stand-in worker lost")
        active = 0
        for r in self.runs.values():
            if r[2] < r[1]:
                r[2] = min(r[1], r[2] + k)
                active += 1
        self.log.append(("advance", -1, active))
        return active

    def finished(self):
        return [s for s, r in self.runs.items() if r[2] >= r[1]]

    def diagnostics(self, slot, first, count):
        self.reads += 1
        if self.reads == self.lose_on_read:
            raise serve.WorkerLost("stand-in worker lost while reading a result")
        rows = np.zeros(count, dtype=[("step", "i8"), ("field", "f8")])
        rows["step"] = np.arange(first, first + count)
        return rows

    def get_state(self, slot):
        n = self.runs[slot][0].npart
        return np.zeros(n, np.float32), np.zeros(n, np.float32)

    def get_field(self, slot):
        return dict(E=np.zeros(self.runs[slot][0].ncell))

    def release(self, slot):
        r = self.runs.pop(slot)
        self.used -= r[3]
        self.released[slot] = r[2]
        self.log.append(("release", slot, len(self.runs)))

    def close(self):
        self.closed = True


def make_server(pool, k, make_pool=None):
    srv = serve.Server.__new__(serve.Server)    # no device pool
    srv.pool, srv.k, srv.history = pool, k, pool.history
    srv.make_pool = make_pool
    return srv


def request(rid, arrival, npart, ncell, steps):
    return serve.Request(rid, arrival, Params(npart=npart, ncell=ncell, length=1.0),
                         Loading(v0=0.1, vth=0.0, seed=rid), steps)


def test_every_request_finishes_with_its_steps():
    pool = FakePool(budget=10 ** 9)
    reqs = [request(i, 0.002 * i, 1000 + 10 * i, 64, 30 + 7 * i) for i in range(12)]
    recs, stats = make_server(pool, 10).serve(reqs)
    assert [r.rid for r in recs] == list(range(12))
    for r, q in zip(recs, reqs):
        assert r.steps == q.steps and r.npart == q.params.npart
        assert r.finished >= r.admitted >= r.arrival - 1e-9
        assert int(r.result["step"]) == q.steps              # the last history row
    assert stats["requests"] == 12 and stats["particle_steps"] == sum(
        q.params.npart * q.steps for q in reqs)
    assert not pool.runs and pool.used == 0                   # everything released


def test_a_head_that_does_not_fit_does_not_block():
    resident = request(0, 0.0, 900, 64, 200)
    big = request(1, 0.0, 1000, 64, 20)
    small = request(2, 0.0, 100, 64, 20)
    # the budget holds `resident` + `small`, or `big` alone, not `resident` + `big`
    budget = FakePool.bytes_of(resident.params) + FakePool.bytes_of(small.params) + 1
    assert FakePool.bytes_of(big.params) <= budget
    pool = FakePool(budget=budget)
    recs, stats = make_server(pool, 10).serve([resident, big, small])
    admitted = [s for e, s, _ in pool.log if e == "admit"]
    # slots in admission order: resident (0), small (1) while big waits, big (2)
    assert admitted == [0, 1, 2]
    assert recs[2].admitted < recs[1].admitted               # small passed big
    assert recs[1].admitted >= recs[0].finished - 1e-9       # big after resident left
    assert stats["rejected"] == 0


def test_a_request_larger_than_the_pool_is_rejected():
    pool = FakePool(budget=10 ** 5)
    reqs = [request(0, 0.0, 10 ** 6, 64, 20), request(1, 0.001, 100, 64, 20)]
    recs, stats = make_server(pool, 10).serve(reqs)
    assert recs[0].rejected and recs[0].result is None
    assert not recs[1].rejected and int(recs[1].result["step"]) == 20
    assert stats["rejected"] == 1 and stats["particle_steps"] == 100 * 20


def test_an_invalid_request_is_rejected_not_fatal():
    pool = FakePool(budget=10 ** 9)
    reqs = [request(0, 0.0, 100, 8192, 20), request(1, 0.0, 100, 64, 20)]
    recs, stats = make_server(pool, 10).serve(reqs)
    assert recs[0].rejected and not recs[1].rejected
    assert stats["rejected"] == 1


def test_late_arrivals_join_running_advances():
    pool = FakePool(budget=10 ** 9)
    reqs = [request(0, 0.0, 1000, 64, 400)] + [
        request(i, 0.01 + 0.002 * i, 500, 64, 40) for i in range(1, 6)]
    recs, stats = make_server(pool, 5).serve(reqs)
    # some advance moved the first run together with later ones
    assert max(a for e, _, a in pool.log if e == "advance") >= 2
    assert all(r.finished < recs[0].finished for r in recs[1:])
    assert stats["mean_active"] > 1.0


def test_kept_requests_return_state_field_and_history():
    pool = FakePool(budget=10 ** 9, history=64)
    reqs = [request(0, 0.0, 300, 32, 20), request(1, 0.0, 300, 32, 20)]
    recs, _ = make_server(pool, 7).serve(reqs, keep={1})
    (x, v), field, hist = recs[1].result
    assert x.shape == (300,) and field["E"].shape == (32,)
    assert hist["step"].tolist() == list(range(21))
    assert int(recs[0].result["step"]) == 20


def test_a_server_that_never_advances_is_refused():
    # checked before any device pool is made
    with pytest.raises(ValueError):
        serve.Server(arena_bytes=1 << 20, advance_steps=0)


def test_cancelled_requests_leave_the_queue_or_give_back_their_slot():
    pool = FakePool(budget=10 ** 9)
    long = request(0, 0.0, 1000, 64, 10 ** 5)
    long.cancel_at = 0.03                       # resident by then, far from done
    late = request(1, 0.04, 500, 64, 30)
    late.cancel_at = 0.0                        # cancelled as it arrives
    plain = request(2, 0.0, 700, 64, 40)
    log = io.StringIO()
    recs, stats = make_server(pool, 10).serve([long, late, plain], log=log)
    assert recs[0].outcome == "cancelled" and recs[0].cancelled >= 0.03
    assert 0 < pool.released[0] < long.steps    # released mid-flight
    assert recs[1].outcome == "cancelled" and recs[1].admitted == -1.0
    assert recs[2].outcome == "finished" and int(recs[2].result["step"]) == 40
    assert stats["cancelled"] == 2 and stats["particle_steps"] == 700 * 40
    assert not pool.runs and pool.used == 0
    lines = [json.loads(l) for l in log.getvalue().splitlines()]
    assert sorted(d["rid"] for d in lines) == [0, 1, 2]
    assert {d["rid"]: d["outcome"] for d in lines} == {0: "cancelled", 1: "cancelled",
                                                      2: "finished"}


@pytest.mark.parametrize("how", ["pool", "injected"])
def test_a_lost_worker_resubmits_its_resident_requests(how):
    pools = []

    def make_pool():
        pools.append(FakePool(budget=10 ** 9))
        return pools[-1]

    first = FakePool(budget=10 ** 9, lose_on_advance=3 if how == "pool" else None)
    pools.append(first)
    reqs = [request(i, 0.0, 100 * (i + 1), 64, 50) for i in range(4)]
    reqs.append(request(4, 0.2, 300, 64, 20))    # arrives after the loss
    log = io.StringIO()
    srv = make_server(first, 10, make_pool)
    recs, stats = srv.serve(reqs, log=log, crash_after={3} if how == "injected" else ())
    assert stats["worker_crashes"] == 1 and len(pools) == 2 and first.closed
    assert [r.restarts for r in recs] == [1, 1, 1, 1, 0]
    for r, q in zip(recs, reqs):
        assert r.outcome == "finished" and int(r.result["step"]) == q.steps
    # the reruns went through the new pool from their start
    assert [s for e, s, _ in pools[1].log if e == "admit"] == [0, 1, 2, 3, 4]
    assert stats["restarts"] == 4 and stats["particle_steps"] == sum(
        q.params.npart * q.steps for q in reqs)
    lines = [json.loads(l) for l in log.getvalue().splitlines()]
    assert {d["rid"]: d["restarts"] for d in lines} == {0: 1, 1: 1, 2: 1, 3: 1, 4: 0}
    assert all(d["latency"] > 0 and d["particle_steps"] == d["npart"] * d["steps"]
               for d in lines)


def test_log_lines_of_rejected_requests():
    pool = FakePool(budget=10 ** 5)
    log = io.StringIO()
    recs, stats = make_server(pool, 10).serve(
        [request(0, 0.0, 10 ** 6, 64, 20), request(1, 0.0, 100, 64, 20)], log=log)
    lines = {json.loads(l)["rid"]: json.loads(l) for l in log.getvalue().splitlines()}
    assert lines[0]["outcome"] == "rejected" and "latency" not in lines[0]
    assert lines[1]["outcome"] == "finished" and math.isfinite(lines[1]["latency"])


def test_a_worker_lost_while_reading_results_keeps_the_unread_ones():
    pools = []

    def make_pool():
        pools.append(FakePool(budget=10 ** 9))
        return pools[-1]

    first = FakePool(budget=10 ** 9, lose_on_read=2)     # the second result read fails
    pools.append(first)
    reqs = [request(i, 0.0, 100 * (i + 1), 64, 20) for i in range(3)]   # all finish together
    recs, stats = make_server(first, 10, make_pool).serve(reqs)
    assert stats["worker_crashes"] == 1
    assert [r.restarts for r in recs] == [0, 1, 1]        # the first was read and retired
    assert all(r.outcome == "finished" and int(r.result["step"]) == 20 for r in recs)
