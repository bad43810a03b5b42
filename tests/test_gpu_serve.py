"""The serving loop: every request finishes, and a request's result is the
same (bit for bit in particles and field) alone and in the mix."""
import math

import numpy as np
import pytest

import paper_1108_1954_gb300 as pic  # noqa: E402
import torch  # noqa: E402,F401
import workloads as W
from paper_1108_1954_gb300 import serve

pytestmark = pytest.mark.gpu


def small_stream(n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        npart = int(rng.integers(1000, 200000))
        ncell = int(rng.choice([64, 100, 256, 1000, 1024]))
        steps = int(rng.integers(20, 60))
        L = 4 * math.pi
        reqs.append(serve.Request(i, 0.003 * i,
                                  pic.Params(npart=npart, ncell=ncell, length=L, dt=0.1),
                                  pic.Loading(v0=0.2, vth=0.01, seed=1000 + i,
                                              modes=W.two_stream_modes_1_to_8(1e-4, i)),
                                  steps))
    return reqs


def test_served_results_equal_alone():
    reqs = small_stream(24, 1)
    keep = [0, 5, 11, 23]
    srv = serve.Server(arena_bytes=1 << 30, max_slots=6, ncell_max=1024, history=64,
                       advance_steps=7, device="cuda:0")
    recs, stats = srv.serve(reqs, keep=keep)
    assert stats["requests"] == 24
    assert all(r.finished >= r.admitted >= r.arrival - 1e-9 for r in recs)
    assert stats["p99_s"] >= stats["p50_s"] > 0
    for rid in keep:
        req = reqs[rid]
        (xs, vs), f, hist = recs[rid].result
        run = pic.Run(pic.Params(npart=req.params.npart, ncell=req.params.ncell,
                                 length=req.params.length, dt=0.1, history=64), device="cuda:0")
        run.init_loaded(req.loading)
        run.step_n(req.steps)
        x, v = run.get_state()
        g = run.get_field()
        assert np.array_equal(xs, x) and np.array_equal(vs, v)
        assert np.array_equal(f["E"], g["E"]) and np.array_equal(f["rho_q"], g["rho_q"])
        d = run.diagnostics(0, req.steps + 1)
        assert np.allclose(hist["field"], d["field"], rtol=1e-12, atol=0)
        run.close()
    # every request's last row is its final step
    for r in recs:
        if r.rid not in keep:
            assert int(r.result["step"]) == r.steps
    srv.close()


def test_resubmitted_requests_after_a_lost_worker_give_the_same_results():
    # the worker is taken as lost after the second advance (injected on the
    # host); the new pool reruns the resident requests from their seeds
    reqs = small_stream(10, 2)
    srv = serve.Server(arena_bytes=1 << 30, max_slots=6, ncell_max=1024, history=64,
                       advance_steps=7, device="cuda:0")
    base, _ = srv.serve(reqs)
    again, stats = srv.serve(reqs, crash_after={2})
    assert stats["worker_crashes"] == 1 and stats["restarts"] >= 1
    assert any(r.restarts == 1 for r in again)
    for a, b in zip(base, again):
        assert a.outcome == b.outcome == "finished"
        assert a.result.tobytes() == b.result.tobytes()      # the last row, bit for bit
    srv.close()


def test_a_cancelled_resident_request_frees_its_memory():
    reqs = small_stream(4, 3)
    reqs[0].steps = 100000                       # would run for a long time
    reqs[0].cancel_at = 0.05
    srv = serve.Server(arena_bytes=1 << 30, max_slots=6, ncell_max=1024, history=64,
                       advance_steps=7, device="cuda:0")
    recs, stats = srv.serve(reqs)
    assert recs[0].outcome == "cancelled" and recs[0].admitted >= 0.0
    assert all(r.outcome == "finished" for r in recs[1:])
    assert stats["cancelled"] == 1
    assert srv.pool.usage()[0] == 0              # every slot and byte given back
    srv.close()
