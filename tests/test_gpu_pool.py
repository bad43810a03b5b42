"""Batched and served runs against the same runs alone.

The pool advances many runs in one cluster launch; each run's particles,
field and fixed-point density must be bit-identical to the single-run path
(same operations on the same numbers), whatever the launch shape, the mix of
runs or the moment a run was admitted.  Diagnostics sum in another order and
agree to rounding.
"""
import math

import numpy as np
import pytest

import paper_1108_1954_gb300 as pic  # noqa: E402
import torch  # noqa: E402,F401
import workloads as W

pytestmark = pytest.mark.gpu
L4PI = 4.0 * math.pi
GIB = 1 << 30


def run_set():
    """Runs of different sizes, grids and beams (ragged N, tiny N and NG)."""
    specs = [(20000, 64, 0.2, 0.01), (100003, 2048, 0.35, 0.02), (4099, 200, 0.1, 0.0),
             (5, 16, 0.3, 0.05), (1, 1, 0.2, 0.0), (77777, 512, 0.05, 0.001),
             (250001, 1024, 0.5, 0.03), (3, 7, 0.2, 0.01), (65537, 4096, 0.2, 0.01)]
    out = []
    for i, (n, ng, v0, vth) in enumerate(specs):
        x, v = W.two_stream(n, L4PI, v0, vth, 100 + i)
        x32, v32 = W.to_f32_state(x, v, L4PI)
        out.append((pic.Params(npart=n, ncell=ng, length=L4PI, dt=0.1), x32, v32))
    return out


def alone(p, x32, v32, steps):
    run = pic.Run(pic.Params(npart=p.npart, ncell=p.ncell, length=p.length, dt=p.dt,
                             sort_interval=p.sort_interval, history=512), device="cuda:0")
    run.init(x32, v32)
    run.step_n(steps)
    x, v = run.get_state()
    f = run.get_field()
    d = run.diagnostics(0, steps + 1)
    run.close()
    return x, v, f, d


def assert_same(pool, slot, ref, steps):
    x, v, f, d = ref
    xs, vs = pool.get_state(slot)
    assert np.array_equal(xs, x) and np.array_equal(vs, v)
    fs = pool.get_field(slot)
    assert np.array_equal(fs["rho_q"], f["rho_q"])
    assert np.array_equal(fs["E"], f["E"])
    assert np.array_equal(fs["rho"], f["rho"])
    np.testing.assert_allclose(fs["phi"], f["phi"], rtol=0, atol=1e-12 * max(1e-300, np.abs(f["phi"]).max()))
    ds = pool.diagnostics(slot, 0, steps + 1)
    assert ds["step"].tolist() == d["step"].tolist()
    assert (ds["charge_q"] == d["charge_q"]).all()
    # field energy: float64 node sums in another order
    a, b = ds["field"], d["field"]
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * max(np.abs(b).max(), 1e-300))
    # kinetic energy and momentum: float32 per-thread partial sums over a
    # different split of the particles, float64 across threads
    p = pool.params[slot]
    m = p.length / p.npart
    vabs = m * np.abs(vs.astype(np.float64)).sum()
    a, b = ds["kinetic"][:-1], d["kinetic"][:-1]
    assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * max(np.abs(b).max(), 1e-300)), "kinetic"
    a, b = ds["momentum"][:-1], d["momentum"][:-1]
    assert np.allclose(a, b, rtol=0, atol=1e-5 * vabs + 1e-300), "momentum"
    assert np.isnan(ds["kinetic"][-1]) and np.isnan(d["kinetic"][-1])
    np.testing.assert_allclose(ds["mode"], d["mode"], rtol=1e-4, atol=1e-6 * max(1e-300, np.abs(d["mode"]).max()))


@pytest.mark.parametrize("variant,cluster,block,ncell_max",
                         [(2, 8, 256, 2048), (1, 8, 256, 2048), (5, 4, 512, 2048),
                          (2, 2, 512, 1024), (2, 1, 512, 512), (1, 4, 256, 1024),
                          (2 + 16, 8, 512, 4096), (5 + 16, 8, 256, 2048)])
def test_batched_equals_alone(variant, cluster, block, ncell_max):
    runs = [r for r in run_set() if r[0].ncell <= ncell_max]
    steps = 23
    pool = pic.Pool(max_slots=16, ncell_max=ncell_max, arena_bytes=GIB, history=512,
                    variant=variant, cluster=cluster, block=block, device="cuda:0")
    slots = [pool.admit(p, x, v, steps) for p, x, v in runs]
    assert None not in slots
    pool.advance(7)
    pool.advance(100)          # each run stops at its own 23
    assert sorted(pool.finished()) == sorted(slots)
    for (p, x, v), s in zip(runs, slots):
        assert pool.step_count(s) == steps
        assert_same(pool, s, alone(p, x, v, steps), steps)


@pytest.mark.parametrize("variant,cluster,block,ncell_max,intervals",
                         [(1 + 16, 8, 256, 2048, (5, 3, 1, 7)), (5, 4, 512, 2048, (4, 9)),
                          (2, 2, 512, 1024, (6,)), (6, 1, 512, 512, (2, 5))])
def test_batched_with_sorting_equals_alone(variant, cluster, block, ncell_max, intervals):
    # Runs that sort every S steps (S differing between runs, sorts falling
    # on both sides of launch boundaries) give the same particles, density
    # and field as the same runs alone, bit for bit: the in-cluster counting
    # sort yields the unique stable order by cell of the single run's sort.
    runs = [r for r in run_set() if r[0].ncell <= ncell_max]
    for i, (p, _, _) in enumerate(runs):
        p.sort_interval = intervals[i % len(intervals)]
    steps = 23
    pool = pic.Pool(max_slots=16, ncell_max=ncell_max, arena_bytes=GIB, history=512,
                    variant=variant, cluster=cluster, block=block, device="cuda:0")
    slots = [pool.admit(p, x, v, steps) for p, x, v in runs]
    assert None not in slots
    pool.advance(3)
    pool.advance(8)
    pool.advance(100)
    for (p, x, v), s in zip(runs, slots):
        assert pool.step_count(s) == steps
        assert_same(pool, s, alone(p, x, v, steps), steps)


def test_pool_sort_needs_a_second_buffer():
    p = pic.Params(npart=100000, ncell=256, length=L4PI)
    q = pic.Params(npart=100000, ncell=256, length=L4PI, sort_interval=20)
    assert pic.pool_run_bytes(q, 64) - pic.pool_run_bytes(p, 64) >= 8 * 100000


def test_staggered_admission_equals_alone():
    # requests admitted while others are mid-run (continuous batching)
    runs = run_set()[:5]
    runs[1][0].sort_interval = 4           # one run sorts
    pool = pic.Pool(max_slots=8, ncell_max=2048, arena_bytes=GIB, history=512, device="cuda:0")
    plan = [(0, 30), (1, 17), (2, 25), (3, 9), (4, 12)]
    slots = {}
    slots[0] = pool.admit(runs[0][0], runs[0][1], runs[0][2], plan[0][1])
    pool.advance(6)
    slots[1] = pool.admit(runs[1][0], runs[1][1], runs[1][2], plan[1][1])
    slots[2] = pool.admit(runs[2][0], runs[2][1], runs[2][2], plan[2][1])
    pool.advance(5)
    slots[3] = pool.admit(runs[3][0], runs[3][1], runs[3][2], plan[3][1])
    pool.advance(11)
    slots[4] = pool.admit(runs[4][0], runs[4][1], runs[4][2], plan[4][1])
    for _ in range(10):
        pool.advance(4)
    for i, steps in plan:
        assert pool.step_count(slots[i]) == steps
        p, x, v = runs[i]
        assert_same(pool, slots[i], alone(p, x, v, steps), steps)


def test_admission_by_memory_and_slots():
    p = pic.Params(npart=100000, ncell=256, length=L4PI)
    per = pic.pool_run_bytes(p, 64)
    assert per >= 8 * 100000
    x, v = W.two_stream(100000, L4PI, 0.2, 0.01, 3)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    # room for the tables (a few KB for 4 slots) and exactly two runs
    pool = pic.Pool(max_slots=4, ncell_max=256, arena_bytes=2 * per + per // 2 + 4096,
                    history=64, device="cuda:0")
    a = pool.admit(p, x32, v32, 5)
    b = pool.admit(p, x32, v32, 5)
    assert a is not None and b is not None
    assert pool.admit(p, x32, v32, 5) is None            # arena full
    pool.advance(5)
    assert sorted(pool.finished()) == sorted([a, b])
    xa, _ = pool.get_state(a)
    pool.release(a)
    c = pool.admit(p, x32, v32, 5)                        # space reused
    assert c is not None
    pool.advance(5)
    xc, _ = pool.get_state(c)
    assert np.array_equal(xa, xc)
    used, free = pool.usage()
    assert used == 2 * per
    # slots run out before memory
    small = pic.Params(npart=10, ncell=8, length=1.0)
    pool2 = pic.Pool(max_slots=2, ncell_max=8, arena_bytes=1 << 24, history=8, device="cuda:0")
    xs = np.linspace(0, 1, 10, endpoint=False).astype(np.float32)
    vs = np.zeros(10, np.float32)
    assert pool2.admit(small, xs, vs, 1) is not None
    assert pool2.admit(small, xs, vs, 1) is not None
    assert pool2.admit(small, xs, vs, 1) is None


def test_pool_rejects_bad_input():
    pool = pic.Pool(max_slots=2, ncell_max=64, arena_bytes=1 << 24, history=8, device="cuda:0")
    p = pic.Params(npart=10, ncell=128, length=1.0)          # NG above the pool's limit
    xs = np.linspace(0, 1, 10, endpoint=False).astype(np.float32)
    with pytest.raises(pic.PicError):
        pool.admit(p, xs, np.zeros(10, np.float32), 1)
    p = pic.Params(npart=10, ncell=8, length=1.0)
    bad = xs.copy()
    bad[3] = 1.0
    with pytest.raises(pic.PicError):
        pool.admit(p, bad, np.zeros(10, np.float32), 1)
    with pytest.raises(pic.PicError):
        pool.configure(2, 3, 256)                            # cluster of 3
    with pytest.raises(pic.PicError):
        pool.configure(3, 8, 256)                            # packed variant
    with pytest.raises(pic.PicError):
        pool.configure(2, 1, 32)                             # 64 nodes > 32 threads


def test_pool_run_against_the_oracle():
    """A pooled run checked directly against the FP64 oracle, not only
    against the single-run path: the density of E^0's set-up and of one step
    bit for bit against orc_deposit_fixed of the pool's own float32
    positions, E against the oracle's direct solve of that density, and the
    step's particles within the one-step tolerances."""
    import oracle as O
    from test_gpu_parity import check_field_against_oracle, periodic_dist
    from units import to_cells
    n, ng, L = 100003, 1024, L4PI
    modes = W.two_stream_modes_1_to_8(1e-4, 21)
    x, v = W.two_stream(n, L, 0.2, 0.01, 21, modes=modes)
    x32, v32 = W.to_f32_state(x, v, L)
    pool = pic.Pool(max_slots=4, ncell_max=2048, arena_bytes=1 << 28, history=8,
                    device="cuda:0")
    # a second run shares the launch
    xo, vo = W.to_f32_state(*W.two_stream(5003, L, 0.3, 0.02, 22), L)
    pool.admit(pic.Params(npart=5003, ncell=300, length=L), xo, vo, 1)
    s = pool.admit(pic.Params(npart=n, ncell=ng, length=L), x32, v32, 1)
    pool.advance(0)
    f0 = pool.get_field(s)
    u0, _ = pool.get_cells(s)
    assert np.array_equal(u0, to_cells(x32, ng, L))
    assert np.array_equal(f0["rho_q"], O.deposit_fixed(ng, u0))
    check_field_against_oracle(f0, n, ng, L)
    pool.advance(1)
    x1, v1 = pool.get_state(s)
    ref = O.State(O.params(ng, n, L, 0.1), x32.astype(np.float64), v32.astype(np.float64))
    ref.step()
    assert periodic_dist(x1, ref.x, L).max() <= 1e-5 * L
    vscale = np.maximum(np.abs(ref.v), 0.2 + 0.01)
    assert (np.abs(v1 - ref.v) <= 1e-5 * vscale).all()
    f1 = pool.get_field(s)
    assert np.array_equal(f1["rho_q"], O.deposit_fixed(ng, pool.get_cells(s)[0]))
    check_field_against_oracle(f1, n, ng, L)
    pool.close()
