"""Multi-step runs on the GPU judged by invariants and growth rates (the
trajectories themselves are chaotic after saturation), the counting sort, and
checkpoint/restore."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from units import to_cells

import paper_1108_1954_gb300 as pic  # noqa: E402
import torch  # noqa: E402,F401

pytestmark = pytest.mark.gpu
L4PI = 4.0 * math.pi
L_FAST = 2 * math.pi * 0.2 / math.sqrt(0.375)


def make_run(n, ng, L, **kw):
    return pic.Run(pic.Params(npart=n, ncell=ng, length=L, **kw), device="cuda:0")


def c1_state(seed=11):
    x, v = W.two_stream(20000, L4PI, 0.2, 0.01, seed)
    return W.to_f32_state(x, v, L4PI)


@pytest.mark.parametrize("sort_interval", [0, 20])
def test_c1_conservation(sort_interval):
    # the Sec. 4 run: 20,000 electrons, 64 cells, 200 steps
    x32, v32 = c1_state()
    run = make_run(20000, 64, L4PI, sort_interval=sort_interval)
    run.init(x32, v32)
    run.step_n(200)
    d = run.diagnostics(0, 200)
    assert (d["charge_q"] == 20000 << O.FIX_BITS).all()
    assert np.abs(d["charge"]).max() < 1e-12
    tot = d["kinetic"] + d["field"]
    assert (tot.max() - tot.min()) / tot[0] < 0.01
    m = L4PI / 20000
    assert np.abs(d["momentum"] - d["momentum"][0]).max() <= 1e-6 * m * np.abs(v32).sum()
    assert d["field"][-1] > 100 * d["field"][0]
    # the oracle's run from the same state lands on the same energy budget
    ref = O.State(O.params(64, 20000, L4PI), x32.astype(np.float64), v32.astype(np.float64))
    h = ref.run(200)
    ke_ref = 0.5 * ref.mass * h[:, 0]
    assert abs(ke_ref[0] - d["kinetic"][0]) <= 1e-5 * ke_ref[0]
    # linear phase (t <= 5): field energy follows the oracle's closely
    fe_ref = h[:, 2]
    assert np.abs(d["field"][:50] - fe_ref[:50]).max() <= 1e-3 * fe_ref[:50].max()


@pytest.mark.parametrize("lx,vth", [(L4PI, 0.0), (L_FAST, 0.0), (L_FAST, 0.01)])
def test_two_stream_growth_rate(lx, vth):
    n, v0, dt = 20000, 0.2, 0.1
    k = 2 * math.pi / lx
    gamma = W.cold_two_stream_gamma(k, v0)
    x, v = W.two_stream_eigenmode(n, lx, v0, vth, 1e-3, 1, 5)
    run = make_run(n, 64, lx)
    run.init(*W.to_f32_state(x, v, lx))
    run.step_n(122)
    d = run.diagnostics(0, 122)
    t = np.arange(122) * dt
    sel = (t >= 2.0) & (t <= 12.0)
    rate = np.polyfit(t[sel], np.log(d["mode"][sel, 0]), 1)[0]
    assert abs(rate - gamma) / gamma < 0.05, (rate, gamma)


def test_langmuir_frequency():
    n, dt = 20000, 0.1
    x, v = W.cold_langmuir(n, L4PI, 1e-3, 1)
    run = make_run(n, 64, L4PI)
    run.init(*W.to_f32_state(x, v, L4PI))
    run.step_n(400)
    fe = run.diagnostics(0, 400)["field"]
    peaks = []
    for i in range(1, fe.size - 1):
        if fe[i] > fe[i - 1] and fe[i] >= fe[i + 1]:
            a, b, c = fe[i - 1], fe[i], fe[i + 1]
            peaks.append((i + 0.5 * (a - c) / (a - 2 * b + c)) * dt)
    omega = math.pi / ((peaks[-1] - peaks[0]) / (len(peaks) - 1))
    assert abs(omega - 1.0) < 0.01


def _keys(u, ng):
    """The sort key of a cell coordinate: trunc(u), clamped to the grid."""
    return np.clip(u.astype(np.float64), 0, ng - 1).astype(np.int64)


def test_sort_is_a_stable_permutation():
    n, ng, L = 200003, 1024, L4PI
    rng = np.random.default_rng(2)
    x32 = rng.uniform(0, L, n).astype(np.float32)
    v32 = (np.arange(n) * 1e-6).astype(np.float32)   # original order, recoverable
    run = make_run(n, ng, L)
    run.init(x32, v32)
    f0 = run.get_field()
    u32 = to_cells(x32, ng, L)
    run.sort()
    xs, vs = run.get_cells()
    k = _keys(xs, ng)
    assert (np.diff(k) >= 0).all()
    # same multiset of (u, v) pairs
    a = np.lexsort((v32, u32))
    b = np.lexsort((vs, xs))
    assert np.array_equal(u32[a], xs[b]) and np.array_equal(v32[a], vs[b])
    # stable: within a cell the original order (increasing v) is kept
    same = np.diff(k) == 0
    assert (np.diff(vs)[same] > 0).all()
    run.deposit()
    run.solve_field()
    assert np.array_equal(run.get_field()["rho_q"], f0["rho_q"])


def test_sorted_and_unsorted_runs_hold_the_same_particles():
    n, ng = 100001, 256
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, 8)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    a = make_run(n, ng, L4PI, sort_interval=5)
    b = make_run(n, ng, L4PI, sort_interval=0)
    a.init(x32, v32)
    b.init(x32, v32)
    a.step_n(23)
    b.step_n(23)
    assert np.array_equal(a.get_field()["rho_q"], b.get_field()["rho_q"])
    xa, va = a.get_cells()
    xb, vb = b.get_cells()
    ia, ib = np.lexsort((va, xa)), np.lexsort((vb, xb))
    assert np.array_equal(xa[ia], xb[ib]) and np.array_equal(va[ia], vb[ib])


def test_checkpoint_restore_is_bit_identical():
    # a checkpoint in cell coordinates (get_cells / set_cells) continues bit
    # for bit; one in physical units (get_state / set_state) continues to the
    # float32 rounding of the two conversions
    n, ng = 50001, 128
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, 6)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    a = make_run(n, ng, L4PI, sort_interval=7)
    a.init(x32, v32)
    a.step_n(40)
    b = make_run(n, ng, L4PI, sort_interval=7)
    b.init(x32, v32)
    b.step_n(19)
    us, vs = b.get_cells()
    c = make_run(n, ng, L4PI, sort_interval=7)
    c.set_cells(us, vs, 19)
    c.step_n(21)
    xa, va = a.get_state()
    xc, vc = c.get_state()
    assert np.array_equal(xa, xc) and np.array_equal(va, vc)
    assert np.array_equal(a.get_cells()[0], c.get_cells()[0])
    assert np.array_equal(a.get_field()["rho_q"], c.get_field()["rho_q"])
    xs, vs = b.get_state()
    d = make_run(n, ng, L4PI, sort_interval=7)
    d.set_state(xs, vs, 19)
    ud, _ = d.get_cells()
    # the round trip moves a cell coordinate by at most two float32 steps
    # (periodically: a coordinate within a step of NG may come back as 0)
    du = np.abs(ud.astype(np.float64) - us)
    assert np.minimum(du, ng - du).max() <= 2.0 ** -22 * ng
    assert d.step == 19
    with pytest.raises(pic.PicError) as e:        # coordinates outside [0, NG)
        bad = us.copy()
        bad[3] = np.float32(ng)
        d.set_cells(bad, vs, 0)
    assert e.value.code == pic.PIC_EINVAL


def test_graph_replay_equals_single_steps():
    n, ng = 20000, 64
    x32, v32 = c1_state(3)
    a = make_run(n, ng, L4PI, sort_interval=4)
    a.init(x32, v32)
    a.step_n(37)                     # graph periods + single steps
    b = make_run(n, ng, L4PI, sort_interval=4)
    b.init(x32, v32)
    for i in range(37):
        if i > 0 and i % 4 == 0:
            b.sort()
        b.push()
        b.solve_field()
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    da, db = a.diagnostics(0, 37), b.diagnostics(0, 37)
    assert np.array_equal(da["field"], db["field"])


@pytest.mark.parametrize("layout", ["sorted_jitter", "sorted_blocks_reversed", "mixed"])
def test_sort_matches_stable_argsort(layout):
    # The scatter has two paths: tiles whose keys span few cells (the state a
    # periodic sort leaves behind) and tiles that span many.  Both must give
    # exactly the stable order by cell.
    n, ng, L = 300007, 4096, L4PI
    rng = np.random.default_rng(3)
    base = np.sort(rng.uniform(0, L, n))
    if layout == "sorted_jitter":
        x = base + rng.normal(0, 2.0 * L / ng, n)
    elif layout == "sorted_blocks_reversed":
        x = np.concatenate([b[::-1] for b in np.array_split(base, 97)])
    else:
        x = base.copy()
        wild = rng.random(n) < 0.002
        x[wild] = rng.uniform(0, L, wild.sum())
    x32, _ = W.to_f32_state(np.mod(x, L), np.zeros(n), L)
    v32 = (np.arange(n) * 1e-6).astype(np.float32)
    run = make_run(n, ng, L)
    run.init(x32, v32)
    u32 = to_cells(x32, ng, L)
    run.sort()
    xs, vs = run.get_cells()
    perm = np.argsort(_keys(u32, ng), kind="stable")
    assert np.array_equal(xs, u32[perm]) and np.array_equal(vs, v32[perm])
    run.sort()
    xs2, vs2 = run.get_cells()
    assert np.array_equal(xs2, xs) and np.array_equal(vs2, vs)


def test_sort_interval_tuner_leaves_the_state_and_adopts():
    n, ng = 400003, 1024
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, 21)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    a = make_run(n, ng, L4PI, sort_interval=10)
    b = make_run(n, ng, L4PI, sort_interval=10)
    a.init(x32, v32)
    b.init(x32, v32)
    a.step_n(13)
    b.step_n(13)
    best, table = a.tune_sort_interval((0, 3, 10, 40), adopt=False)
    assert best in (0, 3, 10, 40) and set(table) == {0, 3, 10, 40}
    assert all(t > 0 for t in table.values())
    assert table[best] == min(table.values())
    assert a.p.sort_interval == 10
    ua, va = a.get_cells()
    ub, vb = b.get_cells()
    assert np.array_equal(ua, ub) and np.array_equal(va, vb)
    # adopting: the run then sorts at the chosen interval, exactly like a run
    # created with it from the same state
    best, _ = a.tune_sort_interval((3,), adopt=True)
    assert best == 3 and a.p.sort_interval == 3
    c = make_run(n, ng, L4PI, sort_interval=3)
    c.set_cells(ua, va, 13)
    a.step_n(11)
    c.step_n(11)
    assert np.array_equal(a.get_cells()[0], c.get_cells()[0])
    assert np.array_equal(a.get_field()["rho_q"], c.get_field()["rho_q"])
