"""Nearest-grid-point shape (PIC_SHAPE_NGP; Sec. 2, reading R13) on the GPU:
the fixed-point density bit for bit against the oracle's fixed-point NGP
deposit of the same float32 positions, one step against the FP64 oracle's
NGP step, momentum conservation, sort invariance and the API's guards."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1108_1954_gb300 as pic  # noqa: E402
import torch  # noqa: E402,F401
import workloads as W

pytestmark = pytest.mark.gpu
L4PI = 4.0 * math.pi


def make_run(n, ng, L, **kw):
    return pic.Run(pic.Params(npart=n, ncell=ng, length=L, shape=pic.PIC_SHAPE_NGP, **kw),
                   device="cuda:0")


def state(n, L, seed, v0=0.2, vth=0.01):
    x, v = W.two_stream(n, L, v0, vth, seed, modes=W.two_stream_modes_1_to_8(1e-3, seed))
    return W.to_f32_state(x, v, L)


@pytest.mark.parametrize("n,ng", [(1, 16), (5, 16), (20000, 64), (20003, 256),
                                  (262147, 4096), (50000, 8192)])
def test_ngp_density_bit_exact(n, ng):
    x32, v32 = state(n, L4PI, n + ng)
    run = make_run(n, ng, L4PI)
    run.init(x32, v32)
    f = run.get_field()
    assert np.array_equal(f["rho_q"], O.deposit_fixed_ngp(ng, L4PI, x32))
    assert int(f["rho_q"].sum()) == n << O.FIX_BITS
    run.step_n(3)
    xs, _ = run.get_state()
    assert np.array_equal(run.get_field()["rho_q"], O.deposit_fixed_ngp(ng, L4PI, xs))


@pytest.mark.parametrize("n,ng", [(20000, 64), (100003, 1024)])
def test_ngp_one_step_parity(n, ng):
    x32, v32 = state(n, L4PI, 7 * n + ng)
    run = make_run(n, ng, L4PI)
    run.init(x32, v32)
    ref = O.State(O.params(ng, n, L4PI, 0.1, shape=O.NGP), x32.astype(np.float64),
                  v32.astype(np.float64))
    run.push()
    run.solve_field()
    x1, v1 = run.get_state()
    ref.step()
    # a position within rounding of a cell boundary may fall in the other
    # cell in float32 (floor(x c)) than in float64 (trunc(x / dx)); those
    # few particles see the neighbouring node's field
    c32 = np.float32(ng / L4PI)
    cell32 = np.floor(x32 * c32).astype(np.int64) % ng
    cell64 = np.floor(x32.astype(np.float64) / (L4PI / ng)).astype(np.int64) % ng
    same = cell32 == cell64
    assert same.mean() > 0.999
    d = np.abs(x1 - ref.x)
    d = np.minimum(d, L4PI - d)
    assert d[same].max() <= 1e-5 * L4PI
    vscale = np.maximum(np.abs(ref.v), 0.21)
    assert (np.abs(v1 - ref.v)[same] <= 1e-5 * vscale[same]).all()
    assert np.array_equal(run.get_field()["rho_q"], O.deposit_fixed_ngp(ng, L4PI, x1))


def test_ngp_momentum_conserved_and_sort_invariant():
    n, ng = 100001, 256
    x32, v32 = state(n, L4PI, 11)
    a = make_run(n, ng, L4PI, sort_interval=7, history=256)
    b = make_run(n, ng, L4PI, sort_interval=0, history=256)
    a.init(x32, v32)
    b.init(x32, v32)
    a.step_n(150)
    b.step_n(150)
    assert np.array_equal(a.get_field()["rho_q"], b.get_field()["rho_q"])
    d = a.diagnostics(0, 150)
    m = L4PI / n
    mom = d["momentum"]
    assert np.abs(mom - mom[0]).max() <= 1e-5 * m * np.abs(v32).sum()
    assert d["field"][-1] > 10 * d["field"][0]          # the instability grows


def test_ngp_guards():
    n, ng = 1000, 64
    x32, v32 = state(n, L4PI, 1)
    with pytest.raises(pic.PicError):
        pic.Run(pic.Params(npart=n, ncell=ng, length=L4PI, shape=pic.PIC_SHAPE_NGP,
                           precision=pic.PIC_FP64), device="cuda:0")
    run = make_run(n, ng, L4PI)
    run.init(x32, v32)
    with pytest.raises(pic.PicError):
        run.set_launch(variant=pic.PIC_DEPOSIT_ATOMIC)
    run.set_launch(block=256)
    tune = run.autotune(reps=2)
    assert len(tune) > 0 and (tune["variant"] == 15).all()     # the NGP kernel
    pool = pic.Pool(max_slots=2, ncell_max=64, arena_bytes=1 << 24, history=4)
    with pytest.raises(pic.PicError):
        pool.admit(pic.Params(npart=n, ncell=ng, length=L4PI, shape=pic.PIC_SHAPE_NGP),
                   x32, v32, 10)
    pool.close()
