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
from units import to_cells

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
    assert np.array_equal(f["rho_q"], O.deposit_fixed_ngp(ng, to_cells(x32, ng, L4PI)))
    assert int(f["rho_q"].sum()) == n << O.FIX_BITS
    run.step_n(3)
    us, _ = run.get_cells()
    assert np.array_equal(run.get_field()["rho_q"], O.deposit_fixed_ngp(ng, us))


@pytest.mark.parametrize("n,ng", [(20000, 64), (100003, 1024)])
def test_ngp_one_step_parity(n, ng):
    # With nearest-grid-point weighting one particle in the neighbouring cell
    # changes E at a node by a whole particle charge, so the oracle starts
    # from the device's own positions (its cell coordinates times dx, in
    # float64) and every particle must then be in the same cell on both sides.
    x32, v32 = state(n, L4PI, 7 * n + ng)
    run = make_run(n, ng, L4PI)
    run.init(x32, v32)
    u0, _ = run.get_cells()
    dx = L4PI / ng
    x0 = u0.astype(np.float64) * dx
    ref = O.State(O.params(ng, n, L4PI, 0.1, shape=O.NGP), x0, v32.astype(np.float64))
    cell_dev = np.floor(u0).astype(np.int64) % ng
    cell_orc = (x0 / dx).astype(np.int64) % ng
    assert np.array_equal(cell_dev, cell_orc)
    f0 = run.get_field()
    assert np.abs(f0["E"] - ref.E).max() <= 1e-9 * np.abs(ref.E).max()
    run.push()
    run.solve_field()
    x1, v1 = run.get_state()
    ref.step()
    d = np.abs(x1 - ref.x)
    d = np.minimum(d, L4PI - d)
    assert d.max() <= 1e-5 * L4PI
    vscale = np.maximum(np.abs(ref.v), 0.21)
    assert (np.abs(v1 - ref.v) <= 1e-5 * vscale).all()
    assert np.array_equal(run.get_field()["rho_q"], O.deposit_fixed_ngp(ng, run.get_cells()[0]))


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
