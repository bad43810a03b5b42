"""Combinations of the run options (precision mode x field solver x shape x
sort interval) against the invariants that hold for all of them: exact
charge, conserved momentum to the mode's rounding, graphs equal to single
launches, and the checkpoint round trip."""
import math

import numpy as np
import pytest

import paper_1108_1954_gb300 as pic  # noqa: E402
import torch  # noqa: E402,F401
import workloads as W

pytestmark = pytest.mark.gpu
L4PI = 4.0 * math.pi


def _state(n, precision, seed):
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, seed, modes=((1, 1e-2, 0.0), (3, 1e-2, 1.0)))
    if precision == pic.PIC_FP64:
        return x, v
    return W.to_f32_state(x, v, L4PI)


@pytest.mark.parametrize("precision,solver,shape,sort", [
    (pic.PIC_FP32_FIXED, pic.PIC_SOLVER_CG, pic.PIC_SHAPE_CIC, 5),
    (pic.PIC_FP32_FIXED, pic.PIC_SOLVER_CG, pic.PIC_SHAPE_NGP, 5),
    (pic.PIC_FP32_FIXED, pic.PIC_SOLVER_EXACT, pic.PIC_SHAPE_NGP, 0),
    (pic.PIC_FP32_ATOMIC, pic.PIC_SOLVER_CG, pic.PIC_SHAPE_CIC, 7),
    (pic.PIC_FP64, pic.PIC_SOLVER_CG, pic.PIC_SHAPE_CIC, 7),
    (pic.PIC_FP64, pic.PIC_SOLVER_EXACT, pic.PIC_SHAPE_CIC, 0),
])
def test_option_combinations(precision, solver, shape, sort):
    n, ng, steps = 30001, 128, 40
    x, v = _state(n, precision, 3)
    p = pic.Params(npart=n, ncell=ng, length=L4PI, precision=precision, field_solver=solver,
                   shape=shape, sort_interval=sort, history=64)
    a = pic.Run(p, device="cuda:0")
    a.init(x, v)
    a.step_n(steps)
    d = a.diagnostics(0, steps)
    m = L4PI / n
    vabs = m * np.abs(np.asarray(v, dtype=np.float64)).sum()
    tol = 1e-12 if precision == pic.PIC_FP64 else 1e-5
    assert np.abs(d["momentum"] - d["momentum"][0]).max() <= tol * vabs + 1e-300
    if precision == pic.PIC_FP32_FIXED:
        assert (d["charge_q"] == n << 24).all()
        assert (d["charge"] == 0.0).all()                # sum_g R_g = 0 exactly
    else:
        # float sums of N weights: ~N eps relative, times NG nodes
        eps = 1e-7 if precision == pic.PIC_FP32_ATOMIC else 1e-15
        assert np.abs(d["charge"]).max() <= 10 * eps * ng * L4PI
    # graphs (step_n) and single launches give the same state
    b = pic.Run(p, device="cuda:0")
    b.init(x, v)
    for _ in range(steps):
        b.step_n(1)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    if precision == pic.PIC_FP32_FIXED:
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    else:
        # float atomics sum in a launch-dependent order: the positions differ
        # at the rounding level, and a sort may then order two neighbours of
        # a cell boundary differently, so the particles are compared as sets
        # (ordered by position, then velocity)
        ia, ib = np.lexsort((va, xa)), np.lexsort((vb, xb))
        assert np.abs(xa[ia] - xb[ib]).max() <= 1e-3 * L4PI
    # checkpoint round trip: restore the state at step `steps` (as the device
    # holds it: cell coordinates in the float32 modes) and go on
    c = pic.Run(p, device="cuda:0")
    if precision == pic.PIC_FP64:
        c.set_state(xa, va, steps)
    else:
        c.set_cells(*a.get_cells(), steps)
    c.step_n(5)
    a.step_n(5)
    xc, vc = c.get_state()
    xa2, va2 = a.get_state()
    if precision == pic.PIC_FP32_FIXED:
        assert np.array_equal(xc, xa2) and np.array_equal(vc, va2)
    for r in (a, b, c):
        r.close()
