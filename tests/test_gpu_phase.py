"""Phase-space snapshots (the Sec. 4 two-stream test, Fig. 1): the device
histogram against the oracle's counts (orc_phase_space, the same float32 bin
rule) of the run's own particles, and the paper's observation that the beams
mix by t = 20."""
import math

import numpy as np
import pytest

import paper_1108_1954_gb300 as pic  # noqa: E402
import torch  # noqa: E402,F401
import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
L4PI = 4.0 * math.pi


@pytest.mark.parametrize("nx,nv", [(64, 64), (128, 100), (1, 1)])
def test_phase_space_counts(nx, nv):
    n = 100003
    x, v = W.two_stream(n, L4PI, 0.2, 0.05, 3)
    run = pic.Run(pic.Params(npart=n, ncell=64, length=L4PI), device="cuda:0")
    run.init(*W.to_f32_state(x, v, L4PI))
    run.step_n(7)
    us, vs = run.get_cells()
    got = run.phase_space(nx, nv, -0.5, 0.5)
    # the bin rule on the stored cell coordinates: a box of length NG
    assert np.array_equal(got, O.phase_space(nx, nv, 64, -0.5, 0.5, us, vs))
    with pytest.raises(pic.PicError):
        run.phase_space(200, 200, -1.0, 1.0)           # above the bin limit


def test_two_stream_beams_mix_by_t20():
    # Fig. 1: at t = 0 two lines at v = +-0.2; by t = 20 the instability has
    # moved beam particles to velocities near zero.  The slow fraction is a
    # coarse phase-space statistic, so it is compared with the oracle's run
    # from the same state (8.9% of the particles at |v| < 0.1 at step 200).
    n, ng = 20000, 64
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, 11)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    run = pic.Run(pic.Params(npart=n, ncell=ng, length=L4PI), device="cuda:0")
    run.init(x32, v32)
    f0 = run.phase_space(64, 40, -0.4, 0.4)
    run.step_n(200)
    f20 = run.phase_space(64, 40, -0.4, 0.4)
    slow = slice(15, 25)                       # |v| < 0.1
    assert f0[slow].sum() == 0
    assert f0.sum() == n and f20.sum() <= n
    st = O.State(O.params(ng, n, L4PI, 0.1), x32.astype(np.float64), v32.astype(np.float64))
    for _ in range(200):
        st.step()
    frac_oracle = float(np.mean(np.abs(st.v) < 0.1))
    frac_gpu = f20[slow].sum() / n
    assert frac_oracle > 0.05
    assert abs(frac_gpu - frac_oracle) < 0.01
