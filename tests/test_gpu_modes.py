"""The mode amplitudes of the diagnostics rows (the |E_m| the Sec. 4
two-stream test follows in time) against the oracle's orc_mode_amplitudes of
the GPU's own field, element by element for m = 1..8.

The device forms the modes of node g from the float32 copy of E with float32
twiddles (one sincospi of 2 pi g/NG, then the rotation e^{-i theta} applied m
times), sums them in float32 over the nodes of a block (a warp tree of depth 5,
then the warps in order) and in float64 over the blocks.  Each of those steps
rounds at most once per level, so every mode sum is off by at most
sum_g |E_g| (2 m + 3 + 5 + 16) 2^-24 (twiddle, rounding of E, warp tree, at
most 16 warps), and the amplitude 2 |sum| / NG by sqrt(2) times that times
2/NG.  The test takes (2/NG) sum_g |E_g| 64 2^-24, above that bound for
m <= 8, and far below a wrong normalisation or phase sign."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

import paper_1108_1954_gb300 as pic  # noqa: E402
import torch  # noqa: E402,F401

pytestmark = pytest.mark.gpu
L4PI = 4.0 * math.pi


def check_modes(row, E, ng, n, L):
    ref = O.mode_amplitudes(O.params(ng, n, L), E, 8)
    tol = (2.0 / ng) * np.abs(E).sum() * 64 * 2.0 ** -24
    assert np.abs(row["mode"] - ref).max() <= tol, (row["mode"], ref, tol)
    return ref


@pytest.mark.parametrize("ng,n,modes", [
    (64, 20000, ((3, 0.05, 0.0),)),                       # one clean cosine
    (64, 20001, ((1, 0.02, 0.7), (2, 0.01, -1.3))),       # two modes, phases
    (4096, 1 << 20, None),                                # config-2 recipe
])
def test_mode_amplitudes_match_the_oracle(ng, n, modes):
    seed = 7 + ng
    if modes is None:
        modes = W.two_stream_modes_1_to_8(1e-4, seed)
        x, v = W.two_stream(n, L4PI, 0.2, 0.01, seed, modes=modes)
    else:
        x, v = W.two_stream(n, L4PI, 0.0, 0.0, seed, modes=modes)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    run = pic.Run(pic.Params(npart=n, ncell=ng, length=L4PI, history=64), device="cuda:0")
    run.init(x32, v32)
    ref0 = check_modes(run.diagnostics(0, 1)[0], run.get_field()["E"], ng, n, L4PI)
    # the seeded modes carry the field: a lone mode dominates, and two modes
    # stand far above the rest
    seeded = [m - 1 for m, _, _ in modes]
    if len(modes) <= 2:
        rest = np.delete(ref0, seeded)
        assert ref0[seeded].min() > 10 * rest.max()
    run.step_n(3)
    check_modes(run.diagnostics(3, 1)[0], run.get_field()["E"], ng, n, L4PI)
    run.close()


def test_mode_amplitude_of_a_cosine_density():
    """A cold lattice displaced by xi = -(eps/k) sin(k x0) carries the charge
    density rho = -eps cos(k x) on the ion background (to first order), whose
    field by Gauss's law is E = -(eps/k) sin(k x): amplitude eps/k in mode m.
    The grid changes it by the factors of the linear weighting (deposit),
    the Eq. 6 operator and the Eq. 7 difference, together
    sin(k dx)/(k dx) = 0.994 at k dx = 0.196 here; 2% covers that."""
    ng, n, m, eps = 64, 64000, 2, 1e-3
    x, v = W.cold_langmuir(n, L4PI, eps, mode=m)
    x32, v32 = W.to_f32_state(x, v, L4PI)
    run = pic.Run(pic.Params(npart=n, ncell=ng, length=L4PI, history=8), device="cuda:0")
    run.init(x32, v32)
    row = run.diagnostics(0, 1)[0]
    ref = check_modes(row, run.get_field()["E"], ng, n, L4PI)
    k = 2 * math.pi * m / L4PI
    assert abs(row["mode"][m - 1] - eps / k) <= 0.02 * eps / k
    # the second harmonic of the displacement is of relative order eps/4
    assert np.delete(row["mode"], m - 1).max() < 2e-3 * eps / k
    assert abs(ref[m - 1] - eps / k) <= 0.02 * eps / k
    run.close()
