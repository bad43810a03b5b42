"""Pins of the oracle's nearest-grid-point weighting (Sec. 2: the density at
a grid point counts the particles of its cell; a particle feels the field of
its cell; reading R13): brute force against the nearest node by distance,
the cell-boundary convention, the invariants that make momentum conserved,
and the fixed-point form."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from units import to_cells

L4PI = 4.0 * math.pi


def _nearest_node(x, ng, lx):
    """Index of the node (cell centre) nearest to each x, by periodic distance."""
    dx = lx / ng
    nodes = (np.arange(ng) + 0.5) * dx
    d = np.abs(x[:, None] - nodes[None, :])
    d = np.minimum(d, lx - d)
    return np.argmin(d, axis=1)


def _away_from_boundaries(x, ng, lx, tol=1e-9):
    u = x / (lx / ng)
    return np.abs(u - np.rint(u)) > tol


@pytest.mark.parametrize("ng,npart", [(1, 5), (4, 7), (8, 3), (16, 200)])
def test_ngp_deposit_matches_nearest_node(ng, npart):
    rng = np.random.default_rng(ng * 100 + npart)
    x = rng.uniform(0, L4PI, npart)
    x = x[_away_from_boundaries(x, ng, L4PI)]
    p = O.params(ng, x.size, L4PI, shape=O.NGP)
    rho = O.deposit(p, x)
    counts = np.bincount(_nearest_node(x, ng, L4PI), minlength=ng)
    q_over_dx = -L4PI / x.size / (L4PI / ng)
    np.testing.assert_allclose(rho, 1.0 + q_over_dx * counts, rtol=0, atol=1e-13)


def test_ngp_gather_matches_nearest_node():
    ng = 16
    rng = np.random.default_rng(4)
    x = rng.uniform(0, L4PI, 300)
    x = x[_away_from_boundaries(x, ng, L4PI)]
    p = O.params(ng, x.size, L4PI, shape=O.NGP)
    E = rng.standard_normal(ng)
    assert np.array_equal(O.gather(p, x, E), E[_nearest_node(x, ng, L4PI)])


def test_ngp_cell_boundaries_belong_to_the_right_cell():
    # x = k dx starts cell k; x = L is the periodic image of 0
    ng, lx = 8, 8.0
    x = np.array([0.0, 1.0, 3.0, 7.0, 8.0])
    p = O.params(ng, x.size, lx, shape=O.NGP)
    E = np.arange(ng, dtype=float) + 10.0
    assert np.array_equal(O.gather(p, x, E), [10.0, 11.0, 13.0, 17.0, 10.0])


def test_ngp_total_force_on_particles_vanishes():
    # NGP deposit + Eq. 6 + Eq. 7 + NGP gather: sum_p E(x_p) = (N/NG) sum_g
    # (1 - rho_g) E_g = 0, since sum_g E_g = 0 and sum_g rho_g E_g = 0 for
    # the discrete Poisson operator; the total momentum is conserved.
    rng = np.random.default_rng(6)
    for ng, npart in ((8, 3), (64, 1000), (256, 5000)):
        x = rng.uniform(0, L4PI, npart)
        p = O.params(ng, npart, L4PI, shape=O.NGP)
        rho = O.deposit(p, x)
        _, E = O.field(p, rho)
        Ex = O.gather(p, x, E)
        assert abs(Ex.sum()) <= 1e-12 * max(1.0, np.abs(Ex).sum())


def test_ngp_single_particle_moves_freely():
    # a lone particle's field is odd about its own node, so E there is 0
    lx, dt = L4PI, 0.1
    x0, v0 = 1.234, 0.37
    s = O.State(O.params(64, 1, lx, dt, shape=O.NGP), [x0], [v0])
    for n in range(1, 301):
        s.step()
        want = math.fmod(x0 + n * v0 * dt, lx)
        d = abs(s.x[0] - want)
        assert min(d, lx - d) < 1e-12
        assert abs(s.v[0] - v0) < 1e-12


def test_ngp_two_stream_momentum_and_growth():
    # the Sec. 4 run with NGP weighting: momentum conserved to rounding, the
    # instability still grows
    n = 20000
    x, v = W.two_stream(n, L4PI, 0.2, 0.01, 11)
    s = O.State(O.params(64, n, L4PI, shape=O.NGP), x, v)
    h = s.run(200)
    m = s.mass
    mom = m * h[:, 1]
    assert np.abs(mom - mom[0]).max() <= 1e-12 * m * np.abs(v).sum()
    assert h[-1, 2] > 100 * h[0, 2]


def test_ngp_fixed_deposit_counts():
    ng, n = 64, 100003
    x, _ = W.two_stream(n, L4PI, 0.2, 0.01, 7)
    x32, _ = W.to_f32_state(x, np.zeros(n), L4PI)
    u = to_cells(x32, ng, L4PI)
    rq = O.deposit_fixed_ngp(ng, u)
    assert rq.sum() == n << O.FIX_BITS
    assert (rq % (1 << O.FIX_BITS) == 0).all()
    # away from cell boundaries the float32 cell is the float64 cell
    x64 = x32.astype(np.float64)
    ok = _away_from_boundaries(x64, ng, L4PI, 1e-5)
    counts = np.bincount(np.floor(x64[ok] * ng / L4PI).astype(int) % ng, minlength=ng)
    rq_ok = O.deposit_fixed_ngp(ng, u[ok])
    assert np.array_equal(rq_ok >> O.FIX_BITS, counts)
    # and the recipe itself on hand-picked coordinates: the cell is floor(u)
    for uv in (0.0, np.nextafter(np.float32(ng), np.float32(0.0)), 1.0, 0.99999994, 17.5):
        want = int(np.floor(np.float32(uv))) % ng
        got = np.nonzero(O.deposit_fixed_ngp(ng, np.array([uv], dtype=np.float32)))[0]
        assert list(got) == [want]
