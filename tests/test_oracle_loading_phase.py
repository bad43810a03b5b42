"""Pins of the oracle's initial loading (Sec. 2 set-up, Appendix A lattice,
Sec. 4 beams; reading R6) and of its phase-space counts (Sec. 4, Fig. 1),
each against something other than the oracle itself: the generator's
published test vector, the Box-Muller moments, the closed-form lattice, the
first-order Fourier amplitude and phase of the density perturbation, numpy's
2-D histogram and hand-worked bins."""
import math

import numpy as np

import oracle as O


def test_splitmix64_published_vector():
    # SplitMix64 (Steele, Lea & Flood 2014), seed 1234567: the first five
    # outputs of the reference implementation
    got = [O.splitmix64(1234567, k) for k in range(1, 6)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_cold_unperturbed_loading_is_the_lattice_with_two_equal_beams():
    n, L = 1001, 3.0
    x, v = O.load_two_stream(n, L, 0.25, 0.0, 7)
    assert np.array_equal(x, (np.arange(n) + 0.5) * (L / n))
    assert np.array_equal(v[0::2], np.full((n + 1) // 2, 0.25))
    assert np.array_equal(v[1::2], np.full(n // 2, -0.25))


def test_box_muller_spread_moments():
    n, vth = 400000, 0.01
    x, v = O.load_two_stream(n, 4 * math.pi, 0.2, vth, 99)
    g = (v - np.where(np.arange(n) % 2 == 0, 0.2, -0.2)) / vth
    se = 1.0 / math.sqrt(n)
    assert abs(g.mean()) < 5 * se
    assert abs(g.var() - 1.0) < 5 * math.sqrt(2.0) * se
    assert abs(np.mean(np.abs(g) < 1.0) - 0.682689) < 5 * 0.47 * se
    assert abs(np.mean(g ** 4) - 3.0) < 0.05                 # Gaussian kurtosis
    # both beams carry the same spread
    assert abs(g[0::2].std() - g[1::2].std()) < 0.01


def test_density_perturbation_amplitude_and_phase():
    # x = x0 - (eps/k) sin(k x0 + phase) gives density 1 + eps cos(k x + phase)
    # to first order, whose Fourier coefficient mean(exp(-i k x)) is
    # (eps/2) exp(i phase)
    n, L = 200000, 4 * math.pi
    for m, eps, ph in ((1, 1e-3, 0.0), (3, 2e-3, 1.1), (5, 1e-3, -2.0)):
        x, _ = O.load_two_stream(n, L, 0.2, 0.0, 1, modes=((m, eps, ph),))
        assert (x >= 0).all() and (x < L).all()
        k = 2 * math.pi * m / L
        c = np.exp(-1j * k * x).mean()
        assert abs(c - 0.5 * eps * np.exp(1j * ph)) < 0.02 * eps
        # the other modes stay at the lattice's level
        c2 = np.exp(-1j * (2 * math.pi * (m + 1) / L) * x).mean()
        assert abs(c2) < 0.02 * eps


def test_phase_space_equals_histogram2d_away_from_bin_edges():
    rng = np.random.default_rng(4)
    nx, nv, L, vmin, vmax = 32, 20, 4.0, -0.5, 0.5          # dyadic bin widths
    # bin-interior values: the float32 rule and the real-number rule agree
    ix = rng.integers(0, nx, 5000)
    iv = rng.integers(-2, nv + 2, 5000)                      # some out of range
    fx = rng.uniform(0.05, 0.95, 5000)
    fv = rng.uniform(0.05, 0.95, 5000)
    x = ((ix + fx) * (L / nx)).astype(np.float32)
    v = (vmin + (iv + fv) * ((vmax - vmin) / nv)).astype(np.float32)
    got = O.phase_space(nx, nv, L, vmin, vmax, x, v)
    ref, _, _ = np.histogram2d(v.astype(np.float64), x.astype(np.float64),
                               bins=[nv, nx], range=[[vmin, vmax], [0.0, L]])
    assert np.array_equal(got, ref.astype(np.uint32))
    assert got.sum() == np.sum((iv >= 0) & (iv < nv))


def test_phase_space_hand_worked_bins():
    # L = 1, nx = 4, [vmin, vmax) = [-1, 1), nv = 2: every value below is
    # exact in float32
    x = np.float32([0.0, 0.25, 0.99999994, 0.5, 0.5, 0.5])
    v = np.float32([-1.0, 0.0, 0.9999999, 1.0, -1.0000001, 0.5])
    got = O.phase_space(4, 2, 1.0, -1.0, 1.0, x, v)
    want = np.zeros((2, 4), dtype=np.uint32)
    want[0, 0] += 1          # (0, -1): the lower corner is in
    want[1, 1] += 1          # (0.25, 0): v = 0 opens the upper half
    want[1, 3] += 1          # x just below L: the last column
    want[1, 2] += 1          # (0.5, 0.5)
    assert np.array_equal(got, want)    # v = vmax and v < vmin are left out
