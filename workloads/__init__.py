"""Seeded synthetic inputs for the 1D electrostatic electron PIC runs.

This module is the one piece of code that both sides of the parity check use:
the CUDA library's tests and benchmark, and the FP64 oracle's tests.  It holds
the particle loading (lattice "quiet start" positions and Maxwellian
velocities, Sec. 2 and the Appendix A set-up), the two-stream set-up of the
verification test (Sec. 4), the run-parameter draws of the batched ensemble
and the request stream of the serving loop.  It contains none of the step's
arithmetic (no gather, push, deposit or field solve).

Readings of the paper taken here:
  * beams are assigned by particle parity (even index +v0, odd -v0), so the
    two beams hold exactly half the particles each; the Appendix A listing
    draws the sign at random, which leaves the beams unequal;
  * the Maxwellian spread uses numpy's normal generator (the listing uses the
    polar Box-Muller method on libc rand(), unseeded);
  * a "sinusoidal perturbation of mode m with amplitude eps" is a density
    perturbation dn/n = eps*cos(k x + phase), imposed by displacing the
    lattice by xi(x0) = -(eps/k) sin(k x0 + phase).
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def lattice_positions(n: int, length: float) -> np.ndarray:
    """Uniform lattice x_j = (j + 1/2) L / n (the quiet start of Appendix A)."""
    return (np.arange(n, dtype=np.float64) + 0.5) * (length / n)


def fold(x: np.ndarray, length: float) -> np.ndarray:
    """Fold initial positions into [0, L)."""
    y = np.mod(x, length)
    y[y >= length] = 0.0
    return y


def beam_signs(n: int) -> np.ndarray:
    """+1 for even particle index, -1 for odd."""
    return np.where(np.arange(n) % 2 == 0, 1.0, -1.0)


def random_phases(nmodes: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, 0x5EED])
    return rng.uniform(0.0, TWO_PI, nmodes)


def two_stream(n: int, length: float, v0: float, vth: float, seed: int,
               modes=((1, 1e-3, 0.0),)):
    """Two counter-streaming electron beams at +-v0 with thermal spread vth.

    `modes` is a sequence of (m, eps, phase): density perturbation
    eps*cos(2 pi m x / L + phase) per mode.  Returns float64 (x, v).
    """
    rng = np.random.default_rng(seed)
    x0 = lattice_positions(n, length)
    xi = np.zeros(n)
    for m, eps, phase in modes:
        k = TWO_PI * m / length
        xi -= (eps / k) * np.sin(k * x0 + phase)
    x = fold(x0 + xi, length)
    v = beam_signs(n) * v0
    if vth > 0.0:
        v = v + vth * rng.standard_normal(n)
    return x, v


def two_stream_modes_1_to_8(eps: float, seed: int):
    """Modes 1..8 at amplitude eps with seeded random phases."""
    ph = random_phases(8, seed)
    return tuple((m, eps, float(ph[m - 1])) for m in range(1, 9))


def cold_two_stream_gamma(k: float, v0: float) -> float:
    """Growth rate of the cold symmetric two-stream instability.

    Two beams at +-v0, each with plasma frequency^2 = 1/2 (omega_p = 1):
    1 = (1/2)/(w - k v0)^2 + (1/2)/(w + k v0)^2, whose unstable root is
    gamma^2 = (sqrt(1 + 8 a^2) - 1 - 2 a^2) / 2 with a = k v0 (0 for a >= 1).
    """
    a2 = (k * v0) ** 2
    g2 = 0.5 * (math.sqrt(1.0 + 8.0 * a2) - 1.0 - 2.0 * a2)
    return math.sqrt(g2) if g2 > 0.0 else 0.0


def two_stream_eigenmode(n: int, length: float, v0: float, vth: float,
                         eps: float, mode: int, seed: int):
    """Two-stream beams seeded with the growing eigenmode of mode `mode`.

    Cold-fluid linear theory: for beam s with drift u_s the Lagrangian
    displacement is xi_s = Re[c/(i gamma - k u_s)^2 e^{i k x0}] and the
    velocity perturbation is d xi_s/dt = Re[(gamma + i k u_s) xi_hat_s
    e^{i k x0}], with c scaled so that each beam's density perturbation has
    amplitude eps (k |xi_hat| = eps).
    """
    rng = np.random.default_rng(seed)
    k = TWO_PI * mode / length
    gamma = cold_two_stream_gamma(k, v0)
    x0 = lattice_positions(n, length)
    sgn = beam_signs(n)
    u = sgn * v0
    denom = (1j * gamma - k * u) ** 2
    c = (eps / k) * abs(1j * gamma - k * v0) ** 2
    xi_hat = c / denom
    phase = np.exp(1j * k * x0)
    x = fold(x0 + np.real(xi_hat * phase), length)
    v = u + np.real((gamma + 1j * k * u) * xi_hat * phase)
    if vth > 0.0:
        v = v + vth * rng.standard_normal(n)
    return x, v


def cold_langmuir(n: int, length: float, eps: float, mode: int = 1):
    """Cold plasma at rest with density perturbation eps*cos(k x)."""
    k = TWO_PI * mode / length
    x0 = lattice_positions(n, length)
    x = fold(x0 - (eps / k) * np.sin(k * x0), length)
    return x, np.zeros(n)


def maxwellian(n: int, length: float, vth: float, v0: float, seed: int):
    """Maxwellian plasma of the weak-scaling runs (Sec. 5.2): lattice
    positions, drift v0, thermal velocity vth."""
    rng = np.random.default_rng(seed)
    x = lattice_positions(n, length)
    v = v0 + vth * rng.standard_normal(n)
    return x, v


def to_f32_state(x: np.ndarray, v: np.ndarray, length: float):
    """Round a float64 state to the float32 state of the FP32 path.

    Positions that round up to L (as float32) are the point 0.
    """
    x32 = x.astype(np.float32)
    x32[x32 >= np.float32(length)] = np.float32(0.0)
    x32[x32 < 0] = np.float32(0.0)
    return x32, v.astype(np.float32)


# --- batched ensemble and request stream ---------------------------------

def ensemble_runs(nrun: int, seed: int, ncell_range=(64, 2048),
                  npart_range=(1e4, 1e6), v0_range=(0.05, 0.5),
                  vth_range=(0.001, 0.05), length=4.0 * math.pi, dt=0.1):
    """Run parameters of an ensemble of independent runs: cells and
    particles log-uniform, beam and thermal velocities uniform."""
    rng = np.random.default_rng([seed, 0xE45])
    lo, hi = math.log(ncell_range[0]), math.log(ncell_range[1])
    ncell = np.rint(np.exp(rng.uniform(lo, hi, nrun))).astype(np.int64)
    lo, hi = math.log(npart_range[0]), math.log(npart_range[1])
    npart = np.rint(np.exp(rng.uniform(lo, hi, nrun))).astype(np.int64)
    v0 = rng.uniform(*v0_range, nrun)
    vth = rng.uniform(*vth_range, nrun)
    runs = []
    for r in range(nrun):
        runs.append(dict(ncell=int(ncell[r]), npart=int(npart[r]),
                         length=float(length), dt=float(dt),
                         v0=float(v0[r]), vth=float(vth[r]),
                         seed=int(seed * 100003 + r)))
    return runs


def request_stream(nreq: int, rate: float, seed: int, ncell_range=(64, 4096),
                   npart_range=(1e4, 4e6), steps_range=(100, 2000),
                   v0=0.2, vth=0.01, length=4.0 * math.pi, dt=0.1):
    """Poisson arrivals (exponential gaps, mean 1/rate) of run requests."""
    rng = np.random.default_rng([seed, 0x5E4E])
    gaps = rng.exponential(1.0 / rate, nreq)
    t = np.cumsum(gaps)
    lo, hi = math.log(ncell_range[0]), math.log(ncell_range[1])
    ncell = np.rint(np.exp(rng.uniform(lo, hi, nreq))).astype(np.int64)
    lo, hi = math.log(npart_range[0]), math.log(npart_range[1])
    npart = np.rint(np.exp(rng.uniform(lo, hi, nreq))).astype(np.int64)
    steps = rng.integers(steps_range[0], steps_range[1] + 1, nreq)
    reqs = []
    for i in range(nreq):
        reqs.append(dict(arrival=float(t[i]), ncell=int(ncell[i]),
                         npart=int(npart[i]), steps=int(steps[i]),
                         length=float(length), dt=float(dt), v0=float(v0),
                         vth=float(vth), seed=int(seed * 1000003 + i)))
    return reqs
