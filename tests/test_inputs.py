"""The seeded input generators: the counter-based generator against its
published test vector, and the statistics of the loadings it feeds."""
import math

import numpy as np

import workloads as W


def test_splitmix64_published_vector():
    # SplitMix64 (Steele, Lea & Flood 2014), seed 1234567: the reference
    # implementation's first five outputs
    got = W.splitmix64(1234567, np.arange(1, 6, dtype=np.uint64)).tolist()
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_counter_loading_statistics():
    n, L = 400000, 4 * math.pi
    x, v = W.counter_two_stream(n, L, 0.2, 0.01, 99, modes=((1, 1e-3, 0.0),))
    assert x.dtype == np.float32 and (x >= 0).all() and (x < np.float32(L)).all()
    vp, vm = v[0::2].astype(np.float64), v[1::2].astype(np.float64)
    se = 0.01 / math.sqrt(n / 2)
    assert abs(vp.mean() - 0.2) < 5 * se and abs(vm.mean() + 0.2) < 5 * se
    assert abs(vp.std() / 0.01 - 1.0) < 0.01
    # the density perturbation of mode 1 has amplitude eps
    k = 2 * math.pi / L
    amp = 2 * abs(np.exp(-1j * k * x.astype(np.float64)).mean())
    assert abs(amp - 1e-3) < 1e-4


def test_ensemble_and_request_draws():
    runs = W.ensemble_runs(512, 3)
    assert len(runs) == 512
    ng = np.array([r["ncell"] for r in runs])
    npart = np.array([r["npart"] for r in runs])
    assert ng.min() >= 64 and ng.max() <= 2048
    assert npart.min() >= 10000 and npart.max() <= 1000000
    # log-uniform: the median sits near the geometric mean of the range
    assert 0.6e5 < np.median(npart) < 1.6e5
    reqs = W.request_stream(2000, 200.0, 5)
    t = np.array([r["arrival"] for r in reqs])
    assert (np.diff(t) > 0).all()
    assert abs(2000 / t[-1] - 200.0) < 20.0
