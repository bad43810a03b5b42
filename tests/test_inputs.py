"""The seeded input generators: the draws of the batched ensemble and of the
request stream."""
import math

import numpy as np

import workloads as W


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
