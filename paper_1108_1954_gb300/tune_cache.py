"""A file of launch shapes the push autotuner adopted, so that a later run of
the same kind on the same GPU model takes the shape without timing again.

Runs share an entry when they have the same GPU model, precision mode,
particle shape and sort interval, NG in the same power-of-two bucket and N
in the same power-of-two bucket (the push's cost per particle depends on
the density tile and on how many particles share a cell).  The file is one
JSON object, {key: {"variant", "block", "unroll", "ms"}}, rewritten whole
through a temporary file and a rename, so that a reader never sees half of
it.
"""
from __future__ import annotations

import json
import math
import os
import tempfile


def bucket(n: int) -> int:
    """The power of two at or above n (n >= 1)."""
    return 1 << max(0, math.ceil(math.log2(max(1, int(n)))))


def key(gpu: str, npart: int, ncell: int, sort_interval: int, precision: int,
        shape: int) -> str:
    return "%s|prec%d|shape%d|S%d|ng%d|n%d" % (gpu.strip(), int(precision), int(shape),
                                               int(sort_interval), bucket(ncell), bucket(npart))


def load(path: str) -> dict:
    """The cache's entries ({} if the file is missing or unreadable)."""
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def lookup(path: str, k: str):
    """The entry for key k, or None."""
    e = load(path).get(k)
    if not isinstance(e, dict) or not all(f in e for f in ("variant", "block", "unroll")):
        return None
    return e


def store(path: str, k: str, variant: int, block: int, unroll: int, ms: float) -> None:
    """Add or replace the entry for key k."""
    d = load(path)
    d[k] = {"variant": int(variant), "block": int(block), "unroll": int(unroll),
            "ms": float(ms)}
    folder = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".tune_cache.", dir=folder)
    try:
        with os.fdopen(fd, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise
