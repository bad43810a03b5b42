"""The library's conversion of float32 positions to cell coordinates (stated
in include/pic.h): u = (float)((double)x (NG/L)), a u rounding to NG is 0.
Tests that build the device's starting state without a GPU use it; GPU tests
read the device's own coordinates back with get_cells."""
import numpy as np


def to_cells(x32, ng, length):
    u = (np.asarray(x32, dtype=np.float32).astype(np.float64) * (ng / length)).astype(np.float32)
    u[u >= np.float32(ng)] = np.float32(0.0)
    return u
