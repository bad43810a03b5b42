"""Device-side loading against the oracle's float64 statement of the same
loading (orc_load_two_stream), and runs started from it against runs started
from the same state uploaded from the host."""
import math

import numpy as np
import pytest

import paper_1108_1954_gb300 as pic  # noqa: E402
import torch  # noqa: E402
import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
L4PI = 4.0 * math.pi


@pytest.mark.parametrize("n,modes", [(1, ()), (7, ((1, 1e-3, 0.0),)),
                                     (1000003, W.two_stream_modes_1_to_8(1e-4, 2))])
def test_loader_matches_the_oracle(n, modes):
    ld = pic.Loading(v0=0.2, vth=0.01, seed=1234 + n, modes=modes)
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    v = torch.empty(n, dtype=torch.float32, device="cuda")
    pic.load_two_stream(ld, n, L4PI, x, v)
    torch.cuda.synchronize()
    xh, vh = O.load_two_stream(n, L4PI, 0.2, 0.01, 1234 + n, modes)
    xd, vd = x.cpu().numpy(), v.cpu().numpy()
    # the device rounds x to float32 (half an ulp of L, 4.8e-7) after a
    # float32 perturbation sum (below 1e-9 here)
    d = np.abs(xd.astype(np.float64) - xh)
    d = np.minimum(d, L4PI - d)
    assert d.max() <= 4e-7 * L4PI
    # float32 Box-Muller (a few ulps of |g| <= 6, times vth) and the float32
    # rounding of v and v0
    assert np.abs(vd.astype(np.float64) - vh).max() <= 2e-6 * 0.01 * 8 + 1e-7
    assert (xd >= 0).all() and (xd < np.float32(L4PI)).all()


def test_init_loaded_equals_uploaded_state():
    # the loader's physical output, uploaded, gives the same run as loading
    # on the device: both go through the same conversion to cell units
    n, ng = 200001, 512
    ld = pic.Loading(v0=0.2, vth=0.01, seed=77, modes=((1, 1e-3, 0.0),))
    a = pic.Run(pic.Params(npart=n, ncell=ng, length=L4PI), device="cuda:0")
    a.init_loaded(ld)
    xd = torch.empty(n, dtype=torch.float32, device="cuda")
    vd = torch.empty(n, dtype=torch.float32, device="cuda")
    pic.load_two_stream(ld, n, L4PI, xd, vd)
    torch.cuda.synchronize()
    x, v = xd.cpu().numpy(), vd.cpu().numpy()
    b = pic.Run(pic.Params(npart=n, ncell=ng, length=L4PI), device="cuda:0")
    b.init(x, v)
    assert np.array_equal(a.get_cells()[0], b.get_cells()[0])
    a.step_n(10)
    b.step_n(10)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_pool_admit_loaded_equals_alone():
    n, ng = 50003, 256
    ld = pic.Loading(v0=0.3, vth=0.02, seed=5, modes=W.two_stream_modes_1_to_8(1e-4, 5))
    p = pic.Params(npart=n, ncell=ng, length=L4PI)
    pool = pic.Pool(max_slots=4, ncell_max=256, arena_bytes=1 << 28, history=64, device="cuda:0")
    s = pool.admit_loaded(p, ld, 15)
    pool.advance(15)
    run = pic.Run(pic.Params(npart=n, ncell=ng, length=L4PI, history=64), device="cuda:0")
    run.init_loaded(ld)
    run.step_n(15)
    xa, va = pool.get_state(s)
    xb, vb = run.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(pool.get_field(s)["E"], run.get_field()["E"])
