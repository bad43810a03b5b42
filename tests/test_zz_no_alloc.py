"""pic_sort_noalloc: the counting sort for callers that cannot allocate device
memory (a framework whose caching allocator owns the device, a fixed memory
reservation, code that cannot pay for cudaMalloc's synchronisation).  Its
scratch lives in a device array inside the library, shared by every call.

The test calls the entry point through the C ABI on caller-owned device
buffers, several times in a row with different inputs, and compares each
result with pic_sort of a run holding the same particles and with numpy's
stable argsort of the cell keys.  A stable sort by cell has one answer, so
all three must agree bit for bit.  Bad pointers (misaligned, overlapping) are refused on the
host before anything is launched.  This file is collected last."""
import ctypes as C
import math

import numpy as np
import pytest

import paper_1108_1954_gb300 as pic  # noqa: E402
import torch  # noqa: E402

pytestmark = pytest.mark.gpu
L = 4.0 * math.pi


def _entry():
    lib = C.CDLL(pic.LIB_PATH)
    fn = lib.pic_sort_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p] * 4 + [C.c_int64, C.c_int32, C.c_double, C.c_void_p]
    return fn


def _sorted_by_pic_sort(x, v, ncell):
    """A run holding the particles, sorted by pic_sort: its cell coordinates
    u = x NG/L before and after the sort."""
    run = pic.Run(pic.Params(npart=x.size, ncell=ncell, length=L), device="cuda:0")
    run.init(x, v)
    u, _ = run.get_cells()
    run.sort()
    us, vs = run.get_cells()
    run.close()
    return u, us, vs


def _stable_argsort_by_cell(x, ncell, length):
    """The documented key: trunc(x c), c = (float)(NG/L), clamped to [0, NG-1],
    all in float32; numpy's stable argsort of it."""
    c = np.float32(ncell / length)
    u = x.astype(np.float32) * c
    u = np.where(u > 0, u, np.float32(0))
    u = np.minimum(u, np.float32(ncell - 1))
    return np.argsort(u.astype(np.uint32), kind="stable")


def test_noalloc_sort_matches_pic_sort_and_argsort_twice():
    # A run keeps its positions as cell coordinates u in [0, NG), so the
    # entry point sorts those with L = NG (the cell of u is trunc(u)), the
    # key pic_sort uses; a second call sorts physical positions, compared
    # with numpy alone.
    fn = _entry()
    stream = torch.cuda.current_stream()
    for call, (n, ncell) in enumerate([(300001, 1024), (2_000_003, 4096)]):
        rng = np.random.default_rng(100 + call)
        x = rng.uniform(0, L, n).astype(np.float32)
        x[x >= np.float32(L)] = 0.0
        v = rng.standard_normal(n).astype(np.float32)
        u, ur, vr = _sorted_by_pic_sort(x, v, ncell)
        for pos, length in ((u, float(ncell)), (x, L)):
            xd = torch.from_numpy(pos).to("cuda")
            vd = torch.from_numpy(v).to("cuda")
            xo = torch.empty_like(xd)
            vo = torch.empty_like(vd)
            rc = fn(xd.data_ptr(), vd.data_ptr(), xo.data_ptr(), vo.data_ptr(), n, ncell,
                    length, stream.cuda_stream)
            assert rc == pic.PIC_OK
            torch.cuda.synchronize()
            got_x, got_v = xo.cpu().numpy(), vo.cpu().numpy()
            if pos is u:
                assert np.array_equal(got_x, ur)
                assert np.array_equal(got_v, vr)
            order = _stable_argsort_by_cell(pos, ncell, length)
            assert np.array_equal(got_x, pos[order])
            assert np.array_equal(got_v, v[order])


def test_noalloc_sort_rejects_sizes_beyond_its_limits():
    fn = _entry()
    xd = torch.zeros(16, dtype=torch.float32, device="cuda")
    xo = torch.zeros(16, dtype=torch.float32, device="cuda")
    vo = torch.zeros(16, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert fn(xd.data_ptr(), xd.data_ptr(), xo.data_ptr(), vo.data_ptr(), 16,
              pic.PIC_NCELL_MAX + 1, L, s) == pic.PIC_EINVAL
    assert fn(xd.data_ptr(), xd.data_ptr(), xo.data_ptr(), vo.data_ptr(), 0, 64, L,
              s) == pic.PIC_EINVAL
    assert fn(xd.data_ptr(), xd.data_ptr(), xo.data_ptr(), vo.data_ptr(), 16, 64,
              float("inf"), s) == pic.PIC_EINVAL


def test_noalloc_sort_refuses_bad_pointers_on_the_host():
    """The bad cases are refused by the host checks, so no kernel ever sees them."""
    fn = _entry()
    s = torch.cuda.current_stream().cuda_stream
    buf = torch.zeros(4 * 64, dtype=torch.float32, device="cuda")
    base = buf.data_ptr()
    assert base % 16 == 0
    n = 32
    x, v, xo, vo = base, base + 4 * 64, base + 8 * 64, base + 12 * 64
    ok = [x, v, xo, vo]
    # a position array one element past a 16-byte boundary (a slice x[1:])
    assert fn(x + 4, v, xo, vo, n, 64, L, s) == pic.PIC_EINVAL
    # outputs on an input, on each other, or partly overlapping
    assert fn(x, v, x, vo, n, 64, L, s) == pic.PIC_EINVAL
    assert fn(x, v, xo, v, n, 64, L, s) == pic.PIC_EINVAL
    assert fn(x, v, v, x, n, 64, L, s) == pic.PIC_EINVAL
    assert fn(x, v, xo, xo, n, 64, L, s) == pic.PIC_EINVAL
    assert fn(x, v, xo, xo + 4 * (n - 1), n, 64, L, s) == pic.PIC_EINVAL
    # an output at a 4-byte (not 16-byte) boundary is allowed
    assert fn(x, v, xo + 4, vo, n, 64, L, s) == pic.PIC_OK
    torch.cuda.synchronize()
    assert fn(*ok, n, 64, L, s) == pic.PIC_OK
    torch.cuda.synchronize()
