"""pic_sort_noalloc: the counting sort for callers that cannot allocate device
memory (a framework whose caching allocator owns the device, a fixed memory
reservation, code that cannot pay for cudaMalloc's synchronisation).  Its
scratch lives in a device array inside the library, shared by every call.

The test calls the entry point through the C ABI on caller-owned device
buffers, twice in a row with different inputs, and compares each result with
pic_sort of a run holding the same particles.  A stable sort by cell has one
answer, so the two must agree bit for bit.  This file is collected last."""
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
    run = pic.Run(pic.Params(npart=x.size, ncell=ncell, length=L), device="cuda:0")
    run.init(x, v)
    run.sort()
    xs, vs = run.get_state()
    run.close()
    return xs, vs


def test_noalloc_sort_matches_pic_sort_twice():
    fn = _entry()
    stream = torch.cuda.current_stream()
    for call, (n, ncell) in enumerate([(300001, 1024), (2_000_003, 4096)]):
        rng = np.random.default_rng(100 + call)
        x = rng.uniform(0, L, n).astype(np.float32)
        x[x >= np.float32(L)] = 0.0
        v = rng.standard_normal(n).astype(np.float32)
        xd = torch.from_numpy(x).to("cuda")
        vd = torch.from_numpy(v).to("cuda")
        xo = torch.empty_like(xd)
        vo = torch.empty_like(vd)
        rc = fn(xd.data_ptr(), vd.data_ptr(), xo.data_ptr(), vo.data_ptr(), n, ncell, L,
                stream.cuda_stream)
        assert rc == pic.PIC_OK
        torch.cuda.synchronize()
        xr, vr = _sorted_by_pic_sort(x, v, ncell)
        assert np.array_equal(xo.cpu().numpy(), xr)
        assert np.array_equal(vo.cpu().numpy(), vr)


def test_noalloc_sort_rejects_sizes_beyond_its_limits():
    fn = _entry()
    xd = torch.zeros(16, dtype=torch.float32, device="cuda")
    xo = torch.zeros(16, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert fn(xd.data_ptr(), xd.data_ptr(), xo.data_ptr(), xo.data_ptr(), 16,
              pic.PIC_NCELL_MAX + 1, L, s) == pic.PIC_EINVAL
    assert fn(xd.data_ptr(), xd.data_ptr(), xo.data_ptr(), xo.data_ptr(), 0, 64, L, s) == pic.PIC_EINVAL
    assert fn(xd.data_ptr(), xd.data_ptr(), xd.data_ptr(), xo.data_ptr(), 16, 64, L, s) == pic.PIC_EINVAL
