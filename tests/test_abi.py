"""The C-ABI library loads, exports every function include/pic.h declares, and
rejects bad parameters -- host-side checks that need no GPU."""
import ctypes as C
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_1954_gb300 as pic
    return pic


def test_library_exports_every_header_function(pic):
    names = pic.header_functions(os.path.join(ROOT, "include", "pic.h"))
    assert len(names) >= 19
    lib = C.CDLL(pic.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_text(pic):
    assert pic._lib.pic_version() == 1
    assert pic.strerror(pic.PIC_EINVAL) == "invalid argument"
    assert pic.strerror(pic.PIC_EDEVICE).startswith("kernel flagged")
    assert pic.strerror(12345) == "unknown error"


def _params(pic, **kw):
    base = dict(npart=1000, ncell=64, length=4 * math.pi, dt=0.1)
    base.update(kw)
    return pic.Params(**base)


def test_workspace_size_scales_with_particles(pic):
    a = pic.workspace_size(_params(pic, npart=1 << 20))
    b = pic.workspace_size(_params(pic, npart=1 << 21))
    # four float32 particle arrays (state + sort buffer), 16 B per particle
    assert 16 * (1 << 20) <= b - a <= 16 * (1 << 20) + (1 << 20)
    d = pic.workspace_size(_params(pic, npart=1 << 20, precision=pic.PIC_FP64))
    assert d - a >= 16 * (1 << 20)


@pytest.mark.parametrize("bad", [
    dict(npart=0), dict(ncell=0), dict(ncell=8193), dict(qm=1.0), dict(qm=0.0),
    dict(dt=0.0), dict(length=float("nan")), dict(length=-1.0),
    dict(rho_ion=0.0), dict(block_size=33), dict(block_size=2048),
    dict(block_size=1024), dict(unroll=3),
    dict(deposit_variant=10), dict(deposit_variant=3), dict(deposit_variant=4),
    dict(deposit_variant=7), dict(precision=7), dict(sort_interval=-1),
    dict(npart=1 << 33)])
def test_invalid_parameters_rejected(pic, bad):
    with pytest.raises(pic.PicError) as e:
        pic.workspace_size(_params(pic, **bad))
    assert e.value.code == pic.PIC_EINVAL


def test_create_rejects_missing_or_small_workspace(pic):
    p = _params(pic).c()
    h = C.c_void_p()
    assert pic._lib.pic_create(C.byref(p), None, 0, None, C.byref(h)) == pic.PIC_EINVAL
    # misaligned workspace pointer
    assert pic._lib.pic_create(C.byref(p), C.c_void_p(16), 1 << 30, None,
                               C.byref(h)) == pic.PIC_EINVAL
    assert pic._lib.pic_create(None, C.c_void_p(256), 1, None, C.byref(h)) == pic.PIC_EINVAL


def test_calls_on_null_run_are_rejected(pic):
    lib = pic._lib
    assert lib.pic_push(None) == pic.PIC_EINVAL
    assert lib.pic_step_n(None, 1) == pic.PIC_EINVAL
    assert lib.pic_solve_field(None) == pic.PIC_EINVAL
    assert lib.pic_step_count(None) == -1


@pytest.mark.parametrize("bad", [
    dict(qm=float("inf")), dict(dt=float("inf")), dict(rho_ion=-1.0), dict(history=-1),
    dict(blocks_per_sm=-1), dict(blocks_per_sm=33), dict(unroll=8), dict(field_solver=2),
    dict(cg_iterations=-1), dict(cg_iterations=100001), dict(shape=2),
    dict(shape=1, precision=2), dict(shape=1, precision=1)])
def test_more_invalid_parameters_rejected(pic, bad):
    with pytest.raises(pic.PicError) as e:
        pic.workspace_size(_params(pic, **bad))
    assert e.value.code == pic.PIC_EINVAL


def test_reserved_word_must_be_zero(pic):
    p = _params(pic).c()
    n = C.c_size_t(0)
    assert pic._lib.pic_workspace_size(C.byref(p), C.byref(n)) == pic.PIC_OK
    p.reserved = 1
    assert pic._lib.pic_workspace_size(C.byref(p), C.byref(n)) == pic.PIC_EINVAL


def test_pool_run_bytes(pic):
    a = pic.pool_run_bytes(_params(pic, npart=1 << 20), 8)
    b = pic.pool_run_bytes(_params(pic, npart=1 << 21), 8)
    # x and v in float32: 8 B per particle, plus alignment
    assert 8 * (1 << 20) <= b - a <= 8 * (1 << 20) + 4096
    c = pic.pool_run_bytes(_params(pic, npart=1 << 20), 1000)
    assert c > a                                       # history rows
    for bad, h in [(dict(precision=pic.PIC_FP64), 8), (dict(precision=pic.PIC_FP32_ATOMIC), 8),
                   (dict(field_solver=1), 8), (dict(shape=1), 8), ({}, 0), (dict(npart=0), 8)]:
        with pytest.raises(pic.PicError) as e:
            pic.pool_run_bytes(_params(pic, **bad), h)
        assert e.value.code == pic.PIC_EINVAL


def test_pool_table_bytes(pic):
    def table(*cfg):
        c = pic.CPoolConfig(*cfg)
        n = C.c_size_t(0)
        rc = pic._lib.pic_pool_table_bytes(C.byref(c), C.byref(n))
        return rc, n.value
    rc1, t1 = table(16, 4096, 8, 0, 0, 0)
    rc2, t2 = table(1024, 4096, 8, 0, 0, 0)
    assert rc1 == rc2 == pic.PIC_OK and t2 > t1 > 0
    for bad in [(0, 4096, 8, 0, 0, 0), (16, 0, 8, 0, 0, 0), (16, 8193, 8, 0, 0, 0),
                (16, 4096, 0, 0, 0, 0)]:
        assert table(*bad)[0] == pic.PIC_EINVAL
    assert pic._lib.pic_pool_table_bytes(None, None) == pic.PIC_EINVAL


def test_binding_checks_host_arrays(pic):
    import numpy as np
    import torch
    f = pic._host_array
    # reading: numpy input is converted, length checked
    assert f(np.arange(4.0), np.float32, 4, "x").dtype == np.float32
    with pytest.raises(ValueError):
        f(np.zeros(5, np.float32), np.float32, 4, "x")
    # writing: the caller's numpy array must already be the right buffer
    with pytest.raises(TypeError):
        f(np.zeros(4, np.float64), np.float32, 4, "x", writable=True)
    with pytest.raises(TypeError):
        f(np.zeros(8, np.float32)[::2], np.float32, 4, "x", writable=True)
    # torch: CPU, contiguous, the run's dtype, the run's length
    assert f(torch.zeros(4), np.float32, 4, "x") is not None
    with pytest.raises(TypeError):
        f(torch.zeros(4, dtype=torch.float64), np.float32, 4, "x")
    with pytest.raises(TypeError):
        f(torch.zeros(8)[::2], np.float32, 4, "x")
    with pytest.raises(ValueError):
        f(torch.zeros(3), np.float32, 4, "x")
    with pytest.raises(TypeError):
        f([0.0] * 4, np.float32, 4, "x")
