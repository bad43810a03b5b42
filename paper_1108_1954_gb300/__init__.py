"""Python binding of libpic, the GB300 (sm_103a) library for the 1D
electrostatic electron Particle-in-Cell step of Markidis & Lapenta (PGAS10).

This module marshals arguments only: every step of the method runs in the
CUDA kernels behind the C ABI of `include/pic.h`.  PyTorch supplies the device
memory (one workspace tensor per run) and the CUDA stream.  There is no CPU
fallback: importing this package fails if `_build/libpic.so` has not been
built (`python -c "import __graft_entry__ as g; g.build()"`).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpic.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libpic.so is not built (%s); build it with paper_1108_1954_gb300.build"
        " or __graft_entry__.build() -- there is no CPU fallback" % LIB_PATH)

_lib = C.CDLL(LIB_PATH)

# --- constants of include/pic.h ------------------------------------------------
PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA = 0, -1, -2, -3
PIC_ETIMEOUT, PIC_EDEVICE, PIC_ESTATE = -4, -5, -6
PIC_FP32_FIXED, PIC_FP32_ATOMIC, PIC_FP64 = 0, 1, 2
PIC_DEPOSIT_AUTO, PIC_DEPOSIT_ATOMIC, PIC_DEPOSIT_MATCH = 0, 1, 2
PIC_DEPOSIT_QUAD, PIC_DEPOSIT_PAIR = 5, 6
PIC_DEPOSIT_QUAD8, PIC_DEPOSIT_PAIR8 = 8, 9
PIC_SOLVER_EXACT, PIC_SOLVER_CG = 0, 1
PIC_SHAPE_CIC, PIC_SHAPE_NGP = 0, 1
PIC_CG_DEFAULT_ITERATIONS = 150
PIC_NCELL_MAX = 8192
PIC_NMODES = 8
FIX_BITS = 24

VARIANT_NAMES = {PIC_DEPOSIT_ATOMIC: "atomic", PIC_DEPOSIT_MATCH: "match",
                 PIC_DEPOSIT_QUAD: "quad", PIC_DEPOSIT_PAIR: "pair",
                 PIC_DEPOSIT_QUAD8: "quad8", PIC_DEPOSIT_PAIR8: "pair8"}


class CParams(C.Structure):
    _fields_ = [("npart", C.c_int64), ("ncell", C.c_int32),
                ("precision", C.c_int32), ("length", C.c_double),
                ("dt", C.c_double), ("qm", C.c_double),
                ("rho_ion", C.c_double), ("sort_interval", C.c_int32),
                ("history", C.c_int32), ("deposit_variant", C.c_int32),
                ("block_size", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("unroll", C.c_int32), ("field_solver", C.c_int32),
                ("cg_iterations", C.c_int32), ("shape", C.c_int32),
                ("reserved", C.c_int32)]


class CDiagRow(C.Structure):
    _fields_ = [("step", C.c_int64), ("kinetic", C.c_double),
                ("momentum", C.c_double), ("field", C.c_double),
                ("charge", C.c_double), ("charge_q", C.c_int64),
                ("mode", C.c_double * PIC_NMODES)]


TUNE_DTYPE = np.dtype([("variant", np.int32), ("block", np.int32),
                       ("unroll", np.int32), ("grid", np.int32), ("ms", np.float32)])

DIAG_DTYPE = np.dtype([("step", np.int64), ("kinetic", np.float64),
                       ("momentum", np.float64), ("field", np.float64),
                       ("charge", np.float64), ("charge_q", np.int64),
                       ("mode", np.float64, (PIC_NMODES,))])
assert DIAG_DTYPE.itemsize == C.sizeof(CDiagRow)

_P = C.POINTER(CParams)
_VP = C.c_void_p
_SIG = {
    "pic_version": (C.c_int, []),
    "pic_strerror": (C.c_char_p, [C.c_int]),
    "pic_workspace_size": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
    "pic_create": (C.c_int, [_P, _VP, C.c_size_t, _VP, C.POINTER(_VP)]),
    "pic_destroy": (None, [_VP]),
    "pic_init": (C.c_int, [_VP, _VP, _VP]),
    "pic_deposit": (C.c_int, [_VP]),
    "pic_solve_field": (C.c_int, [_VP]),
    "pic_push": (C.c_int, [_VP]),
    "pic_sort": (C.c_int, [_VP]),
    "pic_step_n": (C.c_int, [_VP, C.c_int64]),
    "pic_sync": (C.c_int, [_VP]),
    "pic_diagnostics": (C.c_int, [_VP, C.c_int64, C.c_int32, _VP]),
    "pic_step_count": (C.c_int64, [_VP]),
    "pic_get_state": (C.c_int, [_VP, _VP, _VP]),
    "pic_set_state": (C.c_int, [_VP, _VP, _VP, C.c_int64]),
    "pic_get_field": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "pic_get_cells": (C.c_int, [_VP, _VP, _VP]),
    "pic_set_cells": (C.c_int, [_VP, _VP, _VP, C.c_int64]),
    "pic_pool_get_cells": (C.c_int, [_VP, C.c_int32, _VP, _VP]),
    "pic_device_arrays": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(_VP),
                                    C.POINTER(_VP)]),
    "pic_launch_shape": (C.c_int, [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "pic_autotune": (C.c_int, [_VP, C.c_int32, _VP, C.c_int32, C.POINTER(C.c_int32)]),
    "pic_set_launch": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "pic_set_shard": (C.c_int, [_VP, C.c_int64]),
    "pic_device_density": (C.c_int, [_VP, C.POINTER(_VP)]),
    "pic_tune_sort_interval": (C.c_int, [_VP, _VP, C.c_int32, _VP, C.POINTER(C.c_int32),
                                         C.c_int32]),
    "pic_phase_space": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_double, C.c_double, _VP]),
    "pic_load_two_stream": (C.c_int, [_VP, C.c_int64, C.c_double, _VP, _VP, _VP]),
    "pic_init_loaded": (C.c_int, [_VP, _VP]),
    "pic_pool_admit_loaded": (C.c_int, [_VP, _P, _VP, C.c_int64, C.POINTER(C.c_int32)]),
    "pic_pool_run_bytes": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_size_t)]),
    "pic_pool_table_bytes": (C.c_int, [_VP, C.POINTER(C.c_size_t)]),
    "pic_pool_create": (C.c_int, [_VP, _VP, C.c_size_t, _VP, C.POINTER(_VP)]),
    "pic_pool_destroy": (None, [_VP]),
    "pic_pool_configure": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32]),
    "pic_pool_admit": (C.c_int, [_VP, _P, _VP, _VP, C.c_int64, C.POINTER(C.c_int32)]),
    "pic_pool_advance": (C.c_int, [_VP, C.c_int64, C.POINTER(C.c_int32)]),
    "pic_pool_finished": (C.c_int, [_VP, _VP, C.c_int32, C.POINTER(C.c_int32)]),
    "pic_pool_step_count": (C.c_int, [_VP, C.c_int32, C.POINTER(C.c_int64)]),
    "pic_pool_get_state": (C.c_int, [_VP, C.c_int32, _VP, _VP]),
    "pic_pool_get_field": (C.c_int, [_VP, C.c_int32, _VP, _VP, _VP, _VP]),
    "pic_pool_diagnostics": (C.c_int, [_VP, C.c_int32, C.c_int64, C.c_int32, _VP]),
    "pic_pool_release": (C.c_int, [_VP, C.c_int32]),
    "pic_pool_sync": (C.c_int, [_VP]),
    "pic_pool_usage": (C.c_int, [_VP, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
}
for _name, (_res, _args) in _SIG.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

assert _lib.pic_version() == 1, "libpic ABI version mismatch"


class PicError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, strerror(code), code))


def strerror(code: int) -> str:
    return _lib.pic_strerror(int(code)).decode()


def _check(rc: int, what: str):
    if rc != PIC_OK:
        raise PicError(rc, what)


def _ptr(a) -> int:
    """Address of a C-contiguous numpy array or a torch tensor's storage."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


def _host_array(a, dtype, n: int, what: str, writable: bool = False):
    """Check a host argument of n values of `dtype`: a numpy array (converted
    to a C-contiguous copy of that dtype when reading, required exactly when
    it is written to) or a contiguous CPU torch tensor of that dtype."""
    if isinstance(a, np.ndarray):
        if writable:
            if a.dtype != dtype or not a.flags["C_CONTIGUOUS"] or not a.flags["WRITEABLE"]:
                raise TypeError("%s: need a writable C-contiguous %s array" % (what, np.dtype(dtype)))
        else:
            a = np.ascontiguousarray(a, dtype=dtype)
        if a.size != n:
            raise ValueError("%s: %d values given, %d expected" % (what, a.size, n))
        return a
    import torch
    if not isinstance(a, torch.Tensor):
        raise TypeError("%s: a numpy array or a CPU torch tensor" % what)
    want = torch.float64 if np.dtype(dtype) == np.float64 else torch.float32
    if a.device.type != "cpu" or a.dtype != want or not a.is_contiguous():
        raise TypeError("%s: need a contiguous CPU torch tensor of %s" % (what, want))
    if a.numel() != n:
        raise ValueError("%s: %d values given, %d expected" % (what, a.numel(), n))
    return a


@dataclass
class Params:
    """Run parameters (pic_params of include/pic.h)."""
    npart: int
    ncell: int
    length: float
    dt: float = 0.1
    qm: float = -1.0
    rho_ion: float = 1.0
    precision: int = PIC_FP32_FIXED
    sort_interval: int = 0
    history: int = 0
    deposit_variant: int = PIC_DEPOSIT_AUTO
    block_size: int = 0
    blocks_per_sm: int = 0
    unroll: int = 0
    field_solver: int = 0          # PIC_SOLVER_EXACT
    cg_iterations: int = 0         # 0: the paper's 150
    shape: int = 0                 # PIC_SHAPE_CIC

    def c(self) -> CParams:
        return CParams(int(self.npart), int(self.ncell), int(self.precision),
                       float(self.length), float(self.dt), float(self.qm),
                       float(self.rho_ion), int(self.sort_interval),
                       int(self.history), int(self.deposit_variant),
                       int(self.block_size), int(self.blocks_per_sm),
                       int(self.unroll), int(self.field_solver),
                       int(self.cg_iterations), int(self.shape), 0)

    @property
    def dtype(self):
        return np.float64 if self.precision == PIC_FP64 else np.float32


def workspace_size(p: Params) -> int:
    n = C.c_size_t(0)
    cp = p.c()
    _check(_lib.pic_workspace_size(C.byref(cp), C.byref(n)), "pic_workspace_size")
    return int(n.value)


class Run:
    """One PIC run on a CUDA device; its workspace is a torch uint8 tensor."""

    def __init__(self, p: Params, device=None, stream=None):
        import torch
        self.p = p
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = workspace_size(p)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            handle = _VP()
            cp = p.c()
            _check(_lib.pic_create(C.byref(cp), _VP(self.workspace.data_ptr()),
                                   nbytes, _VP(self.stream.cuda_stream),
                                   C.byref(handle)), "pic_create")
        self._h = handle

    # --- lifecycle ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _lib.pic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _host(self, a, what="x", writable=False):
        return _host_array(a, self.p.dtype, self.p.npart, what, writable)

    # --- the C ABI, one method per entry point -------------------------------
    def init(self, x0, v0):
        x0, v0 = self._host(x0, "x0"), self._host(v0, "v0")
        _check(_lib.pic_init(self._h, _VP(_ptr(x0)), _VP(_ptr(v0))), "pic_init")

    def init_loaded(self, ld: Loading):
        cl = ld.c()
        _check(_lib.pic_init_loaded(self._h, C.byref(cl)), "pic_init_loaded")

    def set_state(self, x, v, step: int):
        x, v = self._host(x, "x"), self._host(v, "v")
        _check(_lib.pic_set_state(self._h, _VP(_ptr(x)), _VP(_ptr(v)), int(step)),
               "pic_set_state")

    def deposit(self):
        _check(_lib.pic_deposit(self._h), "pic_deposit")

    def solve_field(self):
        _check(_lib.pic_solve_field(self._h), "pic_solve_field")

    def push(self):
        _check(_lib.pic_push(self._h), "pic_push")

    def sort(self):
        _check(_lib.pic_sort(self._h), "pic_sort")

    def step_n(self, n: int):
        _check(_lib.pic_step_n(self._h, int(n)), "pic_step_n")

    def sync(self):
        _check(_lib.pic_sync(self._h), "pic_sync")

    @property
    def step(self) -> int:
        return int(_lib.pic_step_count(self._h))

    def diagnostics(self, first: int = 0, count: int | None = None) -> np.ndarray:
        if count is None:
            count = self.step - first + 1
        out = np.zeros(count, dtype=DIAG_DTYPE)
        _check(_lib.pic_diagnostics(self._h, int(first), int(count), _VP(out.ctypes.data)),
               "pic_diagnostics")
        return out

    def get_state(self, x=None, v=None):
        x = np.empty(self.p.npart, dtype=self.p.dtype) if x is None else \
            self._host(x, "x", writable=True)
        v = np.empty(self.p.npart, dtype=self.p.dtype) if v is None else \
            self._host(v, "v", writable=True)
        _check(_lib.pic_get_state(self._h, _VP(_ptr(x)), _VP(_ptr(v))), "pic_get_state")
        return x, v

    def get_cells(self, u=None, v=None):
        """The float32 state as the device holds it: (u, v), u = x NG/L."""
        n = self.p.npart
        u = np.empty(n, np.float32) if u is None else _host_array(u, np.float32, n, "u", True)
        v = np.empty(n, np.float32) if v is None else _host_array(v, np.float32, n, "v", True)
        _check(_lib.pic_get_cells(self._h, _VP(_ptr(u)), _VP(_ptr(v))), "pic_get_cells")
        return u, v

    def set_cells(self, u, v, step: int):
        """Restore a state from get_cells (continues bit for bit)."""
        u = _host_array(u, np.float32, self.p.npart, "u")
        v = _host_array(v, np.float32, self.p.npart, "v")
        _check(_lib.pic_set_cells(self._h, _VP(_ptr(u)), _VP(_ptr(v)), int(step)),
               "pic_set_cells")

    def get_field(self):
        ng = self.p.ncell
        rho, phi, E = np.zeros(ng), np.zeros(ng), np.zeros(ng)
        rq = np.zeros(ng, dtype=np.int64)
        _check(_lib.pic_get_field(self._h, _VP(rho.ctypes.data), _VP(phi.ctypes.data),
                                  _VP(E.ctypes.data), _VP(rq.ctypes.data)), "pic_get_field")
        return dict(rho=rho, phi=phi, E=E, rho_q=rq)

    def phase_space(self, nx: int, nv: int, vmin: float, vmax: float) -> np.ndarray:
        """f(x, v) counts, shape (nv, nx): row iv, column ix."""
        out = np.zeros((int(nv), int(nx)), dtype=np.uint32)
        _check(_lib.pic_phase_space(self._h, int(nx), int(nv), float(vmin), float(vmax),
                                    _VP(out.ctypes.data)), "pic_phase_space")
        return out

    def device_arrays(self):
        """Torch views (x, v, E32) of the current device arrays (positions in
        cell units in the float32 modes)."""
        import torch
        x, v, e = _VP(), _VP(), _VP()
        _check(_lib.pic_device_arrays(self._h, C.byref(x), C.byref(v), C.byref(e)),
               "pic_device_arrays")
        base = self.workspace.data_ptr()
        tdt = torch.float64 if self.p.precision == PIC_FP64 else torch.float32
        es = 8 if self.p.precision == PIC_FP64 else 4
        n = self.p.npart

        def view(addr, count, dt, size):
            off = addr - base
            return self.workspace[off:off + count * size].view(dt)
        return (view(x.value, n, tdt, es), view(v.value, n, tdt, es),
                view(e.value, self.p.ncell, torch.float32, 4))

    def set_launch(self, variant: int = 0, block: int = 0, unroll: int = 0,
                   blocks_per_sm: int = 0):
        _check(_lib.pic_set_launch(self._h, int(variant), int(block), int(unroll),
                                   int(blocks_per_sm)), "pic_set_launch")

    def autotune(self, reps: int = 5, cache: str | None = None) -> np.ndarray:
        """Time the candidate push shapes on a copy of the state and adopt
        the fastest; returns the timings.  With `cache` (a file path), a
        shape already adopted for a run of this kind on this GPU model is
        taken from the file without timing (an empty table is returned), and
        a newly adopted shape is added to it."""
        k = None
        if cache is not None:
            import torch
            from . import tune_cache
            k = tune_cache.key(torch.cuda.get_device_name(self.device), self.p.npart,
                               self.p.ncell, self.p.sort_interval, self.p.precision,
                               self.p.shape)
            hit = tune_cache.lookup(cache, k)
            if hit is not None:
                self.set_launch(hit["variant"], hit["block"], hit["unroll"])
                return np.zeros(0, dtype=TUNE_DTYPE)
        out = np.zeros(64, dtype=TUNE_DTYPE)
        n = C.c_int32(0)
        _check(_lib.pic_autotune(self._h, int(reps), _VP(out.ctypes.data), 64, C.byref(n)),
               "pic_autotune")
        table = out[:n.value]
        if k is not None and len(table):
            from . import tune_cache
            _, block, variant, unroll = self.launch_shape()
            best = table[(table["variant"] == variant) & (table["block"] == block) &
                         (table["unroll"] == unroll)]
            tune_cache.store(cache, k, variant, block, unroll,
                             float(best["ms"][0]) if len(best) else float("nan"))
        return table

    def set_shard(self, npart_total: int):
        """This run holds one rank's particles of a plasma of npart_total."""
        _check(_lib.pic_set_shard(self._h, int(npart_total)), "pic_set_shard")

    def density(self):
        """Torch int64 view of the device density accumulator (NG sums)."""
        import torch
        d = _VP()
        _check(_lib.pic_device_density(self._h, C.byref(d)), "pic_device_density")
        off = d.value - self.workspace.data_ptr()
        return self.workspace[off:off + 8 * self.p.ncell].view(torch.int64)

    def tune_sort_interval(self, intervals=(0, 5, 10, 20, 40, 80), adopt: bool = False):
        """Modelled step cost (ms) of each candidate sort interval on a copy
        of the state; returns (best interval, {S: ms}).  adopt: make the run
        sort at the best interval from now on."""
        iv = np.ascontiguousarray(intervals, dtype=np.int32)
        ms = np.zeros(iv.size, dtype=np.float32)
        best = C.c_int32(0)
        _check(_lib.pic_tune_sort_interval(self._h, _VP(iv.ctypes.data), iv.size,
                                           _VP(ms.ctypes.data), C.byref(best), int(adopt)),
               "pic_tune_sort_interval")
        if adopt:
            self.p.sort_interval = int(best.value)
        return int(best.value), {int(k): float(t) for k, t in zip(iv, ms)}

    def launch_shape(self):
        """(grid, block, variant, unroll) of the fused push."""
        g, b, v, u = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(_lib.pic_launch_shape(self._h, C.byref(g), C.byref(b), C.byref(v), C.byref(u)),
               "pic_launch_shape")
        return int(g.value), int(b.value), int(v.value), int(u.value)


PIC_LOAD_MAX_MODES = 8


class CLoading(C.Structure):
    _fields_ = [("v0", C.c_double), ("vth", C.c_double), ("seed", C.c_uint64),
                ("nmodes", C.c_int32), ("reserved", C.c_int32),
                ("mode", C.c_int32 * PIC_LOAD_MAX_MODES),
                ("eps", C.c_double * PIC_LOAD_MAX_MODES),
                ("phase", C.c_double * PIC_LOAD_MAX_MODES)]


@dataclass
class Loading:
    """Device-side two-stream loading (pic_loading): beams +-v0, spread vth,
    SplitMix64 seed, density modes [(m, eps, phase), ...]."""
    v0: float
    vth: float
    seed: int
    modes: tuple = ()

    def c(self) -> CLoading:
        ld = CLoading()
        ld.v0, ld.vth, ld.seed = float(self.v0), float(self.vth), int(self.seed)
        ld.nmodes = len(self.modes)
        ld.reserved = 0
        for i, (m, eps, ph) in enumerate(self.modes):
            ld.mode[i], ld.eps[i], ld.phase[i] = int(m), float(eps), float(ph)
        return ld


def load_two_stream(ld: Loading, n: int, length: float, x, v, stream=None):
    """Fill device tensors x, v (float32, n each) on the device."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    cl = ld.c()
    _check(_lib.pic_load_two_stream(C.byref(cl), int(n), float(length), _VP(x.data_ptr()),
                                    _VP(v.data_ptr()), _VP(s.cuda_stream)),
           "pic_load_two_stream")


class CPoolConfig(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("ncell_max", C.c_int32),
                ("history", C.c_int32), ("variant", C.c_int32),
                ("cluster", C.c_int32), ("block", C.c_int32)]


def pool_run_bytes(p: Params, history: int) -> int:
    n = C.c_size_t(0)
    cp = p.c()
    _check(_lib.pic_pool_run_bytes(C.byref(cp), int(history), C.byref(n)), "pic_pool_run_bytes")
    return int(n.value)


class Pool:
    """An ensemble of independent runs advanced together by one persistent
    cluster launch per advance (the batched and served forms)."""

    def __init__(self, max_slots: int, ncell_max: int, arena_bytes: int, history: int = 256,
                 variant: int = 0, cluster: int = 0, block: int = 0, device=None, stream=None):
        import torch
        self.device = torch.device(device if device is not None else "cuda")
        self.cfg = CPoolConfig(int(max_slots), int(ncell_max), int(history), int(variant),
                               int(cluster), int(block))
        self.history = int(history)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=self.device)
            h = _VP()
            _check(_lib.pic_pool_create(C.byref(self.cfg), _VP(self.arena.data_ptr()),
                                        int(arena_bytes), _VP(self.stream.cuda_stream),
                                        C.byref(h)), "pic_pool_create")
        self._h = h
        self.params = {}

    def close(self):
        if getattr(self, "_h", None):
            _lib.pic_pool_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, variant: int, cluster: int, block: int):
        _check(_lib.pic_pool_configure(self._h, int(variant), int(cluster), int(block)),
               "pic_pool_configure")

    def admit(self, p: Params, x0, v0, steps: int):
        """Slot of the admitted run, or None when the arena or slots are full."""
        x0 = _host_array(x0, np.float32, p.npart, "x0")
        v0 = _host_array(v0, np.float32, p.npart, "v0")
        slot = C.c_int32(-1)
        cp = p.c()
        rc = _lib.pic_pool_admit(self._h, C.byref(cp), _VP(_ptr(x0)), _VP(_ptr(v0)),
                                 int(steps), C.byref(slot))
        if rc == PIC_ENOMEM:
            return None
        _check(rc, "pic_pool_admit")
        self.params[slot.value] = p
        return int(slot.value)

    def admit_loaded(self, p: Params, ld: Loading, steps: int):
        """Slot of a run generated on the device, or None when full."""
        slot = C.c_int32(-1)
        cp, cl = p.c(), ld.c()
        rc = _lib.pic_pool_admit_loaded(self._h, C.byref(cp), C.byref(cl), int(steps),
                                        C.byref(slot))
        if rc == PIC_ENOMEM:
            return None
        _check(rc, "pic_pool_admit_loaded")
        self.params[slot.value] = p
        return int(slot.value)

    def advance(self, k: int) -> int:
        n = C.c_int32(0)
        _check(_lib.pic_pool_advance(self._h, int(k), C.byref(n)), "pic_pool_advance")
        return int(n.value)

    def finished(self):
        buf = np.zeros(int(self.cfg.max_slots), dtype=np.int32)
        n = C.c_int32(0)
        _check(_lib.pic_pool_finished(self._h, _VP(buf.ctypes.data), buf.size, C.byref(n)),
               "pic_pool_finished")
        return buf[:n.value].tolist()

    def step_count(self, slot: int) -> int:
        s = C.c_int64(0)
        _check(_lib.pic_pool_step_count(self._h, int(slot), C.byref(s)), "pic_pool_step_count")
        return int(s.value)

    def get_state(self, slot: int, x=None, v=None):
        n = self.params[slot].npart
        x = np.empty(n, np.float32) if x is None else _host_array(x, np.float32, n, "x", True)
        v = np.empty(n, np.float32) if v is None else _host_array(v, np.float32, n, "v", True)
        _check(_lib.pic_pool_get_state(self._h, int(slot), _VP(_ptr(x)), _VP(_ptr(v))),
               "pic_pool_get_state")
        return x, v

    def get_cells(self, slot: int):
        """(u, v) of the run in `slot` as the device holds them."""
        n = self.params[slot].npart
        u, v = np.empty(n, np.float32), np.empty(n, np.float32)
        _check(_lib.pic_pool_get_cells(self._h, int(slot), _VP(_ptr(u)), _VP(_ptr(v))),
               "pic_pool_get_cells")
        return u, v

    def get_field(self, slot: int):
        ng = self.params[slot].ncell
        rho, phi, E = np.zeros(ng), np.zeros(ng), np.zeros(ng)
        rq = np.zeros(ng, dtype=np.int64)
        _check(_lib.pic_pool_get_field(self._h, int(slot), _VP(rho.ctypes.data),
                                       _VP(phi.ctypes.data), _VP(E.ctypes.data),
                                       _VP(rq.ctypes.data)), "pic_pool_get_field")
        return dict(rho=rho, phi=phi, E=E, rho_q=rq)

    def diagnostics(self, slot: int, first: int = 0, count: int | None = None):
        if count is None:
            count = self.step_count(slot) - first + 1
        out = np.zeros(count, dtype=DIAG_DTYPE)
        _check(_lib.pic_pool_diagnostics(self._h, int(slot), int(first), int(count),
                                         _VP(out.ctypes.data)), "pic_pool_diagnostics")
        return out

    def release(self, slot: int):
        _check(_lib.pic_pool_release(self._h, int(slot)), "pic_pool_release")
        self.params.pop(slot, None)

    def sync(self):
        _check(_lib.pic_pool_sync(self._h), "pic_pool_sync")

    def usage(self):
        u, f = C.c_size_t(0), C.c_size_t(0)
        _check(_lib.pic_pool_usage(self._h, C.byref(u), C.byref(f)), "pic_pool_usage")
        return int(u.value), int(f.value)


def header_functions(header_path: str | None = None):
    """Names of the functions include/pic.h declares."""
    import re
    if header_path is None:
        header_path = os.path.join(os.path.dirname(_HERE), "include", "pic.h")
    text = open(header_path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z0-9_]+)\s*\(", text)))
