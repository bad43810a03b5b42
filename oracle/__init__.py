"""FP64 CPU oracle of the 1D electrostatic electron PIC step (test infrastructure).

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline
leg may import this package.  The CUDA library does not, and this package does
not import the library: the two share no code.  The arithmetic lives in
`pic_oracle.c` (plain C, built with gcc into `_build/liboracle.so`); this
module only marshals numpy arrays.  Each wrapper names the paper passage its C
function restates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

FIX_BITS = 24


def build(force: bool = False) -> str:
    """Compile pic_oracle.c with gcc (no fused multiply-add)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    """orc_params: the Appendix A parameter block."""
    _fields_ = [("ng", C.c_int32), ("shape", C.c_int32), ("np", C.c_int64),
                ("lx", C.c_double), ("dt", C.c_double),
                ("qoms0", C.c_double), ("rho_init0", C.c_double)]


CIC, NGP = 0, 1


def params(ng, np_, lx, dt=0.1, qoms0=-1.0, rho_init0=1.0, shape=CIC) -> Params:
    """shape: CIC (the listing's two-cell weighting) or NGP (nearest grid
    point: the particle's own cell)."""
    return Params(int(ng), int(shape), int(np_), float(lx), float(dt), float(qoms0),
                  float(rho_init0))


_P = C.POINTER(Params)
_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)
_L = C.POINTER(C.c_int64)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            sig = {
                "orc_particle_mass": (C.c_double, [_P]),
                "orc_deposit": (C.c_int, [_P, _D, _D]),
                "orc_field_solve": (C.c_int, [_P, _D, _D, _D]),
                "orc_field_cg": (C.c_int, [_P, _D, C.c_int, _D, _D]),
                "orc_efield": (None, [_P, _D, _D]),
                "orc_gather": (C.c_int, [_P, _D, _D, _D]),
                "orc_kick": (None, [_P, _D, _D]),
                "orc_drift": (None, [_P, _D, _D]),
                "orc_field": (C.c_int, [_P, _D, _D, _D, _D]),
                "orc_prepare": (C.c_int, [_P, _D, _D, _D, _D, _D]),
                "orc_step": (C.c_int, [_P, _D, _D, _D, _D, _D, _D, _D]),
                "orc_step_threads": (C.c_int, [_P, _D, _D, _D, _D, _D, _D, _D,
                                               C.POINTER(C.c_int32), C.c_int]),
                "orc_run_paper_order": (C.c_int, [_P, _D, _D, _D, _D, _D,
                                                  C.c_int64, _D]),
                "orc_run": (C.c_int, [_P, _D, _D, _D, _D, _D, C.c_int64,
                                      C.c_int, _D, _D]),
                "orc_field_energy": (C.c_double, [_P, _D]),
                "orc_mode_amplitudes": (None, [_P, _D, C.c_int, _D]),
                "orc_deposit_fixed": (C.c_int, [C.c_int32, C.c_int64, _F, _L]),
                "orc_deposit_fixed_ngp": (C.c_int, [C.c_int32, C.c_int64, _F, _L]),
                "orc_rho_from_fixed": (None, [_P, _L, _D]),
                "orc_fix_bits": (C.c_int, []),
                "orc_splitmix64": (C.c_uint64, [C.c_uint64, C.c_uint64]),
                "orc_load_two_stream": (C.c_int, [C.c_int64, C.c_double, C.c_double,
                                                  C.c_double, C.c_uint64, C.c_int,
                                                  C.POINTER(C.c_int32), _D, _D, _D, _D]),
                "orc_phase_space": (C.c_int, [C.c_int32, C.c_int32, C.c_double,
                                              C.c_double, C.c_double, C.c_int64, _F, _F,
                                              C.POINTER(C.c_uint32)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            assert lib.orc_fix_bits() == FIX_BITS
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed (code %d)" % (what, rc))


class State:
    """One run's FP64 state (x^n, v^{n-1/2}, rho^n, phi^n, E^n)."""

    def __init__(self, p: Params, x, v):
        self.p = p
        self.x = _f64(x).copy()
        self.v = _f64(v).copy()
        assert self.x.shape == (p.np,) and self.v.shape == (p.np,)
        ng = p.ng
        self.rho = np.zeros(ng)
        self.phi = np.zeros(ng)
        self.E = np.zeros(ng)
        self._work = np.zeros(p.np + 3 * ng + 8)
        _check(_load().orc_prepare(C.byref(p), _d(self.x), _d(self.rho),
                                   _d(self.phi), _d(self.E), _d(self._work)),
               "prepare")

    def step(self):
        """One step in the library order; returns (sum v_old v_new, sum v_new)."""
        sums = np.zeros(2)
        _check(_load().orc_step(C.byref(self.p), _d(self.x), _d(self.v),
                                _d(self.rho), _d(self.phi), _d(self.E),
                                _d(self._work), _d(sums)), "step")
        return float(sums[0]), float(sums[1])

    def step_threads(self, nthreads: int):
        """orc_step on nthreads host threads (the same state bit for bit; the
        two sums grouped by thread).  For timing the oracle on all cores."""
        if getattr(self, "_ig", None) is None:
            self._ig = np.zeros(self.p.np, dtype=np.int32)
        sums = np.zeros(2)
        _check(_load().orc_step_threads(C.byref(self.p), _d(self.x), _d(self.v),
                                        _d(self.rho), _d(self.phi), _d(self.E),
                                        _d(self._work), _d(sums),
                                        self._ig.ctypes.data_as(C.POINTER(C.c_int32)),
                                        int(nthreads)), "threaded step")
        return float(sums[0]), float(sums[1])

    def run(self, nsteps: int, nmodes: int = 8) -> np.ndarray:
        """nsteps steps; returns the per-step history rows
        [sum v^{n-1/2}v^{n+1/2}, sum v^{n+1/2}, field energy, modes...]."""
        hist = np.zeros((nsteps, 3 + nmodes))
        _check(_load().orc_run(C.byref(self.p), _d(self.x), _d(self.v),
                               _d(self.rho), _d(self.phi), _d(self.E),
                               int(nsteps), int(nmodes), _d(hist),
                               _d(self._work)), "run")
        return hist

    def run_paper_order(self, nt: int):
        _check(_load().orc_run_paper_order(C.byref(self.p), _d(self.x),
                                           _d(self.v), _d(self.rho),
                                           _d(self.phi), _d(self.E), int(nt),
                                           _d(self._work)), "paper order")

    @property
    def mass(self) -> float:
        return particle_mass(self.p)


def particle_mass(p: Params) -> float:
    return _load().orc_particle_mass(C.byref(p))


def deposit(p: Params, x) -> np.ndarray:
    """Sec. 2.3 charge deposit with the ion background: rho[NG]."""
    x = _f64(x)
    rho = np.zeros(p.ng)
    _check(_load().orc_deposit(C.byref(p), _d(x), _d(rho)), "deposit")
    return rho


def field_solve(p: Params, rho) -> np.ndarray:
    """Eq. 6 solved exactly with Phi_0 = 0: phi[NG]."""
    rho = _f64(rho)
    phi = np.zeros(p.ng)
    work = np.zeros(2 * p.ng + 2)
    _check(_load().orc_field_solve(C.byref(p), _d(rho), _d(phi), _d(work)),
           "field solve")
    return phi


def field_cg(p: Params, rho, maxit: int):
    """The Appendix A CG with maxit iterations: (phi, iterations done)."""
    rho = _f64(rho)
    phi = np.zeros(p.ng)
    work = np.zeros(3 * p.ng + 2)
    it = _load().orc_field_cg(C.byref(p), _d(rho), int(maxit), _d(phi),
                              _d(work))
    return phi, it


def efield(p: Params, phi) -> np.ndarray:
    """Eq. 7 central difference with periodic ends."""
    phi = _f64(phi)
    E = np.zeros(p.ng)
    _load().orc_efield(C.byref(p), _d(phi), _d(E))
    return E


def field(p: Params, rho):
    """rho -> (phi, E)."""
    phi = field_solve(p, rho)
    return phi, efield(p, phi)


def gather(p: Params, x, E) -> np.ndarray:
    """Sec. 2.3 field at the particles."""
    x = _f64(x)
    E = _f64(E)
    Ex = np.zeros(p.np)
    _check(_load().orc_gather(C.byref(p), _d(x), _d(E), _d(Ex)), "gather")
    return Ex


def kick(p: Params, Ex, v) -> np.ndarray:
    v = _f64(v).copy()
    _load().orc_kick(C.byref(p), _d(_f64(Ex)), _d(v))
    return v


def drift(p: Params, v, x) -> np.ndarray:
    x = _f64(x).copy()
    _load().orc_drift(C.byref(p), _d(_f64(v)), _d(x))
    return x


def field_energy(p: Params, E) -> float:
    return _load().orc_field_energy(C.byref(p), _d(_f64(E)))


def mode_amplitudes(p: Params, E, nmodes: int = 8) -> np.ndarray:
    amp = np.zeros(nmodes)
    _load().orc_mode_amplitudes(C.byref(p), _d(_f64(E)), int(nmodes), _d(amp))
    return amp


def deposit_fixed(ng: int, u32) -> np.ndarray:
    """Fixed-point deposit (reading R5) of float32 cell coordinates
    u = x/dx: int64 rho_q."""
    u32 = np.ascontiguousarray(u32, dtype=np.float32)
    rho_q = np.zeros(int(ng), dtype=np.int64)
    _check(_load().orc_deposit_fixed(int(ng), u32.size, u32.ctypes.data_as(_F),
                                     rho_q.ctypes.data_as(_L)),
           "fixed deposit")
    return rho_q


def deposit_fixed_ngp(ng: int, u32) -> np.ndarray:
    """Fixed-point nearest-grid-point deposit (R13) of float32 cell
    coordinates."""
    u32 = np.ascontiguousarray(u32, dtype=np.float32)
    rho_q = np.zeros(int(ng), dtype=np.int64)
    _check(_load().orc_deposit_fixed_ngp(int(ng), u32.size, u32.ctypes.data_as(_F),
                                         rho_q.ctypes.data_as(_L)),
           "fixed NGP deposit")
    return rho_q


def rho_from_fixed(p: Params, rho_q) -> np.ndarray:
    rho_q = np.ascontiguousarray(rho_q, dtype=np.int64)
    rho = np.zeros(p.ng)
    _load().orc_rho_from_fixed(C.byref(p), rho_q.ctypes.data_as(_L), _d(rho))
    return rho


def splitmix64(seed: int, k: int) -> int:
    """Output k >= 1 of SplitMix64 seeded with `seed` (its published definition)."""
    return int(_load().orc_splitmix64(int(seed) & (2**64 - 1), int(k) & (2**64 - 1)))


def load_two_stream(n: int, lx: float, v0: float, vth: float, seed: int, modes=()):
    """The counter-based two-stream loading (Sec. 2 set-up, Sec. 4 beams,
    reading R6) in float64: lattice positions displaced by the density modes
    [(m, eps, phase), ...], beams +-v0 by parity, Box-Muller spread from
    SplitMix64 outputs 2j+1 and 2j+2.  Returns float64 (x, v)."""
    nm = len(modes)
    mode = (C.c_int32 * max(nm, 1))(*[int(m) for m, _, _ in modes])
    eps = np.array([float(e) for _, e, _ in modes] or [0.0])
    ph = np.array([float(f) for _, _, f in modes] or [0.0])
    x = np.zeros(int(n))
    v = np.zeros(int(n))
    _check(_load().orc_load_two_stream(int(n), float(lx), float(v0), float(vth),
                                       int(seed) & (2**64 - 1), nm, mode, _d(eps), _d(ph),
                                       _d(x), _d(v)), "load")
    return x, v


def phase_space(nx: int, nv: int, lx: float, vmin: float, vmax: float, x32, v32) -> np.ndarray:
    """Counts of the float32 bin rule of the phase-space snapshot (Sec. 4,
    Fig. 1), shape (nv, nx): row iv, column ix."""
    x32 = np.ascontiguousarray(x32, dtype=np.float32)
    v32 = np.ascontiguousarray(v32, dtype=np.float32)
    out = np.zeros((int(nv), int(nx)), dtype=np.uint32)
    _check(_load().orc_phase_space(int(nx), int(nv), float(lx), float(vmin), float(vmax),
                                   x32.size, x32.ctypes.data_as(_F), v32.ctypes.data_as(_F),
                                   out.ctypes.data_as(C.POINTER(C.c_uint32))), "phase space")
    return out
