"""FP64 CPU oracle of the Hermite-4 block-time-step N-body method (ctypes over oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline / reference arm of ``bench.py`` may import this package.
It shares no code with the CUDA library (``paper_astro_ph_0702058_gb300``)
and never imports it.

Each wrapper cites the passage of Portegies Zwart, Belleman & Geldof (2007)
whose arithmetic the C function follows (see ``oracle.h``).  Arrays are
numpy float64 (n, 3) for vectors, int64 ticks of dt_min = 2^-lmax for times
and int8 levels with dt = 2^-level.

Parity pins (see ``tests/test_oracle_pins.py``): every function here is
checked against something other than itself -- closed forms (two-body
Kepler orbit, circular-orbit time-step criterion, polynomial trajectories
for predictor and corrector), finite differences, exact rational brute force
at N <= 16, conservation laws and hand-built block schedules.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_I32 = C.POINTER(C.c_int32)
_I8 = C.POINTER(C.c_int8)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no FP contraction)."""
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-Wextra", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # NBODY_ORACLE_LIB points the tests' mutation check at a deliberately
            # broken copy of this oracle; normal use builds and loads liboracle.so.
            alt = os.environ.get("NBODY_ORACLE_LIB")
            if not alt:
                build()
            L = C.CDLL(alt or _LIB)
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            L.orc_force.argtypes = [C.c_int64, _D, _D, _D, C.c_double, C.c_int64, _I32, _D, _D, _D]
            L.orc_force_fp32_terms.argtypes = [C.c_int64, _D, _D, _D, C.c_double, C.c_int64, _I32, _D, _D, _D]
            L.orc_force_sorted_fp32.argtypes = [C.c_int64, _D, _D, _D, C.c_double, C.c_int64, _I32, _D, _D, _D]
            L.orc_rsqrt_rn_f32.argtypes = [C.c_float]
            L.orc_rsqrt_rn_f32.restype = C.c_float
            L.orc_predict.argtypes = [C.c_int64, _D, _D, _D, _D, _I64, C.c_int64, C.c_int, _D, _D]
            L.orc_dt_initial.argtypes = [_D, _D, C.c_double]
            L.orc_dt_initial.restype = C.c_double
            L.orc_dt_aarseth.argtypes = [_D, _D, _D, _D, C.c_double]
            L.orc_dt_aarseth.restype = C.c_double
            L.orc_level_floor.argtypes = [C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int)]
            L.orc_level_floor.restype = C.c_int
            L.orc_next_level.argtypes = [C.c_int, C.c_int, C.c_int64, C.c_int, C.c_int]
            L.orc_next_level.restype = C.c_int
            L.orc_schedule.argtypes = [C.c_int64, _I64, _I8, C.c_int, _I64, _I32]
            L.orc_schedule.restype = C.c_int64
            L.orc_correct.argtypes = [C.c_int64, _I32, _D, _D, _D, _D, _I64, _I8, _D, _D, _D, _D,
                                      C.c_int64, C.c_double, C.c_int, C.c_int, _D, _I64]
            L.orc_correct.restype = C.c_int64
            L.orc_init.argtypes = [C.c_int64, _D, _D, _D, C.c_double, C.c_double, C.c_int, C.c_int,
                                   _D, _D, _I64, _I8, _I64]
            L.orc_energy.argtypes = [C.c_int64, _D, _D, _D, C.c_double, _D, _D]
            L.orc_evolve.argtypes = [C.c_int64, _D, _D, _D, _D, _D, _I64, _I8, C.c_double,
                                     C.c_double, C.c_int, C.c_int, C.c_int64, C.c_int64,
                                     _I64, _I64, _I32, C.c_int64, _I64]
            L.orc_evolve.restype = C.c_int64
            _lib = L
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def force(m, x, v, eps2, active=None):
    """(acc, jerk, pot) on the listed particles: Eq. (Force) with the Appendix A pair term."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    act = np.arange(n, dtype=np.int32) if active is None else np.ascontiguousarray(active, dtype=np.int32)
    na = act.shape[0]
    acc = np.zeros((na, 3))
    jerk = np.zeros((na, 3))
    pot = np.zeros(na)
    lib().orc_force(n, _p(m, _D), _p(x, _D), _p(v, _D), float(eps2), na, _p(act, _I32),
                    _p(acc, _D), _p(jerk, _D), _p(pot, _D))
    return acc, jerk, pot


def force_fp32_terms(m, x, v, eps2, active=None):
    """(acc, jerk, pot) as the FP64 sums of the FP32 pair terms of the compensated pair term
    formed with correctly rounded operations in a fixed order (the summation check)."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    act = np.arange(n, dtype=np.int32) if active is None else np.ascontiguousarray(active, dtype=np.int32)
    na = act.shape[0]
    acc = np.zeros((na, 3))
    jerk = np.zeros((na, 3))
    pot = np.zeros(na)
    lib().orc_force_fp32_terms(n, _p(m, _D), _p(x, _D), _p(v, _D), float(eps2), na, _p(act, _I32),
                               _p(acc, _D), _p(jerk, _D), _p(pot, _D))
    return acc, jerk, pot


def force_sorted_fp32(m, x, v, eps2, active=None):
    """(acc, jerk, pot) of the sorted-summation ablation: plain FP32 pair terms (correctly
    rounded, fixed order) added in FP32 by increasing magnitude (Sect. 6 of the paper)."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    act = np.arange(n, dtype=np.int32) if active is None else np.ascontiguousarray(active, dtype=np.int32)
    na = act.shape[0]
    acc = np.zeros((na, 3))
    jerk = np.zeros((na, 3))
    pot = np.zeros(na)
    lib().orc_force_sorted_fp32(n, _p(m, _D), _p(x, _D), _p(v, _D), float(eps2), na, _p(act, _I32),
                                _p(acc, _D), _p(jerk, _D), _p(pot, _D))
    return acc, jerk, pot


def rsqrt_rn_f32(r2):
    """Correctly rounded single-precision 1/sqrt(r2)."""
    return np.float32(lib().orc_rsqrt_rn_f32(float(np.float32(r2))))


def predict(x, v, a, k, t_tick, t_new, lmax):
    """Predicted (x_p, v_p) of every particle at tick t_new (Sect. 2 predictor)."""
    x = _f64(x)
    n = x.shape[0]
    v, a, k = _f64(v, (n, 3)), _f64(a, (n, 3)), _f64(k, (n, 3))
    t = np.ascontiguousarray(t_tick, dtype=np.int64)
    xp = np.empty((n, 3))
    vp = np.empty((n, 3))
    lib().orc_predict(n, _p(x, _D), _p(v, _D), _p(a, _D), _p(k, _D), _p(t, _I64), int(t_new),
                      int(lmax), _p(xp, _D), _p(vp, _D))
    return xp, vp


def dt_initial(a, k, eta):
    return float(lib().orc_dt_initial(_p(_f64(a), _D), _p(_f64(k), _D), float(eta)))


def dt_aarseth(a1, k1, a2e, a3, eta):
    return float(lib().orc_dt_aarseth(_p(_f64(a1), _D), _p(_f64(k1), _D), _p(_f64(a2e), _D),
                                      _p(_f64(a3), _D), float(eta)))


def level_floor(dt, lmin, lmax):
    """(level, below_min) for a time step dt (power-of-two quantisation)."""
    bm = C.c_int(0)
    L = lib().orc_level_floor(float(dt), int(lmin), int(lmax), C.byref(bm))
    return int(L), bool(bm.value)


def next_level(l_old, l_crit, t_new, lmin, lmax):
    return int(lib().orc_next_level(int(l_old), int(l_crit), int(t_new), int(lmin), int(lmax)))


def schedule(t_tick, level, lmax):
    """(t_blk, active) of the next block (Sect. 2 step list)."""
    t = np.ascontiguousarray(t_tick, dtype=np.int64)
    lv = np.ascontiguousarray(level, dtype=np.int8)
    n = t.shape[0]
    act = np.empty(max(n, 1), dtype=np.int32)
    tb = C.c_int64(0)
    na = lib().orc_schedule(n, _p(t, _I64), _p(lv, _I8), int(lmax), C.byref(tb), _p(act, _I32))
    return int(tb.value), act[:na].copy()


class State:
    """FP64 particle state of the oracle integrator (all arrays owned here)."""

    def __init__(self, m, x, v, eps2, eta, *, eta_init=None, lmin=6, lmax=26):
        self.m = _f64(m).copy()
        self.n = self.m.shape[0]
        self.x = _f64(x, (self.n, 3)).copy()
        self.v = _f64(v, (self.n, 3)).copy()
        self.a = np.zeros((self.n, 3))
        self.k = np.zeros((self.n, 3))
        self.t = np.zeros(self.n, dtype=np.int64)
        self.level = np.zeros(self.n, dtype=np.int8)
        self.eps2 = float(eps2)
        self.eta = float(eta)
        self.eta_init = float(eta if eta_init is None else eta_init)
        self.lmin, self.lmax = int(lmin), int(lmax)
        self.n_below_min = 0

    def ptrs(self):
        return (_p(self.m, _D), _p(self.x, _D), _p(self.v, _D), _p(self.a, _D), _p(self.k, _D),
                _p(self.t, _I64), _p(self.level, _I8))

    def init(self):
        """Full force at t = 0 and initial levels from Eq. (initTimestep)."""
        bm = C.c_int64(0)
        m, x, v, a, k, t, lv = self.ptrs()
        lib().orc_init(self.n, m, x, v, self.eps2, self.eta_init, self.lmin, self.lmax, a, k, t,
                       lv, C.byref(bm))
        self.n_below_min += bm.value
        return self

    def schedule(self):
        return schedule(self.t, self.level, self.lmax)

    def predict(self, t_new):
        return predict(self.x, self.v, self.a, self.k, self.t, t_new, self.lmax)

    def correct(self, active, xp, vp, acc, jerk, t_new):
        """Corrector + new levels for ``active``; returns dt_crit per active particle."""
        act = np.ascontiguousarray(active, dtype=np.int32)
        na = act.shape[0]
        acc = _f64(acc, (na, 3))
        jerk = _f64(jerk, (na, 3))
        xp, vp = _f64(xp, (self.n, 3)), _f64(vp, (self.n, 3))
        dtc = np.empty(max(na, 1))
        bm = C.c_int64(0)
        _, x, v, a, k, t, lv = self.ptrs()
        bad = lib().orc_correct(na, _p(act, _I32), x, v, a, k, t, lv, _p(xp, _D), _p(vp, _D),
                                _p(acc, _D), _p(jerk, _D), int(t_new), self.eta, self.lmin,
                                self.lmax, _p(dtc, _D), C.byref(bm))
        self.n_below_min += bm.value
        if bad:
            raise FloatingPointError(f"oracle corrector: {bad} non-finite particles")
        return dtc[:na]

    def step(self):
        """One block step; returns (t_blk, active, acc, jerk, pot, dt_crit)."""
        t_blk, act = self.schedule()
        xp, vp = self.predict(t_blk)
        acc, jerk, pot = force(self.m, xp, vp, self.eps2, act)
        dtc = self.correct(act, xp, vp, acc, jerk, t_blk)
        return t_blk, act, acc, jerk, pot, dtc

    def evolve(self, t_end_tick, max_blocks=1 << 40, record_lists=0):
        """Block steps up to t_end_tick in C; returns (blk_t, blk_n, lists)."""
        cap = int(max_blocks) if max_blocks < (1 << 24) else (1 << 24)
        bt = np.zeros(cap, dtype=np.int64)
        bn = np.zeros(cap, dtype=np.int64)
        lists = np.zeros(max(int(record_lists), 1), dtype=np.int32)
        bm = C.c_int64(0)
        m, x, v, a, k, t, lv = self.ptrs()
        nb = lib().orc_evolve(self.n, m, x, v, a, k, t, lv, self.eps2, self.eta, self.lmin,
                              self.lmax, int(t_end_tick), min(int(max_blocks), cap),
                              _p(bt, _I64), _p(bn, _I64),
                              _p(lists, _I32) if record_lists else None, int(record_lists),
                              C.byref(bm))
        self.n_below_min += bm.value
        if nb < 0:
            raise FloatingPointError(f"oracle run stopped on a non-finite state after {-nb - 1} blocks")
        cs = np.cumsum(bn[:nb])
        used = int(cs[cs <= int(record_lists)][-1]) if record_lists and (cs <= int(record_lists)).any() else 0
        return bt[:nb].copy(), bn[:nb].copy(), (lists[:used].copy() if record_lists else None)

    def energy(self):
        return energy(self.m, self.x, self.v, self.eps2)

    def time(self):
        return np.ldexp(self.t.astype(np.float64), -self.lmax)


def energy(m, x, v, eps2):
    """(E_kin, E_pot) with the softened potential, excluding self-terms."""
    m = _f64(m)
    n = m.shape[0]
    x, v = _f64(x, (n, 3)), _f64(v, (n, 3))
    ek, ep = C.c_double(0), C.c_double(0)
    lib().orc_energy(n, _p(m, _D), _p(x, _D), _p(v, _D), float(eps2), C.byref(ek), C.byref(ep))
    return float(ek.value), float(ep.value)
