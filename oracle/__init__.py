"""Plain FP64 CPU oracle (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It never imports the product package
and the product never imports it: the two share nothing but the seeded
input records the tests hand to both.

The arithmetic lives in ``oracle.c`` (plain C, FP64, Neumaier sums, OpenMP
over independent rows); this module only compiles it with gcc and marshals
numpy arrays.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)


def compile_oracle(force: bool = False) -> str:
    """Build ``liboracle.so`` with gcc (no -march flags: same results on x86 and Arm)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = [
        "gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
        "-shared", "-fPIC", "-o", tmp, _SRC, "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(compile_oracle())
        lib.oracle_force_rows.argtypes = [ctypes.c_int64, _i64p, _f32p, ctypes.c_int64, _f32p,
                                          ctypes.c_float, _f64p, _f64p]
        lib.oracle_force_rows.restype = None
        lib.oracle_force_rows_eps_i.argtypes = [ctypes.c_int64, _i64p, _f32p, ctypes.c_int64, _f32p, _f64p, _f64p]
        lib.oracle_force_rows_eps_i.restype = None
        lib.oracle_potential_energy.argtypes = [ctypes.c_int64, _f32p, _f64p]
        lib.oracle_potential_energy.restype = ctypes.c_double
        lib.oracle_adjoint_rows.argtypes = [ctypes.c_int64, _i64p, ctypes.c_int64, _f32p,
                                            ctypes.c_float, _f32p, _f64p, _f64p]
        lib.oracle_adjoint_rows.restype = None
        lib.oracle_loss_k.argtypes = [ctypes.c_int64, _f32p, ctypes.c_float, _f32p, ctypes.c_int64,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.oracle_loss_k.restype = ctypes.c_double
        lib.oracle_fp32_study.argtypes = [ctypes.c_int64, _i64p, _f32p, ctypes.c_int64, _f32p,
                                          ctypes.c_float, ctypes.c_int, ctypes.c_int64, _f64p]
        lib.oracle_fp32_study.restype = None
        lib.oracle_force_jerk_rows.argtypes = [ctypes.c_int64, _i64p, _f32p, _f32p, ctypes.c_int64, _f32p, _f32p,
                                               ctypes.c_float, _f64p, _f64p, _f64p]
        lib.oracle_force_jerk_rows.restype = None
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = None
        _lib = lib
        return lib


def _rec(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 4:
        raise ValueError("particle records must be float32 (n, 4)")
    return a


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def force(pos_i, pos_mass_j, eps2, rows=None, potential: bool = True):
    """Eq. 1 acceleration (and potential) in FP64 for all i, or the listed rows.

    Returns ``(acc[n_rows, 3], pot[n_rows] or None)`` as float64.
    """
    lib = _load()
    pi = _rec(pos_i)
    pj = _rec(pos_mass_j)
    if rows is None:
        n_rows, rp = pi.shape[0], None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        if rows.size and (rows.min() < 0 or rows.max() >= pi.shape[0]):
            raise IndexError("row index out of range")
        n_rows, rp = rows.shape[0], rows
    acc = np.zeros((n_rows, 3), dtype=np.float64)
    pot = np.zeros(n_rows, dtype=np.float64) if potential else None
    lib.oracle_force_rows(n_rows, _ptr(rp, _i64p), _ptr(pi, _f32p), pj.shape[0], _ptr(pj, _f32p),
                          float(np.float32(eps2)), _ptr(acc, _f64p), _ptr(pot, _f64p))
    return acc, pot


def force_eps_i(pos_eps_i, pos_mass_j, rows=None, potential: bool = True):
    """Eq. 1 with a softening per i-particle, taken from the 4th component of
    its record (x, y, z, eps2_i) as in the appendix's force driver.

    Returns ``(acc[n_rows, 3], pot[n_rows] or None)`` as float64.
    """
    lib = _load()
    pi = _rec(pos_eps_i)
    pj = _rec(pos_mass_j)
    if rows is None:
        n_rows, rp = pi.shape[0], None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        if rows.size and (rows.min() < 0 or rows.max() >= pi.shape[0]):
            raise IndexError("row index out of range")
        n_rows, rp = rows.shape[0], rows
    acc = np.zeros((n_rows, 3), dtype=np.float64)
    pot = np.zeros(n_rows, dtype=np.float64) if potential else None
    lib.oracle_force_rows_eps_i(n_rows, _ptr(rp, _i64p), _ptr(pi, _f32p), pj.shape[0], _ptr(pj, _f32p),
                                _ptr(acc, _f64p), _ptr(pot, _f64p))
    return acc, pot


def force_jerk(pos_i, vel_i, pos_mass_j, vel_j, eps2, rows=None, potential: bool = True):
    """Acceleration, jerk (d a / dt along straight-line motion) and potential in FP64.

    Returns ``(acc[n_rows, 3], jerk[n_rows, 3], pot[n_rows] or None)``.
    """
    lib = _load()
    pi, vi = _rec(pos_i), _rec(vel_i)
    pj, vj = _rec(pos_mass_j), _rec(vel_j)
    if vi.shape[0] != pi.shape[0] or vj.shape[0] != pj.shape[0]:
        raise ValueError("velocity records must match the position records")
    if rows is None:
        n_rows, rp = pi.shape[0], None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        n_rows, rp = rows.shape[0], rows
    acc = np.zeros((n_rows, 3), dtype=np.float64)
    jerk = np.zeros((n_rows, 3), dtype=np.float64)
    pot = np.zeros(n_rows, dtype=np.float64) if potential else None
    lib.oracle_force_jerk_rows(n_rows, _ptr(rp, _i64p), _ptr(pi, _f32p), _ptr(vi, _f32p), pj.shape[0],
                               _ptr(pj, _f32p), _ptr(vj, _f32p), float(np.float32(eps2)), _ptr(acc, _f64p),
                               _ptr(jerk, _f64p), _ptr(pot, _f64p))
    return acc, jerk, pot


def potential_energy(pos_mass, pot) -> float:
    """W = 1/2 sum_i m_i phi_i in FP64."""
    pm = _rec(pos_mass)
    pot = np.ascontiguousarray(pot, dtype=np.float64)
    if pot.shape[0] != pm.shape[0]:
        raise ValueError("pot length mismatch")
    return float(_load().oracle_potential_energy(pm.shape[0], _ptr(pm, _f32p), _ptr(pot, _f64p)))


def adjoint(pos_mass, eps2, w, rows=None):
    """Analytic dL/dx and dL/dm for L = sum_i w_i . a_i (FP64)."""
    lib = _load()
    pm = _rec(pos_mass)
    w = np.ascontiguousarray(w, dtype=np.float32)
    if w.shape != (pm.shape[0], 3):
        raise ValueError("w must be float32 (n, 3)")
    if rows is None:
        n_rows, rp = pm.shape[0], None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        n_rows, rp = rows.shape[0], rows
    gp = np.zeros((n_rows, 3), dtype=np.float64)
    gm = np.zeros(n_rows, dtype=np.float64)
    lib.oracle_adjoint_rows(n_rows, _ptr(rp, _i64p), pm.shape[0], _ptr(pm, _f32p),
                            float(np.float32(eps2)), _ptr(w, _f32p), _ptr(gp, _f64p), _ptr(gm, _f64p))
    return gp, gm


def loss_k(pos_mass, eps2, w, k: int, xk, mk: float) -> float:
    """Terms of L = sum_i w_i . a_i that involve particle k, with k at ``xk`` (FP64) and mass ``mk``."""
    pm = _rec(pos_mass)
    w = np.ascontiguousarray(w, dtype=np.float32)
    return float(_load().oracle_loss_k(pm.shape[0], _ptr(pm, _f32p), float(np.float32(eps2)),
                                       _ptr(w, _f32p), int(k), float(xk[0]), float(xk[1]),
                                       float(xk[2]), float(mk)))


FP32_DIRECT = 0
FP32_FORCE_LOOP = 1
FP32_EXACT_SUM = 2


def fp32_study(pos_i, pos_mass_j, eps2, mode: int, n_jb: int = 512, rows=None) -> np.ndarray:
    """FP32 pair terms summed DIRECT, FORCE-LOOP (J-BAG of ``n_jb``) or exactly."""
    lib = _load()
    pi = _rec(pos_i)
    pj = _rec(pos_mass_j)
    if rows is None:
        n_rows, rp = pi.shape[0], None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        n_rows, rp = rows.shape[0], rows
    acc = np.zeros((n_rows, 3), dtype=np.float64)
    lib.oracle_fp32_study(n_rows, _ptr(rp, _i64p), _ptr(pi, _f32p), pj.shape[0], _ptr(pj, _f32p),
                          float(np.float32(eps2)), int(mode), int(n_jb), _ptr(acc, _f64p))
    return acc


def rel_errors(a_test, a_ref) -> np.ndarray:
    """Per-particle |a_test - a_ref| / |a_ref| (the quantity maximised in Eq. 3)."""
    a_test = np.asarray(a_test, dtype=np.float64)
    a_ref = np.asarray(a_ref, dtype=np.float64)
    num = np.linalg.norm(a_test - a_ref, axis=-1)
    den = np.linalg.norm(a_ref, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def e_max(a_test, a_ref) -> float:
    """E_max of Eq. 3: the largest per-particle relative error."""
    e = rel_errors(a_test, a_ref)
    return float(e.max()) if e.size else 0.0
