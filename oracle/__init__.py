"""FP64 CPU oracle for the direct-sum Hermite block-timestep method.

TEST INFRASTRUCTURE ONLY: the independent reference that the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA library (``paper_0709_4552_gb300``) and
imports nothing from it.

The arithmetic lives in ``nbody_oracle.c`` (plain C, IEEE FP64, no fast-math,
no FP contraction, OpenMP over active particles only); this module compiles it
with gcc on first use and marshals numpy arrays through ctypes.  Vectors are
row-major ``[n, 3]`` float64.

Functions follow the single-node loop of Sec. 4.1 (steps 2-5) of Groen et al.:
``forces`` (step 4, Eq. 3), ``predict`` (step 3), ``correct`` + ``aarseth_dt``
+ ``block_dt`` (step 5, block steps of Sec. 2), ``hermite_run`` (steps 2-6) and
``energy`` (diagnostic; the paper is silent on it).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbody_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.c_double
_i64 = ctypes.c_int64
_int = ctypes.c_int
_pd = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)
_pint = ctypes.POINTER(ctypes.c_int)


class Stats(ctypes.Structure):
    _fields_ = [("block_steps", ctypes.c_int64), ("particle_steps", ctypes.c_int64),
                ("interactions", ctypes.c_double), ("dt_underflows", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile ``nbody_oracle.c`` into ``liboracle.so`` (gcc, -O2, OpenMP)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-std=c11", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path):
    """Load an oracle shared library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    if True:  # (indented block kept flat for readability of the signatures)
        lib.orc_forces.argtypes = [_i64, _pd, _pd, _pd, _d, _i64, _pi64, _pd, _pd, _pd, _int, _int]
        lib.orc_forces.restype = None
        lib.orc_predict.argtypes = [_i64, _pd, _pd, _pd, _pd, _pd, _d, _pd, _pd]
        lib.orc_predict.restype = None
        lib.orc_correct.argtypes = [_i64] + [_pd] * 13
        lib.orc_correct.restype = None
        lib.orc_aarseth_dt.argtypes = [_pd, _pd, _pd, _pd, _d]
        lib.orc_aarseth_dt.restype = _d
        lib.orc_block_dt.argtypes = [_d, _d, _d, _d, _d, _pint]
        lib.orc_block_dt.restype = _d
        lib.orc_initial_dt.argtypes = [_pd, _pd, _d, _d, _d]
        lib.orc_initial_dt.restype = _d
        lib.orc_pow2_floor.argtypes = [_d]
        lib.orc_pow2_floor.restype = _d
        lib.orc_energy.argtypes = [_i64, _pd, _pd, _pd, _d, _int, _pd, _pd]
        lib.orc_energy.restype = None
        lib.orc_hermite_run.argtypes = [_i64, _pd, _pd, _pd, _pd, _pd, _pd, _pd, _pd, _d, _d, _d, _d, _d,
                                        _int, _int, _int, _i64, ctypes.POINTER(Stats)]
        lib.orc_hermite_run.restype = _i64
        lib.orc_max_threads.argtypes = []
        lib.orc_max_threads.restype = _int
    return lib


_override = threading.local()


def _load():
    lib = getattr(_override, "lib", None)
    if lib is not None:
        return lib
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
        return _lib


class using:
    """Context manager: run the wrappers below on another build of
    ``nbody_oracle.c`` (used by the tests that plant mistakes in a copy of
    the oracle source to show that the pins catch them)."""

    def __init__(self, so_path):
        self.lib = _bind(so_path)

    def __enter__(self):
        self.prev = getattr(_override, "lib", None)
        _override.lib = self.lib
        return self

    def __exit__(self, *exc):
        _override.lib = self.prev
        return False


def compile_source(src_text: str, out_path: str) -> str:
    """Compile C source text (a copy of ``nbody_oracle.c``) with the oracle's
    flags into ``out_path``."""
    c_path = out_path[:-3] + ".c" if out_path.endswith(".so") else out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fno-fast-math", "-std=c11", "-w", "-o", out_path, c_path, "-lm"], check=True)
    return out_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a):
    return a.ctypes.data_as(_pd)


def max_threads() -> int:
    """OpenMP threads the oracle uses by default (all host cores)."""
    return int(_load().orc_max_threads())


def forces(m, x, v, eps, idx=None, compensated=False, threads=0):
    """Acceleration, jerk and potential on particles ``idx`` (all if None)
    from all N particles at (x, v); j == i excluded.  Sec. 4.1 step 4."""
    lib = _load()
    m = _f64(m)
    N = m.shape[0]
    x = _f64(x, (N, 3))
    v = _f64(v, (N, 3))
    if idx is None:
        n, pidx = N, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        if idx.size and (idx.min() < 0 or idx.max() >= N):
            raise IndexError("active index out of range")
        n, pidx = idx.shape[0], idx.ctypes.data_as(_pi64)
    acc = np.zeros((n, 3))
    jerk = np.zeros((n, 3))
    pot = np.zeros(n)
    if n:
        lib.orc_forces(N, _p(m), _p(x), _p(v), float(eps), n, pidx, _p(acc), _p(jerk), _p(pot),
                       int(bool(compensated)), int(threads))
    return acc, jerk, pot


def predict(x, v, a, jk, t_i, t):
    """Taylor prediction of all particles to time t.  Sec. 4.1 step 3."""
    lib = _load()
    t_i = _f64(t_i)
    N = t_i.shape[0]
    x, v, a, jk = (_f64(q, (N, 3)) for q in (x, v, a, jk))
    xp = np.empty((N, 3))
    vp = np.empty((N, 3))
    lib.orc_predict(N, _p(x), _p(v), _p(a), _p(jk), _p(t_i), float(t), _p(xp), _p(vp))
    return xp, vp


def correct(x0, v0, a0, j0, xp, vp, a1, j1, h):
    """Hermite corrector (Sec. 4.1 step 5).  Returns x1, v1, a2_end, a3."""
    lib = _load()
    h = _f64(np.atleast_1d(h))
    n = h.shape[0]
    arrs = [_f64(q, (n, 3)) for q in (x0, v0, a0, j0, xp, vp, a1, j1)]
    x1, v1, a2, a3 = (np.empty((n, 3)) for _ in range(4))
    lib.orc_correct(n, *[_p(q) for q in arrs], _p(h), _p(x1), _p(v1), _p(a2), _p(a3))
    return x1, v1, a2, a3


def aarseth_dt(a, j, a2, a3, eta):
    lib = _load()
    a, j, a2, a3 = (_f64(q, (3,)) for q in (a, j, a2, a3))
    return float(lib.orc_aarseth_dt(_p(a), _p(j), _p(a2), _p(a3), float(eta)))


def block_dt(dt_crit, dt_old, t, dt_min, dt_max):
    """Returns (new_dt, underflow_flag).  Block rule of Sec. 2."""
    lib = _load()
    uf = ctypes.c_int(0)
    r = lib.orc_block_dt(float(dt_crit), float(dt_old), float(t), float(dt_min), float(dt_max),
                         ctypes.byref(uf))
    return float(r), int(uf.value)


def initial_dt(a, j, eta, dt_min, dt_max):
    lib = _load()
    a, j = _f64(a, (3,)), _f64(j, (3,))
    return float(lib.orc_initial_dt(_p(a), _p(j), float(eta), float(dt_min), float(dt_max)))


def pow2_floor(x):
    return float(_load().orc_pow2_floor(float(x)))


def energy(m, x, v, eps, threads=0):
    """(kinetic, potential) energy with the softened pairwise potential."""
    lib = _load()
    m = _f64(m)
    N = m.shape[0]
    x, v = _f64(x, (N, 3)), _f64(v, (N, 3))
    ek, ep = _d(0), _d(0)
    lib.orc_energy(N, _p(m), _p(x), _p(v), float(eps), int(threads), ctypes.byref(ek), ctypes.byref(ep))
    return float(ek.value), float(ep.value)


def hermite_run(m, x, v, eps, eta, dt_min, dt_max, t_end, state=None, compensated=False,
                threads=0, max_block_steps=-1):
    """Block-timestep Hermite integration (Sec. 4.1 steps 2-6) to t_end.

    ``state`` (optional dict with a, jerk, pot, t, dt) continues a run;
    otherwise forces and initial steps are computed at t = 0.
    Returns a dict with x, v, a, jerk, pot, t, dt and the run statistics."""
    lib = _load()
    m = _f64(m)
    N = m.shape[0]
    x = _f64(x, (N, 3)).copy()
    v = _f64(v, (N, 3)).copy()
    if state is None:
        a, jk, pot = np.zeros((N, 3)), np.zeros((N, 3)), np.zeros(N)
        t_i, dt = np.zeros(N), np.zeros(N)
        init = 1
    else:
        a = _f64(state["a"], (N, 3)).copy()
        jk = _f64(state["jerk"], (N, 3)).copy()
        pot = _f64(state["pot"]).copy()
        t_i = _f64(state["t"]).copy()
        dt = _f64(state["dt"]).copy()
        init = 0
    st = Stats()
    r = lib.orc_hermite_run(N, _p(m), _p(x), _p(v), _p(a), _p(jk), _p(pot), _p(t_i), _p(dt),
                            float(eps), float(eta), float(dt_min), float(dt_max), float(t_end),
                            init, int(bool(compensated)), int(threads), int(max_block_steps),
                            ctypes.byref(st))
    if r < 0:
        raise ValueError("bad integrator arguments (t_end must be a multiple of dt_max)")
    return dict(x=x, v=v, a=a, jerk=jk, pot=pot, t=t_i, dt=dt, block_steps=st.block_steps,
                particle_steps=st.particle_steps, interactions=st.interactions,
                dt_underflows=st.dt_underflows)
