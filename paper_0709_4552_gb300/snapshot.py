"""Binary snapshots of an N-body state (the input snapshot read and the output
snapshot written by the integration loop of Sec. 4.1 steps 1 and 7).

Layout, little-endian:
  8 bytes  magic  b"NBSNAP01"
  int64    N
  float64  t_sys, eps, eta, dt_min, dt_max
  float64  m[N], x[N][3], v[N][3], a[N][3], jerk[N][3], pot[N], t[N], dt[N]

A snapshot holds everything the block-step loop needs to continue (positions,
velocities, the last acceleration and jerk, every particle's own time and
block step), so loading it into a context and stepping on gives the same
block schedule as the run that wrote it; on the FP64 path the continuation
is bitwise identical.  Host-side file I/O only: the state moves through
``nb_get_particles`` / ``nb_set_j_particles``.
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"NBSNAP01"
_HEAD = struct.Struct("<8sq5d")
_FIELDS = (("m", 1), ("x", 3), ("v", 3), ("a", 3), ("jerk", 3), ("pot", 1), ("t", 1), ("dt", 1))


def write(path, state, eps, eta, dt_min, dt_max):
    """Write a state dict (keys m, x, v, a, jerk, pot, t, dt; host arrays) to path."""
    N = int(np.asarray(state["m"]).shape[0])
    t_sys = float(np.min(state["t"])) if N else 0.0
    with open(path, "wb") as f:
        f.write(_HEAD.pack(MAGIC, N, t_sys, float(eps), float(eta), float(dt_min), float(dt_max)))
        for k, w in _FIELDS:
            a = np.ascontiguousarray(state[k], dtype="<f8")
            if a.size != N * w:
                raise ValueError(f"snapshot field {k}: {a.size} values, expected {N * w}")
            f.write(a.tobytes())


def read(path):
    """Returns (state dict, params dict) from a snapshot file."""
    with open(path, "rb") as f:
        head = f.read(_HEAD.size)
        if len(head) != _HEAD.size:
            raise ValueError("snapshot: truncated header")
        magic, N, t_sys, eps, eta, dt_min, dt_max = _HEAD.unpack(head)
        if magic != MAGIC or N < 0:
            raise ValueError("snapshot: not a snapshot file")
        state = {}
        for k, w in _FIELDS:
            buf = f.read(8 * N * w)
            if len(buf) != 8 * N * w:
                raise ValueError(f"snapshot: truncated field {k}")
            a = np.frombuffer(buf, dtype="<f8").astype(np.float64)
            state[k] = a.reshape(N, 3) if w == 3 else a
        if f.read(1):
            raise ValueError("snapshot: trailing bytes")
    return state, dict(t_sys=t_sys, eps=eps, eta=eta, dt_min=dt_min, dt_max=dt_max)


def save(ctx, path):
    """Snapshot of a single-system context (an ``nbody.NBody`` or a raw handle)."""
    from . import nbody
    ctx = getattr(ctx, "ctx", ctx)
    N = nbody.nb_get_n(ctx)
    st = nbody.nb_get_particles(ctx, 0, N)
    p = nbody.nb_get_params(ctx)
    write(path, st, p["eps"], p["eta"], p["dt_min"], p["dt_max"])


def load(ctx, path):
    """Load a snapshot into a single-system context (parameters and particles)."""
    from . import nbody
    ctx = getattr(ctx, "ctx", ctx)
    st, p = read(path)
    nbody.nb_set_params(ctx, p["eps"], p["eta"], p["dt_min"], p["dt_max"])
    nbody.nb_set_j_particles(ctx, 0, st["m"], st["x"], st["v"], st["a"], st["jerk"], st["t"], st["dt"])
    return st, p
