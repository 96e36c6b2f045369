"""Thin ctypes binding to libnbody.so, the CUDA C-ABI library of this package.

Every ``nb_*`` function here has the name and meaning of the C entry point in
``include/nbody.h`` and only marshals arguments: numpy arrays (and CPU torch
tensors) are passed as host pointers (``NB_PTR_HOST``), CUDA torch tensors as
device pointers (``NB_PTR_DEVICE``) on the context's stream.  A non-zero
status raises :class:`NBodyError`.  All computation happens in the library's
CUDA kernels: there is no Python or CPU fallback, and loading fails loudly
when ``libnbody.so`` has not been built (``paper_0709_4552_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnbody.so")
# the autotuner's table measured on a GB300 (152 SMs), shipped with the
# package; contexts load it through NB_TUNE_FILE unless the caller set that
# (the library refuses a table measured on a GPU with another SM count)
DEFAULT_TUNE_FILE = os.path.join(HERE, "tuning", "gb300_152sm.json")

NB_OK, NB_EINVAL, NB_ENOMEM, NB_ECUDA, NB_ENUMERIC, NB_EDTMIN, NB_ETIMEOUT, NB_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
NB_FP64, NB_MIXED = 0, 1
NB_PTR_HOST, NB_PTR_DEVICE = 0, 1
NB_ENSEMBLE_PERSISTENT, NB_ENSEMBLE_PER_CLUSTER = 0, 1
NB_LOOP_HOST, NB_LOOP_GRAPH, NB_LOOP_PERSISTENT, NB_LOOP_CLUSTER, NB_LOOP_AUTO = 0, 1, 2, 3, 4
NB_PERSISTENT_MAX_N, NB_PERSISTENT_MAX_N_FP64 = 262144, 65536
NB_CLUSTER_MAX_N = 16384
NB_JPREDICT_AUTO = -1

# every symbol include/nbody.h declares
EXPORTS = (
    "nb_create", "nb_destroy", "nb_set_params", "nb_get_params", "nb_default_params", "nb_set_precision",
    "nb_set_j_particles", "nb_set_n", "nb_get_n", "nb_get_particles", "nb_next_block", "nb_predict",
    "nb_compute_forces", "nb_compute_forces_at", "nb_get_particles_idx", "nb_set_particles_idx",
    "nb_get_predicted", "nb_forces_on", "nb_set_forces", "nb_set_initial_forces", "nb_set_jpredict", "nb_get_jpredict", "nb_correct", "nb_initial_forces_and_dt", "nb_step", "nb_integrate",
    "nb_energy", "nb_get_timings", "nb_get_counters", "nb_check_device_status", "nb_check_grid_barrier",
    "nb_last_error", "nb_clear_error",
    "nb_set_tuning", "nb_set_far_tiles", "nb_get_far_tiles", "nb_selftest_corrector", "nb_autotune", "nb_autotune_list", "nb_ensemble_autotune", "nb_tune_save", "nb_tune_load", "nb_tune_count", "nb_tune_clear",
    "nb_measure_peaks", "nb_measure_fp64_issue", "nb_ensemble_create", "nb_ensemble_initial_forces_and_dt",
    "nb_ensemble_integrate", "nb_ensemble_energy", "nb_forces_fp64_noalloc", "nb_strerror", "nb_version",
)


class NBodyError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {_strerror(code)} ({code})" if what else f"{_strerror(code)} ({code})")


_lib = None
_vp = ctypes.c_void_p
_d = ctypes.c_double
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_int = ctypes.c_int
_pd = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)
_pint = ctypes.POINTER(ctypes.c_int)


def lib():
    """The loaded libnbody.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_0709_4552_gb300.build` (needs nvcc); there is no fallback")
    if "NB_TUNE_FILE" not in os.environ and os.path.exists(DEFAULT_TUNE_FILE):
        os.environ["NB_TUNE_FILE"] = DEFAULT_TUNE_FILE
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "nb_create": (_int, [ctypes.POINTER(_vp), _i64, _int, _int, _vp]),
        "nb_destroy": (None, [_vp]),
        "nb_set_params": (_int, [_vp, _d, _d, _d, _d]),
        "nb_get_params": (_int, [_vp, _vp, _vp, _vp, _vp]),
        "nb_default_params": (None, [_pd, _pd, _pd, _pd]),
        "nb_set_precision": (_int, [_vp, _int]),
        "nb_set_j_particles": (_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _int]),
        "nb_set_n": (_int, [_vp, _i64]),
        "nb_get_n": (_int, [_vp, _pi64]),
        "nb_get_particles": (_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _int]),
        "nb_next_block": (_int, [_vp, _pd, _vp, _pi64]),
        "nb_predict": (_int, [_vp, _d]),
        "nb_compute_forces": (_int, [_vp, _vp, _i64, _vp, _vp, _vp, _int]),
        "nb_compute_forces_at": (_int, [_vp, _d, _vp, _i64, _vp, _vp, _vp, _int]),
        "nb_set_jpredict": (_int, [_vp, _i64]),
        "nb_get_particles_idx": (_int, [_vp, _vp, _i64] + [_vp] * 8 + [_int]),
        "nb_set_particles_idx": (_int, [_vp, _vp, _i64] + [_vp] * 8 + [_int]),
        "nb_get_predicted": (_int, [_vp, _vp, _i64, _vp, _vp, _int]),
        "nb_forces_on": (_int, [_vp, _i64, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _int, _int]),
        "nb_set_forces": (_int, [_vp, _vp, _i64, _vp, _vp, _vp, _int]),
        "nb_set_initial_forces": (_int, [_vp, _vp, _vp, _vp, _int]),
        "nb_get_jpredict": (_int, [_vp, _pi64]),
        "nb_correct": (_int, [_vp, _vp, _i64, _d, _int]),
        "nb_initial_forces_and_dt": (_int, [_vp]),
        "nb_step": (_int, [_vp, _pd, _pi64]),
        "nb_integrate": (_int, [_vp, _d, _int]),
        "nb_energy": (_int, [_vp, _pd, _pd]),
        "nb_get_timings": (_int, [_vp, _pd, _pd, _pd, _pd, _int]),
        "nb_get_counters": (_int, [_vp, _pi64, _pi64]),
        "nb_check_device_status": (_int, [_vp, _pi64]),
        "nb_check_grid_barrier": (_int, [_vp, _int, _d]),
        "nb_last_error": (_int, [_vp]),
        "nb_clear_error": (None, [_vp]),
        "nb_set_tuning": (_int, [_vp, _int, _int, _int, _int]),
        "nb_set_far_tiles": (_int, [_vp, _int]),
        "nb_get_far_tiles": (_int, [_vp, _pint]),
        "nb_selftest_corrector": (_int, [_int, _i64, ctypes.c_uint64, ctypes.POINTER(_i64)]),
        "nb_autotune": (_int, [_vp, _i64, _pint, _pint, _pint, _pint]),
        "nb_autotune_list": (_int, [_vp, _vp, _i64, _int, _pint, _pint, _pint, _pint]),
        "nb_ensemble_autotune": (_int, [_vp, _i64, _pint, _pint, _pd, _pd]),
        "nb_tune_save": (_int, [_vp, ctypes.c_char_p]),
        "nb_tune_load": (_int, [_vp, ctypes.c_char_p]),
        "nb_tune_count": (_int, [_vp, _pint]),
        "nb_tune_clear": (_int, [_vp]),
        "nb_ensemble_create": (_int, [ctypes.POINTER(_vp), _i32, _vp, _vp, _int, _int, _vp]),
        "nb_measure_peaks": (_int, [_vp, _pd, _pd, _pd]),
        "nb_measure_fp64_issue": (_int, [_vp, _pd, _pd, _pd, _pd]),
        "nb_ensemble_initial_forces_and_dt": (_int, [_vp]),
        "nb_ensemble_integrate": (_int, [_vp, _d, _int]),
        "nb_ensemble_energy": (_int, [_vp, _vp, _vp]),
        "nb_forces_fp64_noalloc": (_int, [_i64, _vp, _vp, _vp, _d, _vp, _i64, _vp, _vp, _vp, _vp]),
        "nb_strerror": (ctypes.c_char_p, [_int]),
        "nb_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _strerror(code):
    try:
        return lib().nb_strerror(int(code)).decode()
    except Exception:  # library unavailable while formatting an error
        return "error"


def _check(code, what=""):
    if code != NB_OK:
        raise NBodyError(code, what)


# ---------------------------------------------------------------- marshalling
def _kind_ptr(a, dtype):
    """(ptr_kind, pointer, keep-alive) for a numpy array or torch tensor."""
    if a is None:
        return None, None, None
    mod = type(a).__module__
    if mod.startswith("torch"):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return (NB_PTR_DEVICE if a.is_cuda else NB_PTR_HOST), ctypes.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return NB_PTR_HOST, ctypes.c_void_p(arr.ctypes.data), arr


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream


def _stream(stream):
    """cudaStream_t for a torch stream / raw handle; torch's default stream
    (handle 0) is passed as cudaStreamLegacy because NULL asks the library
    for a stream of its own."""
    if stream is None:
        return None
    h = int(getattr(stream, "cuda_stream", stream))
    return _vp(h if h != 0 else CUDA_STREAM_LEGACY)


def _marshal(arrays, dtypes):
    kinds, ptrs, keep = set(), [], []
    for a, dt in zip(arrays, dtypes):
        k, p, kp = _kind_ptr(a, dt)
        if k is not None:
            kinds.add(k)
        ptrs.append(p)
        keep.append(kp)
    if len(kinds) > 1:
        raise TypeError("mix of host and device buffers in one call")
    return (kinds.pop() if kinds else NB_PTR_HOST), ptrs, keep


# ------------------------------------------------------------ C entry points
def nb_version():
    return lib().nb_version().decode()


def nb_strerror(code):
    return lib().nb_strerror(int(code)).decode()


def nb_default_params():
    v = [_d() for _ in range(4)]
    lib().nb_default_params(*[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)


def nb_create(n_max, precision=NB_MIXED, device=0, stream=None):
    h = _vp()
    s = _stream(stream)
    _check(lib().nb_create(ctypes.byref(h), int(n_max), int(precision), int(device), s), "nb_create")
    return h


def nb_destroy(ctx):
    lib().nb_destroy(ctx)


def nb_set_params(ctx, eps, eta, dt_min, dt_max):
    _check(lib().nb_set_params(ctx, eps, eta, dt_min, dt_max), "nb_set_params")


def nb_get_params(ctx):
    vals = [_d() for _ in range(4)]
    _check(lib().nb_get_params(ctx, *[ctypes.byref(x) for x in vals]), "nb_get_params")
    return dict(zip(("eps", "eta", "dt_min", "dt_max"), (x.value for x in vals)))


def nb_set_precision(ctx, precision):
    _check(lib().nb_set_precision(ctx, int(precision)), "nb_set_precision")


def nb_set_j_particles(ctx, first, m, x, v, a=None, jerk=None, t=None, dt=None):
    count = int(m.shape[0])
    kind, p, keep = _marshal([m, x, v, a, jerk, t, dt], [np.float64] * 7)
    _check(lib().nb_set_j_particles(ctx, int(first), count, *p, kind), "nb_set_j_particles")
    del keep


def nb_set_n(ctx, n):
    _check(lib().nb_set_n(ctx, int(n)), "nb_set_n")


def nb_get_n(ctx):
    n = _i64()
    _check(lib().nb_get_n(ctx, ctypes.byref(n)), "nb_get_n")
    return n.value


def nb_get_particles(ctx, first, count, out=None):
    """Returns a dict of host arrays (or fills ``out``: dict of arrays/tensors
    with keys m, x, v, a, jerk, pot, t, dt; missing keys are skipped)."""
    if out is None:
        out = dict(m=np.empty(count), x=np.empty((count, 3)), v=np.empty((count, 3)),
                   a=np.empty((count, 3)), jerk=np.empty((count, 3)), pot=np.empty(count),
                   t=np.empty(count), dt=np.empty(count))
    keys = ["m", "x", "v", "a", "jerk", "pot", "t", "dt"]
    kind, p, keep = _marshal([out.get(k) for k in keys], [np.float64] * 8)
    _check(lib().nb_get_particles(ctx, int(first), int(count), *p, kind), "nb_get_particles")
    # numpy outputs that were copied to a contiguous buffer are returned as such
    for k, kp in zip(keys, keep):
        if k in out and isinstance(kp, np.ndarray) and kp is not out[k]:
            out[k][...] = kp
    return out


def nb_next_block(ctx, want_indices=True):
    t = _d()
    n = _i64()
    N = nb_get_n(ctx)
    idx = np.empty(N, dtype=np.int32) if want_indices else None
    _check(lib().nb_next_block(ctx, ctypes.byref(t), None if idx is None else idx.ctypes.data_as(_vp),
                               ctypes.byref(n)), "nb_next_block")
    return t.value, n.value, (idx[: n.value].copy() if idx is not None else None)


def nb_predict(ctx, t):
    _check(lib().nb_predict(ctx, float(t)), "nb_predict")


def nb_compute_forces(ctx, i_idx, acc=None, jerk=None, pot=None):
    """Forces on the active list i_idx.  With numpy/host inputs and no
    outputs given, returns new host arrays (acc[n,3], jerk[n,3], pot[n])."""
    n = int(i_idx.shape[0])
    ret = False
    if acc is None and jerk is None and pot is None and type(i_idx).__module__ != "torch":
        acc, jerk, pot = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
        ret = True
    kind, p, keep = _marshal([i_idx, acc, jerk, pot], [np.int32, np.float64, np.float64, np.float64])
    _check(lib().nb_compute_forces(ctx, p[0], n, p[1], p[2], p[3], kind), "nb_compute_forces")
    if ret:
        return keep[1], keep[2], keep[3]
    return acc, jerk, pot


def nb_compute_forces_at(ctx, t, i_idx, acc=None, jerk=None, pot=None):
    """GRAPE-style forces on i_idx at time t: the list predicted alone, the
    j-particles predicted inside the force kernel (no nb_predict needed).
    Returns like nb_compute_forces."""
    n = int(i_idx.shape[0])
    ret = False
    if acc is None and jerk is None and pot is None and type(i_idx).__module__ != "torch":
        acc, jerk, pot = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
        ret = True
    kind, p, keep = _marshal([i_idx, acc, jerk, pot], [np.int32, np.float64, np.float64, np.float64])
    _check(lib().nb_compute_forces_at(ctx, float(t), p[0], n, p[1], p[2], p[3], kind), "nb_compute_forces_at")
    if ret:
        return keep[1], keep[2], keep[3]
    return acc, jerk, pot


_STATE_KEYS = ("m", "x", "v", "a", "jerk", "pot", "t", "dt")
_STATE_SHAPE = dict(m=(), x=(3,), v=(3,), a=(3,), jerk=(3,), pot=(), t=(), dt=())


def nb_get_particles_idx(ctx, idx, out=None, keys=_STATE_KEYS):
    """Particles idx (ascending) of the state, list order: a dict of host
    arrays for `keys`, or fills `out` (arrays/tensors; missing keys skipped)."""
    n = int(idx.shape[0])
    if out is None:
        out = {k: np.empty((n,) + _STATE_SHAPE[k]) for k in keys}
    kind, p, keep = _marshal([idx] + [out.get(k) for k in _STATE_KEYS], [np.int32] + [np.float64] * 8)
    _check(lib().nb_get_particles_idx(ctx, p[0], n, *p[1:], kind), "nb_get_particles_idx")
    for k, kp in zip(_STATE_KEYS, keep[1:]):
        if k in out and isinstance(kp, np.ndarray) and kp is not out[k]:
            out[k][...] = kp
    return out


def nb_set_particles_idx(ctx, idx, values):
    """Write particles idx (ascending) from a dict of list-ordered arrays
    (keys of m, x, v, a, jerk, pot, t, dt; missing keys stay unchanged)."""
    n = int(idx.shape[0])
    kind, p, keep = _marshal([idx] + [values.get(k) for k in _STATE_KEYS], [np.int32] + [np.float64] * 8)
    _check(lib().nb_set_particles_idx(ctx, p[0], n, *p[1:], kind), "nb_set_particles_idx")
    del keep


def nb_get_predicted(ctx, idx, xp=None, vp=None):
    n = int(idx.shape[0])
    if xp is None and vp is None and type(idx).__module__ != "torch":
        xp, vp = np.empty((n, 3)), np.empty((n, 3))
    kind, p, keep = _marshal([idx, xp, vp], [np.int32, np.float64, np.float64])
    _check(lib().nb_get_predicted(ctx, p[0], n, p[1], p[2], kind), "nb_get_predicted")
    return (keep[1] if isinstance(keep[1], np.ndarray) else xp), (keep[2] if isinstance(keep[2], np.ndarray) else vp)


def nb_forces_on(ctx, xi, vi, gid=None, gid_base=0, acc=None, jerk=None, pot=None, accumulate=False):
    """Forces on particles held elsewhere (predicted xi, vi [n,3]) from this
    context's j-particles; gid (int64, nullable) excludes the self pair.
    Host inputs without outputs return new arrays."""
    n = int(xi.shape[0])
    if acc is None and jerk is None and pot is None and type(xi).__module__ != "torch":
        acc, jerk, pot = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    kind, p, keep = _marshal([xi, vi, gid, acc, jerk, pot],
                             [np.float64, np.float64, np.int64, np.float64, np.float64, np.float64])
    _check(lib().nb_forces_on(ctx, n, p[0], p[1], p[2], int(gid_base), p[3], p[4], p[5], int(bool(accumulate)),
                              kind), "nb_forces_on")
    for dst, kp in ((acc, keep[3]), (jerk, keep[4]), (pot, keep[5])):
        if isinstance(dst, np.ndarray) and isinstance(kp, np.ndarray) and kp is not dst:
            dst[...] = kp
    return acc, jerk, pot


def nb_set_forces(ctx, idx, acc, jerk, pot):
    n = int(idx.shape[0])
    kind, p, keep = _marshal([idx, acc, jerk, pot], [np.int32, np.float64, np.float64, np.float64])
    _check(lib().nb_set_forces(ctx, p[0], n, p[1], p[2], p[3], kind), "nb_set_forces")


def nb_set_initial_forces(ctx, acc, jerk, pot):
    kind, p, keep = _marshal([acc, jerk, pot], [np.float64] * 3)
    _check(lib().nb_set_initial_forces(ctx, p[0], p[1], p[2], kind), "nb_set_initial_forces")


def nb_set_jpredict(ctx, max_n):
    _check(lib().nb_set_jpredict(ctx, int(max_n)), "nb_set_jpredict")


def nb_get_jpredict(ctx):
    v = _i64()
    _check(lib().nb_get_jpredict(ctx, ctypes.byref(v)), "nb_get_jpredict")
    return v.value


def nb_correct(ctx, i_idx, t):
    n = int(i_idx.shape[0])
    kind, p, keep = _marshal([i_idx], [np.int32])
    _check(lib().nb_correct(ctx, p[0], n, float(t), kind), "nb_correct")


def nb_initial_forces_and_dt(ctx):
    _check(lib().nb_initial_forces_and_dt(ctx), "nb_initial_forces_and_dt")


def nb_step(ctx):
    t = _d()
    n = _i64()
    _check(lib().nb_step(ctx, ctypes.byref(t), ctypes.byref(n)), "nb_step")
    return t.value, n.value


def nb_integrate(ctx, t_end, use_graph=False, loop=None):
    """Block steps to t_end.  loop: NB_LOOP_HOST, NB_LOOP_GRAPH,
    NB_LOOP_PERSISTENT, NB_LOOP_CLUSTER or NB_LOOP_AUTO (the fastest for the
    context's size); without it, use_graph picks the graph or host loop."""
    if loop is None:
        loop = NB_LOOP_GRAPH if use_graph else NB_LOOP_HOST
    _check(lib().nb_integrate(ctx, float(t_end), int(loop)), "nb_integrate")


def nb_energy(ctx):
    k, w = _d(), _d()
    _check(lib().nb_energy(ctx, ctypes.byref(k), ctypes.byref(w)), "nb_energy")
    return k.value, w.value


def nb_get_timings(ctx, reset=False):
    v = [_d() for _ in range(4)]
    _check(lib().nb_get_timings(ctx, *[ctypes.byref(x) for x in v], int(bool(reset))), "nb_get_timings")
    return dict(ms_pred=v[0].value, ms_force=v[1].value, ms_corr=v[2].value, interactions=v[3].value)


def nb_get_counters(ctx):
    k, s = _i64(), _i64()
    _check(lib().nb_get_counters(ctx, ctypes.byref(k), ctypes.byref(s)), "nb_get_counters")
    return dict(kernel_launches=k.value, block_steps=s.value)


def nb_check_device_status(ctx):
    """(status code, dt underflow count) -- does not raise."""
    u = _i64()
    code = lib().nb_check_device_status(ctx, ctypes.byref(u))
    return code, u.value


def nb_check_grid_barrier(ctx, phantom=False, wait_ms=100.0):
    """Status code of the persistent loop's bounded grid-barrier wait on the
    device (NB_ETIMEOUT expected with phantom=True) -- does not raise."""
    return lib().nb_check_grid_barrier(ctx, int(bool(phantom)), float(wait_ms))


def nb_last_error(ctx):
    return lib().nb_last_error(ctx)


def nb_clear_error(ctx):
    lib().nb_clear_error(ctx)


def nb_set_tuning(ctx, i_per_thread=0, threads=0, j_tile=0, n_split=0):
    _check(lib().nb_set_tuning(ctx, int(i_per_thread), int(threads), int(j_tile), int(n_split)), "nb_set_tuning")


def nb_set_far_tiles(ctx, enable=True):
    _check(lib().nb_set_far_tiles(ctx, int(bool(enable))), "nb_set_far_tiles")


def nb_get_far_tiles(ctx):
    v = _int()
    _check(lib().nb_get_far_tiles(ctx, ctypes.byref(v)), "nb_get_far_tiles")
    return bool(v.value)


def nb_autotune(ctx, n):
    v = [_int() for _ in range(4)]
    _check(lib().nb_autotune(ctx, int(n), *[ctypes.byref(x) for x in v]), "nb_autotune")
    return dict(i_per_thread=v[0].value, threads=v[1].value, j_tile=v[2].value, n_split=v[3].value)


def nb_selftest_corrector(samples=1 << 20, seed=1, device=0):
    """Mismatches of the corrector's exponent forms against their FP64
    expressions on `samples` random operand sets (0 expected)."""
    out = _i64()
    _check(lib().nb_selftest_corrector(int(device), int(samples), int(seed), ctypes.byref(out)),
           "nb_selftest_corrector")
    return int(out.value)


def nb_autotune_list(ctx, i_idx):
    """nb_autotune timed on the active list i_idx (host or device)."""
    v = [_int() for _ in range(4)]
    n = int(i_idx.shape[0])
    kind, p, keep = _marshal([i_idx], [np.int32])
    _check(lib().nb_autotune_list(ctx, p[0], n, kind, *[ctypes.byref(x) for x in v]), "nb_autotune_list")
    return dict(i_per_thread=v[0].value, threads=v[1].value, j_tile=v[2].value, n_split=v[3].value)


def nb_ensemble_autotune(ctx, steps=16):
    """Times the device-driven item shapes on `steps` block steps of the
    context's state (restored) and keeps the fastest in its tuning table."""
    it, w = _int(), _int()
    mb, md = _d(), _d()
    _check(lib().nb_ensemble_autotune(ctx, int(steps), ctypes.byref(it), ctypes.byref(w), ctypes.byref(mb),
                                      ctypes.byref(md)), "nb_ensemble_autotune")
    return dict(i_tile=it.value, item_waves=w.value, ms_best=mb.value, ms_default=md.value)


def nb_tune_save(ctx, path):
    _check(lib().nb_tune_save(ctx, os.fsencode(path)), "nb_tune_save")


def nb_tune_load(ctx, path):
    _check(lib().nb_tune_load(ctx, os.fsencode(path)), "nb_tune_load")


def nb_tune_count(ctx):
    v = _int()
    _check(lib().nb_tune_count(ctx, ctypes.byref(v)), "nb_tune_count")
    return v.value


def nb_tune_clear(ctx):
    _check(lib().nb_tune_clear(ctx), "nb_tune_clear")


def nb_measure_peaks(ctx):
    v = [_d() for _ in range(3)]
    _check(lib().nb_measure_peaks(ctx, *[ctypes.byref(x) for x in v]), "nb_measure_peaks")
    return dict(fp32_tflops=v[0].value, fp64_tflops=v[1].value, rsqrt_tops=v[2].value)


def nb_measure_fp64_issue(ctx):
    v = [_d() for _ in range(4)]
    _check(lib().nb_measure_fp64_issue(ctx, *[ctypes.byref(x) for x in v]), "nb_measure_fp64_issue")
    return dict(dep32_cycles=v[0].value, dep1_cycles=v[1].value, indep4_cycles=v[2].value,
                sm16_cycles_per_warp_instr=v[3].value)


def nb_ensemble_create(offsets, eps, precision=NB_MIXED, device=0, stream=None):
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    h = _vp()
    s = _stream(stream)
    _check(lib().nb_ensemble_create(ctypes.byref(h), int(offsets.shape[0] - 1), offsets.ctypes.data_as(_vp),
                                    eps.ctypes.data_as(_vp), int(precision), int(device), s),
           "nb_ensemble_create")
    return h


def nb_ensemble_initial_forces_and_dt(ctx):
    _check(lib().nb_ensemble_initial_forces_and_dt(ctx), "nb_ensemble_initial_forces_and_dt")


def nb_ensemble_integrate(ctx, t_end, mode=NB_ENSEMBLE_PERSISTENT):
    _check(lib().nb_ensemble_integrate(ctx, float(t_end), int(mode)), "nb_ensemble_integrate")


def nb_ensemble_energy(ctx, n_clusters):
    """(kinetic[n_clusters], potential[n_clusters]) host arrays."""
    k = np.empty(int(n_clusters))
    w = np.empty(int(n_clusters))
    _check(lib().nb_ensemble_energy(ctx, k.ctypes.data_as(_vp), w.ctypes.data_as(_vp)), "nb_ensemble_energy")
    return k, w


def nb_forces_fp64_noalloc(m, x, v, eps, i_idx, acc=None, jerk=None, pot=None, stream=None):
    """FP64 forces from caller-owned CUDA tensors without any device
    allocation by the library (for callers that manage all device memory
    themselves).  m[N], x[N,3], v[N,3], i_idx[n] (int32) and the outputs
    acc[n,3], jerk[n,3], pot[n] must be contiguous CUDA tensors; the work is
    enqueued on ``stream`` (default: the legacy default stream)."""
    n = int(i_idx.shape[0])
    kind, p, keep = _marshal([m, x, v, i_idx, acc, jerk, pot],
                             [np.float64, np.float64, np.float64, np.int32, np.float64, np.float64, np.float64])
    if kind != NB_PTR_DEVICE:
        raise TypeError("nb_forces_fp64_noalloc takes device (CUDA) tensors only")
    s = _stream(stream)
    _check(lib().nb_forces_fp64_noalloc(int(m.shape[0]), p[0], p[1], p[2], float(eps), p[3], n, p[4], p[5],
                                        p[6], s), "nb_forces_fp64_noalloc")


class Ensemble:
    """Owning wrapper around an ensemble context (clusters stored back to back)."""

    def __init__(self, offsets, eps, precision=NB_MIXED, device=0, stream=None):
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.ctx = nb_ensemble_create(self.offsets, eps, precision, device, stream)

    @property
    def n_clusters(self):
        return len(self.offsets) - 1

    def close(self):
        if self.ctx is not None:
            nb_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def energy(self):
        return nb_ensemble_energy(self.ctx, self.n_clusters)

    def __getattr__(self, name):
        for pre in ("nb_ensemble_", "nb_"):
            f = globals().get(pre + name)
            if f is not None:
                return lambda *a, **k: f(self.ctx, *a, **k)
        raise AttributeError(name)


class NBody:
    """Owning convenience wrapper around one context (same calls, fewer args)."""

    def __init__(self, n_max, precision=NB_MIXED, device=0, stream=None):
        self.ctx = nb_create(n_max, precision, device, stream)
        # the cudaStream_t handle the context works on as torch reports it
        # (0 = torch's default stream), None for a stream of the library's own
        self.stream_handle = None if stream is None else int(getattr(stream, "cuda_stream", stream))

    def close(self):
        if self.ctx is not None:
            nb_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __getattr__(self, name):
        f = globals().get("nb_" + name)
        if f is None:
            raise AttributeError(name)
        return lambda *a, **k: f(self.ctx, *a, **k)
