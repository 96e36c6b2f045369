"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/nbody.h declares; the host-only calls answer without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nbody.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_0709_4552_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("nb_create", "nb_set_j_particles", "nb_predict", "nb_compute_forces", "nb_correct",
                 "nb_next_block", "nb_integrate", "nb_ensemble_integrate"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared in nbody.h but not exported"


def test_binding_covers_every_symbol():
    from paper_0709_4552_gb300 import nbody
    assert sorted(nbody.EXPORTS) == _declared()


def test_binding_constants_match_header():
    from paper_0709_4552_gb300 import nbody
    src = open(os.path.join(ROOT, "include", "nbody.h")).read()
    defs = dict(re.findall(r"#define\s+(NB_[A-Z0-9_]+)\s+(-?\d+)\b", src))
    names = [n for n in defs if hasattr(nbody, n)]
    for must in ("NB_OK", "NB_ETIMEOUT", "NB_FP64", "NB_MIXED", "NB_LOOP_HOST", "NB_LOOP_GRAPH",
                 "NB_LOOP_PERSISTENT", "NB_PERSISTENT_MAX_N", "NB_PERSISTENT_MAX_N_FP64",
                 "NB_ENSEMBLE_PER_CLUSTER"):
        assert must in names
    for n in names:
        assert getattr(nbody, n) == int(defs[n]), n


def test_host_only_calls(lib):
    from paper_0709_4552_gb300 import nbody as nb
    assert nb.nb_version().startswith("libnbody")
    assert nb.nb_strerror(nb.NB_EINVAL) == "invalid argument"
    eps, eta, dmin, dmax = nb.nb_default_params()
    assert (eps, dmin, dmax) == (2.0 ** -8, 2.0 ** -22, 2.0 ** -3)   # Sec. 2 values
    assert eta == 0.01


def test_null_arguments_rejected(lib):
    from paper_0709_4552_gb300 import nbody as nb
    L = nb.lib()
    assert L.nb_create(None, 10, 0, 0, None) == nb.NB_EINVAL
    assert L.nb_set_params(None, 0.1, 0.01, 2.0 ** -22, 0.125) == nb.NB_EINVAL
    assert L.nb_step(None, None, None) == nb.NB_EINVAL
    for loop in (nb.NB_LOOP_HOST, nb.NB_LOOP_GRAPH, nb.NB_LOOP_PERSISTENT):
        assert L.nb_integrate(None, 0.125, loop) == nb.NB_EINVAL
    assert L.nb_check_grid_barrier(None, 1, 50.0) == nb.NB_EINVAL
    h = ctypes.c_void_p()
    assert L.nb_create(ctypes.byref(h), 0, 0, 0, None) == nb.NB_EINVAL       # n_max < 1
    assert L.nb_create(ctypes.byref(h), 10, 7, 0, None) == nb.NB_EINVAL      # bad precision
    assert not h.value


def test_sources_target_sm103a_only():
    from paper_0709_4552_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
