"""Device-driven block steps: the CUDA-graph integration loop of one system
(nb_integrate with use_graph) and the batched ensemble of independent
clusters (nb_ensemble_*), against the host-driven path and the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_0709_4552_gb300 import inputs
from _util import rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


def _single(nb, prec, m, x, v, eps, dt_min, dt_max):
    s = nb.NBody(len(m), prec, 0)
    s.set_params(eps, 0.01, dt_min, dt_max)
    s.set_j_particles(0, m, x, v)
    s.initial_forces_and_dt()
    return s


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_loop_matches_host_loop(nbl, prec):
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    N, eps, t_end = 1500, 1 / 256, 2.0 ** -5
    m, x, v = inputs.plummer(N, 401, "salpeter")
    with _single(nbl, P, m, x, v, eps, 2.0 ** -22, t_end) as s:
        s.integrate(t_end, use_graph=False)
        a = s.get_particles(0, N)
        ca = s.get_counters()
    with _single(nbl, P, m, x, v, eps, 2.0 ** -22, t_end) as s:
        s.integrate(t_end, use_graph=True)
        b = s.get_particles(0, N)
        cb = s.get_counters()
    assert np.all(a["t"] == t_end) and np.all(b["t"] == t_end)
    if P == nbl.NB_FP64:
        assert cb["block_steps"] == ca["block_steps"]
        assert np.array_equal(a["dt"], b["dt"])
        assert np.abs(a["x"] - b["x"]).max() < 1e-12
        assert np.abs(a["v"] - b["v"]).max() < 1e-11
    else:
        # the two mixed runs sum in different orders (the host loop uses the
        # spatial j-order), so a criterion near a power of two can pick a
        # different step for a few particles: same physics, not the same bits
        assert abs(cb["block_steps"] - ca["block_steps"]) <= 0.05 * ca["block_steps"]
        assert np.mean(a["dt"] == b["dt"]) > 0.95
        assert np.abs(a["x"] - b["x"]).max() < 1e-5


def _ensemble_ics(sizes, seed):
    ms, xs, vs, eps = [], [], [], []
    for q, n in enumerate(sizes):
        m, x, v = inputs.plummer(int(n), seed + q, "salpeter")
        ms.append(m)
        xs.append(x)
        vs.append(v)
        eps.append(1.0 / (4.0 * n ** (1.0 / 3.0)))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return off, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), np.array(eps)


def _ens(nb, prec, off, m, x, v, eps, t_end):
    e = nb.Ensemble(off, eps, prec, 0)
    e.set_params(0.01, 0.01, 2.0 ** -22, t_end)   # eps per cluster comes from nb_ensemble_create
    e.set_j_particles(0, m, x, v)
    e.initial_forces_and_dt()
    return e


@pytest.mark.parametrize("prec,far", [("fp64", True), ("mixed", True), ("mixed", False)])
def test_ensemble_initial_forces_are_per_cluster(nbl, prec, far):
    # the mixed ensemble keeps each cluster in spatial order on its own rows;
    # particle indices at the ABI are unchanged.  far=False: double-single
    # differences on every tile (nb_set_far_tiles)
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    tol = 1e-12 if prec == "fp64" else 1e-5
    sizes = [100, 37, 512, 256, 1, 3000, 129]
    off, m, x, v, eps = _ensemble_ics(sizes, 500)
    e = nbl.Ensemble(off, eps, P, 0)
    e.set_far_tiles(far)
    e.set_params(0.01, 0.01, 2.0 ** -22, 2.0 ** -6)
    e.set_j_particles(0, m, x, v)
    e.initial_forces_and_dt()
    with e:
        st = e.get_particles(0, int(off[-1]))
    assert np.array_equal(st["x"], x) and np.array_equal(st["m"], m)
    for q in range(len(sizes)):
        a, b = off[q], off[q + 1]
        ar, jr, pr = oracle.forces(m[a:b], x[a:b], v[a:b], eps[q], compensated=True)
        if b - a > 1:
            errs = (rel_vec(st["a"][a:b], ar), rel_vec(st["jerk"][a:b], jr), rel_scalar(st["pot"][a:b], pr))
            for e_ in errs:
                assert e_.max() <= tol
                if P == nbl.NB_MIXED:
                    assert np.median(e_) <= 1e-6
        else:
            assert np.all(st["a"][a:b] == 0.0) and np.all(st["pot"][a:b] == 0.0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_persistent_matches_per_cluster(nbl, prec):
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    sizes = inputs.ensemble_sizes(12, 64, 1024, seed=7)
    off, m, x, v, eps = _ensemble_ics(sizes, 600)
    t_end = 2.0 ** -6
    N = int(off[-1])
    with _ens(nbl, P, off, m, x, v, eps, t_end) as e:
        e.integrate(t_end, nbl.NB_ENSEMBLE_PERSISTENT)
        a = e.get_particles(0, N)
    with _ens(nbl, P, off, m, x, v, eps, t_end) as e:
        e.integrate(t_end, nbl.NB_ENSEMBLE_PER_CLUSTER)
        b = e.get_particles(0, N)
    assert np.all(a["t"] == t_end) and np.all(b["t"] == t_end)
    if P == nbl.NB_FP64:
        assert np.array_equal(a["dt"], b["dt"])
        assert np.abs(a["x"] - b["x"]).max() < 1e-12
    else:
        assert np.abs(a["x"] - b["x"]).max() < 1e-6


def test_ensemble_matches_oracle(nbl):
    # every cluster integrated independently by the oracle (FP64, block steps)
    sizes = [300, 90, 700, 128]
    off, m, x, v, eps = _ensemble_ics(sizes, 700)
    t_end = 2.0 ** -5
    N = int(off[-1])
    with _ens(nbl, nbl.NB_FP64, off, m, x, v, eps, t_end) as e:
        e.integrate(t_end)
        st = e.get_particles(0, N)
        ek, ep = e.energy()
    for q in range(len(sizes)):
        a, b = off[q], off[q + 1]
        r = oracle.hermite_run(m[a:b], x[a:b], v[a:b], eps[q], 0.01, 2.0 ** -22, t_end, t_end, compensated=True)
        assert np.array_equal(st["dt"][a:b], r["dt"])
        assert np.abs(st["x"][a:b] - r["x"]).max() < 1e-11
        k0, w0 = oracle.energy(m[a:b], st["x"][a:b], st["v"][a:b], eps[q])
        assert abs(ek[q] - k0) < 1e-13 * abs(k0) and abs(ep[q] - w0) < 1e-12 * abs(w0)


def test_ensemble_energy_drift_within_oracle(nbl):
    # batched mixed-precision ensemble: per-cluster energy drift vs the oracle's own
    sizes = [400, 200]
    off, m, x, v, eps = _ensemble_ics(sizes, 800)
    t_end = 2.0 ** -4
    N = int(off[-1])
    with _ens(nbl, nbl.NB_MIXED, off, m, x, v, eps, t_end) as e:
        e.integrate(t_end)
        st = e.get_particles(0, N)
    for q in range(len(sizes)):
        a, b = off[q], off[q + 1]
        E0 = sum(oracle.energy(m[a:b], x[a:b], v[a:b], eps[q]))
        r = oracle.hermite_run(m[a:b], x[a:b], v[a:b], eps[q], 0.01, 2.0 ** -22, t_end, t_end)
        d_orc = abs(sum(oracle.energy(m[a:b], r["x"], r["v"], eps[q])) - E0) / abs(E0)
        d_gpu = abs(sum(oracle.energy(m[a:b], st["x"][a:b], st["v"][a:b], eps[q])) - E0) / abs(E0)
        print(f"cluster {q}: |dE/E| gpu {d_gpu:.3e} oracle {d_orc:.3e}")
        assert d_gpu <= 2 * d_orc + 1e-9


def test_ensemble_rejects_single_system_calls(nbl):
    off, m, x, v, eps = _ensemble_ics([50, 60], 900)
    with _ens(nbl, nbl.NB_MIXED, off, m, x, v, eps, 2.0 ** -6) as e:
        with pytest.raises(nbl.NBodyError) as err:
            e.step()
        assert err.value.code == nbl.NB_ESTATE
        with pytest.raises(nbl.NBodyError):
            e.integrate(2.0 ** -6 * 1.5)   # not a multiple of dt_max
