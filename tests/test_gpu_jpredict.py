"""On-the-fly prediction of the j-particles inside the force kernel, GRAPE's
split of a block step (Sec. 4.4 steps 3-5: the host predicts the n active
particles, the board predicts every j-particle as it loads it):
nb_compute_forces_at and the host loop's small blocks (nb_set_jpredict),
against the FP64 oracle predicting all N first (Sec. 4.1 steps 3-4)."""
import numpy as np
import pytest

import oracle
from paper_0709_4552_gb300 import inputs
from _util import rel_scalar, rel_vec

pytestmark = pytest.mark.gpu

MIX_MED, MIX_MAX = 1e-6, 1e-5


def _block_state(nb, N, seed, eps, T):
    """A state of the block-step schedule at block time T: the initial
    forces and steps of a Plummer sphere, each particle's time the last
    multiple of its step before T (t_i < T <= t_i + dt_i), so the particles
    are predicted over h = T - t_i up to a whole step."""
    m, x, v = inputs.plummer(N, seed)
    with nb.NBody(N, nb.NB_MIXED, 0) as s:   # (the mixed forces: quick at N = 2^20)
        s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
        s.set_j_particles(0, m, x, v)
        s.initial_forces_and_dt()
        st = s.get_particles(0, N)
    ti = (np.ceil(T / st["dt"]) - 1.0) * st["dt"]
    assert np.all(ti < T) and np.all(T <= ti + st["dt"])
    return m, x, v, st["a"], st["jerk"], ti, st["dt"]


def _ctx(nb, prec, state, eps):
    m, x, v, a, j, ti, dt = state
    s = nb.NBody(len(m), prec, 0)
    s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
    s.set_j_particles(0, m, x, v, a, j, ti, dt)
    return s


def _oracle_at(state, eps, T, idx):
    m, x, v, a, j, ti, dt = state
    xp, vp = oracle.predict(x, v, a, j, ti, T)
    return oracle.forces(m, xp, vp, eps, idx=np.asarray(idx, dtype=np.int64), compensated=True)


def _check(got, ref):
    errs = (rel_vec(got[0], ref[0]), rel_vec(got[1], ref[1]), rel_scalar(got[2], ref[2]))
    for name, e in zip(("acc", "jerk", "pot"), errs):
        assert np.median(e) <= MIX_MED, (name, np.median(e))
        assert e.max() <= MIX_MAX, (name, e.max())
    return errs


@pytest.mark.parametrize("N,n", [((1 << 17) + 77, 1), ((1 << 17) + 77, 31), ((1 << 17) + 77, 256),
                                 ((1 << 17) + 77, 4096), (1 << 20, 256)])
def test_forces_at_matches_oracle(nbl, N, n):
    eps, T = 1.0 / 4096, 2.0 ** -4
    state = _block_state(nbl, N, 3, eps, T)
    idx = inputs.sample_indices(N, n, 1003 + n).astype(np.int32)
    ref = _oracle_at(state, eps, T, idx)
    with _ctx(nbl, nbl.NB_MIXED, state, eps) as s:
        got = s.compute_forces_at(T, idx)
        # the separate FP64 predictor of all N, then the same forces
        s.predict(T)
        sep = s.compute_forces(idx)
    e = _check(got, ref)
    _check(sep, ref)
    print(f"N={N} n={n}: on-the-fly acc {np.median(e[0]):.2e}/{e[0].max():.2e} "
          f"jerk {np.median(e[1]):.2e}/{e[1].max():.2e} pot {e[2].max():.2e}")


def test_forces_at_strict_and_fp64(nbl):
    # without the far-tile pass, and on the FP64 path (which predicts all N)
    N, eps, T = 20000, 1.0 / 1024, 2.0 ** -5
    state = _block_state(nbl, N, 5, eps, T)
    idx = inputs.sample_indices(N, 700, 6).astype(np.int32)
    ref = _oracle_at(state, eps, T, idx)
    with _ctx(nbl, nbl.NB_MIXED, state, eps) as s:
        s.set_far_tiles(False)
        _check(s.compute_forces_at(T, idx), ref)
    with _ctx(nbl, nbl.NB_FP64, state, eps) as s:
        a, j, p = s.compute_forces_at(T, idx)
    assert rel_vec(a, ref[0]).max() <= 1e-12 and rel_vec(j, ref[1]).max() <= 1e-12
    assert rel_scalar(p, ref[2]).max() <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_correct_after_forces_at(nbl, prec):
    # nb_next_block -> nb_compute_forces_at(t, block) -> nb_correct(block, t)
    # takes the same block step as nb_step (FP64: bit for bit, its forces
    # use the full prediction; mixed: within the mixed bounds)
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    N, eps = 3000, 1.0 / 256
    m, x, v = inputs.plummer(N, 41, "salpeter")
    runs = []
    for api in (False, True):
        with nbl.NBody(N, P, 0) as s:
            s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
            s.set_j_particles(0, m, x, v)
            s.initial_forces_and_dt()
            for _ in range(30):
                if api:
                    t, n, idx = s.next_block()
                    s.compute_forces_at(t, idx)
                    s.correct(idx, t)
                else:
                    s.step()
            runs.append(s.get_particles(0, N))
    a, b = runs
    assert np.array_equal(a["t"], b["t"])
    if P == nbl.NB_FP64:
        for k in ("x", "v", "a", "jerk", "dt"):
            assert np.array_equal(a[k], b[k]), k
    else:
        assert np.mean(a["dt"] == b["dt"]) > 0.99
        assert np.abs(a["x"] - b["x"]).max() < 1e-9


def test_host_loop_small_blocks_on_the_fly(nbl):
    # every block of the host loop through the on-the-fly path (max_n = N):
    # the same schedule and energy drift as predicting all N each step
    N, eps, t_end = 6000, 1 / 256, 2.0 ** -5
    m, x, v = inputs.plummer(N, 700 + N, "salpeter")
    out = {}
    for mode in (0, N):
        with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
            s.set_params(eps, 0.01, 2.0 ** -22, t_end)
            s.set_j_particles(0, m, x, v)
            s.initial_forces_and_dt()
            s.set_jpredict(mode)
            assert s.get_jpredict() == mode
            k0, w0 = s.energy()
            c0 = s.get_counters()
            s.integrate(t_end)
            c1 = s.get_counters()
            k1, w1 = s.energy()
            out[mode] = (s.get_particles(0, N), c1["block_steps"] - c0["block_steps"],
                         abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0))
    (a, ca, da), (b, cb, db) = out[0], out[N]
    assert np.all(a["t"] == t_end) and np.all(b["t"] == t_end)
    assert abs(cb - ca) <= 0.05 * ca
    assert np.mean(a["dt"] == b["dt"]) > 0.95
    assert np.abs(a["x"] - b["x"]).max() < 1e-5
    assert db <= 2 * da + 1e-9, (da, db)


def test_jpredict_rejects_bad_arguments(nbl):
    with nbl.NBody(100, nbl.NB_MIXED, 0) as s:
        with pytest.raises(nbl.NBodyError):
            s.set_jpredict(-2)
        s.set_jpredict(nbl.NB_JPREDICT_AUTO)
        assert s.get_jpredict() > 0
