"""Pins of the oracle's integrator (Sec. 4.1 steps 2-6, block steps of Sec. 2)
against closed forms and invariants that do not come from its own formulas.

* predictor: hand-computed cubic;
* corrector: exact for a quintic trajectory (a cubic acceleration), and
  algebraically equal to the Hut-Makino form of the same Hermite scheme;
* time-step criterion: sqrt(eta)/omega on a circular orbit;
* block rule: hand cases (shrink, grow only when commensurate, clamps);
* Kepler two-body orbit against Kepler's equation, 4th-order convergence;
* momentum conservation with shared steps, Plummer energy drift, block-step
  invariants (powers of two, t_i a multiple of dt_i).
"""
import math

import numpy as np
import pytest

from paper_0709_4552_gb300 import inputs


def test_predictor_hand_cubic(orc):
    # x0=1, v0=2, a0=3, j0=6, h=0.5: xp = 1+1+0.375+0.125 = 2.5, vp = 2+1.5+0.75 = 4.25
    x = np.array([[1.0, 0.0, -1.0]])
    v = np.array([[2.0, 0.0, 0.0]])
    a = np.array([[3.0, 0.0, 0.0]])
    j = np.array([[6.0, 0.0, 0.0]])
    xp, vp = orc.predict(x, v, a, j, np.array([0.25]), 0.75)
    assert xp[0].tolist() == [2.5, 0.0, -1.0]
    assert vp[0].tolist() == [4.25, 0.0, 0.0]


def _quintic(seed):
    rng = np.random.default_rng(seed)
    c = rng.normal(size=(3, 6))          # x_k(t) = sum_p c[k,p] t^p
    P = [np.polynomial.Polynomial(c[k]) for k in range(3)]
    return P


@pytest.mark.parametrize("h", [0.5, 2.0 ** -6, 2.0 ** -12])
def test_corrector_exact_for_quintic(orc, h):
    P = _quintic(5)

    def ev(d, t):
        return np.array([[P[k].deriv(d)(t) if d else P[k](t) for k in range(3)]])

    x0, v0, a0, j0 = ev(0, 0.0), ev(1, 0.0), ev(2, 0.0), ev(3, 0.0)
    xp, vp = orc.predict(x0, v0, a0, j0, np.array([0.0]), h)
    a1, j1 = ev(2, h), ev(3, h)
    x1, v1, a2e, a3 = orc.correct(x0, v0, a0, j0, xp, vp, a1, j1, [h])
    sc = np.abs(ev(0, h)).max() + 1
    assert np.abs(x1 - ev(0, h)).max() < 1e-13 * sc
    assert np.abs(v1 - ev(1, h)).max() < 1e-12 * (np.abs(ev(1, h)).max() + 1)
    # 2nd derivative of a at the end and the (constant) 3rd derivative
    assert np.abs(a2e - ev(4, h)).max() < 1e-9 * (np.abs(ev(4, h)).max() + 1) / min(1.0, h)
    assert np.abs(a3 - ev(5, 0.0)).max() < 1e-8 * (np.abs(ev(5, 0.0)).max() + 1) / min(1.0, h) ** 2


def test_corrector_equals_hut_makino_form(orc):
    # v1 = v0 + (a0+a1) h/2 + (j0-j1) h^2/12 ; x1 = x0 + (v0+v1) h/2 + (a0-a1) h^2/12
    rng = np.random.default_rng(9)
    n = 200
    x0, v0, a0, j0, a1, j1 = (rng.normal(size=(n, 3)) for _ in range(6))
    h = 2.0 ** -rng.integers(3, 12, size=n).astype(float)
    xp, vp = orc.predict(x0, v0, a0, j0, np.zeros(n), 0.0)  # h = 0: xp = x0
    # predictor to each particle's own h
    xp = x0 + v0 * h[:, None] + a0 * (h ** 2 / 2)[:, None] + j0 * (h ** 3 / 6)[:, None]
    vp = v0 + a0 * h[:, None] + j0 * (h ** 2 / 2)[:, None]
    x1, v1, _, a3 = orc.correct(x0, v0, a0, j0, xp, vp, a1, j1, h)
    H = h[:, None]
    v1_hm = v0 + (a0 + a1) * H / 2 + (j0 - j1) * H ** 2 / 12
    x1_hm = x0 + (v0 + v1_hm) * H / 2 + (a0 - a1) * H ** 2 / 12
    # velocities: the two forms are the same polynomial in h
    assert np.abs(v1 - v1_hm).max() < 1e-14 * (np.abs(v1).max() + 1)
    # positions: they differ by exactly the 5th-order term a3 h^5 / 720
    # (h^2/120 (2 (a0-a1) + h (j0+j1)) written out by hand)
    d = H ** 2 / 120 * (2 * (a0 - a1) + H * (j0 + j1))
    assert np.abs((x1 - x1_hm) - d).max() < 1e-14 * (np.abs(x1).max() + 1)
    assert np.abs(d - a3 * H ** 5 / 720).max() < 1e-14 * (np.abs(d).max() + 1e-300)


@pytest.mark.parametrize("r,eta", [(1.0, 0.01), (0.2, 0.02), (3.0, 0.005)])
def test_aarseth_circular_orbit(orc, r, eta):
    # x = r (cos wt, sin wt, 0): a = -w^2 x, j = -w^2 v, a2 = w^4 x, a3 = w^4 v
    w = math.sqrt(1.0 / r ** 3)
    th = 0.3
    x = r * np.array([math.cos(th), math.sin(th), 0.0])
    v = r * w * np.array([-math.sin(th), math.cos(th), 0.0])
    dt = orc.aarseth_dt(-w * w * x, -w * w * v, w ** 4 * x, w ** 4 * v, eta)
    assert dt == pytest.approx(math.sqrt(eta) / w, rel=1e-14)


def test_pow2_floor(orc):
    assert orc.pow2_floor(1.0) == 1.0
    assert orc.pow2_floor(0.75) == 0.5
    assert orc.pow2_floor(2.0 ** -22 * 1.5) == 2.0 ** -22
    assert orc.pow2_floor(3.0) == 2.0
    assert orc.pow2_floor(1e-300) == 2.0 ** math.floor(math.log2(1e-300))


@pytest.mark.parametrize("crit,old,t,expect,uf", [
    (2.0 ** -9 * 1.3, 2.0 ** -5, 0.5, 2.0 ** -9, 0),      # shrink freely
    (1.0, 2.0 ** -5, 2.0 ** -4, 2.0 ** -4, 0),            # grow x2: t multiple of 2 dt_old
    (1.0, 2.0 ** -5, 3 * 2.0 ** -5, 2.0 ** -5, 0),        # not commensurate: keep
    (1.9 * 2.0 ** -5, 2.0 ** -5, 2.0 ** -4, 2.0 ** -5, 0),  # crit < 2 dt_old: keep
    (1.0, 2.0 ** -3, 1.0, 2.0 ** -3, 0),                  # capped at dt_max
    (1e-12, 2.0 ** -10, 0.5, 2.0 ** -22, 1),              # underflow: clamp + flag
])
def test_block_rule(orc, crit, old, t, expect, uf):
    got, flag = orc.block_dt(crit, old, t, 2.0 ** -22, 2.0 ** -3)
    assert got == expect and flag == uf


def test_initial_dt(orc):
    # eta |a|/|j| = 0.01 * 2 / 0.001 = 20 -> capped at 1/8 ; 0.01*1/64 -> 2^-13 floor
    assert orc.initial_dt([2, 0, 0], [0.001, 0, 0], 0.01, 2.0 ** -22, 0.125) == 0.125
    assert orc.initial_dt([1, 0, 0], [0, 64, 0], 0.01, 2.0 ** -22, 0.125) == 2.0 ** -13


# ------------------------------------------------------------------ Kepler
def _kepler_pair(e=0.5, m1=0.5, m2=0.5):
    # pericentre on the x axis, semi-major axis 1, G M = 1 -> period 2 pi
    M = m1 + m2
    rp = 1.0 - e
    vp = math.sqrt(M * (1 + e) / rp)
    m = np.array([m1, m2])
    x = np.array([[-m2 / M * rp, 0, 0], [m1 / M * rp, 0, 0]])
    v = np.array([[0, -m2 / M * vp, 0], [0, m1 / M * vp, 0]])
    return m, x, v


def _kepler_sep(t, e=0.5):
    # Kepler's equation E - e sin E = t (mean motion 1), Newton iteration
    Mq = math.fmod(t, 2 * math.pi)
    E = Mq if e < 0.8 else math.pi
    for _ in range(60):
        E -= (E - e * math.sin(E) - Mq) / (1 - e * math.cos(E))
    return np.array([math.cos(E) - e, math.sqrt(1 - e * e) * math.sin(E), 0.0])


def _run_kepler(orc, dt, t_end, eta=0.01, dt_min=None):
    m, x, v = _kepler_pair()
    dtmin = dt if dt_min is None else dt_min
    r = orc.hermite_run(m, x, v, 0.0, eta, dtmin, dt, t_end)
    sep = r["x"][1] - r["x"][0]
    return sep, r


def test_kepler_closed_form(orc):
    t_end = 64.0                      # ~10.2 orbits
    sep, r = _run_kepler(orc, 2.0 ** -9, t_end)
    ref = _kepler_sep(t_end)
    assert np.linalg.norm(sep - ref) < 1e-6
    assert np.all(r["t"] == t_end)


def test_kepler_block_steps(orc):
    # individual (block) steps with the Aarseth criterion still follow Kepler
    sep, r = _run_kepler(orc, 2.0 ** -3, 64.0, eta=0.0025, dt_min=2.0 ** -22)
    ref = _kepler_sep(64.0)
    assert np.linalg.norm(sep - ref) < 1e-4
    assert r["block_steps"] > 64 * 8  # steps shrank below dt_max near pericentre


def test_fourth_order_convergence(orc):
    t_end = 8.0
    ref = _kepler_sep(t_end)
    e1 = np.linalg.norm(_run_kepler(orc, 2.0 ** -5, t_end)[0] - ref)
    e2 = np.linalg.norm(_run_kepler(orc, 2.0 ** -6, t_end)[0] - ref)
    e3 = np.linalg.norm(_run_kepler(orc, 2.0 ** -7, t_end)[0] - ref)
    assert 12.0 < e1 / e2 < 20.0
    assert 12.0 < e2 / e3 < 20.0


# ------------------------------------------------------------- N-body runs
def test_shared_step_momentum_conservation(orc):
    m, x, v = inputs.plummer(256, 81)
    r = orc.hermite_run(m, x, v, 1.0 / 256, 0.01, 2.0 ** -10, 2.0 ** -10, 2.0 ** -5, compensated=True)
    assert r["block_steps"] == 32
    P = (m[:, None] * r["v"]).sum(axis=0)
    assert np.abs(P).max() < 1e-14
    assert np.all(r["t"] == 2.0 ** -5)


def _invariants(r, t_end, dt_min, dt_max):
    dt, t = r["dt"], r["t"]
    k = np.log2(dt)
    assert np.all(k == np.round(k))
    assert np.all((dt >= dt_min) & (dt <= dt_max))
    assert np.all(np.fmod(t, dt) == 0.0)
    assert np.all(t == t_end)


@pytest.mark.slow
def test_plummer_energy_drift_one_time_unit(orc):
    # one N-body time unit, block steps 2^-22..2^-3, eps = 2^-8 (Sec. 2)
    N, eps = 256, 2.0 ** -8
    m, x, v = inputs.plummer(N, 91)
    ek0, ep0 = orc.energy(m, x, v, eps)
    E0 = ek0 + ep0
    r = orc.hermite_run(m, x, v, eps, 0.01, 2.0 ** -22, 2.0 ** -3, 1.0)
    _invariants(r, 1.0, 2.0 ** -22, 2.0 ** -3)
    ek1, ep1 = orc.energy(m, r["x"], r["v"], eps)
    dE = abs((ek1 + ep1 - E0) / E0)
    assert dE < 1e-6
    # smaller eta -> smaller error (4th order in dt ~ sqrt(eta))
    r2 = orc.hermite_run(m, x, v, eps, 0.0025, 2.0 ** -22, 2.0 ** -3, 1.0)
    ek2, ep2 = orc.energy(m, r2["x"], r2["v"], eps)
    dE2 = abs((ek2 + ep2 - E0) / E0)
    assert dE2 < dE
    assert r2["particle_steps"] > 1.5 * r["particle_steps"]


def test_block_schedule_invariants_short(orc):
    m, x, v = inputs.plummer(128, 92, "salpeter")
    r = orc.hermite_run(m, x, v, 1.0 / 128, 0.01, 2.0 ** -22, 2.0 ** -6, 2.0 ** -6)
    _invariants(r, 2.0 ** -6, 2.0 ** -22, 2.0 ** -6)
    # continuing a run from its state equals running straight through
    a = orc.hermite_run(m, x, v, 1.0 / 128, 0.01, 2.0 ** -22, 2.0 ** -6, 2.0 ** -5)
    b = orc.hermite_run(m, r["x"], r["v"], 1.0 / 128, 0.01, 2.0 ** -22, 2.0 ** -6, 2.0 ** -5, state=r)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["dt"], b["dt"])


def test_bad_arguments(orc):
    m, x, v = inputs.plummer(8, 1)
    with pytest.raises(ValueError):
        orc.hermite_run(m, x, v, 0.01, 0.01, 2.0 ** -22, 2.0 ** -3, 1.0 / 16)
