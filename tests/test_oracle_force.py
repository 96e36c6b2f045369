"""Pins of the oracle's direct-sum force (Sec. 4.1 step 4, Eq. 3) against
facts that do not come from the oracle's own formulas.

* symbolic brute force: acceleration and jerk obtained by differentiating the
  softened pair potential (sympy, 40 digits) for N <= 6;
* closed forms: a two-body pair with hand-computed numbers, a symmetric
  octahedral shell, a circular orbit's jerk = -omega^2 v;
* invariants: Newton's third law for acceleration and jerk, finite-difference
  gradient of the potential, finite-difference time derivative of the
  acceleration along straight-line motion;
* the virial ratio of a Plummer sphere;
* compensated summation recovering a sum that plain summation loses.
"""
import math

import numpy as np
import pytest

from paper_0709_4552_gb300 import inputs


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ----------------------------------------------------------------- closed forms
def test_two_body_hand_values(orc):
    # j of mass 2 at (3, 4, 0) relative to i at the origin, eps = 0:
    # |r| = 5, acc = 2 (3,4,0)/125, pot = -2/5.
    m = np.array([1.0, 2.0])
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    v = np.zeros((2, 3))
    a, j, p = orc.forces(m, x, v, 0.0)
    assert np.allclose(a[0], [0.048, 0.064, 0.0], rtol=0, atol=1e-17)
    assert p[0] == pytest.approx(-0.4, rel=1e-15)
    # and i of mass 1 pulls j back with acc (−3,−4,0)/125
    assert np.allclose(a[1], [-0.024, -0.032, 0.0], rtol=0, atol=1e-17)
    assert p[1] == pytest.approx(-0.2, rel=1e-15)
    assert np.all(j == 0.0)
    # softened: eps = 5 doubles s^2 -> s = 5 sqrt(2)
    a, j, p = orc.forces(m, x, v, 5.0)
    s3 = (50.0) ** 1.5
    assert a[0] == pytest.approx([6.0 / s3, 8.0 / s3, 0.0], rel=1e-15, abs=1e-18)
    assert p[0] == pytest.approx(-2.0 / math.sqrt(50.0), rel=1e-15)


def test_octahedral_shell(orc):
    # six equal masses M/6 at distance R on the axes; the centre feels no net
    # force and sits in the potential -M / sqrt(R^2 + eps^2).
    R, M, eps = 0.75, 3.0, 0.1
    pts = [[R, 0, 0], [-R, 0, 0], [0, R, 0], [0, -R, 0], [0, 0, R], [0, 0, -R]]
    x = np.array([[0.0, 0.0, 0.0]] + pts)
    m = np.array([1.0] + [M / 6.0] * 6)
    v = np.zeros_like(x)
    v[0] = [0.3, -0.2, 0.1]
    a, j, p = orc.forces(m, x, v, eps, idx=[0])
    assert np.abs(a[0]).max() < 1e-15
    assert p[0] == pytest.approx(-M / math.sqrt(R * R + eps * eps), rel=1e-15)
    # a moving test particle at the centre of a static shell: jerk = -G M v (...)
    # is not a closed form we use; but the shell's jerk must be antiparallel to v
    # along each axis by symmetry: jerk_k = c * v_k with one c for all k.
    c = j[0] / v[0]
    assert np.allclose(c, c[0], rtol=1e-13)
    assert c[0] < 0


def test_circular_orbit_jerk(orc):
    # unit mass at rest in the origin; test particle on a circular orbit of
    # radius r: v = sqrt(1/r), omega^2 = 1/r^3; a = -omega^2 x, jerk = -omega^2 v.
    r = 0.37
    vc = math.sqrt(1.0 / r)
    m = np.array([1.0, 1e-30])
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    v = np.array([[0.0, 0.0, 0.0], [0.0, vc, 0.0]])
    a, j, p = orc.forces(m, x, v, 0.0, idx=[1])
    w2 = 1.0 / r ** 3
    assert rel(a[0], -w2 * x[1]) < 1e-15
    assert rel(j[0], -w2 * v[1]) < 1e-15
    assert p[0] == pytest.approx(-1.0 / r, rel=1e-15)


# ----------------------------------------------------------- symbolic brute force
def _symbolic_forces(m, x, v, eps, i, digits=40):
    sp = pytest.importorskip("sympy")
    t = sp.Symbol("t")
    X = sp.symbols("X0:3")
    R = sp.Rational
    e2 = R(eps) ** 2
    phi = 0
    for jj in range(len(m)):
        if jj == i:
            continue
        d2 = sum((R(x[jj, k]) + R(v[jj, k]) * t - X[k]) ** 2 for k in range(3))
        phi += -R(m[jj]) / sp.sqrt(d2 + e2)
    on_orbit = {X[k]: R(x[i, k]) + R(v[i, k]) * t for k in range(3)}
    acc_t = [(-sp.diff(phi, X[k])).subs(on_orbit) for k in range(3)]
    acc = [float(a.subs(t, 0).evalf(digits)) for a in acc_t]
    jerk = [float(sp.diff(a, t).subs(t, 0).evalf(digits)) for a in acc_t]
    pot = float(phi.subs(on_orbit).subs(t, 0).evalf(digits))
    return np.array(acc), np.array(jerk), pot


@pytest.mark.parametrize("N,eps,seed", [(2, 0.0, 3), (3, 1.0 / 256, 4), (5, 0.05, 5), (6, 0.0, 6)])
@pytest.mark.parametrize("compensated", [False, True])
def test_symbolic_brute_force(orc, N, eps, seed, compensated):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(N, 3))
    v = rng.normal(size=(N, 3))
    m = rng.uniform(0.1, 1.0, size=N)
    a, j, p = orc.forces(m, x, v, eps, compensated=compensated)
    for i in range(N):
        sa, sj, sp_ = _symbolic_forces(m, x, v, eps, i)
        assert rel(a[i], sa) < 1e-14
        assert rel(j[i], sj) < 1e-14
        assert p[i] == pytest.approx(sp_, rel=1e-14)


def test_active_subset_matches_full(orc):
    m, x, v = inputs.plummer(300, 11)
    idx = inputs.sample_indices(300, 37, 12)
    a, j, p = orc.forces(m, x, v, 0.01)
    a2, j2, p2 = orc.forces(m, x, v, 0.01, idx=idx)
    assert np.array_equal(a[idx], a2) and np.array_equal(j[idx], j2) and np.array_equal(p[idx], p2)


# ------------------------------------------------------------------- invariants
@pytest.mark.parametrize("masses", ["equal", "salpeter"])
def test_newton_third_law(orc, masses):
    m, x, v = inputs.plummer(2048, 21, masses)
    a, j, p = orc.forces(m, x, v, 1.0 / 256, compensated=True)
    F = (m[:, None] * a).sum(axis=0)
    scale = np.abs(m[:, None] * a).sum()
    assert np.abs(F).max() <= 1e-14 * scale
    G = (m[:, None] * j).sum(axis=0)
    gscale = np.abs(m[:, None] * j).sum()
    assert np.abs(G).max() <= 1e-14 * gscale


def test_jerk_is_time_derivative_of_acc(orc):
    # straight-line motion x(t) = x + v t: central difference of acc
    m, x, v = inputs.plummer(64, 31)
    eps, h = 1.0 / 64, 1e-5
    a0, j0, _ = orc.forces(m, x, v, eps, compensated=True)
    ap, _, _ = orc.forces(m, x + v * h, v, eps, compensated=True)
    am, _, _ = orc.forces(m, x - v * h, v, eps, compensated=True)
    fd = (ap - am) / (2 * h)
    assert rel(fd, j0) < 1e-7
    # per particle as well (excluding none)
    per = np.linalg.norm(fd - j0, axis=1) / np.linalg.norm(j0, axis=1)
    assert np.median(per) < 1e-7


def test_potential_gradient_is_acc(orc):
    m, x, v = inputs.plummer(48, 41)
    eps, h = 1.0 / 32, 1e-5
    a0, _, _ = orc.forces(m, x, v, eps, compensated=True)
    for i in (0, 7, 23, 47):
        g = np.zeros(3)
        for k in range(3):
            xp_, xm_ = x.copy(), x.copy()
            xp_[i, k] += h
            xm_[i, k] -= h
            _, _, pp = orc.forces(m, xp_, v, eps, idx=[i], compensated=True)
            _, _, pm = orc.forces(m, xm_, v, eps, idx=[i], compensated=True)
            g[k] = -(pp[0] - pm[0]) / (2 * h)
        assert rel(g, a0[i]) < 1e-7


def test_plummer_virial_ratio(orc):
    # analytic virial scaling: W -> -1/2, K -> 1/4 (N^-1/2 sampling noise)
    m, x, v = inputs.plummer(16384, 51)
    ek, ep = orc.energy(m, x, v, 0.0)
    assert ep == pytest.approx(-0.5, abs=0.03)
    assert ek == pytest.approx(0.25, abs=0.02)
    assert ek + ep == pytest.approx(-0.25, abs=0.03)


def test_energy_matches_pairwise_sum(orc):
    # W = sum over unordered pairs of -m_i m_j / s_ij (brute force, small N)
    m, x, v = inputs.plummer(40, 61, "salpeter")
    eps = 0.02
    W = 0.0
    for i in range(40):
        for j in range(i + 1, 40):
            W -= m[i] * m[j] / math.sqrt(((x[i] - x[j]) ** 2).sum() + eps * eps)
    K = 0.5 * float((m * (v * v).sum(axis=1)).sum())
    ek, ep = orc.energy(m, x, v, eps)
    assert ep == pytest.approx(W, rel=1e-14)
    assert ek == pytest.approx(K, rel=1e-14)


def test_compensated_sum_recovers_lost_term(orc):
    # i at the origin; j0 (m=1e16) at +x, j1 (m=4) at 2x, j2 (m=1e16) at -x.
    # acc_x terms in j order: +1e16, +1, -1e16.  Plain FP64 loses the 1.
    m = np.array([1.0, 1e16, 4.0, 1e16])
    x = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0], [-1.0, 0, 0]])
    v = np.zeros((4, 3))
    a_plain, _, _ = orc.forces(m, x, v, 0.0, idx=[0])
    a_comp, _, _ = orc.forces(m, x, v, 0.0, idx=[0], compensated=True)
    assert a_plain[0, 0] == 0.0
    assert a_comp[0, 0] == 1.0


def test_plain_and_compensated_agree_on_plummer(orc):
    m, x, v = inputs.plummer(4096, 71, "salpeter")
    a, j, p = orc.forces(m, x, v, 1.0 / 1024)
    ac, jc, pc = orc.forces(m, x, v, 1.0 / 1024, compensated=True)
    assert np.median(np.linalg.norm(a - ac, axis=1) / np.linalg.norm(ac, axis=1)) < 1e-14
    assert np.max(np.abs(p - pc) / np.abs(pc)) < 1e-13
