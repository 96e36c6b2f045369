"""The oracle's pins must catch plausible mistakes.

Each case below plants one mistake (a dropped term, a wrong sign, index or
coefficient, a transposed operand) in a COPY of the oracle's C source, builds
it on the CPU, and runs a quick battery of the pins used in
test_oracle_force.py / test_oracle_hermite.py.  The unmodified source passes
every check; every mutant must fail at least one.
"""
import math
import os

import numpy as np
import pytest

from paper_0709_4552_gb300 import inputs

MUTANTS = {
    "jerk_drop_factor_3": ("3.0 * rw / s2", "rw / s2"),
    "jerk_sign": ("(w0 - c_jrk * r0)", "(w0 + c_jrk * r0)"),
    "acc_uses_m_i": ("const double mj = m[j];", "const double mj = m[self];"),
    "r_sign_x": ("x[3 * j + 0] - xi[0]", "xi[0] - x[3 * j + 0]"),
    "drop_softening": ("r2 * r2 + eps2;", "r2 * r2;"),
    "pot_sign": ("-mj * inv_s", "mj * inv_s"),
    "wrong_power": ("inv_s / s2;", "inv_s / s;"),
    "no_self_exclusion": ("if (j == self) continue;", ""),
    "dv_uses_x": ("v[3 * j + 1] - vi[1]", "v[3 * j + 1] - xi[1]"),
    "pred_x_half": ("a[q] * (h * h / 2.0)", "a[q] * (h * h)"),
    "pred_jerk_coeff": ("jk[q] * (h * h * h / 6.0)", "jk[q] * (h * h * h / 2.0)"),
    "pred_v_missing_jerk": ("vp[q] = v[q] + a[q] * h + jk[q] * (h * h / 2.0);", "vp[q] = v[q] + a[q] * h;"),
    "corr_a2_transposed": ("h * (4.0 * j0[q] + 2.0 * j1[q])", "h * (2.0 * j0[q] + 4.0 * j1[q])"),
    "corr_a3_coeff": ("(12.0 * da + 6.0", "(6.0 * da + 6.0"),
    "corr_x_coeff": ("a3 * h5 / 120.0", "a3 * h5 / 24.0"),
    "corr_v_drop_a3": ("v1[q] = vp[q] + a2 * h3 / 6.0 + a3 * h4 / 24.0;", "v1[q] = vp[q] + a2 * h3 / 6.0;"),
    "corr_a2_end_sign": ("a2_end[q] = a2 + a3 * h;", "a2_end[q] = a2 - a3 * h;"),
    "aarseth_swapped": ("na * n2 + nj * nj", "na * n3 + nj * nj"),
    "aarseth_no_sqrt": ("return sqrt(eta * num / den);", "return eta * num / den;"),
    "block_grow_any_time": ("fmod(t, 2.0 * dt_old) == 0.0", "1"),
    "forces_unpredicted": ("orc_forces(N, m, xp, vp, eps, n, act", "orc_forces(N, m, x, v, eps, n, act"),
    "neumaier_branch": ("a->c += (a->s - t) + x;", "a->c += (x - t) + a->s;"),
}


def _battery(o):
    """Quick pins; returns the list of failed check names."""
    failed = []

    def check(name, ok):
        if not ok:
            failed.append(name)

    def rel(a, b):
        return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)

    # two-body hand values (eps 0 and 5)
    m = np.array([1.0, 2.0])
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    v = np.zeros((2, 3))
    a, j, p = o.forces(m, x, v, 0.0)
    check("two_body", np.allclose(a[0], [0.048, 0.064, 0.0], atol=1e-15) and abs(p[0] + 0.4) < 1e-15)
    a, j, p = o.forces(m, x, v, 5.0)
    check("two_body_soft", abs(a[0, 0] - 6.0 / 50.0 ** 1.5) < 1e-15 and abs(p[0] + 2 / math.sqrt(50)) < 1e-15)
    # circular orbit jerk
    r = 0.37
    mm = np.array([1.0, 1e-30])
    xx = np.array([[0.0, 0, 0], [r, 0, 0]])
    vv = np.array([[0.0, 0, 0], [0, math.sqrt(1 / r), 0]])
    a, j, p = o.forces(mm, xx, vv, 0.0, idx=[1])
    check("circular_jerk", rel(j[0], -vv[1] / r ** 3) < 1e-14)
    # Newton III, FD jerk, potential gradient on a small Plummer model
    m, x, v = inputs.plummer(48, 3, "salpeter")
    eps = 1.0 / 32
    a, j, p = o.forces(m, x, v, eps, compensated=True)
    check("newton3", np.abs((m[:, None] * a).sum(0)).max() < 1e-14 * np.abs(m[:, None] * a).sum())
    check("newton3_jerk", np.abs((m[:, None] * j).sum(0)).max() < 1e-14 * np.abs(m[:, None] * j).sum())
    h = 1e-5
    ap, _, _ = o.forces(m, x + v * h, v, eps, compensated=True)
    am, _, _ = o.forces(m, x - v * h, v, eps, compensated=True)
    check("fd_jerk", rel((ap - am) / (2 * h), j) < 1e-7)
    i = 5
    g = np.zeros(3)
    for k in range(3):
        xp_, xm_ = x.copy(), x.copy()
        xp_[i, k] += h
        xm_[i, k] -= h
        g[k] = -(o.forces(m, xp_, v, eps, idx=[i])[2][0] - o.forces(m, xm_, v, eps, idx=[i])[2][0]) / (2 * h)
    check("pot_gradient", rel(g, a[i]) < 1e-7)
    # octahedral shell: potential at the centre
    R, M = 0.75, 3.0
    pts = [[R, 0, 0], [-R, 0, 0], [0, R, 0], [0, -R, 0], [0, 0, R], [0, 0, -R]]
    xs = np.array([[0.0, 0, 0]] + pts)
    ms = np.array([1.0] + [M / 6] * 6)
    a, j, p = o.forces(ms, xs, np.zeros_like(xs), 0.1, idx=[0])
    check("shell_pot", abs(p[0] + M / math.sqrt(R * R + 0.01)) < 1e-14)
    # compensated sum recovers the lost term
    mc = np.array([1.0, 1e16, 4.0, 1e16])
    xc = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0], [-1.0, 0, 0]])
    a, _, _ = o.forces(mc, xc, np.zeros((4, 3)), 0.0, idx=[0], compensated=True)
    check("compensated", a[0, 0] == 1.0)
    # predictor hand cubic
    xp, vp = o.predict([[1.0, 0, 0]], [[2.0, 0, 0]], [[3.0, 0, 0]], [[6.0, 0, 0]], [0.25], 0.75)
    check("predictor", xp[0, 0] == 2.5 and vp[0, 0] == 4.25)
    # corrector exact on a quintic
    rng = np.random.default_rng(5)
    c = rng.normal(size=(3, 6))
    P = [np.polynomial.Polynomial(c[k]) for k in range(3)]

    def ev(d, t):
        return np.array([[P[k].deriv(d)(t) if d else P[k](t) for k in range(3)]])

    hh = 0.5
    x0, v0, a0, j0 = ev(0, 0), ev(1, 0), ev(2, 0), ev(3, 0)
    xq, vq = o.predict(x0, v0, a0, j0, [0.0], hh)
    x1, v1, a2e, a3 = o.correct(x0, v0, a0, j0, xq, vq, ev(2, hh), ev(3, hh), [hh])
    check("corrector_quintic", np.abs(x1 - ev(0, hh)).max() < 1e-12 and np.abs(v1 - ev(1, hh)).max() < 1e-12
          and np.abs(a2e - ev(4, hh)).max() < 1e-8)
    # Aarseth on a circular orbit
    ro = 0.2
    w = math.sqrt(1.0 / ro ** 3)
    xo = np.array([ro, 0, 0])
    vo = np.array([0, ro * w, 0])
    dto = o.aarseth_dt(-w * w * xo, -w * w * vo, w ** 4 * xo, w ** 4 * vo, 0.01)
    check("aarseth_circular", abs(dto - 0.1 / w) < 1e-14 / w)
    # block rule: no growth off the 2 dt_old grid
    check("block_rule", o.block_dt(1.0, 2.0 ** -5, 3 * 2.0 ** -5, 2.0 ** -22, 0.125)[0] == 2.0 ** -5)
    # Kepler with block steps and Aarseth steps
    e = 0.5
    mk = np.array([0.5, 0.5])
    xk = np.array([[-0.25, 0, 0], [0.25, 0, 0]])
    vpk = math.sqrt(3.0)
    vk = np.array([[0, -vpk / 2, 0], [0, vpk / 2, 0]])
    rr = o.hermite_run(mk, xk, vk, 0.0, 0.0025, 2.0 ** -22, 0.125, 8.0, max_block_steps=20000)
    E = 8.0
    for _ in range(60):
        E -= (E - e * math.sin(E) - 8.0) / (1 - e * math.cos(E))
    ref = np.array([math.cos(E) - e, math.sqrt(1 - e * e) * math.sin(E), 0.0])
    check("kepler", np.linalg.norm((rr["x"][1] - rr["x"][0]) - ref) < 1e-5)
    return failed


@pytest.fixture(scope="module")
def built_mutants(tmp_path_factory, orc):
    src = orc.source()
    d = tmp_path_factory.mktemp("mutants")
    paths = {}
    for name, (old, new) in MUTANTS.items():
        assert src.count(old) >= 1, f"mutation site for {name} not found"
        paths[name] = orc.compile_source(src.replace(old, new, 1 if name != "jerk_sign" else -1),
                                         os.path.join(str(d), f"{name}.so"))
    return paths


def test_unmodified_oracle_passes_battery(orc):
    assert _battery(orc) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(orc, built_mutants, name):
    with orc.using(built_mutants[name]):
        failed = _battery(orc)
    assert failed, f"planted mistake {name} passed every pin"
