"""Parity of the CUDA integrator (Sec. 4.1 steps 1-6: block selection,
predictor, forces, Hermite corrector, power-of-two block steps of Sec. 2)
with the FP64 oracle on the same seeded inputs."""
import math

import numpy as np
import pytest

import oracle
from paper_0709_4552_gb300 import inputs
from _util import rel_scalar, rel_vec

pytestmark = pytest.mark.gpu


def _ctx(nb, m, x, v, eps, eta, dt_min, dt_max, prec=None, state=None):
    s = nb.NBody(len(m), nb.NB_FP64 if prec is None else prec, 0)
    s.set_params(eps, eta, dt_min, dt_max)
    if state is None:
        s.set_j_particles(0, m, x, v)
        s.initial_forces_and_dt()
    else:
        s.set_j_particles(0, m, state["x"], state["v"], state["a"], state["jerk"], state["t"], state["dt"])
    return s


def _state(s, N):
    return s.get_particles(0, N)


def test_initial_steps_match(nbl):
    N, eps = 700, 1 / 256
    m, x, v = inputs.plummer(N, 201, "salpeter")
    r = oracle.hermite_run(m, x, v, eps, 0.01, 2.0 ** -22, 2.0 ** -3, 2.0 ** -3, max_block_steps=0,
                           compensated=True)
    with _ctx(nbl, m, x, v, eps, 0.01, 2.0 ** -22, 2.0 ** -3) as s:
        st = _state(s, N)
    assert rel_vec(st["a"], r["a"]).max() < 1e-12
    assert rel_vec(st["jerk"], r["jerk"]).max() < 1e-12
    assert np.array_equal(st["dt"], r["dt"])
    assert np.all(st["t"] == 0.0)


@pytest.mark.parametrize("steps", [1, 40])
def test_block_steps_match(nbl, steps):
    # same block schedule (t, dt exactly) and state (FP64) after k block steps
    N, eps = 1000, 1 / 256
    m, x, v = inputs.plummer(N, 202, "salpeter")
    r = oracle.hermite_run(m, x, v, eps, 0.01, 2.0 ** -22, 2.0 ** -3, 1.0, max_block_steps=steps,
                           compensated=True)
    with _ctx(nbl, m, x, v, eps, 0.01, 2.0 ** -22, 2.0 ** -3) as s:
        for _ in range(steps):
            s.step()
        st = _state(s, N)
    assert np.array_equal(st["t"], r["t"])
    assert np.array_equal(st["dt"], r["dt"])
    assert np.abs(st["x"] - r["x"]).max() < 1e-12
    assert np.abs(st["v"] - r["v"]).max() < 1e-11


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_next_block_matches_definition(nbl, prec):
    N = 3000
    m, x, v = inputs.plummer(N, 203, "salpeter")
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    with _ctx(nbl, m, x, v, 1 / 512, 0.01, 2.0 ** -22, 2.0 ** -3, prec=P) as s:
        for _ in range(5):
            st = _state(s, N)
            t, n, idx = s.next_block()
            due = st["t"] + st["dt"]
            assert t == due.min()
            assert np.array_equal(idx, np.nonzero(due == t)[0].astype(np.int32))
            assert n == len(idx)
            s.step()


def _energy(m, st, eps):
    k, w = oracle.energy(m, st["x"], st["v"], eps)
    return k + w


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_config1_shared_steps(nbl, prec):
    # Plummer N=1024, eps=1/256, shared dt=2^-10, 128 steps (full i=j each step)
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    N, eps, dt = 1024, 1 / 256, 2.0 ** -10
    m, x, v = inputs.plummer(N, 1)
    E0 = _energy(m, dict(x=x, v=v), eps)
    r = oracle.hermite_run(m, x, v, eps, 0.01, dt, dt, 128 * dt, compensated=True)
    assert r["block_steps"] == 128
    dE_orc = abs(_energy(m, r, eps) - E0) / abs(E0)
    with _ctx(nbl, m, x, v, eps, 0.01, dt, dt, prec=P) as s:
        for k in range(128):
            t, n = s.step()
            assert n == N and t == (k + 1) * dt
            if (k + 1) % 16 == 0:
                # forces on the GPU's own state vs the oracle on that state
                st = _state(s, N)
                s.predict(t)
                a, j, p = s.compute_forces(np.arange(N, dtype=np.int32))
                ar, jr, pr = oracle.forces(m, st["x"], st["v"], eps, compensated=True)
                errs = {"acc": rel_vec(a, ar), "jerk": rel_vec(j, jr), "pot": rel_scalar(p, pr)}
                for name, e in errs.items():
                    if P == nbl.NB_FP64:
                        assert e.max() <= 1e-12, (k, name, e.max())
                    else:
                        # the mixed path's bounds: median <= 1e-6, max <= 1e-5
                        assert np.median(e) <= 1e-6, (k, name, np.median(e))
                        assert e.max() <= 1e-5, (k, name, e.max())
        st = _state(s, N)
    dE_gpu = abs(_energy(m, st, eps) - E0) / abs(E0)
    print(f"config1 {prec}: |dE/E| gpu {dE_gpu:.3e} oracle {dE_orc:.3e}")
    assert dE_gpu <= 2 * dE_orc + 1e-13
    P_mom = (m[:, None] * st["v"]).sum(0)
    assert np.abs(P_mom).max() < (1e-14 if P == nbl.NB_FP64 else 1e-9)
    if P == nbl.NB_FP64:
        assert np.abs(st["x"] - r["x"]).max() < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_timings_count_interactions(nbl, prec):
    # nb_get_timings: the interaction count is the sum of n N over the block
    # steps (Eq. 3's n N per force call), and every phase took device time
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    N = 2000
    m, x, v = inputs.plummer(N, 207, "salpeter")
    with _ctx(nbl, m, x, v, 1 / 256, 0.01, 2.0 ** -22, 2.0 ** -3, prec=P) as s:
        tim = s.get_timings(reset=True)
        assert tim["interactions"] == float(N) * N   # the initial full i = j evaluation
        assert s.get_timings()["interactions"] == 0.0
        total, c0 = 0, s.get_counters()
        for _ in range(25):
            t, n = s.step()
            total += n * N
        tim = s.get_timings(reset=True)
        c1 = s.get_counters()
        assert c1["block_steps"] - c0["block_steps"] == 25
        assert tim["interactions"] == float(total)
        assert tim["ms_pred"] > 0 and tim["ms_force"] > 0 and tim["ms_corr"] > 0
        if P != nbl.NB_FP64:
            return
        # host-loop integration: n N per block step, checked against a replay
        # of the same steps through nb_step (FP64: the replay takes the same
        # steps bit for bit)
        st = _state(s, N)
        s.integrate(2.0 ** -3)
        tim = s.get_timings(reset=True)
        replay = 0
        with _ctx(nbl, m, x, v, 1 / 256, 0.01, 2.0 ** -22, 2.0 ** -3, prec=P, state=st) as r:
            while True:
                t, n_next, _ = r.next_block(want_indices=False)
                if t > 2.0 ** -3:
                    break
                t, n = r.step()
                replay += n * N
        assert tim["interactions"] == float(replay)


def _kepler():
    e, rp = 0.5, 0.5
    vp = math.sqrt(3.0)
    m = np.array([0.5, 0.5])
    x = np.array([[-rp / 2, 0, 0], [rp / 2, 0, 0]])
    v = np.array([[0, -vp / 2, 0], [0, vp / 2, 0]])
    return m, x, v


def _kepler_sep(t, e=0.5):
    Mq = math.fmod(t, 2 * math.pi)
    E = Mq
    for _ in range(60):
        E -= (E - e * math.sin(E) - Mq) / (1 - e * math.cos(E))
    return np.array([math.cos(E) - e, math.sqrt(1 - e * e) * math.sin(E), 0.0])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-6), ("mixed", 1e-4)])
def test_kepler_orbit(nbl, prec, tol):
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    m, x, v = _kepler()
    with _ctx(nbl, m, x, v, 0.0, 0.01, 2.0 ** -9, 2.0 ** -9, prec=P) as s:
        s.integrate(64.0)
        st = _state(s, 2)
    sep = st["x"][1] - st["x"][0]
    assert np.linalg.norm(sep - _kepler_sep(64.0)) < tol


def test_integrate_equals_steps(nbl):
    N, eps = 800, 1 / 256
    m, x, v = inputs.plummer(N, 204)
    with _ctx(nbl, m, x, v, eps, 0.01, 2.0 ** -22, 2.0 ** -5) as s:
        s.integrate(2.0 ** -5)
        a = _state(s, N)
    with _ctx(nbl, m, x, v, eps, 0.01, 2.0 ** -22, 2.0 ** -5) as s:
        while True:
            st = _state(s, N)
            if np.all(st["t"] == 2.0 ** -5):
                break
            s.step()
        b = _state(s, N)
    for k in ("x", "v", "a", "jerk", "t", "dt"):
        assert np.array_equal(a[k], b[k]), k


def test_checkpoint_resume_bitwise(nbl):
    N, eps = 900, 1 / 256
    m, x, v = inputs.plummer(N, 205, "salpeter")
    with _ctx(nbl, m, x, v, eps, 0.01, 2.0 ** -22, 2.0 ** -4) as s:
        for _ in range(30):
            s.step()
        mid = _state(s, N)
        for _ in range(30):
            s.step()
        ref = _state(s, N)
    with _ctx(nbl, m, x, v, eps, 0.01, 2.0 ** -22, 2.0 ** -4, state=mid) as s:
        for _ in range(30):
            s.step()
        got = _state(s, N)
    for k in ("x", "v", "a", "jerk", "t", "dt"):
        assert np.array_equal(got[k], ref[k]), k


def test_energy_matches_oracle(nbl):
    N, eps = 2000, 1 / 256
    m, x, v = inputs.plummer(N, 206, "salpeter")
    k0, w0 = oracle.energy(m, x, v, eps)
    with nbl.NBody(N, nbl.NB_FP64, 0) as s:
        s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
        s.set_j_particles(0, m, x, v)
        k, w = s.energy()
    assert abs(k - k0) / abs(k0) < 1e-13
    assert abs(w - w0) / abs(w0) < 1e-12


@pytest.mark.slow
def test_config2_reduced_energy_drift(nbl):
    # config-2 physics at N=16384 (Salpeter, eps=1/1024, eta=0.01, 2^-22..2^-3) to t=1/64
    N, eps, t_end = 16384, 1 / 1024, 2.0 ** -6
    m, x, v = inputs.plummer(N, 2, "salpeter")
    E0 = _energy(m, dict(x=x, v=v), eps)
    r = oracle.hermite_run(m, x, v, eps, 0.01, 2.0 ** -22, t_end, t_end)
    dE_orc = abs(_energy(m, r, eps) - E0) / abs(E0)
    with _ctx(nbl, m, x, v, eps, 0.01, 2.0 ** -22, t_end) as s:
        s.integrate(t_end)
        st = _state(s, N)
        idx = inputs.sample_indices(N, 4096, 1002)
        s.predict(t_end)
        a, j, p = s.compute_forces(idx.astype(np.int32))
    ar, jr, pr = oracle.forces(m, st["x"], st["v"], eps, idx=idx, compensated=True)
    assert rel_vec(a, ar).max() < 1e-12 and rel_vec(j, jr).max() < 1e-12
    dE_gpu = abs(_energy(m, st, eps) - E0) / abs(E0)
    print(f"config2@16k: |dE/E| gpu {dE_gpu:.3e} oracle {dE_orc:.3e}")
    assert dE_gpu <= 2 * dE_orc + 1e-13


def test_nan_input_reported(nbl):
    torch = pytest.importorskip("torch")
    N = 256
    m, x, v = inputs.plummer(N, 207)
    v = v.copy()
    v[17, 0] = np.nan
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        s.set_j_particles(0, dev(m), dev(x), dev(v))   # device input: not validated
        torch.cuda.synchronize()
        with pytest.raises(nbl.NBodyError) as e:
            s.initial_forces_and_dt()
        assert e.value.code == nbl.NB_ENUMERIC
        code, _ = s.check_device_status()
        assert code == nbl.NB_ENUMERIC
        s.clear_error()
        assert s.check_device_status()[0] == nbl.NB_OK


def test_dt_underflow_counted(nbl):
    # a tight unsoftened binary: its criterion falls below dt_min = 2^-12
    m = np.array([0.5, 0.5, 1e-3])
    x = np.array([[-1e-4, 0, 0], [1e-4, 0, 0], [1.0, 0, 0]])
    vb = math.sqrt(0.5 / 2e-4) / 2 * 2
    v = np.array([[0, -vb / 2, 0], [0, vb / 2, 0], [0, 0.5, 0]])
    with _ctx(nbl, m, x, v, 0.0, 0.01, 2.0 ** -12, 2.0 ** -6) as s:
        s.step()
        code, under = s.check_device_status()
        st = _state(s, 3)
    assert code == nbl.NB_OK and under >= 2
    assert st["dt"][0] == 2.0 ** -12 and st["dt"][1] == 2.0 ** -12


def test_resident_order_round_trip(nbl):
    # a mixed context keeps its arrays in the spatial order of the particles;
    # every ABI call still speaks particle indices
    N, eps = 5000, 1 / 256
    m, x, v = inputs.plummer(N, 207, "salpeter")
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
        s.set_j_particles(0, m, x, v)
        s.initial_forces_and_dt()  # computes the order and reorders the arrays
        st = s.get_particles(0, N)
        for k, ref in (("m", m), ("x", x), ("v", v), ("t", np.zeros(N))):
            assert np.array_equal(st[k], ref), k
        a_ref, j_ref, p_ref = oracle.forces(m, x, v, eps)
        assert rel_vec(st["a"], a_ref).max() < 1e-5 and rel_scalar(st["pot"], p_ref).max() < 1e-6
        sub = s.get_particles(1234, 100)
        assert np.array_equal(sub["m"], m[1234:1334]) and np.array_equal(sub["x"], x[1234:1334])
        # device outputs take the same gather
        torch = pytest.importorskip("torch")
        dx = torch.empty((N, 3), dtype=torch.float64, device="cuda")
        s.get_particles(0, N, out=dict(x=dx))
        torch.cuda.synchronize()
        assert np.array_equal(dx.cpu().numpy(), x)
        # forces on a caller's list come back in the caller's order
        idx = inputs.sample_indices(N, 900, 5)
        s.predict(0.0)
        a, _, p = s.compute_forces(idx.astype(np.int32))
        assert rel_vec(a, a_ref[idx]).max() < 1e-5 and rel_scalar(p, p_ref[idx]).max() < 1e-6
        for _ in range(3):
            s.step()
        st = s.get_particles(0, N)
        t, n, act = s.next_block()
        due = st["t"] + st["dt"]
        assert t == due.min() and np.array_equal(act, np.nonzero(due == t)[0].astype(np.int32))
        # overwrite a range: the rest keeps its state, the range reads back as written
        x2 = x[100:200] * 1.5
        s.set_j_particles(100, m[100:200], x2, v[100:200])
        st2 = s.get_particles(0, N)
        assert np.array_equal(st2["x"][100:200], x2)
        keep = np.r_[0:100, 200:N]
        for k in ("x", "v", "a", "t", "dt"):
            assert np.array_equal(st2[k][keep], st[k][keep]), k
        s.initial_forces_and_dt()
        s.set_n(N - 10)
        st3 = s.get_particles(0, N - 10)
        assert np.array_equal(st3["m"], m[: N - 10]) and np.array_equal(st3["x"][100:200], x2)


def test_snapshot_file_resume_bitwise(nbl, tmp_path):
    # the binary snapshot holds what the block-step loop needs: an FP64 run
    # resumed from the file repeats the uninterrupted run bit for bit
    from paper_0709_4552_gb300 import snapshot
    N, eps = 700, 1 / 256
    m, x, v = inputs.plummer(N, 208, "salpeter")
    path = tmp_path / "mid.nbs"
    with _ctx(nbl, m, x, v, eps, 0.01, 2.0 ** -22, 2.0 ** -4) as s:
        for _ in range(25):
            s.step()
        snapshot.save(s, path)
        for _ in range(25):
            s.step()
        ref = _state(s, N)
    with nbl.NBody(N, nbl.NB_FP64, 0) as s:
        _, prm = snapshot.load(s, path)
        assert prm["eps"] == eps and prm["dt_max"] == 2.0 ** -4
        assert s.get_params() == dict(eps=eps, eta=0.01, dt_min=2.0 ** -22, dt_max=2.0 ** -4)
        for _ in range(25):
            s.step()
        got = _state(s, N)
    for k in ("x", "v", "a", "jerk", "t", "dt"):
        assert np.array_equal(got[k], ref[k]), k


def test_invalid_parameters_rejected(nbl):
    with nbl.NBody(16, nbl.NB_MIXED, 0) as s:
        for bad in ((-1.0, 0.01, 2.0 ** -22, 2.0 ** -3), (0.01, 0.0, 2.0 ** -22, 2.0 ** -3),
                    (0.01, 0.01, 3e-7, 2.0 ** -3), (0.01, 0.01, 2.0 ** -3, 2.0 ** -22),
                    (float("nan"), 0.01, 2.0 ** -22, 2.0 ** -3)):
            with pytest.raises(nbl.NBodyError) as e:
                s.set_params(*bad)
            assert e.value.code == nbl.NB_EINVAL
        s.clear_error()
        with pytest.raises(nbl.NBodyError):
            s.set_j_particles(0, np.ones(3), np.array([[0.0, 0, 0], [np.inf, 0, 0], [1, 1, 1]]), np.zeros((3, 3)))


def test_resident_order_random_api_sequence(nbl):
    # a seeded random sequence of ABI calls on a mixed context (whose arrays
    # are kept in spatial order): every read-back and every force result must
    # be the one of the particles the caller names
    N, eps = 2500, 1 / 256
    rng = np.random.default_rng(209)
    m, x, v = inputs.plummer(N, 209, "salpeter")
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -4)
        s.set_j_particles(0, m, x, v)
        s.initial_forces_and_dt()
        for it in range(12):
            op = it % 4
            if op == 0:          # block steps (the order is renewed every 64)
                for _ in range(int(rng.integers(1, 40))):
                    s.step()
            elif op == 1:        # forces on a random caller list at the current block time
                st = s.get_particles(0, N)
                t, n, act = s.next_block()
                idx = np.sort(rng.choice(N, int(rng.integers(1, N)), replace=False)).astype(np.int32)
                s.predict(t)
                a, j, p = s.compute_forces(idx)
                # the oracle on the same predicted state, particle by particle
                h = (t - st["t"])[:, None]
                xp = st["x"] + h * (st["v"] + h * (0.5 * st["a"] + h * st["jerk"] / 6))
                vp = st["v"] + h * (st["a"] + h * 0.5 * st["jerk"])
                ar, jr, pr = oracle.forces(st["m"], xp, vp, eps, idx=idx.astype(np.int64))
                assert rel_vec(a, ar).max() < 1e-5 and rel_scalar(p, pr).max() < 1e-5
            elif op == 2:        # overwrite a random range, read everything back
                lo = int(rng.integers(0, N - 10))
                cnt = int(rng.integers(1, N - lo))
                st = s.get_particles(0, N)
                x2 = st["x"][lo:lo + cnt] + 1e-3 * rng.normal(size=(cnt, 3))
                s.set_j_particles(lo, st["m"][lo:lo + cnt], x2, st["v"][lo:lo + cnt], st["a"][lo:lo + cnt],
                                  st["jerk"][lo:lo + cnt], st["t"][lo:lo + cnt], st["dt"][lo:lo + cnt])
                got = s.get_particles(0, N)
                want = st["x"].copy()
                want[lo:lo + cnt] = x2
                assert np.array_equal(got["x"], want)
                for k in ("m", "v", "t", "dt"):
                    assert np.array_equal(got[k], st[k]), k
            else:                # sub-range reads agree with the full read
                st = s.get_particles(0, N)
                lo = int(rng.integers(0, N - 1))
                cnt = int(rng.integers(1, N - lo + 1))
                sub = s.get_particles(lo, cnt)
                for k in ("m", "x", "v", "a", "jerk", "t", "dt"):
                    assert np.array_equal(sub[k], st[k][lo:lo + cnt]), k


def test_corrector_exponent_forms_bitwise(nbl):
    # the corrector's shortcuts (powers of a power-of-two step, the step rule
    # from exponents) give their FP64 expressions' bits on 4M random operand
    # sets, boundary and non-finite cases included
    assert nbl.nb_selftest_corrector(1 << 22, seed=11) == 0
    assert nbl.nb_selftest_corrector(1 << 20, seed=12) == 0
