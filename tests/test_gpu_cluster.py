"""The cluster loop (nb_integrate with NB_LOOP_CLUSTER): the whole block-step
loop of a small mixed system on one thread-block cluster, the ring algorithm
of Sec. 4.3 on one chip (each CTA holds a slice of the particles, predicted
on the fly; the active block visits every CTA through distributed shared
memory).  Checked against the host-driven loop, whose steps the oracle pins,
and the oracle's own energy drift."""
import numpy as np
import pytest

import oracle
from paper_0709_4552_gb300 import inputs

pytestmark = pytest.mark.gpu


def _single(nb, prec, m, x, v, eps, dt_min, dt_max, eta=0.01):
    s = nb.NBody(len(m), prec, 0)
    s.set_params(eps, eta, dt_min, dt_max)
    s.set_j_particles(0, m, x, v)
    s.initial_forces_and_dt()
    return s


def _run(nb, ics, eps, t_end, loop):
    m, x, v = ics
    with _single(nb, nb.NB_MIXED, m, x, v, eps, 2.0 ** -22, t_end) as s:
        c0 = s.get_counters()
        t0 = s.get_timings(reset=True)
        s.integrate(t_end, loop=loop)
        c1 = s.get_counters()
        tim = s.get_timings()
        return s.get_particles(0, len(m)), c1["block_steps"] - c0["block_steps"], c1["kernel_launches"] - \
            c0["kernel_launches"], tim["interactions"]


@pytest.mark.parametrize("N", [1, 2, 17, 100, 1500, 6000, 16384])
def test_cluster_matches_host_loop(nbl, N):
    # one row per CTA and fewer (N < 16), ragged slices, the largest system
    ics = inputs.plummer(N, 930 + N, "salpeter")
    eps, t_end = 1 / 256, 2.0 ** -5
    a, sa, _, ia = _run(nbl, ics, eps, t_end, nbl.NB_LOOP_HOST)
    b, sb, lb, ib = _run(nbl, ics, eps, t_end, nbl.NB_LOOP_CLUSTER)
    assert np.all(a["t"] == t_end) and np.all(b["t"] == t_end)
    assert lb <= 3   # the j-memory build and one cluster launch for the whole run
    # different summation orders: a criterion near a power of two can pick a
    # different step for a few particles (same physics, not the same bits)
    assert abs(sb - sa) <= 0.05 * sa + 1
    assert np.sum(a["dt"] != b["dt"]) <= max(1, 0.05 * N)
    assert np.abs(a["x"] - b["x"]).max() < 1e-5
    assert np.abs(a["v"] - b["v"]).max() < 1e-4
    # n N per block step: a multiple of N, close to the host loop's sum
    assert ib % N == 0 and abs(ib - ia) <= 0.05 * ia


def test_cluster_energy_drift_within_oracle(nbl):
    N, eps, t_end = 2048, 1 / 256, 2.0 ** -4
    m, x, v = inputs.plummer(N, 811, "salpeter")
    with _single(nbl, nbl.NB_MIXED, m, x, v, eps, 2.0 ** -22, t_end) as s:
        k0, w0 = s.energy()
        s.integrate(t_end, loop=nbl.NB_LOOP_CLUSTER)
        k1, w1 = s.energy()
        st = s.get_particles(0, N)
    assert np.all(st["t"] == t_end)
    E0 = sum(oracle.energy(m, x, v, eps))
    r = oracle.hermite_run(m, x, v, eps, 0.01, 2.0 ** -22, t_end, t_end)
    d_orc = abs(sum(oracle.energy(m, r["x"], r["v"], eps)) - E0) / abs(E0)
    d_gpu = abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0)
    assert d_gpu <= 2 * d_orc + 1e-9, (d_gpu, d_orc)


def test_cluster_resumes_other_loops(nbl):
    # host loop, cluster loop, host loop again: the j-memory the cluster loop
    # leaves is current for the host loop's on-the-fly blocks
    N, eps = 3000, 1 / 256
    ics = inputs.plummer(N, 944, "salpeter")
    a, *_ = _run(nbl, ics, eps, 2.0 ** -4, nbl.NB_LOOP_HOST)
    m, x, v = ics
    with _single(nbl, nbl.NB_MIXED, m, x, v, eps, 2.0 ** -22, 2.0 ** -6) as s:
        s.integrate(2.0 ** -6, loop=nbl.NB_LOOP_HOST)
        s.integrate(2.0 ** -5, loop=nbl.NB_LOOP_CLUSTER)
        s.integrate(2.0 ** -4, loop=nbl.NB_LOOP_HOST)
        b = s.get_particles(0, N)
    assert np.all(b["t"] == 2.0 ** -4)
    assert np.abs(a["x"] - b["x"]).max() < 1e-5


def test_cluster_numeric_failure_reported(nbl):
    torch = pytest.importorskip("torch")
    N = 300
    m, x, v = inputs.plummer(N, 913)
    with _single(nbl, nbl.NB_MIXED, m, x, v, 1 / 256, 2.0 ** -14, 2.0 ** -8) as s:
        st = s.get_particles(0, N)
        st["v"][41, 1] = np.nan
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()   # device input: not validated
        s.set_j_particles(0, *(dev(st[k]) for k in ("m", "x", "v", "a", "jerk", "t", "dt")))
        torch.cuda.synchronize()
        with pytest.raises(nbl.NBodyError) as e:
            s.integrate(2.0 ** -8, loop=nbl.NB_LOOP_CLUSTER)
        assert e.value.code == nbl.NB_ENUMERIC
        s.clear_error()
        assert s.check_device_status()[0] == nbl.NB_OK


def test_cluster_rejects_bad_arguments(nbl):
    m, x, v = inputs.plummer(500, 917)
    with _single(nbl, nbl.NB_FP64, m, x, v, 1 / 256, 2.0 ** -22, 2.0 ** -3) as s:
        with pytest.raises(nbl.NBodyError) as e:   # mixed path only
            s.integrate(0.125, loop=nbl.NB_LOOP_CLUSTER)
        assert e.value.code == nbl.NB_EINVAL
    N = nbl.NB_CLUSTER_MAX_N + 1
    m, x, v = inputs.plummer(N, 918)
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        s.set_params(1 / 256, 0.01, 2.0 ** -22, 2.0 ** -3)
        s.set_j_particles(0, m, x, v)
        with pytest.raises(nbl.NBodyError) as e:
            s.integrate(0.125, loop=nbl.NB_LOOP_CLUSTER)
        assert e.value.code == nbl.NB_EINVAL
