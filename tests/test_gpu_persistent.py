"""The persistent block-step loop (nb_integrate with NB_LOOP_PERSISTENT: one
cooperative launch per run, grid barriers between the phases of a step)
against the host-driven loop, whose steps the oracle pins, and its bounded
barrier wait."""
import numpy as np
import pytest

from paper_0709_4552_gb300 import inputs

pytestmark = pytest.mark.gpu


def _single(nb, prec, m, x, v, eps, dt_min, dt_max, eta=0.01):
    s = nb.NBody(len(m), prec, 0)
    s.set_params(eps, eta, dt_min, dt_max)
    s.set_j_particles(0, m, x, v)
    s.initial_forces_and_dt()
    return s


def _run(nb, prec, ics, eps, t_end, loops, dt_max=None):
    m, x, v = ics
    with _single(nb, prec, m, x, v, eps, 2.0 ** -22, dt_max or t_end) as s:
        c0 = s.get_counters()
        for t, loop in loops:
            s.integrate(t, loop=loop)
        c1 = s.get_counters()
        c = {k: c1[k] - c0[k] for k in c1}   # of the integration alone
        return s.get_particles(0, len(m)), c


def _close_fp64(a, ca, b, cb, t_end):
    assert np.all(a["t"] == t_end) and np.all(b["t"] == t_end)
    assert cb["block_steps"] == ca["block_steps"]
    assert np.array_equal(a["dt"], b["dt"])
    # the j-split sums group differently: same steps, last-bit differences
    assert np.abs(a["x"] - b["x"]).max() < 1e-12
    assert np.abs(a["v"] - b["v"]).max() < 1e-11


@pytest.mark.parametrize("N", [1, 2, 3, 100, 128, 129, 1000, 2500])
def test_persistent_fp64_matches_host_loop(nbl, N):
    # ragged and tiny systems: one row tile, a tile plus one row, fewer tiles
    # than CTAs, several tiles per j-split
    ics = inputs.plummer(N, 600 + N, "salpeter")
    eps, t_end = 1 / 256, 2.0 ** -5
    a, ca = _run(nbl, nbl.NB_FP64, ics, eps, t_end, [(t_end, nbl.NB_LOOP_HOST)])
    b, cb = _run(nbl, nbl.NB_FP64, ics, eps, t_end, [(t_end, nbl.NB_LOOP_PERSISTENT)])
    _close_fp64(a, ca, b, cb, t_end)
    assert cb["kernel_launches"] == 1   # one cooperative launch for the whole run


@pytest.mark.parametrize("N", [2, 3, 17, 64, 100, 128])
def test_loops_bitwise_equal_when_sums_group_alike(nbl, N):
    # with at most two j-splits every driver sums the same partials in the
    # same order, so the three loops share predictor, forces, corrector and
    # block rule bit for bit (one 64-particle j-tile: all three; two: host
    # and persistent)
    ics = inputs.plummer(N, 640 + N, "salpeter")
    eps, t_end = 1 / 256, 2.0 ** -5
    runs = [nbl.NB_LOOP_HOST, nbl.NB_LOOP_PERSISTENT] + ([nbl.NB_LOOP_GRAPH] if N <= 64 else [])
    out = [_run(nbl, nbl.NB_FP64, ics, eps, t_end, [(t_end, loop)]) for loop in runs]
    (a, ca) = out[0]
    for b, cb in out[1:]:
        assert cb["block_steps"] == ca["block_steps"]
        for k in ("x", "v", "a", "jerk", "pot", "t", "dt"):
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("N", [1500, 6000, 131072])
def test_persistent_mixed_matches_host_loop(nbl, N):
    # several launches: the spatial order is renewed every 64 block steps;
    # 131072 lies above the FP64 loop's bound (a few hundred rows per CTA,
    # full-block force phases of 1.7e10 interactions)
    big = N > nbl.NB_PERSISTENT_MAX_N_FP64
    ics = inputs.plummer(N, 700 + N, "equal" if big else "salpeter")
    eps, t_end = 1 / 256, 2.0 ** (-7 if big else -5)
    a, ca = _run(nbl, nbl.NB_MIXED, ics, eps, t_end, [(t_end, nbl.NB_LOOP_HOST)])
    b, cb = _run(nbl, nbl.NB_MIXED, ics, eps, t_end, [(t_end, nbl.NB_LOOP_PERSISTENT)])
    assert np.all(a["t"] == t_end) and np.all(b["t"] == t_end)
    # different summation orders: a criterion near a power of two can pick
    # a different step for a few particles (same physics, not the same bits)
    assert abs(cb["block_steps"] - ca["block_steps"]) <= 0.05 * ca["block_steps"]
    assert np.mean(a["dt"] == b["dt"]) > 0.95
    assert np.abs(a["x"] - b["x"]).max() < 1e-5
    assert np.abs(a["v"] - b["v"]).max() < 1e-4


def test_persistent_energy_drift_like_host_loop(nbl):
    N, eps, t_end = 2048, 1 / 256, 2.0 ** -4
    ics = inputs.plummer(N, 811, "salpeter")
    drift = {}
    for loop in (nbl.NB_LOOP_HOST, nbl.NB_LOOP_PERSISTENT):
        m, x, v = ics
        with _single(nbl, nbl.NB_MIXED, m, x, v, eps, 2.0 ** -22, t_end) as s:
            k0, w0 = s.energy()
            s.integrate(t_end, loop=loop)
            k1, w1 = s.energy()
        drift[loop] = abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0)
    assert drift[nbl.NB_LOOP_PERSISTENT] <= 2 * drift[nbl.NB_LOOP_HOST] + 1e-9


def test_persistent_resumes_other_loops(nbl):
    # the loops share the state: persistent, host and graph runs in turn end
    # where the host loop alone ends
    ics = inputs.plummer(1200, 901, "salpeter")
    eps, t_end = 1 / 256, 2.0 ** -5
    h = 2.0 ** -7   # every t_end a multiple of dt_max
    a, ca = _run(nbl, nbl.NB_FP64, ics, eps, t_end, [(t_end, nbl.NB_LOOP_HOST)], dt_max=h)
    b, cb = _run(nbl, nbl.NB_FP64, ics, eps, t_end,
                 [(h, nbl.NB_LOOP_PERSISTENT), (2 * h, nbl.NB_LOOP_HOST),
                  (3 * h, nbl.NB_LOOP_GRAPH), (t_end, nbl.NB_LOOP_PERSISTENT)], dt_max=h)
    _close_fp64(a, ca, b, cb, t_end)


def test_persistent_numeric_failure_reported(nbl):
    torch = pytest.importorskip("torch")
    N = 300
    m, x, v = inputs.plummer(N, 913)
    with _single(nbl, nbl.NB_FP64, m, x, v, 1 / 256, 2.0 ** -14, 2.0 ** -8) as s:
        st = s.get_particles(0, N)
        st["v"][41, 1] = np.nan
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()   # device input: not validated
        s.set_j_particles(0, *(dev(st[k]) for k in ("m", "x", "v", "a", "jerk", "t", "dt")))
        torch.cuda.synchronize()
        with pytest.raises(nbl.NBodyError) as e:
            s.integrate(2.0 ** -8, loop=nbl.NB_LOOP_PERSISTENT)
        assert e.value.code == nbl.NB_ENUMERIC
        s.clear_error()
        assert s.check_device_status()[0] == nbl.NB_OK


@pytest.mark.parametrize("prec_name", ["mixed", "fp64"])
def test_persistent_rejects_bad_arguments(nbl, prec_name):
    # one particle above the precision's bound: a full-block force phase
    # would come too close to the barrier wait's limit
    prec = nbl.NB_MIXED if prec_name == "mixed" else nbl.NB_FP64
    N = (nbl.NB_PERSISTENT_MAX_N if prec == nbl.NB_MIXED else nbl.NB_PERSISTENT_MAX_N_FP64) + 1
    m, x, v = inputs.plummer(N, 917)
    with nbl.NBody(N, prec, 0) as s:
        s.set_params(1 / 256, 0.01, 2.0 ** -22, 2.0 ** -3)
        s.set_j_particles(0, m, x, v)
        with pytest.raises(nbl.NBodyError) as e:
            s.integrate(0.125, loop=nbl.NB_LOOP_PERSISTENT)
        assert e.value.code == nbl.NB_EINVAL
        s.clear_error()
        with pytest.raises(nbl.NBodyError) as e:
            s.integrate(0.125, loop=99)
        assert e.value.code == nbl.NB_EINVAL


@pytest.mark.parametrize("loop", ["host", "graph", "persistent", "cluster", "auto"])
def test_state_without_steps_is_refused_promptly(nbl, loop):
    # particles set but no initial forces and steps (dt = 0): the block time
    # never advances; every loop driver stops at once with NB_ESTATE instead of
    # repeating the same block time
    import time
    lp = {"host": nbl.NB_LOOP_HOST, "graph": nbl.NB_LOOP_GRAPH, "persistent": nbl.NB_LOOP_PERSISTENT,
          "cluster": nbl.NB_LOOP_CLUSTER, "auto": nbl.NB_LOOP_AUTO}[loop]
    m, x, v = inputs.plummer(1000, 918)
    with nbl.NBody(1000, nbl.NB_MIXED, 0) as s:
        s.set_params(1 / 256, 0.01, 2.0 ** -22, 2.0 ** -3)
        s.set_j_particles(0, m, x, v)
        t0 = time.perf_counter()
        with pytest.raises(nbl.NBodyError) as e:
            s.integrate(0.125, loop=lp)
        if loop == "cluster" and e.value.code == nbl.NB_ECUDA:
            pytest.skip("this GPU does not co-schedule the cluster")
        assert e.value.code == nbl.NB_ESTATE
        assert time.perf_counter() - t0 < 10.0


def test_grid_barrier_wait_is_bounded(nbl):
    # a barrier that waits for a CTA nobody launched gives up after the
    # limit, reports the timeout, and leaves the context usable
    m, x, v = inputs.plummer(256, 919)
    with _single(nbl, nbl.NB_FP64, m, x, v, 1 / 256, 2.0 ** -22, 2.0 ** -6) as s:
        assert s.check_grid_barrier(False, 100.0) == nbl.NB_OK
        assert s.check_grid_barrier(True, 50.0) == nbl.NB_ETIMEOUT
        assert s.check_device_status()[0] == nbl.NB_ETIMEOUT
        s.clear_error()
        assert s.check_device_status()[0] == nbl.NB_OK
        s.integrate(2.0 ** -6, loop=nbl.NB_LOOP_PERSISTENT)
        assert np.all(s.get_particles(0, 256)["t"] == 2.0 ** -6)


@pytest.mark.parametrize("loop", ["graph", "persistent"])
def test_strict_differences_in_every_loop(nbl, loop):
    # nb_set_far_tiles(0) reaches the graph and persistent loops' force items:
    # they follow the strict host loop as closely as the default ones do
    N, eps, t_end = 6000, 1 / 256, 2.0 ** -5
    m, x, v = inputs.plummer(N, 700 + N, "salpeter")
    L = nbl.NB_LOOP_GRAPH if loop == "graph" else nbl.NB_LOOP_PERSISTENT
    out = []
    for lp in (nbl.NB_LOOP_HOST, L):
        with _single(nbl, nbl.NB_MIXED, m, x, v, eps, 2.0 ** -22, t_end) as s:
            s.set_far_tiles(False)
            c0 = s.get_counters()
            s.integrate(t_end, loop=lp)
            c1 = s.get_counters()
            out.append((s.get_particles(0, N), c1["block_steps"] - c0["block_steps"]))
    (a, ca), (b, cb) = out
    assert np.all(a["t"] == t_end) and np.all(b["t"] == t_end)
    assert abs(cb - ca) <= 0.05 * ca
    assert np.mean(a["dt"] == b["dt"]) > 0.95
    assert np.abs(a["x"] - b["x"]).max() < 1e-5


@pytest.mark.parametrize("prec_name,N,expect", [("mixed", 1024, "cluster"), ("mixed", 3000, "persistent"),
                                                 ("fp64", 1000, "persistent"), ("fp64", 3000, "host"),
                                                 ("mixed", 70000, "persistent"), ("mixed", 140000, "host")])
def test_auto_loop_takes_the_measured_driver(nbl, prec_name, N, expect):
    # NB_LOOP_AUTO resolves to one of the explicit drivers: its run repeats that
    # driver's run bit for bit (the cluster loop where the GPU co-schedules it)
    prec = nbl.NB_MIXED if prec_name == "mixed" else nbl.NB_FP64
    loop = {"cluster": nbl.NB_LOOP_CLUSTER, "persistent": nbl.NB_LOOP_PERSISTENT, "host": nbl.NB_LOOP_HOST}[expect]
    t_end = 2.0 ** -8 if N > 10000 else 2.0 ** -5
    ics = inputs.plummer(N, 31)
    try:
        ref, cr = _run(nbl, prec, ics, 1 / 256, t_end, [(t_end, loop)])
    except nbl.NBodyError:
        if expect == "cluster":
            pytest.skip("this GPU does not co-schedule the cluster")
        raise
    got, cg = _run(nbl, prec, ics, 1 / 256, t_end, [(t_end, nbl.NB_LOOP_AUTO)])
    assert cg["block_steps"] == cr["block_steps"]
    for k in ("x", "v", "a", "jerk", "t", "dt"):
        assert np.array_equal(got[k], ref[k]), k
