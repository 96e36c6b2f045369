"""Parity of the CUDA force kernels (Sec. 4.1 step 4, Eq. 3) with the FP64
oracle, element by element on the same seeded inputs.

Tolerances (per particle, relative to the oracle's compensated FP64 sums):
  FP64 path:  max <= 1e-12 for acceleration, jerk and potential;
  mixed path: median <= 1e-6 and max <= 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_0709_4552_gb300 import inputs
from _util import gpu_forces, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIX_MED, MIX_MAX = 1e-6, 1e-5


def _check(prec, nb, got, ref):
    a, j, p = got
    ar, jr, pr = ref
    ea, ej, ep = rel_vec(a, ar), rel_vec(j, jr), rel_scalar(p, pr)
    if prec == nb.NB_FP64:
        assert ea.max() <= FP64_TOL, ea.max()
        assert ej.max() <= FP64_TOL, ej.max()
        assert ep.max() <= FP64_TOL, ep.max()
    else:
        for name, e in (("acc", ea), ("jerk", ej), ("pot", ep)):
            assert np.median(e) <= MIX_MED, (name, np.median(e))
            assert e.max() <= MIX_MAX, (name, e.max())
    return ea, ej, ep


@pytest.mark.parametrize("N,masses,eps", [(1000, "equal", 1 / 256), (1024, "equal", 1 / 256),
                                          (2500, "salpeter", 1 / 1024), (77, "salpeter", 0.01)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_ij_parity(nbl, N, masses, eps, prec):
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    m, x, v = inputs.plummer(N, 100 + N, masses)
    idx = np.arange(N)
    ref = oracle.forces(m, x, v, eps, compensated=True)
    got = gpu_forces(nbl, P, m, x, v, eps, idx)
    _check(P, nbl, got, ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [1, 2, 31, 256, 1000, 4097])
def test_active_subsets(nbl, prec, n):
    # ragged active blocks of a ragged N: exercises split-j and i-tile tails
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    N, eps = 6007, 1 / 512
    m, x, v = inputs.plummer(N, 7, "salpeter")
    idx = inputs.sample_indices(N, n, 8 + n)
    ref = oracle.forces(m, x, v, eps, idx=idx, compensated=True)
    got = gpu_forces(nbl, P, m, x, v, eps, idx)
    _check(P, nbl, got, ref)


def _supported(nb, prec):
    out = []
    thr = (64, 128, 256)
    if prec == nb.NB_FP64:
        for t in thr:
            for jt in (32, 64, 128):
                out.append(dict(i_per_thread=1, threads=t, j_tile=jt))
    else:
        for t in thr:
            for ipt in (1, 2, 4):
                for jt in (64, 128, 256):
                    out.append(dict(i_per_thread=ipt, threads=t, j_tile=jt))
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_every_tuning_and_split(nbl, prec):
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    N, eps = 3001, 1 / 256
    m, x, v = inputs.plummer(N, 11)
    idx = inputs.sample_indices(N, 700, 12)
    ref = oracle.forces(m, x, v, eps, idx=idx, compensated=True)
    for cfg in _supported(nbl, P):
        for split in (1, 3, 0):
            got = gpu_forces(nbl, P, m, x, v, eps, idx, tuning=dict(cfg, n_split=split))
            _check(P, nbl, got, ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_unsoftened(nbl, prec):
    # eps = 0: the self pair must be excluded exactly (index mask / r = 0 mask)
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    m, x, v = inputs.plummer(513, 21)
    ref = oracle.forces(m, x, v, 0.0, compensated=True)
    got = gpu_forces(nbl, P, m, x, v, 0.0, np.arange(513))
    ea, ej, ep = rel_vec(got[0], ref[0]), rel_vec(got[1], ref[1]), rel_scalar(got[2], ref[2])
    if P == nbl.NB_MIXED:
        print(f"eps=0 mixed: acc {np.median(ea):.2e}/{ea.max():.2e} jerk {np.median(ej):.2e}/{ej.max():.2e} "
              f"pot {np.median(ep):.2e}/{ep.max():.2e}")
    # the same bounds as every softened case: nothing is left unbounded
    _check(P, nbl, got, ref)


def test_two_body_values(nbl):
    # hand values (two-body pair at distance 5): acc = 2 (3,4,0)/125
    m = np.array([1.0, 2.0])
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    v = np.array([[0.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    for P, tol in ((nbl.NB_FP64, 1e-15), (nbl.NB_MIXED, 1e-6)):
        a, j, p = gpu_forces(nbl, P, m, x, v, 0.0, [0, 1])
        assert np.allclose(a[0], [0.048, 0.064, 0.0], rtol=tol, atol=tol * 0.1)
        assert abs(p[0] + 0.4) < tol and abs(p[1] + 0.2) < tol


def test_device_pointers_match_host(nbl):
    torch = pytest.importorskip("torch")
    N, eps = 4000, 1 / 256
    m, x, v = inputs.plummer(N, 31)
    idx = inputs.sample_indices(N, 1500, 32).astype(np.int32)
    for P in (nbl.NB_FP64, nbl.NB_MIXED):
        ah, jh, ph = gpu_forces(nbl, P, m, x, v, eps, idx)
        with nbl.NBody(N, P, 0, stream=torch.cuda.current_stream()) as s:
            s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            s.set_j_particles(0, dev(m), dev(x), dev(v))
            s.predict(0.0)
            a = torch.empty((len(idx), 3), dtype=torch.float64, device="cuda")
            j = torch.empty_like(a)
            p = torch.empty(len(idx), dtype=torch.float64, device="cuda")
            s.compute_forces(dev(idx), a, j, p)
            torch.cuda.synchronize()
            assert np.array_equal(a.cpu().numpy(), ah)
            assert np.array_equal(j.cpu().numpy(), jh)
            assert np.array_equal(p.cpu().numpy(), ph)


def test_deterministic(nbl):
    N, eps = 5000, 1 / 256
    m, x, v = inputs.plummer(N, 41)
    idx = inputs.sample_indices(N, 300, 42)
    for P in (nbl.NB_FP64, nbl.NB_MIXED):
        r1 = gpu_forces(nbl, P, m, x, v, eps, idx)
        r2 = gpu_forces(nbl, P, m, x, v, eps, idx)
        for a, b in zip(r1, r2):
            assert np.array_equal(a, b)


def test_bad_lists_rejected(nbl):
    N = 100
    m, x, v = inputs.plummer(N, 51)
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        s.set_j_particles(0, m, x, v)
        s.predict(0.0)
        for bad in ([3, 2], [0, 0], [-1], [100], list(range(101))):
            with pytest.raises(nbl.NBodyError) as e:
                s.compute_forces(np.array(bad, dtype=np.int32))
            assert e.value.code == nbl.NB_EINVAL
        # forces before any prediction of new data
        s.set_j_particles(0, m, x, v)
        with pytest.raises(nbl.NBodyError) as e:
            s.compute_forces(np.array([1, 2], dtype=np.int32))
        assert e.value.code == nbl.NB_ESTATE
        with pytest.raises(nbl.NBodyError) as e:
            s.set_params(-1.0, 0.01, 2.0 ** -22, 0.125)
        assert e.value.code == nbl.NB_EINVAL
        with pytest.raises(nbl.NBodyError):
            s.set_params(0.01, 0.01, 3e-7, 0.125)   # not a power of two
        bad_x = x.copy()
        bad_x[5, 1] = np.nan
        with pytest.raises(nbl.NBodyError):
            s.set_j_particles(0, m, bad_x, v)


def test_autotune_picks_a_supported_launch(nbl):
    # the autotuner times the supported launches for (N, n) and keeps the fastest
    N, eps, n = 20000, 1 / 512, 700
    m, x, v = inputs.plummer(N, 61)
    idx = inputs.sample_indices(N, n, 62)
    ref = oracle.forces(m, x, v, eps, idx=idx, compensated=True)
    for P in (nbl.NB_FP64, nbl.NB_MIXED):
        with nbl.NBody(N, P, 0) as s:
            s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
            s.set_j_particles(0, m, x, v)
            s.predict(0.0)
            cfg = s.autotune(n)
            assert cfg["threads"] in (64, 128, 256) and cfg["n_split"] >= 0  # 0 = automatic
            assert cfg["i_per_thread"] in ((1,) if P == nbl.NB_FP64 else (1, 2, 4))
            s.predict(0.0)
            got = s.compute_forces(idx.astype(np.int32))
        _check(P, nbl, got, ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_degenerate_sizes(nbl, prec):
    # one particle: no pair, zero force and potential; empty active list: no-op
    P = nbl.NB_FP64 if prec == "fp64" else nbl.NB_MIXED
    with nbl.NBody(4, P, 0) as s:
        s.set_params(0.01, 0.01, 2.0 ** -22, 2.0 ** -3)
        s.set_j_particles(0, np.array([1.0]), np.array([[0.1, 0.2, 0.3]]), np.array([[1.0, 0.0, 0.0]]))
        s.predict(0.0)
        a, j, p = s.compute_forces(np.array([0], dtype=np.int32))
        assert np.all(a == 0.0) and np.all(j == 0.0) and np.all(p == 0.0)
        a, j, p = s.compute_forces(np.zeros(0, dtype=np.int32))
        assert a.shape == (0, 3)
        s.initial_forces_and_dt()
        t, n = s.step()
        assert n == 1 and t == 2.0 ** -3


def test_far_tiles_off_is_strict(nbl):
    # configuration 3's softening on a 2^15-particle sphere: in spatial order
    # most (warp, j-tile) pairs pass the far test and take hi-only
    # differences; with nb_set_far_tiles(0) every difference is double-single.
    # Both stay within the mixed bounds, and the pass does change the bits.
    N, eps = 1 << 15, 1.0 / 4096
    m, x, v = inputs.plummer(N, 3)
    idx = inputs.sample_indices(N, 2048, 1003)
    ref = oracle.forces(m, x, v, eps, idx=idx, compensated=True)
    got = {}
    for far in (True, False):
        with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
            s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
            s.set_j_particles(0, m, x, v)
            s.set_far_tiles(far)
            assert s.get_far_tiles() == far
            s.predict(0.0)
            a, j, p = s.compute_forces(np.arange(N, dtype=np.int32))
        got[far] = (a[idx], j[idx], p[idx])
        ea, ej, ep = _check(nbl.NB_MIXED, nbl, got[far], ref)
        print(f"far tiles {far}: acc {np.median(ea):.2e}/{ea.max():.2e} jerk {np.median(ej):.2e}/{ej.max():.2e}")
    assert not np.array_equal(got[True][0], got[False][0])


def test_fp64_issue_probe_runs(nbl):
    # the FP64 issue probe returns positive cycle counts for every layout, and
    # one warp is not faster with one lane than with 32 (a whole-warp cost)
    with nbl.NBody(1024, nbl.NB_MIXED, 0) as s:
        r = s.measure_fp64_issue()
    assert all(np.isfinite(v) and v > 0 for v in r.values())
    assert r["dep1_cycles"] >= 0.9 * r["dep32_cycles"]
