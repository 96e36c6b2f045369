"""Full-size parity checks for the five workload configurations (Plummer
spheres of Sec. 2; sizes of the precision, batching and large-N runs), on
outputs the oracle computes one by one: sampled particles of a full i = j
force evaluation in the launch configuration the benchmark times.

Tolerances: FP64 GPU path <= 1e-12 (vs the compensated oracle); mixed path
median <= 1e-6 and max <= 1e-5 (vs the oracle) for acceleration, jerk and
potential.  These tests allocate up to ~2 GB of device memory.
"""
import numpy as np
import pytest

import oracle
from paper_0709_4552_gb300 import inputs
from _util import rel_scalar, rel_vec

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

MIX_MED, MIX_MAX = 1e-6, 1e-5


def _check_mixed(got, ref, label):
    for name, e in (("acc", rel_vec(got[0], ref[0])), ("jerk", rel_vec(got[1], ref[1])),
                    ("pot", rel_scalar(got[2], ref[2]))):
        print(f"{label} {name}: median {np.median(e):.2e} max {e.max():.2e}")
        assert np.median(e) <= MIX_MED, (label, name)
        assert e.max() <= MIX_MAX, (label, name)


def _check_fp64(got, ref, label):
    for name, e in (("acc", rel_vec(got[0], ref[0])), ("jerk", rel_vec(got[1], ref[1])),
                    ("pot", rel_scalar(got[2], ref[2]))):
        print(f"{label} {name}: max {e.max():.2e}")
        assert e.max() <= 1e-12, (label, name)


def _full_then_sample(nb, torch, s, N, idx):
    """Full i = j launch on device (the bench's launch), then the sampled rows."""
    ident = torch.arange(N, dtype=torch.int32, device="cuda")
    A = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    J = torch.empty_like(A)
    P = torch.empty(N, dtype=torch.float64, device="cuda")
    s.compute_forces(ident, A, J, P)
    torch.cuda.synchronize()
    ii = torch.from_numpy(idx).cuda()
    return A[ii].cpu().numpy(), J[ii].cpu().numpy(), P[ii].cpu().numpy()


def test_config2_full_ij_fp64(nbl):
    # N = 196608 Salpeter, eps = 1/1024: one full i = j FP64 evaluation, 4096 sampled rows
    torch = pytest.importorskip("torch")
    N, eps = 196608, 1.0 / 1024
    m, x, v = inputs.plummer(N, 2, "salpeter")
    idx = inputs.sample_indices(N, 4096, 1002)
    ref = oracle.forces(m, x, v, eps, idx=idx, compensated=True)
    with nbl.NBody(N, nbl.NB_FP64, 0) as s:
        s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
        s.set_j_particles(0, m, x, v)
        s.predict(0.0)
        got = _full_then_sample(nbl, torch, s, N, idx)
    _check_fp64(got, ref, "config2 fp64")


@pytest.mark.parametrize("n_active", [256, 4096, 65536, 1 << 20])
def test_config3_active_blocks(nbl, n_active):
    # N = 2^20 equal masses, eps = 1/4096: mixed path on active blocks of the
    # sweep (the first n of a seeded shuffle), FP64 GPU path on the sample
    torch = pytest.importorskip("torch")
    N, eps = 1 << 20, 1.0 / 4096
    m, x, v = inputs.plummer(N, 3)
    act = inputs.sample_indices(N, n_active, 1003).astype(np.int32)
    pos = inputs.sample_indices(n_active, min(n_active, 2048), 2003)
    idx = act[pos]
    ref = oracle.forces(m, x, v, eps, idx=idx.astype(np.int64), compensated=True)
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        s.set_params(eps, 0.01, 2.0 ** -10, 2.0 ** -10)
        s.set_j_particles(0, m, x, v)
        s.predict(0.0)
        A = torch.empty((n_active, 3), dtype=torch.float64, device="cuda")
        J = torch.empty_like(A)
        P = torch.empty(n_active, dtype=torch.float64, device="cuda")
        s.compute_forces(torch.from_numpy(act).cuda(), A, J, P)
        torch.cuda.synchronize()
        pp = torch.from_numpy(pos).cuda()
        got = (A[pp].cpu().numpy(), J[pp].cpu().numpy(), P[pp].cpu().numpy())
        _check_mixed(got, ref, f"config3 mixed n={n_active}")
        if n_active == 4096:
            s.set_precision(nbl.NB_FP64)
            s.predict(0.0)
            _check_fp64(s.compute_forces(idx), ref, "config3 fp64 sample")


def test_config5_full_ij_mixed(nbl):
    # N = 4,194,304 Salpeter, eps = 1/8192: one full i = j mixed evaluation, 2048 sampled rows
    torch = pytest.importorskip("torch")
    N, eps = 1 << 22, 1.0 / 8192
    m, x, v = inputs.plummer(N, 5, "salpeter")
    idx = inputs.sample_indices(N, 2048, 1005)
    ref = oracle.forces(m, x, v, eps, idx=idx, compensated=True)
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -6)
        s.set_j_particles(0, m, x, v)
        s.predict(0.0)
        got = _full_then_sample(nbl, torch, s, N, idx)
    _check_mixed(got, ref, "config5 mixed")


def test_config4_ensemble_initial_forces(nbl):
    # 512 clusters, N_c log-uniform in [256, 16384] (seed 7), Salpeter, eps_c = 1/(4 N_c^(1/3));
    # batched initial forces of every cluster, 16 seeded clusters checked row by row
    sizes = inputs.ensemble_sizes(512, 256, 16384, seed=7)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    eps = 1.0 / (4.0 * sizes.astype(np.float64) ** (1.0 / 3.0))
    parts = [inputs.plummer(int(n), 10000 + q, "salpeter") for q, n in enumerate(sizes)]
    m = np.concatenate([p[0] for p in parts])
    x = np.concatenate([p[1] for p in parts])
    v = np.concatenate([p[2] for p in parts])
    pick = np.sort(np.random.default_rng(77).choice(512, 16, replace=False))
    with nbl.Ensemble(off, eps, nbl.NB_MIXED, 0) as e:
        e.set_params(0.01, 0.01, 2.0 ** -22, 2.0 ** -4)
        e.set_j_particles(0, m, x, v)
        e.initial_forces_and_dt()
        st = e.get_particles(0, int(off[-1]))
    for q in pick:
        a, b = off[q], off[q + 1]
        k = inputs.sample_indices(int(b - a), 64, 3000 + int(q))
        ref = oracle.forces(m[a:b], x[a:b], v[a:b], eps[q], idx=k, compensated=True)
        got = (st["a"][a:b][k], st["jerk"][a:b][k], st["pot"][a:b][k])
        _check_mixed(got, ref, f"config4 cluster {q} (N={b - a})")
