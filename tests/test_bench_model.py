"""The Sec. 4.1 performance model as the bench evaluates it (bench.sec41_taus,
bench.sec41_T): Eq. 1 T_integrate = sum over block steps of (t_pred + t_force
+ t_corr), with t_pred = tau_pred N (Eq. 2), t_force = tau_force n N (Eq. 3)
and t_corr = tau_corr n (Eq. 4), checked against the step-by-step sum on the
paper's own machine constants (tests/golden/paper_values.json)."""
import json
import os

import numpy as np
import pytest

import bench
from paper_0709_4552_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _steps(N, k, seed):
    # a block-size sequence around the Sec. 3.2 law n = 0.20 N^0.81
    rng = np.random.default_rng(seed)
    n0 = inputs.block_size(N)
    return np.clip(rng.integers(1, 2 * n0, size=k), 1, N)


@pytest.mark.parametrize("machine", ["vader", "yoda", "obi-wan"])
def test_eq1_matches_the_step_by_step_sum(machine):
    N = GOLD["model_calibration_N"]["value"]
    taus = tuple(GOLD[f"tau_{q}_cpu_us"][machine] * 1e-6 for q in ("pred", "force", "corr"))
    ns = _steps(N, 500, 7)
    direct = 0.0
    for n in ns:   # Eq. 1 term by term
        direct += taus[0] * N + taus[1] * n * N + taus[2] * n
    inter, psteps = float(ns.sum()) * N, float(ns.sum())
    assert bench.sec41_T(taus, N, len(ns), inter, psteps) == pytest.approx(direct, rel=1e-12)
    # the force term dominates a single PC (Sec. 3.1): n N tau_force >> N tau_pred + n tau_corr
    assert taus[1] * inter > 10 * (taus[0] * N * len(ns) + taus[2] * psteps)


def test_taus_invert_the_phase_times():
    N, steps = 196608, 321
    ns = _steps(N, steps, 9)
    taus = (1.5e-10, 9.4e-13, 2.1e-9)
    inter, psteps = float(ns.sum()) * N, float(ns.sum())
    t_pred, t_force, t_corr = taus[0] * N * steps, taus[1] * inter, taus[2] * psteps
    got = bench.sec41_taus(t_pred, t_force, t_corr, N, steps, inter, psteps)
    assert np.allclose(got, taus, rtol=1e-14)
    assert bench.sec41_T(got, N, steps, inter, psteps) == pytest.approx(t_pred + t_force + t_corr, rel=1e-14)


def test_grape_tau_force_against_a_pc():
    # GRAPE-6Af's 4.3e-10 s per interaction against the PCs' tau_force (Sec. 4.1,
    # Sec. 4.4): the accelerator is 250-500x faster per interaction
    g = GOLD["tau_grape_force_s"]["value"]
    for machine, us in GOLD["tau_force_cpu_us"].items():
        if machine == "cite":
            continue
        assert 200 < us * 1e-6 / g < 600
