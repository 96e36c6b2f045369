"""The autotuner as part of the path: nb_autotune (the host-driven force
launch, binned by N and n) and nb_ensemble_autotune (the item shape of the
device-driven loops and ensembles, binned by median cluster size and cluster
count), the table in a JSON file (nb_tune_save / nb_tune_load / NB_TUNE_FILE),
and the integrations under a tuned table against the oracle."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_0709_4552_gb300 import inputs

pytestmark = pytest.mark.gpu


def _ensemble_ics(sizes, seed):
    ms, xs, vs, eps = [], [], [], []
    for q, n in enumerate(sizes):
        m, x, v = inputs.plummer(int(n), seed + q, "salpeter")
        ms.append(m)
        xs.append(x)
        vs.append(v)
        eps.append(1.0 / (4.0 * n ** (1.0 / 3.0)))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return off, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), np.array(eps)


def _ens(nb, prec, off, m, x, v, eps, t_end):
    e = nb.Ensemble(off, eps, prec, 0)
    e.set_params(0.01, 0.01, 2.0 ** -22, t_end)
    e.set_j_particles(0, m, x, v)
    e.initial_forces_and_dt()
    return e


def test_table_file_round_trip(nbl, tmp_path, monkeypatch):
    monkeypatch.setenv("NB_TUNE_FILE", "")   # no shipped table: the contexts start empty
    N = 20000
    m, x, v = inputs.plummer(N, 51)
    path1, path2 = str(tmp_path / "t1.json"), str(tmp_path / "t2.json")
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        s.set_j_particles(0, m, x, v)
        s.predict(0.0)
        cfg = s.autotune(700)
        assert s.tune_count() == 1
        nbl.nb_tune_save(s.ctx, path1)
    doc = json.load(open(path1))
    assert doc["format"] == "libnbody tuning table 1" and len(doc["entries"]) == 1
    ent = doc["entries"][0]
    assert ent["kind"] == "single" and ent["precision"] == "mixed"
    assert ent["N_lo"] <= N < ent["N_hi"] and ent["n_lo"] <= 700 < ent["n_hi"]
    assert (ent["i_per_thread"], ent["threads"], ent["j_tile"], ent["n_split"]) == \
        (cfg["i_per_thread"], cfg["threads"], cfg["j_tile"], cfg["n_split"])
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        assert s.tune_count() == 0
        nbl.nb_tune_load(s.ctx, path1)
        assert s.tune_count() == 1
        nbl.nb_tune_save(s.ctx, path2)
    assert json.load(open(path2)) == doc
    # the environment variable is read when a context is made
    monkeypatch.setenv("NB_TUNE_FILE", path1)
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        assert s.tune_count() == 1


def test_autotune_on_a_caller_list(nbl, monkeypatch):
    # nb_autotune_list times the shapes on the caller's (scattered) block; the
    # entry lands in the table and the tuned forces on that block match the oracle
    monkeypatch.setenv("NB_TUNE_FILE", "")
    torch = pytest.importorskip("torch")
    N, n, eps = 20000, 300, 1.0 / 256
    m, x, v = inputs.plummer(N, 52)
    idx = inputs.sample_indices(N, n, 9).astype(np.int32)
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
        s.set_j_particles(0, m, x, v)
        s.predict(0.0)
        for lst in (idx, torch.from_numpy(idx).cuda()):   # host and device lists
            cfg = s.autotune_list(lst)
            assert cfg["threads"] in (64, 128, 256) and cfg["j_tile"] in (64, 128, 256)
            assert cfg["i_per_thread"] in (1, 2, 4) and 0 <= cfg["n_split"] <= 4096
        assert s.tune_count() == 1   # the same (N, n) bin, replaced
        a, j, p = s.compute_forces(idx)
    ref = oracle.forces(m, x, v, eps, idx=idx.astype(np.int64), compensated=True)
    ea = np.linalg.norm(a - ref[0], axis=1) / np.linalg.norm(ref[0], axis=1)
    ej = np.linalg.norm(j - ref[1], axis=1) / np.linalg.norm(ref[1], axis=1)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5
    assert np.median(ej) <= 1e-6 and ej.max() <= 1e-5
    assert np.abs(p - ref[2]).max() / np.abs(ref[2]).min() <= 1e-5
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:   # a list out of order is refused
        s.set_j_particles(0, m, x, v)
        s.predict(0.0)
        with pytest.raises(nbl.NBodyError):
            s.autotune_list(idx[::-1].copy())


@pytest.mark.parametrize("n", [1, 33, 2000])
def test_autotune_list_edge_sizes(nbl, monkeypatch, n):
    # one particle, a ragged warp, the whole system: a supported launch comes
    # back and the tuned forces still match the oracle
    monkeypatch.setenv("NB_TUNE_FILE", "")
    N, eps = 2000, 1.0 / 256
    m, x, v = inputs.plummer(N, 53)
    idx = (np.arange(N) if n == N else inputs.sample_indices(N, n, 10)).astype(np.int32)
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        s.set_params(eps, 0.01, 2.0 ** -22, 2.0 ** -3)
        s.set_j_particles(0, m, x, v)
        s.predict(0.0)
        cfg = s.autotune_list(idx)
        assert cfg["threads"] in (64, 128, 256) and 0 <= cfg["n_split"] <= 4096
        a, j, p = s.compute_forces(idx)
    ref = oracle.forces(m, x, v, eps, idx=idx.astype(np.int64), compensated=True)
    ea = np.linalg.norm(a - ref[0], axis=1) / np.linalg.norm(ref[0], axis=1)
    assert np.median(ea) <= 1e-6 and ea.max() <= 1e-5


def test_table_refuses_foreign_or_broken_files(nbl, tmp_path, monkeypatch):
    monkeypatch.setenv("NB_TUNE_FILE", "")
    with nbl.NBody(1000, nbl.NB_MIXED, 0) as s:
        good = {"format": "libnbody tuning table 1", "device": "x", "sm_count": 0, "entries": []}
        bad_sm = str(tmp_path / "sm.json")
        json.dump(dict(good, sm_count=1), open(bad_sm, "w"))
        broken = str(tmp_path / "broken.json")
        open(broken, "w").write('{"format": "libnbody tuning table 1", "entries": [')
        for p in (bad_sm, broken, str(tmp_path / "missing.json")):
            with pytest.raises(nbl.NBodyError) as err:
                nbl.nb_tune_load(s.ctx, p)
            assert err.value.code == nbl.NB_EINVAL
        assert s.tune_count() == 0


def test_shipped_table_loads(nbl):
    # the package's GB300 table (when present) is what a new context starts from
    from paper_0709_4552_gb300 import nbody
    if not os.path.exists(nbody.DEFAULT_TUNE_FILE) or os.environ.get("NB_TUNE_FILE") != nbody.DEFAULT_TUNE_FILE:
        pytest.skip("no shipped table in use")
    doc = json.load(open(nbody.DEFAULT_TUNE_FILE))
    with nbl.NBody(1000, nbl.NB_MIXED, 0) as s:
        assert s.tune_count() == len(doc["entries"])


def test_ensemble_autotune_restores_the_state(nbl):
    sizes = [300, 90, 700, 128, 1000]
    off, m, x, v, eps = _ensemble_ics(sizes, 710)
    N = int(off[-1])
    with _ens(nbl, nbl.NB_MIXED, off, m, x, v, eps, 2.0 ** -5) as e:
        e.tune_clear()
        before = e.get_particles(0, N)
        c0 = e.get_counters()
        res = e.autotune(8)
        assert res["i_tile"] in (32, 64, 128) and res["item_waves"] in (2, 4, 8, 16)
        assert 0 < res["ms_best"] <= res["ms_default"]
        assert e.tune_count() == 1
        after = e.get_particles(0, N)
        assert e.get_counters()["block_steps"] == c0["block_steps"]
    for k in ("x", "v", "a", "jerk", "t", "dt"):
        assert np.array_equal(before[k], after[k]), k


def test_ensemble_matches_oracle_under_tuned_table(nbl):
    # the FP64 ensemble of the oracle test, integrated with the tuned item shape
    sizes = [300, 90, 700, 128]
    off, m, x, v, eps = _ensemble_ics(sizes, 700)
    t_end = 2.0 ** -5
    N = int(off[-1])
    with _ens(nbl, nbl.NB_FP64, off, m, x, v, eps, t_end) as e:
        res = e.autotune(8)
        e.integrate(t_end)
        st = e.get_particles(0, N)
    print("tuned shape", res)
    for q in range(len(sizes)):
        a, b = off[q], off[q + 1]
        r = oracle.hermite_run(m[a:b], x[a:b], v[a:b], eps[q], 0.01, 2.0 ** -22, t_end, t_end, compensated=True)
        assert np.array_equal(st["dt"][a:b], r["dt"])
        assert np.abs(st["x"][a:b] - r["x"]).max() < 1e-11


def test_graph_loop_under_tuned_table(nbl):
    # one system's graph loop tuned the same way; mixed drift within 2x the oracle's
    N, eps, t_end = 2048, 1 / 256, 2.0 ** -4
    m, x, v = inputs.plummer(N, 811, "salpeter")
    with nbl.NBody(N, nbl.NB_MIXED, 0) as s:
        s.set_params(eps, 0.01, 2.0 ** -22, t_end)
        s.set_j_particles(0, m, x, v)
        s.initial_forces_and_dt()
        res = nbl.nb_ensemble_autotune(s.ctx, 8)
        assert res["i_tile"] in (32, 64, 128)
        k0, w0 = s.energy()
        s.integrate(t_end, use_graph=True)
        k1, w1 = s.energy()
        st = s.get_particles(0, N)
    assert np.all(st["t"] == t_end)
    E0 = sum(oracle.energy(m, x, v, eps))
    r = oracle.hermite_run(m, x, v, eps, 0.01, 2.0 ** -22, t_end, t_end)
    d_orc = abs(sum(oracle.energy(m, r["x"], r["v"], eps)) - E0) / abs(E0)
    d_gpu = abs((k1 + w1) - (k0 + w0)) / abs(k0 + w0)
    assert d_gpu <= 2 * d_orc + 1e-9, (d_gpu, d_orc)
