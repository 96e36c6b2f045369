"""Binary snapshot format (host logic, no GPU): round trip, and rejection of
damaged files."""
import numpy as np
import pytest

from paper_0709_4552_gb300 import inputs, snapshot


def _state(N, seed):
    rng = np.random.default_rng(seed)
    m, x, v = inputs.plummer(N, seed)
    return dict(m=m, x=x, v=v, a=rng.normal(size=(N, 3)), jerk=rng.normal(size=(N, 3)),
                pot=-rng.random(N), t=np.full(N, 0.125), dt=2.0 ** -rng.integers(3, 22, N))


def test_round_trip_is_exact(tmp_path):
    st = _state(1000, 3)
    p = tmp_path / "s.nbs"
    snapshot.write(p, st, 1 / 256, 0.01, 2.0 ** -22, 2.0 ** -3)
    got, prm = snapshot.read(p)
    for k in st:
        assert np.array_equal(got[k], st[k]), k
    assert prm == dict(t_sys=0.125, eps=1 / 256, eta=0.01, dt_min=2.0 ** -22, dt_max=2.0 ** -3)
    assert p.stat().st_size == 8 + 8 + 5 * 8 + 8 * 1000 * (1 + 3 * 4 + 3)


def test_empty_state(tmp_path):
    st = {k: np.zeros((0, 3) if k in ("x", "v", "a", "jerk") else 0) for k in
          ("m", "x", "v", "a", "jerk", "pot", "t", "dt")}
    p = tmp_path / "e.nbs"
    snapshot.write(p, st, 0.0, 0.01, 2.0 ** -22, 2.0 ** -3)
    got, _ = snapshot.read(p)
    assert got["x"].shape == (0, 3)


@pytest.mark.parametrize("damage", ["magic", "truncate", "trailing"])
def test_damaged_files_rejected(tmp_path, damage):
    st = _state(64, 4)
    p = tmp_path / "d.nbs"
    snapshot.write(p, st, 1 / 256, 0.01, 2.0 ** -22, 2.0 ** -3)
    raw = bytearray(p.read_bytes())
    if damage == "magic":
        raw[0:8] = b"NOTSNAP!"
    elif damage == "truncate":
        raw = raw[:-8]
    else:
        raw += b"\0"
    p.write_bytes(bytes(raw))
    with pytest.raises(ValueError):
        snapshot.read(p)


def test_wrong_field_size_rejected(tmp_path):
    st = _state(10, 5)
    st["v"] = st["v"][:9]
    with pytest.raises(ValueError):
        snapshot.write(tmp_path / "w.nbs", st, 1 / 256, 0.01, 2.0 ** -22, 2.0 ** -3)
