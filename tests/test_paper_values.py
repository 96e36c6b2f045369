"""The few method constants the paper prints (tests/golden/paper_values.json,
each with its citation) against the input generator's helpers."""
import json
import os

from paper_0709_4552_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_block_size_law():
    c, e = GOLD["block_size_law"]["coef"], GOLD["block_size_law"]["exponent"]
    for N in (1024, 32768, 196608, 1 << 20):
        assert inputs.block_size(N) == max(1, int(round(c * N ** e)))
    # Sec. 3.2 law at the largest N run in the paper
    assert 3000 < inputs.block_size(GOLD["n_max_run"]["value"]) < 4500


def test_time_step_bounds_are_powers_of_two():
    assert GOLD["dt_min"]["value"] == 2.0 ** -22
    assert GOLD["dt_max"]["value"] == 2.0 ** -3
    assert GOLD["softening"]["value"] == 2.0 ** -8
