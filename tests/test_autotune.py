"""The batched drill-down's autotuner on the CPU: the search finds the
minimum of cost functions with a known optimum, a cached choice is reused
without measuring, the cache survives a reload from its file, and workload
signatures group batches of about the same shape."""

import itertools

import pytest

from paper_2204_04898_b300 import autotune


def _grid_min(cost, space):
    keys = list(space)
    best = min(itertools.product(*(space[k] for k in keys)), key=lambda v: cost(dict(zip(keys, v))))
    return dict(zip(keys, best))


@pytest.mark.parametrize("target", [{"chunk": 32, "items_per_sm": 2, "stages": 8},
                                    {"chunk": 8, "items_per_sm": 8, "stages": 1},
                                    {"chunk": 16, "items_per_sm": 4, "stages": 4}])
def test_descent_finds_separable_optimum(target):
    def cost(c):
        return sum((c[k] - target[k]) ** 2 for k in c) + 1.0

    best, t, trials = autotune.coordinate_descent(cost)
    assert best == target == _grid_min(cost, autotune.SPACE)
    assert t == 1.0
    assert len(trials) < 3 * 4 * 3  # fewer than the full grid


def test_descent_with_interaction_reaches_a_coordinate_minimum():
    # cost with an interaction term: the result must not improve along any axis
    def cost(c):
        return abs(c["chunk"] * c["items_per_sm"] - 64) + abs(c["stages"] - 2) + 0.01 * c["chunk"]

    best, t, _ = autotune.coordinate_descent(cost)
    for knob, values in autotune.SPACE.items():
        for v in values:
            assert cost({**best, knob: v}) >= t


def test_cache_is_used_and_persisted(tmp_path):
    path = str(tmp_path / "tune.json")
    tuner = autotune.Tuner(cache_path=path)
    sig = autotune.signature(206_571_951, 10_000_000, 500, 4096, 664_362_650, 1000, "B300")
    calls = []

    def measure(c):
        calls.append(c)
        return c["chunk"] / 16 + c["stages"] / 4 + c["items_per_sm"] / 4

    choice = tuner.tune(sig, measure)
    assert choice == {"chunk": 8, "items_per_sm": 2, "stages": 1}
    n = len(calls)

    def never(c):
        raise AssertionError("a cached choice must not be measured again")

    assert tuner.tune(sig, never) == choice and len(calls) == n
    again = autotune.Tuner(cache_path=path)
    assert again.tune(sig, never) == choice


def test_signature_groups_close_shapes():
    a = autotune.signature(100_000_000, 4_850_000, 2000, 4096, 664_000_000, 1000, "B300")
    b = autotune.signature(101_000_000, 4_900_000, 2000, 4096, 650_000_000, 1000, "B300")
    c = autotune.signature(100_000_000, 4_850_000, 2000, 64, 10_000_000, 1000, "B300")
    d = autotune.signature(100_000_000, 4_850_000, 2000, 4096, 664_000_000, 0, "B300")
    assert a == b and a != c and a != d
