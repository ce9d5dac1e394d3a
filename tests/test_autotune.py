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


def test_load_signature_groups_logs_of_about_the_same_shape():
    a = autotune.load_signature(206_571_951, 10_000_000, 500, True, 1000, "B300")
    b = autotune.load_signature(200_000_000, 9_500_000, 480, True, 10, "B300")
    c = autotune.load_signature(206_571_951, 10_000_000, 500, False, 1000, "B300")
    d = autotune.load_signature(20_000_000, 1_000_000, 500, True, 1000, "B300")
    assert a == b
    assert a != c  # row order selects the segment pass
    assert a != d
    assert a.startswith("load|") and a != autotune.signature(206_571_951, 10_000_000, 500, 1, 1, 1, "B300")


def test_load_space_descent_from_the_defaults():
    target = {"clb": 7, "splits": 4, "stream_warps": 16, "stream_off": 0, "edge_table": 0, "part1_items": 4,
              "part2_items": 0, "part_fbits": 9}

    def cost(c):
        return sum((autotune.LOAD_SPACE[k].index(c[k]) - autotune.LOAD_SPACE[k].index(target[k])) ** 2
                   for k in c) + 2.0

    best, t, trials = autotune.coordinate_descent(cost, autotune.LOAD_SPACE, autotune.LOAD_DEFAULTS)
    assert best == target and t == 2.0
    assert trials[0][0] == autotune.LOAD_DEFAULTS  # the defaults are measured first
    assert set(best) == set(autotune.LOAD_KNOBS)


def test_load_choices_are_cached_apart_from_batch_choices(tmp_path):
    tuner = autotune.Tuner(cache_path=str(tmp_path / "t.json"))
    sig = autotune.load_signature(20_000_000, 1_000_000, 50, False, 1000, "B300")
    choice = tuner.tune(sig, lambda c: 1.0 + c["stream_off"] + c["clb"] / 100, autotune.LOAD_SPACE,
                        autotune.LOAD_DEFAULTS)
    assert choice["stream_off"] == 0 and choice["clb"] == 0
    reloaded = autotune.Tuner(cache_path=str(tmp_path / "t.json"))
    assert reloaded.tune(sig, lambda c: (_ for _ in ()).throw(AssertionError("measured again"))) == choice
