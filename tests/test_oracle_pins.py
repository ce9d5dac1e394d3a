"""The CPU oracle against its pins (no GPU): brute force, invariants, closed
forms, replication, shuffles, ties, special cases, filters, golden fixtures."""

import numpy as np
import pytest

import oracle
import pm4g_synth as synth
from tests import oracle_pins as pins


def test_bruteforce_exhaustive(oracle_lib):
    # 12 distinct rows -> 1 + 12 + 144 + 1728 + 20736 logs
    assert pins.check_bruteforce_exhaustive(oracle_lib, max_n=4) == 22621


def test_bruteforce_random_extremes(oracle_lib):
    pins.check_bruteforce_random(oracle_lib, n_logs=800)


def test_tie_swap(oracle_lib):
    pins.check_tie_swap(oracle_lib)


def test_special_cases(oracle_lib):
    pins.check_specials(oracle_lib)


def test_big_durations(oracle_lib):
    pins.check_big_durations(oracle_lib)


@pytest.mark.parametrize("name", ["fine_process_example.json", "signed_ties_example.json"])
def test_golden(oracle_lib, name):
    pins.check_golden(oracle_lib, name)


@pytest.fixture(scope="module")
def logs():
    return pins.small_logs()


def test_invariants_and_closed_form(oracle_lib, logs):
    for log in logs:
        R = pins.check_invariants(oracle_lib, log)
        pins.check_closed_form_sums(oracle_lib, log, R)


def test_replication(oracle_lib, logs):
    for log in logs:
        pins.check_replication(oracle_lib, log, k=3)


def test_shuffle_without_ties(oracle_lib):
    log = synth.generate(synth.single_log(3000))  # exponential gaps: no ties
    pins.check_shuffle(oracle_lib, log)


def test_filters(oracle_lib, logs):
    for log in logs:
        pins.check_filters(oracle_lib, log)
    pins.check_filters_bruteforce(oracle_lib, n_logs=400)


def test_derived_filters(oracle_lib, logs):
    """Paths and case filters: the hand-derived fixture, the definitions on
    random tiny logs, and identities on workload-shaped logs."""
    pins.check_golden_filters(oracle_lib, "filters_fine_process.json")
    pins.check_derived_filters_bruteforce(oracle_lib, n_logs=400)
    for log in logs:
        pins.check_derived_filters(oracle_lib, log)


def test_efg(oracle_lib, logs):
    """Eventually-follows graph and temporal profile: the hand-derived
    fixture, the definition on random tiny logs (exact integer moments, means
    and deviations within a few units in the last place of exact references),
    identities on workload-shaped logs."""
    pins.check_golden_efg(oracle_lib, "efg_fine_process.json")
    pins.check_efg_bruteforce(oracle_lib, n_logs=400)
    for log in logs[:2]:
        pins.check_efg_invariants(oracle_lib, log)


def test_filter_then_summarize_keeps_tie_order(oracle_lib):
    # the sub-log keeps original rows, so ties inside a case resolve as before
    case = [1, 1, 1, 2, 2]
    act = [0, 1, 2, 0, 1]
    ts = [5, 5, 9, 3, 3]
    attr = [4, 4, 4, 6, 6]
    rows = oracle.filter_rows(case, act, ts, attr, 3, [4], 0, 100, oracle.TW_NONE)
    assert rows.tolist() == [0, 1, 2]
    R = oracle.summarize(np.array(case)[rows], np.array(act)[rows], np.array(ts)[rows], 3)
    assert R.variant_seqs() == [(0, 1, 2)]


def test_workload_scale_invariants(oracle_lib):
    log = synth.generate(synth.large_log(20000))
    R = pins.check_invariants(oracle_lib, log)
    pins.check_closed_form_sums(oracle_lib, log, R)
