"""Planted mistakes in copies of the oracle (CPU only): each must fail a pin.

The mistakes are the plausible ones: a dropped tie-break, a transposed edge, a
wrong duration sign, a 64-bit sum, a swapped min/max, wrong end activity,
reversed variant orders, unsigned case ordering, a filter boundary, the case
attribute read at the wrong event, a path across cases or reversed, an open
size bound, a throughput time from the wrong event, the end set read at the
first event, an activity test that skips the last event, eventually-follows
pairs reversed or including an event with itself, a dropped carry in the sums
of squares, a sample instead of a population variance, a truncated mean. The
pristine oracle passes every pin."""

import pytest

import oracle
from tests import oracle_pins as pins

MUTANTS = {
    "no_row_tiebreak": ("std::make_tuple(case_id[a], ts[a], a) < std::make_tuple(case_id[b], ts[b], b)",
                        "std::make_tuple(case_id[a], ts[a], -a) < std::make_tuple(case_id[b], ts[b], -b)"),
    "edge_transposed": ("dfg[std::make_pair(act[x], act[y])]", "dfg[std::make_pair(act[y], act[x])]"),
    "duration_sign": ("(uint64_t)ts[y] - (uint64_t)ts[x]", "(uint64_t)ts[x] - (uint64_t)ts[y]"),
    "sum_64bit": ("g.sum += (u128)delta;", "g.sum = (uint64_t)(g.sum + (u128)delta);"),
    "min_is_max": ("g.min = std::min(g.min, delta);", "g.min = std::max(g.min, delta);"),
    "end_is_start": ("R.end[act[s[e - 1]]] += 1;", "R.end[act[s[b]]] += 1;"),
    "variant_count_ascending": ("return a.second.count > b.second.count;",
                                "return a.second.count < b.second.count;"),
    "variant_min_case_descending": ("return a.second.min_case < b.second.min_case;",
                                    "return a.second.min_case > b.second.min_case;"),
    "unsigned_case_order": ("std::make_tuple(case_id[a], ts[a], a) < std::make_tuple(case_id[b], ts[b], b)",
                            "std::make_tuple((uint32_t)case_id[a], ts[a], a) < std::make_tuple((uint32_t)case_id[b], ts[b], b)"),
    "mean_from_truncated_sum": ("mean[k] = (double)e.second.sum / (double)e.second.count;",
                                "mean[k] = (double)(uint64_t)e.second.sum / (double)e.second.count;"),
    "contained_open_bound": ("case_ok = first >= t_lo && last <= t_hi;",
                             "case_ok = first > t_lo && last <= t_hi;"),
    "attr_at_last_event": ("const int32_t v = attr[s[b]];", "const int32_t v = attr[s[e - 1]];"),
    "freq_skips_last": ("for (int64_t i = b; i < e; ++i) R.freq[act[s[i]]] += 1;",
                        "for (int64_t i = b; i + 1 < e; ++i) R.freq[act[s[i]]] += 1;"),
    "min_case_not_min": ("it->second.min_case = std::min(it->second.min_case, R.case_ids[c]);",
                         "it->second.min_case = std::max(it->second.min_case, R.case_ids[c]);"),
    "path_crosses_cases": ("if (i > 0 && case_id[s[i - 1]] == case_id[s[i]]) {", "if (i > 0) {"),
    "path_reversed": ("const std::pair<int32_t, int32_t> p(act[s[i - 1]], act[s[i]]);",
                      "const std::pair<int32_t, int32_t> p(act[s[i]], act[s[i - 1]]);"),
    "size_bound_open": ("if (min_events >= 0 && len < min_events) ok = false;",
                        "if (min_events >= 0 && len <= min_events) ok = false;"),
    "duration_from_second_event": ("const uint64_t dur = (uint64_t)ts[s[e - 1]] - (uint64_t)ts[s[b]];",
                                   "const uint64_t dur = (uint64_t)ts[s[e - 1]] - (uint64_t)ts[s[b + (e - b > 1)]];"),
    "end_set_reads_first": ("if (n_end > 0 && !in(end_set, n_end, act[s[e - 1]])) ok = false;",
                            "if (n_end > 0 && !in(end_set, n_end, act[s[b]])) ok = false;"),
    "ef_reversed": ("EfAgg &g = (*M)[std::make_pair(act[s[i]], act[s[j]])];",
                    "EfAgg &g = (*M)[std::make_pair(act[s[j]], act[s[i]])];"),
    "ef_self_pairs": ("for (int64_t j = i + 1; j < e; ++j) {", "for (int64_t j = i; j < e; ++j) {"),
    "ef_square_carry_dropped": ("          carry = t >> 64;\n        }\n      }", "          carry = 0;\n        }\n      }"),
    "ef_sample_variance": ("/ (double)g.count / (double)g.count;",
                           "/ (double)g.count / (double)(g.count > 1 ? g.count - 1 : 1);"),
    "ef_mean_truncated": ("mean[k] = (double)g.sum / (double)g.count;\n    const U256",
                          "mean[k] = (double)(uint64_t)(g.sum / g.count);\n    const U256"),
    "contains_skips_last": ("for (int64_t i = b; i < e; ++i) any = any || in(act_set, n_act, act[s[i]]);",
                            "for (int64_t i = b; i + 1 < e; ++i) any = any || in(act_set, n_act, act[s[i]]);"),
}


def test_pristine_oracle_passes_all_pins(oracle_lib):
    pins.run_all(oracle_lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    frm, to = MUTANTS[name]
    lib = oracle.load(oracle.mutant_library(frm, to))
    with pytest.raises(AssertionError):
        pins.run_all(lib)
