"""Planted mistakes in the CPU reference must fail its pins.

Each case copies the reference source, plants one plausible mistake, builds
it on the CPU and checks that the pin meant to guard that spot now fails.
"""
import contextlib
import os
import subprocess

import numpy as np
import pytest

from golden import fixtures
from paper_1711_04556_gb300.instances import Instance

import test_oracle_pins as pins

MUTANTS = {
    # the loop bound printed in Algs. 5-6 (reading R1 replaces it)
    "alg5_alg6_k_lt_M_minus_1": ("for (int k = 0; k < M; ++k)                          /* reading R1 */",
                                 "for (int k = 0; k < M - 1; ++k)"),
    # Eq. 6 range shortened by one position
    "eq6_short_range": ("for (int x = u; x <= v - 1; ++x)", "for (int x = u; x <= v - 2; ++x)"),
    # Alg. 4 line "timeDiff = newTime - max(c, s)" without the max
    "alg4_no_max_with_s": ("int timeDiff = newTime - imax(c[resIdx], s);", "int timeDiff = newTime - c[resIdx];"),
    # Alg. 4 shifted copy taken one element late
    "alg4_copy_offset": ("if (copyIdx >= r) newTime", "if (copyIdx > r) newTime"),
    # Eq. 4 with closed intervals: an activity still uses its resources at its finish time
    "checker_closed_interval": ("if (S[i] <= t && t < S[i] + in->dur[i]) used",
                                "if (S[i] <= t && t <= S[i] + in->dur[i]) used"),
    # Eq. 3 refusing a successor that starts exactly at its predecessor's finish
    "checker_strict_precedence": ("if (S[in->succ[e]] < S[i] + in->dur[i]) return 1;",
                                  "if (S[in->succ[e]] <= S[i] + in->dur[i]) return 1;"),
    # Alg. 4 counting only the entries it touches instead of every loop step
    "alg4_counts_touched_only": ("            }\n            resIdx = resIdx + 1;\n            ++steps;",
                                 "                ++steps;\n            }\n            resIdx = resIdx + 1;"),
    # Alg. 5 window not restarted on an insufficient step
    "alg5_no_restart": ("{ loadTime = 0; sufficient = 0; }", "{ sufficient = 0; }"),
    # Eq. 8 with the quality and intactness weights swapped
    "eq8_weights_swapped": ("double a = 0.8 * quality;", "double a = 0.2 * quality;"),
    # random swap picked by a remainder instead of the scaled draw
    "diversify_by_remainder": ("int pick = (int)(((unsigned long long)w * (unsigned long long)nf) >> 32);",
                               "int pick = (int)(w % (unsigned)nf);"),
    # working-set reads skipping every other slot
    "reads_skip_slots": ("rp = (rp + 1) % F;", "rp = (rp + 2) % F;"),
    # FBI's backward pass decoded on the original network instead of the reversed one
    "fbi_not_reversed": ("int T = fbi_decode(in, &Q, mode, Wb, tau);", "int T = fbi_decode(in, &P, mode, Wb, tau);"),
    # FBI's backward list by finish time, smallest first
    "fbi_backward_order": ("if (fb > fa || (fb == fa && pos[b] > pos[a])) break;",
                           "if (fb < fa || (fb == fa && pos[b] > pos[a])) break;"),
    # a block's improvement not written back to the working set
    "no_write_back": ("if (improved && x->Cbb < f->C) {", "if (improved && x->Cbb < f->C && 0) {"),
    # aspiration admitting a tabu move that only equals the best makespan
    "aspiration_not_strict": ("if (tabu && !(c < Cbest)) continue;", "if (tabu && !(c <= Cbest)) continue;"),
    # ties of equal makespan resolved to the last move instead of the smallest (u, v)
    "tie_break_last": ("if (!found || c < bc) { found = 1;", "if (!found || c <= bc) { found = 1;"),
    # Alg. 3 without clearing the evicted entry's cache bit
    "eviction_keeps_cache": ("tabuCache[uo * N + vo] = 0;", "tabuCache[uo * N + vo] = tabuCache[uo * N + vo];"),
    # a block exchanging once its budget is reached instead of exceeded (reading C3)
    "exchange_timeout_inclusive": ("exch[b] = (char)(improved || x->since > x->assigned);",
                                   "exch[b] = (char)(improved || x->since >= x->assigned);"),
    # a written slot's iterations counter without the IC that was read (reading C4)
    "write_ic_without_read_ic": ("f->IC = x->ICread + x->since;", "f->IC = x->since;"),
    # a block's aspiration threshold its own best instead of C*_max (reading C2)
    "aspiration_block_best": ("if (tabu && !(c < Casp)) continue;", "if (tabu && !(c < x->Cbb)) continue;"),
    # a successor released one step after its predecessor's finish (feasible, but leaves idle steps)
    "precedence_lag": ("es_prec = imax(es_prec, S[j] + in->dur[j]);", "es_prec = imax(es_prec, S[j] + in->dur[j] + 1);"),
    # an empty iteration (no admissible move) does not advance the tabu list
    "empty_move_stalls": ("writeIndex = (writeIndex + 1) % p->tabu_len;\n        if (found && C < Cbest)",
                          "writeIndex = (writeIndex + found) % p->tabu_len;\n        if (found && C < Cbest)"),
}


@contextlib.contextmanager
def mutant(oracle, tmp_path, name):
    src = open(oracle.SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, name
    mut = tmp_path / f"{name}.c"
    mut.write_text(src.replace(old, new))
    (tmp_path / "rcpsp_oracle.h").write_text(open(oracle.HDR).read())
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-pthread", "-o", str(so),
                    str(mut)],
                   check=True)
    saved = oracle._handle
    oracle._handle = oracle.load(str(so))
    try:
        yield
    finally:
        oracle._handle = saved


def table1_cmax(oracle, mode):
    text, vals = fixtures.read("table1_instance.txt")
    inst = Instance.from_text(text)
    return oracle.decode(inst, np.array(vals["W"], np.int32), mode)[0]


def test_mutant_loop_bound_breaks_table1(oracle, tmp_path):
    with mutant(oracle, tmp_path, "alg5_alg6_k_lt_M_minus_1"):
        assert table1_cmax(oracle, 1) != 22


def test_mutant_eq6_breaks_feasibility_pin(oracle, tmp_path):
    with mutant(oracle, tmp_path, "eq6_short_range"):
        with pytest.raises(AssertionError):
            pins.test_eq5_eq6_equal_list_feasibility(oracle)


@pytest.mark.parametrize("name", ["alg4_no_max_with_s", "alg4_copy_offset"])
def test_mutant_alg4_breaks_envelope_pin(oracle, tmp_path, name):
    with mutant(oracle, tmp_path, name):
        with pytest.raises(AssertionError):
            pins.test_alg4_equals_upper_envelope(oracle)
        if name == "alg4_copy_offset":
            with pytest.raises(AssertionError):
                pins.test_fig4_update(oracle)


def test_mutant_alg5_breaks_earliest_fit_pin(oracle, tmp_path):
    with mutant(oracle, tmp_path, "alg5_no_restart"):
        with pytest.raises(AssertionError):
            pins.test_decoders_on_random_lists(oracle)


def test_mutant_precedence_lag_breaks_no_idle_pin(oracle, tmp_path):
    with mutant(oracle, tmp_path, "precedence_lag"):
        with pytest.raises(AssertionError):
            pins.test_serial_sgs_leaves_no_idle_step(oracle)


def test_mutant_eq8_weights_break_closed_forms(oracle, tmp_path):
    import test_oracle_coop as coop
    with mutant(oracle, tmp_path, "eq8_weights_swapped"):
        with pytest.raises(AssertionError):
            coop.test_eq8_prefers_good_and_fresh_solutions(oracle)


def test_mutant_diversify_breaks_drawn_swaps(oracle, tmp_path):
    import test_oracle_coop as coop
    with mutant(oracle, tmp_path, "diversify_by_remainder"):
        with pytest.raises(AssertionError):
            coop.test_diversify_takes_the_drawn_feasible_swaps(oracle)


@pytest.mark.parametrize("name", ["reads_skip_slots", "no_write_back"])
def test_mutant_exchange_breaks_rules(oracle, tmp_path, name):
    import test_oracle_coop as coop
    with mutant(oracle, tmp_path, name):
        with pytest.raises(AssertionError):
            if name == "reads_skip_slots":
                coop.test_exchange_rules(oracle, 4, 8, 1)
            else:
                coop.test_single_block_without_exchanges_is_the_plain_search(oracle, 1)


@pytest.mark.parametrize("name", ["fbi_not_reversed", "fbi_backward_order"])
def test_mutant_fbi_breaks_backward_schedule(oracle, tmp_path, name):
    import test_oracle_coop as coop
    with mutant(oracle, tmp_path, name):
        with pytest.raises(AssertionError):
            coop.test_fbi_backward_schedule_is_a_schedule(oracle)


@pytest.mark.parametrize("name", ["aspiration_not_strict", "tie_break_last", "eviction_keeps_cache",
                                  "empty_move_stalls"])
def test_mutant_tabu_rules_break_restatement(oracle, tmp_path, name):
    with mutant(oracle, tmp_path, name):
        assert sum(pins.restatement_mismatches(oracle, mode)[0] for mode in (1, 2)) > 0


@pytest.mark.parametrize("name", ["exchange_timeout_inclusive", "write_ic_without_read_ic", "aspiration_block_best",
                                  "reads_skip_slots", "fbi_backward_order"])
def test_mutant_cooperation_breaks_restatement(oracle, tmp_path, name):
    import test_oracle_coop_restated as coop
    with mutant(oracle, tmp_path, name):
        assert sum(coop.coop_mismatches(oracle, mode)[0] for mode in (1, 2)) > 0


def test_mutant_alg4_step_count_breaks_work_pins(oracle, tmp_path):
    with mutant(oracle, tmp_path, "alg4_counts_touched_only"):
        with pytest.raises(AssertionError):
            pins.test_capacity_work_counter_matches_envelopes(oracle)
        with pytest.raises(AssertionError):
            pins.test_alg4_equals_upper_envelope(oracle)


@pytest.mark.parametrize("name", ["checker_closed_interval", "checker_strict_precedence"])
def test_mutant_checker_breaks_its_pins(oracle, tmp_path, name):
    with mutant(oracle, tmp_path, name):
        with pytest.raises(AssertionError):
            pins.test_checker_rejects_violations(oracle)
