// Host preparation of instances (validation, critical path, levels,
// evaluator selection, packing) and launch-planning helpers.
#pragma once

#include <string>
#include <vector>

#include "rcpsp_internal.h"

namespace rcpsp {

struct PackedInstance {
    InstHeader h;
    std::vector<int32_t> record;    // h.record_words words
    std::vector<int> initial;       // initial list W (Sec. 4.1)
};

// Validates `in` and packs it; returns RCPSP_OK or a negative RCPSP_E_* code
// with a message in `err`.
int prepare_instance(const rcpsp_instance &in, PackedInstance &out, std::string &err);

// Initial list of a validated precedence graph (Sec. 4.1): activities by
// (level, key, label), key 0 when `keys` is null.
void level_order(int n, const int32_t *succ_off, const int32_t *succ, const int32_t *keys, int32_t *W);

// Evaluator chosen by the selection rule (Sec. 5.4) from the capacities and
// the critical-path length.
int select_evaluator(int m, const int32_t *cap, int critical_path);

// (delta, |tabuList|) by instance size (Table 2).
void default_search_params(int n, int *delta, int *tabu_len);

// Relative cost of one search, for longest-first ordering of the queue.
double estimate_cost(const InstHeader &h, int mode, int iterations, int delta, bool stop_at_cp);

}  // namespace rcpsp
