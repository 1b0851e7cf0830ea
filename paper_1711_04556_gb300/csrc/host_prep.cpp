// Host preparation of an instance before it goes to the device (the host part
// of the paper's homogeneous model, Sec. 6): validation against the problem
// statement (Sec. 2), critical path (Sec. 2), level-ordered initial list
// (Sec. 4.1), evaluator selection (Sec. 5.4) and packing into the record the
// search kernel stages into shared memory.
#include "host_prep.h"

#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

namespace rcpsp {

namespace {

// Selection rule (Sec. 5.4).  The learned JRip rules are not printed in the
// paper (Fig. 5 is lost).  The rule keeps two attributes of Table 3 -- the
// critical path length and the average capacity -- and the direction of
// Sec. 7.2 (capacity-indexed for long schedules with low capacities):
// capacity-indexed iff CP > K * avgCap, compared exactly as CP * M > K * sumR.
// K = 12 was fitted by timing both evaluators on a grid of instances on
// GB300 (selection_study.py), as Sec. 5.4 derives its classes from
// measured run times.
constexpr long long kSelK = 12;

int fail(std::string &err, int code, const std::string &msg) {
    err = msg;
    return code;
}

}  // namespace

void level_order(int n, const int32_t *succ_off, const int32_t *succ, const int32_t *keys, int32_t *W) {
    std::vector<int> indeg(n, 0), order, level(n, 0);
    for (int e = 0; e < succ_off[n]; ++e) ++indeg[succ[e]];
    order.reserve(n);
    for (int i = 0; i < n; ++i)
        if (indeg[i] == 0) order.push_back(i);
    for (size_t h = 0; h < order.size(); ++h) {
        const int i = order[h];
        for (int e = succ_off[i]; e < succ_off[i + 1]; ++e) {
            const int j = succ[e];
            level[j] = std::max(level[j], level[i] + 1);
            if (--indeg[j] == 0) order.push_back(j);
        }
    }
    std::vector<int> w(n);
    std::iota(w.begin(), w.end(), 0);
    std::stable_sort(w.begin(), w.end(), [&](int a, int b) {
        if (level[a] != level[b]) return level[a] < level[b];
        const int ka = keys ? keys[a] : 0, kb = keys ? keys[b] : 0;
        if (ka != kb) return ka < kb;
        return a < b;
    });
    for (int i = 0; i < n; ++i) W[i] = w[i];
}

int select_evaluator(int m, const int32_t *cap, int critical_path) {
    long long sum_r = 0;
    for (int k = 0; k < m; ++k) sum_r += cap[k];
    return static_cast<long long>(critical_path) * m > kSelK * sum_r ? RCPSP_EVAL_CAPACITY : RCPSP_EVAL_TIME;
}

int prepare_instance(const rcpsp_instance &in, PackedInstance &out, std::string &err) {
    const int n = in.n, m = in.m;
    if (n < 3) return fail(err, RCPSP_E_INVALID_ARG, "N must be at least 3");
    if (n > RCPSP_MAX_N) return fail(err, RCPSP_E_TOO_LARGE, "N exceeds RCPSP_MAX_N");
    if (m < 1 || m > RCPSP_MAX_M) return fail(err, RCPSP_E_TOO_LARGE, "M must be in [1, 8]");
    if (!in.dur || !in.cap || !in.req || !in.succ_off || (!in.succ && in.succ_off[n] > 0))
        return fail(err, RCPSP_E_INVALID_ARG, "null array in instance");
    long long horizon = 0;
    for (int i = 0; i < n; ++i) {
        if (in.dur[i] < 0) return fail(err, RCPSP_E_INVALID_ARG, "negative duration");
        horizon += in.dur[i];
    }
    if (in.dur[0] != 0 || in.dur[n - 1] != 0) return fail(err, RCPSP_E_DUMMY, "dummy activities need d = 0");
    if (horizon > RCPSP_MAX_HORIZON) return fail(err, RCPSP_E_TOO_LARGE, "sum of durations exceeds RCPSP_MAX_HORIZON");
    int max_cap = 0;
    for (int k = 0; k < m; ++k) {
        if (in.cap[k] < 1 || in.cap[k] > RCPSP_MAX_CAP)
            return fail(err, in.cap[k] < 1 ? RCPSP_E_INVALID_ARG : RCPSP_E_TOO_LARGE, "capacity out of range");
        max_cap = std::max(max_cap, static_cast<int>(in.cap[k]));
    }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < m; ++k) {
            const int r = in.req[i * m + k];
            if (r < 0) return fail(err, RCPSP_E_INVALID_ARG, "negative demand");
            if (r > in.cap[k]) return fail(err, RCPSP_E_DEMAND_EXCEEDS_CAP, "demand exceeds capacity");
            if ((i == 0 || i == n - 1) && r != 0) return fail(err, RCPSP_E_DUMMY, "dummy activities need r = 0");
        }
    // arcs
    if (in.succ_off[0] != 0) return fail(err, RCPSP_E_INVALID_ARG, "succ_off[0] must be 0");
    for (int i = 0; i < n; ++i)
        if (in.succ_off[i + 1] < in.succ_off[i]) return fail(err, RCPSP_E_INVALID_ARG, "succ_off not monotone");
    const int E = in.succ_off[n];
    std::vector<int> indeg(n, 0), outdeg(n, 0);
    for (int i = 0; i < n; ++i) {
        for (int e = in.succ_off[i]; e < in.succ_off[i + 1]; ++e) {
            const int j = in.succ[e];
            if (j < 0 || j >= n) return fail(err, RCPSP_E_INVALID_ARG, "successor index out of range");
            if (j == i) return fail(err, RCPSP_E_CYCLE, "self loop");
            for (int e2 = in.succ_off[i]; e2 < e; ++e2)
                if (in.succ[e2] == j) return fail(err, RCPSP_E_INVALID_ARG, "duplicate arc");
            indeg[j]++;
            outdeg[i]++;
        }
    }
    if (indeg[0] != 0 || outdeg[n - 1] != 0) return fail(err, RCPSP_E_DUMMY, "0 must be the source and N-1 the sink");
    for (int i = 1; i < n - 1; ++i)
        if (indeg[i] == 0 || outdeg[i] == 0)
            return fail(err, RCPSP_E_DUMMY, "activity " + std::to_string(i) + " lacks a predecessor or a successor");
    // predecessor CSR
    std::vector<int> poff(n + 1, 0), plist(E);
    for (int i = 0; i < n; ++i) poff[i + 1] = poff[i] + indeg[i];
    {
        std::vector<int> fill(n, 0);
        for (int i = 0; i < n; ++i)
            for (int e = in.succ_off[i]; e < in.succ_off[i + 1]; ++e) {
                const int j = in.succ[e];
                plist[poff[j] + fill[j]++] = i;
            }
    }
    // topological order (Kahn); a leftover activity means a cycle
    std::vector<int> order;
    order.reserve(n);
    {
        std::vector<int> deg = indeg;
        for (int i = 0; i < n; ++i)
            if (deg[i] == 0) order.push_back(i);
        for (size_t h = 0; h < order.size(); ++h) {
            const int i = order[h];
            for (int e = in.succ_off[i]; e < in.succ_off[i + 1]; ++e)
                if (--deg[in.succ[e]] == 0) order.push_back(in.succ[e]);
        }
        if (static_cast<int>(order.size()) != n) return fail(err, RCPSP_E_CYCLE, "precedence graph has a cycle");
    }
    // critical path (arc (i,j) weighted d_i) and levels (unit weights)
    std::vector<int> es(n, 0), level(n, 0);
    for (int i : order)
        for (int e = in.succ_off[i]; e < in.succ_off[i + 1]; ++e) {
            const int j = in.succ[e];
            es[j] = std::max(es[j], es[i] + static_cast<int>(in.dur[i]));
            level[j] = std::max(level[j], level[i] + 1);
        }
    // initial list: by (level, key, label)
    std::vector<int> W(n);
    std::iota(W.begin(), W.end(), 0);
    std::stable_sort(W.begin(), W.end(), [&](int a, int b) {
        if (level[a] != level[b]) return level[a] < level[b];
        const int ka = in.level_key ? in.level_key[a] : 0, kb = in.level_key ? in.level_key[b] : 0;
        if (ka != kb) return ka < kb;
        return a < b;
    });
    // SWAR packing of the time-indexed profile: 4 resources of 8 bits per
    // word when every capacity is below 128, else 2 of 16 bits; the high
    // bit of each field stays clear so that a fit test never borrows.
    const int lane_bits = max_cap <= 127 ? 8 : 16;
    const int fields = 32 / lane_bits;
    int wps = (m + fields - 1) / fields;
    wps = wps <= 1 ? 1 : (wps <= 2 ? 2 : 4);
    InstHeader &h = out.h;
    std::memset(&h, 0, sizeof(h));
    h.n = n;
    h.m = m;
    h.ub = static_cast<int>(horizon);
    h.cp = es[n - 1];
    h.sel_mode = select_evaluator(m, in.cap, es[n - 1]);
    h.wps = wps;
    h.lane_bits = lane_bits;
    h.sum_cap = 0;
    for (int k = 0; k < m; ++k) h.sum_cap += in.cap[k];
    h.sum_used = 0;
    for (int i = 0; i < n * m; ++i) h.sum_used += in.req[i] > 0 ? 1 : 0;
    // Does the earliest-start schedule (infinite capacities) respect every
    // capacity?  Then the serial SGS of the level-ordered list places every
    // activity at its earliest start (its predecessors come first, and what
    // is placed before it uses no more than the earliest-start profile), so
    // the initial makespan is the critical path and a search that stops at
    // the critical path ends before its first iteration.  Only the queue
    // order uses this.
    {
        h.es_fits = 1;
        const int horizon_cp = es[n - 1] + 1;
        std::vector<int64_t> prof(static_cast<size_t>(horizon_cp) + 1);
        for (int k = 0; k < m && h.es_fits; ++k) {
            std::fill(prof.begin(), prof.end(), 0);
            for (int i = 0; i < n; ++i) {
                const int r = in.req[i * m + k], d = in.dur[i];
                if (r <= 0 || d <= 0) continue;
                prof[es[i]] += r;
                prof[std::min(es[i] + d, horizon_cp)] -= r;
            }
            int64_t run = 0;
            for (int t = 0; t < horizon_cp && h.es_fits; ++t) {
                run += prof[t];
                if (run > in.cap[k]) h.es_fits = 0;
            }
        }
    }
    h.n_arcs = E;
    const InstLayout L = inst_layout(n, m, wps, E);
    h.inst_words = L.words;
    h.record_words = align4(L.words + n);
    out.record.assign(h.record_words, 0);
    int32_t *r = out.record.data();
    for (int i = 0; i < n; ++i) r[L.dur + i] = in.dur[i];
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < m; ++k) {
            const uint32_t v = static_cast<uint32_t>(in.req[i * m + k]) << ((k % fields) * lane_bits);
            r[L.reqw + i * wps + k / fields] = static_cast<int32_t>(static_cast<uint32_t>(r[L.reqw + i * wps + k / fields]) | v);
        }
    for (int k = 0; k < m; ++k) {
        const uint32_t v = static_cast<uint32_t>(in.cap[k]) << ((k % fields) * lane_bits);
        r[L.capw + k / fields] = static_cast<int32_t>(static_cast<uint32_t>(r[L.capw + k / fields]) | v);
    }
    for (int k = 0, b = 0; k < m; ++k) {
        r[L.cap + k] = in.cap[k];
        r[L.cbase + k] = b;
        b += in.cap[k];
    }
    // per activity, its used resources first, each as r_{i,k} << 3 | k,
    // then zeros (the capacity-indexed decoder's lanes take them in turn)
    for (int i = 0; i < n; ++i)
        for (int k = 0, q = 0; k < m; ++k)
            if (in.req[i * m + k] > 0) r[L.reqk + i * m + q++] = (in.req[i * m + k] << 3) | k;
    for (int i = 0; i <= n; ++i) r[L.poff + i] = poff[i];
    for (int e = 0; e < E; ++e) r[L.plist + e] = plist[e];
    for (int i = 0; i <= n; ++i) r[L.soff + i] = in.succ_off[i];
    for (int e = 0; e < E; ++e) r[L.slist + e] = in.succ[e];
    for (int p = 0; p < n; ++p) r[L.words + p] = W[p];
    out.initial = W;
    return RCPSP_OK;
}

void default_search_params(int n, int *delta, int *tabu_len) {
    // Table 2 (delta, |tabuList|) by instance size; below 45 activities the
    // short swap distance 20 of the single-instance workload is used.
    const int act = n - 2;
    if (act <= 45) { *delta = 20; *tabu_len = 60; }
    else if (act <= 75) { *delta = 60; *tabu_len = 250; }
    else if (act <= 105) { *delta = 60; *tabu_len = 600; }
    else { *delta = 60; *tabu_len = 800; }
}

double estimate_cost(const InstHeader &h, int mode, int iterations, int delta, bool stop_at_cp) {
    const double slots = h.n > 3 ? static_cast<double>(h.n - 3) * delta : 0.0;
    const double per_decode = mode == RCPSP_EVAL_CAPACITY ? h.n * (1.0 + h.sum_cap / 2.0)
                                                          : h.n * 4.0 + 2.0 * h.ub * h.wps;
    // a search that stops at the critical path and starts there does no iteration
    if (stop_at_cp && h.es_fits && mode == RCPSP_EVAL_TIME) iterations = 0;
    return (iterations + 1.0) * (slots * 0.15 + 1.0) * per_decode;
}

}  // namespace rcpsp
