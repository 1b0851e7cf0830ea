/*
 * CPU reference ("oracle") for the parallel tabu search for the RCPSP
 * (Bukata, Sucha, Hanzalek).  TEST INFRASTRUCTURE ONLY: loaded by the tests,
 * the smoke check and the benchmark's CPU-baseline leg, never by the
 * product.  It shares nothing with the CUDA library.
 *
 * Every routine below follows one passage of the paper, in the paper's
 * order and notation, with no blocking, fusion or reordering:
 *   - checker ............ Eqs. 2-4 (Sec. 2.1)
 *   - critical path ...... Sec. 2 (longest path, arc (i,j) weighted d_i)
 *   - levels / W^init .... Sec. 4.1
 *   - move feasibility ... Eqs. 5-6 (Sec. 4.2)
 *   - time-indexed SGS ... Alg. 7 with Alg. 5 and Alg. 6 (Secs. 5.2-5.3)
 *   - capacity-indexed ... Alg. 7 with Eq. 7 and Alg. 4 (Sec. 5.1)
 *   - tabu list .......... Algs. 2-3 (Sec. 4.5)
 *   - search loop ........ Sec. 6 (one block's main loop, no working set)
 *   - FBI ................ Sec. 6 (forward-backward improvement of initial
 *                          solutions; readings F1-F3 beside the code)
 *   - co-operation ....... Sec. 6.1, Eq. 8 (blocks exchanging through the
 *                          working set F; readings C1-C8 beside the code)
 *
 * Readings where the paper is silent, garbled or ambiguous (each one is
 * also listed with the design notes of the repository):
 *   R1  Algs. 5 and 6 print the resource loop bound as k < M-1; read k < M,
 *       as in Alg. 4 (only k < M reproduces C_max = 22 of Table 1).
 *   R2  Inside a level the order is ascending (key, label); key = 0 unless
 *       the caller passes shuffle keys (the shuffling of Sec. 4.1).
 *   R3  The best move is the admissible move with the lexicographically
 *       smallest (C_max, u, v); the enumeration is u-major, v ascending.
 *   R4  Aspiration (Sec. 6: a tabu move is admitted when it gives a new best
 *       makespan): strictly C_uv < C*_max.
 *   R5  No admissible move: W is kept and the empty move (0,0) is added to
 *       the tabu list, so that tabu entries still age.
 *   R6  The stop test (C*_max equal to the critical path) runs before each
 *       iteration; an iteration counts one selection, empty or not.
 *   R7  Duplicate tabu-list entries follow Alg. 3 literally: evicting the
 *       older copy clears the cache entry.
 *   R8  The learned selection rules of Sec. 5.4 are not printed (Fig. 5 is
 *       lost).  The rule used keeps two attributes of Table 3, the critical
 *       path length and the average capacity, and the direction of Sec. 7.2
 *       (capacity-indexed for long schedules with low capacities):
 *       capacity-indexed iff CP > SEL_K * avgCap, compared exactly as
 *       CP * M > SEL_K * sum R_k.  SEL_K = 12 was fitted, as Sec. 5.4 does,
 *       by timing both evaluators on a grid of instances on the target GPU.
 *   R9  "Evaluated schedules" counts neighbour decodes only (every feasible
 *       move, tabu or not); the initial and final decodes are not counted.
 */
#include "rcpsp_oracle.h"

#include <limits.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* Selection constant of reading R8. */
#define SEL_K 12

static int imax(int a, int b) { return a > b ? a : b; }

/* ---------- predecessor lists derived from the successor lists ---------- */
typedef struct {
    int *off;   /* [N+1] */
    int *list;  /* [|E|] */
} preds_t;

static int build_preds(const orc_instance *in, preds_t *p) {
    int N = in->n, E = in->succ_off[N];
    p->off = (int *)calloc((size_t)N + 1, sizeof(int));
    p->list = (int *)malloc(sizeof(int) * (size_t)(E > 0 ? E : 1));
    if (!p->off || !p->list) return -1;
    for (int i = 0; i < N; ++i)
        for (int e = in->succ_off[i]; e < in->succ_off[i + 1]; ++e) p->off[in->succ[e] + 1]++;
    for (int i = 0; i < N; ++i) p->off[i + 1] += p->off[i];
    int *fill = (int *)calloc((size_t)N, sizeof(int));
    if (!fill) return -1;
    for (int i = 0; i < N; ++i)
        for (int e = in->succ_off[i]; e < in->succ_off[i + 1]; ++e) {
            int j = in->succ[e];
            p->list[p->off[j] + fill[j]++] = i;
        }
    free(fill);
    return 0;
}

static void free_preds(preds_t *p) { free(p->off); free(p->list); }

static int is_arc(const orc_instance *in, int i, int j) {
    for (int e = in->succ_off[i]; e < in->succ_off[i + 1]; ++e)
        if (in->succ[e] == j) return 1;
    return 0;
}

/* Kahn's algorithm; returns 0 and a topological order, -1 on a cycle. */
static int topo_order(const orc_instance *in, int *order) {
    int N = in->n, head = 0, tail = 0;
    int *indeg = (int *)calloc((size_t)N, sizeof(int));
    if (!indeg) return -1;
    for (int e = 0; e < in->succ_off[N]; ++e) indeg[in->succ[e]]++;
    for (int i = 0; i < N; ++i) if (indeg[i] == 0) order[tail++] = i;
    while (head < tail) {
        int i = order[head++];
        for (int e = in->succ_off[i]; e < in->succ_off[i + 1]; ++e)
            if (--indeg[in->succ[e]] == 0) order[tail++] = in->succ[e];
    }
    free(indeg);
    return tail == N ? 0 : -1;
}

/* ---------------------------- Eqs. 2-4 ---------------------------------- */
int orc_check_schedule(const orc_instance *in, const int *S, int *cmax) {
    int N = in->n, M = in->m, C = 0;
    for (int i = 0; i < N; ++i) {
        if (S[i] < 0) return 3;
        C = imax(C, S[i] + in->dur[i]);                          /* Eq. 2 */
    }
    if (cmax) *cmax = C;
    for (int i = 0; i < N; ++i)                                  /* Eq. 3 */
        for (int e = in->succ_off[i]; e < in->succ_off[i + 1]; ++e)
            if (S[in->succ[e]] < S[i] + in->dur[i]) return 1;
    for (int k = 0; k < M; ++k)                                  /* Eq. 4 */
        for (int t = 0; t <= C; ++t) {
            int used = 0;
            for (int i = 0; i < N; ++i)
                if (S[i] <= t && t < S[i] + in->dur[i]) used += in->req[i * M + k];
            if (used > in->cap[k]) return 2;
        }
    return 0;
}

/* ------------------------- critical path (Sec. 2) ------------------------ */
int orc_critical_path(const orc_instance *in) {
    int N = in->n;
    int *order = (int *)malloc(sizeof(int) * (size_t)N);
    int *es = (int *)calloc((size_t)N, sizeof(int));
    if (!order || !es || topo_order(in, order) != 0) { free(order); free(es); return -1; }
    for (int a = 0; a < N; ++a) {
        int i = order[a];
        for (int e = in->succ_off[i]; e < in->succ_off[i + 1]; ++e) {
            int j = in->succ[e];
            if (es[i] + in->dur[i] > es[j]) es[j] = es[i] + in->dur[i];
        }
    }
    int cp = es[N - 1];
    free(order); free(es);
    return cp;
}

/* ----------------------------- Sec. 4.1 --------------------------------- */
int orc_levels(const orc_instance *in, int *level) {
    int N = in->n;
    int *order = (int *)malloc(sizeof(int) * (size_t)N);
    if (!order || topo_order(in, order) != 0) { free(order); return -1; }
    for (int i = 0; i < N; ++i) level[i] = 0;
    for (int a = 0; a < N; ++a) {
        int i = order[a];
        for (int e = in->succ_off[i]; e < in->succ_off[i + 1]; ++e) {
            int j = in->succ[e];
            if (level[i] + 1 > level[j]) level[j] = level[i] + 1;
        }
    }
    free(order);
    return 0;
}

int orc_initial_order(const orc_instance *in, int *W) {
    int N = in->n;
    int *level = (int *)malloc(sizeof(int) * (size_t)N);
    if (!level || orc_levels(in, level) != 0) { free(level); return -1; }
    for (int i = 0; i < N; ++i) W[i] = i;
    /* insertion sort by (level, key, label) */
    for (int a = 1; a < N; ++a) {
        int x = W[a], b = a - 1;
        while (b >= 0) {
            int y = W[b];
            int kx = in->level_key ? in->level_key[x] : 0;
            int ky = in->level_key ? in->level_key[y] : 0;
            int before = level[x] < level[y] ||
                         (level[x] == level[y] && (kx < ky || (kx == ky && x < y)));
            if (!before) break;
            W[b + 1] = y;
            --b;
        }
        W[b + 1] = x;
    }
    free(level);
    return 0;
}

/* ----------------------------- Eqs. 5-6 --------------------------------- */
int orc_move_feasible(const orc_instance *in, const int *W, int u, int v) {
    for (int x = u + 1; x <= v; ++x)                             /* Eq. 5 */
        if (is_arc(in, W[u], W[x])) return 0;
    for (int x = u; x <= v - 1; ++x)                             /* Eq. 6 */
        if (is_arc(in, W[x], W[v])) return 0;
    return 1;
}

/* ---------------- Alg. 7 with Alg. 5 / Alg. 6 (time-indexed) ------------ */
static int decode_time(const orc_instance *in, const preds_t *P, const int *W, int *S,
                       long long *work) {
    int N = in->n, M = in->m, UB = 0;
    for (int i = 0; i < N; ++i) UB += in->dur[i];                /* UB = sum d_i */
    int *tau = (int *)malloc(sizeof(int) * (size_t)M * (size_t)(UB > 0 ? UB : 1));
    char *done = (char *)calloc((size_t)N, 1);
    if (!tau || !done) { free(tau); free(done); return -1; }
    for (int k = 0; k < M; ++k)
        for (int t = 0; t < UB; ++t) tau[k * UB + t] = in->cap[k];
    long long steps = 0;
    int Cmax = 0;                                                /* Alg. 7: C_max from 0 */
    for (int u = 0; u < N; ++u) {
        int i = W[u];
        int es_prec = 0;
        for (int e = P->off[i]; e < P->off[i + 1]; ++e) {
            int j = P->list[e];
            if (!done[j]) { Cmax = -1; goto out; }               /* W infeasible */
            es_prec = imax(es_prec, S[j] + in->dur[j]);
        }
        /* Alg. 5: first window of d_i consecutive fitting steps */
        int loadTime = 0, t;
        for (t = es_prec; t < UB && loadTime < in->dur[i]; ++t) {
            int sufficient = 1;
            for (int k = 0; k < M; ++k)                          /* reading R1 */
                if (tau[k * UB + t] < in->req[i * M + k]) { loadTime = 0; sufficient = 0; }
            if (sufficient) ++loadTime;
            ++steps;
        }
        if (loadTime < in->dur[i]) { Cmax = -1; goto out; }      /* cannot happen */
        int es_res = t - loadTime;
        int s = imax(es_prec, es_res);
        /* Alg. 6 */
        for (int k = 0; k < M; ++k)                              /* reading R1 */
            for (int x = s; x < s + in->dur[i]; ++x) tau[k * UB + x] -= in->req[i * M + k];
        S[i] = s;
        done[i] = 1;
        Cmax = imax(Cmax, s + in->dur[i]);
    }
out:
    if (work) *work += steps;
    free(tau); free(done);
    return Cmax;
}

/* ------------------------------ Alg. 4 ---------------------------------- */
int orc_capacity_update(int *c, int R, int r, int d, int s) {
    int *copy = (int *)malloc(sizeof(int) * (size_t)(R > 0 ? R : 1));
    int steps = 0;
    int requiredEffort = r * d;
    if (requiredEffort > 0) {
        int resIdx = 0, copyIdx = 0, newTime = s + d;
        while (requiredEffort > 0 && resIdx < R) {
            if (c[resIdx] < newTime) {
                if (copyIdx >= r) newTime = copy[copyIdx - r];
                int timeDiff = newTime - imax(c[resIdx], s);
                if (requiredEffort - timeDiff > 0) {
                    requiredEffort -= timeDiff;
                    copy[copyIdx++] = c[resIdx];
                    c[resIdx] = newTime;
                } else {
                    c[resIdx] = imax(c[resIdx], s);
                    c[resIdx] += requiredEffort;
                    requiredEffort = 0;
                }
            }
            resIdx = resIdx + 1;
            ++steps;
        }
    }
    free(copy);
    return steps;
}

/* ---------------- Alg. 7 with Eq. 7 / Alg. 4 (capacity-indexed) --------- */
static int decode_capacity(const orc_instance *in, const preds_t *P, const int *W, int *S,
                           long long *work) {
    int N = in->n, M = in->m, tot = 0;
    for (int k = 0; k < M; ++k) tot += in->cap[k];
    int *c = (int *)calloc((size_t)(tot > 0 ? tot : 1), sizeof(int));  /* all zeros */
    int *base = (int *)malloc(sizeof(int) * (size_t)M);
    char *done = (char *)calloc((size_t)N, 1);
    if (!c || !base || !done) { free(c); free(base); free(done); return -1; }
    for (int k = 0, b = 0; k < M; ++k) { base[k] = b; b += in->cap[k]; }
    long long steps = 0;
    int Cmax = 0;
    for (int u = 0; u < N; ++u) {
        int i = W[u];
        int es_prec = 0;
        for (int e = P->off[i]; e < P->off[i + 1]; ++e) {
            int j = P->list[e];
            if (!done[j]) { Cmax = -1; goto out; }
            es_prec = imax(es_prec, S[j] + in->dur[j]);
        }
        int es_res = 0;                                          /* Eq. 7 */
        for (int k = 0; k < M; ++k) {
            int r = in->req[i * M + k];
            if (r > 0) es_res = imax(es_res, c[base[k] + in->cap[k] - r]);
        }
        int s = imax(es_prec, es_res);
        for (int k = 0; k < M; ++k)                              /* Alg. 4 */
            steps += orc_capacity_update(c + base[k], in->cap[k], in->req[i * M + k],
                                         in->dur[i], s);
        S[i] = s;
        done[i] = 1;
        Cmax = imax(Cmax, s + in->dur[i]);
    }
out:
    if (work) *work += steps;
    free(c); free(base); free(done);
    return Cmax;
}

int orc_decode_time(const orc_instance *in, const int *W, int *S, long long *work) {
    preds_t P;
    if (build_preds(in, &P) != 0) return -1;
    int c = decode_time(in, &P, W, S, work);
    free_preds(&P);
    return c;
}

int orc_decode_capacity(const orc_instance *in, const int *W, int *S, long long *work) {
    preds_t P;
    if (build_preds(in, &P) != 0) return -1;
    int c = decode_capacity(in, &P, W, S, work);
    free_preds(&P);
    return c;
}

/* ---------------------- Sec. 5.4 selection (R8) ------------------------- */
int orc_select_mode(const orc_instance *in) {
    long long sumR = 0;
    for (int k = 0; k < in->m; ++k) sumR += in->cap[k];
    const long long cp = orc_critical_path(in);
    /* CP > K * avgCap  <=>  CP * M > K * sumR */
    return cp * in->m > (long long)SEL_K * sumR ? ORC_CAPACITY : ORC_TIME;
}

/* --------------------------- Sec. 6 search ------------------------------ */
int orc_tabu_search(const orc_instance *in, const orc_params *p, orc_result *res) {
    int N = in->n;
    res->status = 0;
    if (N < 2 || p->tabu_len < 1 || p->max_swap_dist < 1 || p->iterations < 0) {
        res->status = -1;
        return -1;
    }
    int mode = p->eval_mode == ORC_AUTO ? orc_select_mode(in) : p->eval_mode;
    preds_t P;
    if (build_preds(in, &P) != 0) { res->status = -1; return -1; }
    int *W = (int *)malloc(sizeof(int) * (size_t)N);
    int *Wc = (int *)malloc(sizeof(int) * (size_t)N);
    int *S = (int *)malloc(sizeof(int) * (size_t)N);
    int *tlU = (int *)calloc((size_t)p->tabu_len, sizeof(int));    /* (0,0) = empty */
    int *tlV = (int *)calloc((size_t)p->tabu_len, sizeof(int));
    char *tabuCache = (char *)calloc((size_t)N * (size_t)N, 1);
    if (!W || !Wc || !S || !tlU || !tlV || !tabuCache || orc_initial_order(in, W) != 0) {
        res->status = -1;
        goto done;
    }
    res->mode = mode;
    res->cp = orc_critical_path(in);
    int C = mode == ORC_TIME ? decode_time(in, &P, W, S, NULL)
                             : decode_capacity(in, &P, W, S, NULL);
    int Cbest = C;
    memcpy(res->best_W, W, sizeof(int) * (size_t)N);
    int writeIndex = 0, it = 0;
    long long evaluated = 0, work = 0;
    while (it < p->iterations) {
        if (p->stop_at_cp && Cbest == res->cp) break;           /* R6 */
        int found = 0, bu = 0, bv = 0, bc = INT_MAX;
        for (int u = 1; u <= N - 2; ++u)
            for (int v = u + 1; v <= N - 2 && v - u <= p->max_swap_dist; ++v) {
                if (!orc_move_feasible(in, W, u, v)) continue;
                memcpy(Wc, W, sizeof(int) * (size_t)N);
                Wc[u] = W[v];
                Wc[v] = W[u];
                int c = mode == ORC_TIME ? decode_time(in, &P, Wc, S, &work)
                                         : decode_capacity(in, &P, Wc, S, &work);
                ++evaluated;
                int tabu = tabuCache[u * N + v];                 /* Alg. 2 */
                if (tabu && !(c < Cbest)) continue;              /* R4 */
                if (!found || c < bc) { found = 1; bu = u; bv = v; bc = c; }  /* R3 */
            }
        if (found) {
            int x = W[bu]; W[bu] = W[bv]; W[bv] = x;
            C = bc;
        } else {
            bu = 0; bv = 0;                                      /* R5 */
        }
        /* Alg. 3 */
        int uo = tlU[writeIndex], vo = tlV[writeIndex];
        tabuCache[uo * N + vo] = 0;
        tlU[writeIndex] = bu;
        tlV[writeIndex] = bv;
        tabuCache[bu * N + bv] = 1;
        writeIndex = (writeIndex + 1) % p->tabu_len;
        if (found && C < Cbest) {
            Cbest = C;
            memcpy(res->best_W, W, sizeof(int) * (size_t)N);
        }
        if (res->trace) {
            res->trace[3 * it + 0] = bu;
            res->trace[3 * it + 1] = bv;
            res->trace[3 * it + 2] = C;
        }
        ++it;
    }
    res->best_cmax = mode == ORC_TIME ? decode_time(in, &P, res->best_W, res->best_S, NULL)
                                      : decode_capacity(in, &P, res->best_W, res->best_S, NULL);
    res->iterations = it;
    res->evaluated = evaluated;
    res->work = work;
    if (res->best_cmax != Cbest) res->status = -2;               /* self-check */
done:
    free(W); free(Wc); free(S); free(tlU); free(tlV); free(tabuCache);
    free_preds(&P);
    return res->status;
}

/* ------------------------ batch over a thread pool ----------------------- */
typedef struct {
    const orc_instance *in;
    const orc_params *p;
    orc_result *res;
    int count;
    int next;
    pthread_mutex_t lock;
} pool_t;

static void *pool_worker(void *arg) {
    pool_t *pl = (pool_t *)arg;
    for (;;) {
        pthread_mutex_lock(&pl->lock);
        int k = pl->next++;
        pthread_mutex_unlock(&pl->lock);
        if (k >= pl->count) break;
        orc_tabu_search(&pl->in[k], pl->p, &pl->res[k]);
    }
    return NULL;
}

int orc_tabu_search_batch(const orc_instance *in, int count, const orc_params *p,
                          orc_result *res, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    pool_t pl = {in, p, res, count, 0, PTHREAD_MUTEX_INITIALIZER};
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) return -1;
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, pool_worker, &pl);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    int rc = 0;
    for (int k = 0; k < count; ++k) if (res[k].status != 0) rc = res[k].status;
    return rc;
}

/* ------------- forward-backward improvement (FBI, Sec. 6) ---------------- */
/*
 * The paper improves every second initial solution by the forward-backward
 * improvement of Li and Willis, which moves the activities of a schedule to
 * the right and back to the left while the makespan falls.  Restated here as
 * the usual justification passes of the
 * serial SGS, with the readings:
 *   F1  Backward pass: the activities ordered by non-increasing finish time
 *       of the forward schedule (ties: later list position first) are
 *       decoded on the reversed network (successors act as predecessors),
 *       with the search's evaluator; tau_i is the reversed start and T the
 *       reversed makespan.  Mirrored, s'_i = T - tau_i - d_i is a schedule
 *       of the original instance of length T.
 *   F2  Forward pass: the activities ordered by non-decreasing s'_i (ties:
 *       earlier position in the current list first) form the new list,
 *       decoded forward.
 *   F3  The passes repeat while the forward makespan gets strictly shorter;
 *       the result is the last list that shortened it (or the input list).
 */
static int fbi_decode(const orc_instance *in, const preds_t *P, int mode, const int *W, int *S) {
    return mode == ORC_TIME ? decode_time(in, P, W, S, NULL) : decode_capacity(in, P, W, S, NULL);
}

int orc_fbi_pass(const orc_instance *in, int mode, const int *W, int *Wnext, int *T_out, int *S_back) {
    const int N = in->n;
    if (mode == ORC_AUTO) mode = orc_select_mode(in);
    preds_t P, Q;                                  /* Q: predecessors of the reversed network */
    if (build_preds(in, &P) != 0) return -1;
    Q.off = (int *)malloc(sizeof(int) * (size_t)(N + 1));
    Q.list = (int *)malloc(sizeof(int) * (size_t)(in->succ_off[N] > 0 ? in->succ_off[N] : 1));
    int *S = (int *)malloc(sizeof(int) * (size_t)N);
    int *tau = (int *)malloc(sizeof(int) * (size_t)N);
    int *pos = (int *)malloc(sizeof(int) * (size_t)N);
    int *Wb = (int *)malloc(sizeof(int) * (size_t)N);
    int C2 = -1;
    if (!Q.off || !Q.list || !S || !tau || !pos || !Wb) goto out;
    for (int i = 0; i <= N; ++i) Q.off[i] = in->succ_off[i];
    for (int e = 0; e < in->succ_off[N]; ++e) Q.list[e] = in->succ[e];
    if (fbi_decode(in, &P, mode, W, S) < 0) goto out;
    for (int p = 0; p < N; ++p) pos[W[p]] = p;
    /* F1: by finish time, largest first; ties: later position first (insertion sort) */
    for (int p = 0; p < N; ++p) {
        int a = W[p], q = p;
        while (q > 0) {
            int b = Wb[q - 1];
            int fa = S[a] + in->dur[a], fb = S[b] + in->dur[b];
            if (fb > fa || (fb == fa && pos[b] > pos[a])) break;
            Wb[q] = b;
            --q;
        }
        Wb[q] = a;
    }
    int T = fbi_decode(in, &Q, mode, Wb, tau);
    if (T_out) *T_out = T;
    if (S_back)
        for (int i = 0; i < N; ++i) S_back[i] = T - tau[i] - in->dur[i];
    /* F2: by mirrored start T - tau - d, smallest first; ties: earlier position first */
    for (int p = 0; p < N; ++p) {
        int a = W[p], q = p;
        int sa = T - tau[a] - in->dur[a];
        while (q > 0) {
            int b = Wnext[q - 1];
            int sb = T - tau[b] - in->dur[b];
            if (sb < sa || (sb == sa && pos[b] < pos[a])) break;
            Wnext[q] = b;
            --q;
        }
        Wnext[q] = a;
    }
    C2 = fbi_decode(in, &P, mode, Wnext, S);
out:
    free(Q.off); free(Q.list); free(S); free(tau); free(pos); free(Wb);
    free_preds(&P);
    return C2;
}

int orc_fbi(const orc_instance *in, int mode, int *W, int *passes) {
    const int N = in->n;
    if (mode == ORC_AUTO) mode = orc_select_mode(in);
    int *Wf = (int *)malloc(sizeof(int) * (size_t)N);
    int *S = (int *)malloc(sizeof(int) * (size_t)N);
    int np = 0, C = -1;
    if (!Wf || !S) goto out;
    C = mode == ORC_TIME ? orc_decode_time(in, W, S, NULL) : orc_decode_capacity(in, W, S, NULL);
    for (;;) {
        int C2 = orc_fbi_pass(in, mode, W, Wf, NULL, NULL);
        if (!(C2 >= 0 && C2 < C)) break;           /* F3 */
        memcpy(W, Wf, sizeof(int) * (size_t)N);
        C = C2;
        ++np;
    }
out:
    if (passes) *passes = np;
    free(Wf); free(S);
    return C;
}

/* -------------- Sec. 6.1: co-operation through a working set ------------ */
/*
 * The paper's blocks run asynchronously and lock the working set, so the
 * order of their exchanges is not defined.  Readings:
 *   C1  The B searches advance in lockstep, one iteration each; after every
 *       iteration come the exchanges: first all writes, then all reads,
 *       each in block order.
 *   C2  C*_max (aspiration threshold, Eq. 8) is the best makespan known when
 *       the iteration starts: the working set's best and every block's best
 *       since its last read.
 *   C3  A block exchanges when its best makespan since its last read is
 *       below the makespan of the solution it read (an improvement), or
 *       when more than I_assigned iterations have passed since that read.
 *   C4  A write goes to the slot the block last read, and only if the
 *       block's best list is better than what the slot holds now; it stores
 *       that list and makespan, the block's tabu list (entries, write index,
 *       cache), IC = the IC read plus the block's iterations since the read,
 *       and clears the slot's read count Phi.  Without a write the slot's IC
 *       grows by the block's iterations since the read.
 *   C5  Reads take slots round robin (one pointer for all blocks, starting
 *       at slot 0), add one to the slot's Phi and copy list, makespan and
 *       tabu state.  If then Phi > Phi_max, Phi_steps random feasible swaps
 *       follow: each takes the block's next random word w and applies the
 *       floor(w * n_f / 2^32)-th of the n_f feasible swaps (u-major order,
 *       v - u <= delta); the new makespan is decoded and not counted.
 *   C6  Eq. 8's quantity factor, printed as (1/5) I_block / I_total, is read
 *       as I_block / 5 (every block reads at least five solutions):
 *       I_assigned = floor(I_block/5 * (0.8 e^{-100 (C^k/C* - 1)} +
 *       0.2 e^{-4 IC^k / I_block})).  e^{-x} is computed as
 *       (sum_{i=0..24} (-x/1024)^i / i!)^(2^10), Horner form, IEEE double
 *       without contraction, 0 for x > 700.  assign_fixed > 0 replaces it.
 *   C7  Slot k starts from the level order with slot k's shuffle keys
 *       (Sec. 4.1); with fbi_every = e > 0 the slots k = e-1, 2e-1, ... are
 *       improved by FBI first (the paper: every second solution, e = 2).
 *   C8  The search ends when the blocks have run I_block iterations each or,
 *       with stop_at_cp, when C* equals the critical path at the start of
 *       an iteration.  The result is the best slot (lowest index), unless a
 *       block's best since its last read is strictly better (lowest block).
 *       Iterations, evaluated schedules and work add up over the blocks.
 */

double orc_exp_neg(double x) {
    if (x > 700.0) return 0.0;
    double y = x / 1024.0;
    double t = 1.0;
    for (int i = 24; i >= 1; --i) t = 1.0 - (y * t) / (double)i;
    for (int k = 0; k < 10; ++k) t = t * t;
    return t;
}

int orc_assigned_iterations(int c_k, int c_star, long long ic_k, int i_block) {
    if (i_block <= 0) return 0;
    double xq = c_star > 0 ? 100.0 * ((double)c_k / (double)c_star - 1.0) : 0.0;
    double xi = 4.0 * ((double)ic_k / (double)i_block);
    double quality = orc_exp_neg(xq);
    double intact = orc_exp_neg(xi);
    double a = 0.8 * quality;
    double b = 0.2 * intact;
    double v = ((double)i_block / 5.0) * (a + b);
    return (int)v;                      /* v >= 0: truncation is the floor */
}

int orc_diversify(const orc_instance *in, int *W, int delta, int steps, const unsigned *words,
                  int P, int *cursor) {
    int N = in->n, done = 0;
    for (int s = 0; s < steps; ++s) {
        int nf = 0;
        for (int u = 1; u <= N - 2; ++u)
            for (int v = u + 1; v <= N - 2 && v - u <= delta; ++v)
                nf += orc_move_feasible(in, W, u, v);
        if (nf == 0) break;
        unsigned w = words[*cursor % P];
        *cursor += 1;
        int pick = (int)(((unsigned long long)w * (unsigned long long)nf) >> 32);
        int k = 0, applied = 0;
        for (int u = 1; u <= N - 2 && !applied; ++u)
            for (int v = u + 1; v <= N - 2 && v - u <= delta; ++v) {
                if (!orc_move_feasible(in, W, u, v)) continue;
                if (k++ == pick) {
                    int x = W[u]; W[u] = W[v]; W[v] = x;
                    applied = 1;
                    break;
                }
            }
        ++done;
    }
    return done;
}

typedef struct {          /* tabu state: Alg. 3's list and cache */
    int *tlU, *tlV;
    char *cache;          /* N x N */
    int widx;
} tabu_t;

typedef struct {          /* one slot k of the working set F */
    int *W;
    tabu_t T;
    int C, phi;
    long long IC;
} slot_t;

typedef struct {          /* one co-operating search (a block) */
    int *W, *Wbb;         /* current list, best list since the last read */
    tabu_t T;
    int C, Cbb;           /* current makespan, best since the last read */
    int slot, Cread, since, assigned, cursor;
    long long ICread;
} cblock_t;

static void tabu_copy(tabu_t *dst, const tabu_t *src, int N, int L) {
    memcpy(dst->tlU, src->tlU, sizeof(int) * (size_t)L);
    memcpy(dst->tlV, src->tlV, sizeof(int) * (size_t)L);
    memcpy(dst->cache, src->cache, (size_t)N * (size_t)N);
    dst->widx = src->widx;
}

static int tabu_alloc(tabu_t *t, int N, int L) {
    t->tlU = (int *)calloc((size_t)L, sizeof(int));
    t->tlV = (int *)calloc((size_t)L, sizeof(int));
    t->cache = (char *)calloc((size_t)N * (size_t)N, 1);
    t->widx = 0;
    return t->tlU && t->tlV && t->cache ? 0 : -1;
}

static void tabu_free(tabu_t *t) { free(t->tlU); free(t->tlV); free(t->cache); }

static void coop_log(orc_coop_event *log, int cap, int *len, int it, int b, int kind, int slot, int c,
                     int assigned, int div, int phi, long long ic) {
    if (!log || *len >= cap) { if (log) ++*len; return; }
    orc_coop_event *e = &log[*len];
    e->iteration = it; e->block = b; e->kind = kind; e->slot = slot; e->cmax = c;
    e->assigned = assigned; e->diversified = div; e->phi = phi; e->ic = ic;
    ++*len;
}

int orc_coop_search(const orc_instance *in, const orc_params *p, const orc_coop_params *cp,
                    const int *const *slot_keys, const unsigned *words, orc_result *res,
                    orc_coop_event *log, int log_cap, int *log_len) {
    const int N = in->n, B = cp->blocks, F = cp->working_set, L = p->tabu_len;
    const int Ib = p->iterations;
    int log_n = 0;
    res->status = 0;
    if (N < 2 || L < 1 || p->max_swap_dist < 1 || Ib < 0 || B < 1 || F < 1 || cp->phi_steps < 0 ||
        (cp->phi_steps > 0 && (!words || cp->words_per_block < 1))) {
        res->status = -1;
        return -1;
    }
    const int mode = p->eval_mode == ORC_AUTO ? orc_select_mode(in) : p->eval_mode;
    preds_t P;
    if (build_preds(in, &P) != 0) { res->status = -1; return -1; }
    slot_t *slot = (slot_t *)calloc((size_t)F, sizeof(slot_t));
    cblock_t *blk = (cblock_t *)calloc((size_t)B, sizeof(cblock_t));
    int *Wc = (int *)malloc(sizeof(int) * (size_t)N);
    int *S = (int *)malloc(sizeof(int) * (size_t)N);
    char *exch = (char *)calloc((size_t)B, 1);
    int ok = slot && blk && Wc && S && exch;
    for (int k = 0; ok && k < F; ++k) {
        slot[k].W = (int *)malloc(sizeof(int) * (size_t)N);
        ok = slot[k].W && tabu_alloc(&slot[k].T, N, L) == 0;
    }
    for (int b = 0; ok && b < B; ++b) {
        blk[b].W = (int *)malloc(sizeof(int) * (size_t)N);
        blk[b].Wbb = (int *)malloc(sizeof(int) * (size_t)N);
        ok = blk[b].W && blk[b].Wbb && tabu_alloc(&blk[b].T, N, L) == 0;
    }
    if (!ok) { res->status = -1; goto done; }
    res->mode = mode;
    res->cp = orc_critical_path(in);
#define DECODE(Wl, work_ptr) (mode == ORC_TIME ? decode_time(in, &P, (Wl), S, (work_ptr)) \
                                               : decode_capacity(in, &P, (Wl), S, (work_ptr)))
    /* C7: the initial working set */
    for (int k = 0; k < F; ++k) {
        orc_instance ik = *in;
        if (slot_keys) ik.level_key = slot_keys[k];
        if (orc_initial_order(&ik, slot[k].W) != 0) { res->status = -1; goto done; }
        if (cp->fbi_every > 0 && k % cp->fbi_every == cp->fbi_every - 1)
            orc_fbi(in, mode, slot[k].W, NULL);                       /* C7 */
        slot[k].C = DECODE(slot[k].W, NULL);
        slot[k].phi = 0;
        slot[k].IC = 0;
    }
    int Cstar = slot[0].C;
    for (int k = 1; k < F; ++k) if (slot[k].C < Cstar) Cstar = slot[k].C;
    int rp = 0, its = 0;
    long long evaluated = 0, work = 0;
    /* C5: a read of block b */
#define READ_SLOT(b_, itlog)                                                              \
    do {                                                                                  \
        cblock_t *x_ = &blk[(b_)];                                                        \
        int k_ = rp;                                                                      \
        rp = (rp + 1) % F;                                                                \
        slot[k_].phi += 1;                                                                \
        memcpy(x_->W, slot[k_].W, sizeof(int) * (size_t)N);                               \
        tabu_copy(&x_->T, &slot[k_].T, N, L);                                             \
        x_->slot = k_;                                                                    \
        x_->Cread = slot[k_].C;                                                           \
        x_->ICread = slot[k_].IC;                                                         \
        x_->since = 0;                                                                    \
        int div_ = 0;                                                                     \
        if (slot[k_].phi > cp->phi_max && cp->phi_steps > 0) {                            \
            div_ = orc_diversify(in, x_->W, p->max_swap_dist, cp->phi_steps,               \
                                 words + (size_t)(b_) * (size_t)cp->words_per_block,      \
                                 cp->words_per_block, &x_->cursor);                        \
            x_->C = DECODE(x_->W, NULL);                                                  \
        } else {                                                                          \
            x_->C = slot[k_].C;                                                           \
        }                                                                                 \
        x_->Cbb = x_->C;                                                                  \
        memcpy(x_->Wbb, x_->W, sizeof(int) * (size_t)N);                                  \
        x_->assigned = cp->assign_fixed > 0 ? cp->assign_fixed                            \
                                            : orc_assigned_iterations(slot[k_].C, Cstar,  \
                                                                      slot[k_].IC, Ib);   \
        coop_log(log, log_cap, &log_n, (itlog), (b_), 2, k_, x_->C, x_->assigned, div_,   \
                 slot[k_].phi, slot[k_].IC);                                              \
    } while (0)

    for (int b = 0; b < B; ++b) READ_SLOT(b, -1);
    for (int b = 0; b < B; ++b) if (blk[b].Cbb < Cstar) Cstar = blk[b].Cbb;   /* C2 */
    while (its < Ib) {
        if (p->stop_at_cp && Cstar == res->cp) break;                 /* C8 */
        const int Casp = Cstar;
        /* one Sec. 6 iteration of every block (as orc_tabu_search) */
        for (int b = 0; b < B; ++b) {
            cblock_t *x = &blk[b];
            int found = 0, bu = 0, bv = 0, bc = INT_MAX;
            for (int u = 1; u <= N - 2; ++u)
                for (int v = u + 1; v <= N - 2 && v - u <= p->max_swap_dist; ++v) {
                    if (!orc_move_feasible(in, x->W, u, v)) continue;
                    memcpy(Wc, x->W, sizeof(int) * (size_t)N);
                    Wc[u] = x->W[v];
                    Wc[v] = x->W[u];
                    int c = DECODE(Wc, &work);
                    ++evaluated;
                    int tabu = x->T.cache[u * N + v];                /* Alg. 2 */
                    if (tabu && !(c < Casp)) continue;              /* aspiration, C2 */
                    if (!found || c < bc) { found = 1; bu = u; bv = v; bc = c; }
                }
            if (found) {
                int t = x->W[bu]; x->W[bu] = x->W[bv]; x->W[bv] = t;
                x->C = bc;
            } else {
                bu = 0; bv = 0;
            }
            int uo = x->T.tlU[x->T.widx], vo = x->T.tlV[x->T.widx];  /* Alg. 3 */
            x->T.cache[uo * N + vo] = 0;
            x->T.tlU[x->T.widx] = bu;
            x->T.tlV[x->T.widx] = bv;
            x->T.cache[bu * N + bv] = 1;
            x->T.widx = (x->T.widx + 1) % L;
            if (x->C < x->Cbb) {
                x->Cbb = x->C;
                memcpy(x->Wbb, x->W, sizeof(int) * (size_t)N);
            }
            x->since += 1;
        }
        its += 1;
        for (int b = 0; b < B; ++b) if (blk[b].Cbb < Cstar) Cstar = blk[b].Cbb;
        /* C3, C4: writes in block order */
        for (int b = 0; b < B; ++b) {
            cblock_t *x = &blk[b];
            int improved = x->Cbb < x->Cread;
            exch[b] = (char)(improved || x->since > x->assigned);
            if (!exch[b]) continue;
            slot_t *f = &slot[x->slot];
            if (improved && x->Cbb < f->C) {
                memcpy(f->W, x->Wbb, sizeof(int) * (size_t)N);
                tabu_copy(&f->T, &x->T, N, L);
                f->C = x->Cbb;
                f->IC = x->ICread + x->since;
                f->phi = 0;
                coop_log(log, log_cap, &log_n, its, b, 1, x->slot, f->C, 0, 0, f->phi, f->IC);
            } else {
                f->IC += x->since;
                if (improved)
                    coop_log(log, log_cap, &log_n, its, b, 3, x->slot, x->Cbb, 0, 0, f->phi, f->IC);
            }
        }
        /* C5: reads in block order */
        if (its < Ib)
            for (int b = 0; b < B; ++b)
                if (exch[b]) READ_SLOT(b, its);
        for (int b = 0; b < B; ++b) if (blk[b].Cbb < Cstar) Cstar = blk[b].Cbb;
    }
    /* C8: the result */
    {
        const int *Wb = slot[0].W;
        int Cb = slot[0].C;
        for (int k = 1; k < F; ++k)
            if (slot[k].C < Cb) { Cb = slot[k].C; Wb = slot[k].W; }
        for (int b = 0; b < B; ++b)
            if (blk[b].Cbb < Cb) { Cb = blk[b].Cbb; Wb = blk[b].Wbb; }
        memcpy(res->best_W, Wb, sizeof(int) * (size_t)N);
        res->best_cmax = mode == ORC_TIME ? decode_time(in, &P, res->best_W, res->best_S, NULL)
                                          : decode_capacity(in, &P, res->best_W, res->best_S, NULL);
        if (res->best_cmax != Cb || Cb != Cstar) res->status = -2;   /* self-check */
    }
    res->iterations = its * B;
    res->evaluated = evaluated;
    res->work = work;
#undef READ_SLOT
#undef DECODE
done:
    if (log_len) *log_len = log_n;
    if (slot)
        for (int k = 0; k < F; ++k) { free(slot[k].W); tabu_free(&slot[k].T); }
    if (blk)
        for (int b = 0; b < B; ++b) { free(blk[b].W); free(blk[b].Wbb); tabu_free(&blk[b].T); }
    free(slot); free(blk); free(Wc); free(S); free(exch);
    free_preds(&P);
    return res->status;
}

/* -------------------- brute force over activity lists -------------------- */
typedef struct {
    const orc_instance *in;
    const preds_t *P;
    int mode;
    int *W;
    int *S;
    char *used;
    int best;
    long long lists;
} bfl_t;

static void bfl_rec(bfl_t *b, int pos) {
    const orc_instance *in = b->in;
    int N = in->n;
    if (pos == N - 1) {
        b->W[pos] = N - 1;
        int c = b->mode == ORC_TIME ? decode_time(in, b->P, b->W, b->S, NULL)
                                    : decode_capacity(in, b->P, b->W, b->S, NULL);
        b->lists++;
        if (c >= 0 && c < b->best) b->best = c;
        return;
    }
    for (int i = 1; i < N - 1; ++i) {
        if (b->used[i]) continue;
        int ok = 1;
        for (int e = b->P->off[i]; e < b->P->off[i + 1]; ++e)
            if (!b->used[b->P->list[e]]) { ok = 0; break; }
        if (!ok) continue;
        b->used[i] = 1;
        b->W[pos] = i;
        bfl_rec(b, pos + 1);
        b->used[i] = 0;
    }
}

int orc_brute_force_lists(const orc_instance *in, int mode, long long *lists) {
    int N = in->n;
    preds_t P;
    if (build_preds(in, &P) != 0) return -1;
    bfl_t b = {in, &P, mode, (int *)malloc(sizeof(int) * (size_t)N),
               (int *)malloc(sizeof(int) * (size_t)N), (char *)calloc((size_t)N, 1), INT_MAX, 0};
    b.W[0] = 0;
    b.used[0] = 1;
    bfl_rec(&b, 1);
    if (lists) *lists = b.lists;
    free(b.W); free(b.S); free(b.used);
    free_preds(&P);
    return b.best;
}

/* --------------- brute force over left-justified start times -------------
 * Any feasible schedule can be shifted left until every activity starts at
 * time 0 or at the finish of an activity that started earlier, without
 * lengthening it.  Enumerating activities in non-decreasing start order and
 * giving each a start from {0} U {finish times so far} therefore reaches an
 * optimal schedule.  Nothing here uses a schedule generation scheme. */
typedef struct {
    const orc_instance *in;
    const preds_t *P;
    int H;
    int *usage;      /* [M*H] */
    int *S;
    char *placed;
    int *tail;       /* longest path from i to the sink, d_i included */
    int best;
} bfs_t;

static void bfs_rec(bfs_t *b, int count, int last_start, int maxfin) {
    const orc_instance *in = b->in;
    int N = in->n, M = in->m;
    if (maxfin >= b->best) return;
    if (count == N) { b->best = maxfin; return; }
    for (int i = 0; i < N; ++i)
        if (!b->placed[i] && last_start + b->tail[i] >= b->best) return;
    for (int i = 0; i < N; ++i) {
        if (b->placed[i]) continue;
        int es = 0, ok = 1;
        for (int e = b->P->off[i]; e < b->P->off[i + 1]; ++e) {
            int j = b->P->list[e];
            if (!b->placed[j]) { ok = 0; break; }
            es = imax(es, b->S[j] + in->dur[j]);
        }
        if (!ok) continue;
        /* candidate starts: 0 and every finish time so far */
        for (int cidx = -1; cidx < N; ++cidx) {
            int s;
            if (cidx < 0) s = 0;
            else if (b->placed[cidx]) s = b->S[cidx] + in->dur[cidx];
            else continue;
            if (s < es || s < last_start) continue;
            int dup = 0;                       /* skip repeated candidate values */
            for (int c2 = -1; c2 < cidx; ++c2) {
                int s2 = c2 < 0 ? 0 : (b->placed[c2] ? b->S[c2] + in->dur[c2] : -1);
                if (s2 == s) { dup = 1; break; }
            }
            if (dup) continue;
            if (s + in->dur[i] > b->H) continue;
            int fits = 1;
            for (int k = 0; k < M && fits; ++k)
                for (int t = s; t < s + in->dur[i]; ++t)
                    if (b->usage[k * b->H + t] + in->req[i * M + k] > in->cap[k]) { fits = 0; break; }
            if (!fits) continue;
            for (int k = 0; k < M; ++k)
                for (int t = s; t < s + in->dur[i]; ++t) b->usage[k * b->H + t] += in->req[i * M + k];
            b->placed[i] = 1;
            b->S[i] = s;
            bfs_rec(b, count + 1, s, imax(maxfin, s + in->dur[i]));
            b->placed[i] = 0;
            for (int k = 0; k < M; ++k)
                for (int t = s; t < s + in->dur[i]; ++t) b->usage[k * b->H + t] -= in->req[i * M + k];
        }
    }
}

int orc_brute_force_starts(const orc_instance *in) {
    int N = in->n, M = in->m, H = 0;
    for (int i = 0; i < N; ++i) H += in->dur[i];
    preds_t P;
    if (build_preds(in, &P) != 0) return -1;
    int *order = (int *)malloc(sizeof(int) * (size_t)N);
    bfs_t b = {in, &P, H > 0 ? H : 1, (int *)calloc((size_t)M * (size_t)(H > 0 ? H : 1), sizeof(int)),
               (int *)calloc((size_t)N, sizeof(int)), (char *)calloc((size_t)N, 1),
               (int *)calloc((size_t)N, sizeof(int)), H + 1};
    if (topo_order(in, order) != 0) { b.best = -1; goto out; }
    for (int a = N - 1; a >= 0; --a) {
        int i = order[a], t = 0;
        for (int e = in->succ_off[i]; e < in->succ_off[i + 1]; ++e) t = imax(t, b.tail[in->succ[e]]);
        b.tail[i] = t + in->dur[i];
    }
    bfs_rec(&b, 0, 0, 0);
out:
    free(order); free(b.usage); free(b.S); free(b.placed); free(b.tail);
    free_preds(&P);
    return b.best;
}
