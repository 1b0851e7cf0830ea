/*
 * CPU reference ("oracle") for the parallel tabu search for the RCPSP.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, literal
 * restatement of the paper's definitions and algorithms that the CUDA path
 * is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it; the product path never does, and it
 * shares no code, header, table or helper with the CUDA library.
 *
 * Notation follows the paper: N activities (dummies 0 and N-1), durations d,
 * M renewable resources with capacities R_k, demands r_{i,k}, precedence
 * arcs E, activity list W, start times S, makespan C_max.
 *
 * Parity status: the decoders, the checker, the critical path and the
 * levels are pinned by the paper's worked example (Table 1, Fig. 4) and by
 * brute force / closed forms in the tests.  The tabu trajectory itself has
 * no external value to compare with (parity unpinned beyond the rules it
 * is made of: Algs. 1-3, Eqs. 5-6 and the selection rule of Sec. 6).
 */
#ifndef RCPSP_ORACLE_H
#define RCPSP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n;                 /* N, dummies included */
    int m;                 /* M */
    const int *dur;        /* [N] */
    const int *cap;        /* [M] */
    const int *req;        /* [N*M] row-major */
    const int *succ_off;   /* [N+1] */
    const int *succ;       /* [|E|] */
    const int *level_key;  /* [N] or NULL: tie-break inside a level */
} orc_instance;

enum { ORC_AUTO = 0, ORC_TIME = 1, ORC_CAPACITY = 2 };

typedef struct {
    int iterations;        /* iteration limit */
    int max_swap_dist;     /* delta (Sec. 4.3) */
    int tabu_len;          /* |tabuList| (Sec. 4.5) */
    int eval_mode;         /* ORC_AUTO / ORC_TIME / ORC_CAPACITY */
    int stop_at_cp;        /* stop when C*_max equals the critical path */
} orc_params;

typedef struct {
    int *best_W;           /* [N] out */
    int *best_S;           /* [N] out */
    int *trace;            /* [3*iterations] out or NULL: u, v, C per iteration */
    int best_cmax;
    int iterations;        /* iterations performed */
    int mode;              /* evaluator used */
    int cp;                /* critical-path length */
    long long evaluated;   /* neighbour schedules decoded */
    long long work;        /* Alg. 5 loop steps (TIME) or Alg. 4 loop steps (CAPACITY) */
    int status;            /* 0 ok, <0 error */
} orc_result;

/* Eq. 2-4: returns 0 if S is feasible, 1 precedence violation, 2 capacity
 * violation, 3 negative start; writes C_max = max(s_i + d_i). */
int orc_check_schedule(const orc_instance *in, const int *S, int *cmax);
/* Sec. 2: longest 0 -> N-1 path with arc (i,j) weighted d_i; -1 on a cycle. */
int orc_critical_path(const orc_instance *in);
/* Sec. 4.1: level = longest unit-weight path from activity 0. */
int orc_levels(const orc_instance *in, int *level);
/* Sec. 4.1: W = levels in ascending order; inside a level by (key, label). */
int orc_initial_order(const orc_instance *in, int *W);
/* Eqs. 5-6 checked literally; 1 feasible, 0 not. */
int orc_move_feasible(const orc_instance *in, const int *W, int u, int v);
/* Alg. 7 with Algs. 5-6 (time-indexed); returns C_max, -1 if W is not a
 * precedence-feasible list.  *work (nullable) += Alg. 5 loop steps. */
int orc_decode_time(const orc_instance *in, const int *W, int *S, long long *work);
/* Alg. 7 with Eq. 7 and Alg. 4 (capacity-indexed).  *work += Alg. 4 steps. */
int orc_decode_capacity(const orc_instance *in, const int *W, int *S, long long *work);
/* Alg. 4 on one resource array c[0..R-1]; returns the loop steps taken. */
int orc_capacity_update(int *c, int R, int r, int d, int s);
/* Sec. 5.3 selection (the printed rules are lost; see the source). */
int orc_select_mode(const orc_instance *in);
/* Sec. 6: one tabu search on one instance. */
int orc_tabu_search(const orc_instance *in, const orc_params *p, orc_result *res);
/* Many independent searches over a pool of nthreads host threads. */
int orc_tabu_search_batch(const orc_instance *in, int count, const orc_params *p,
                          orc_result *res, int nthreads);
/* Minimum C_max over every precedence-feasible list (dummies fixed),
 * decoded with `mode`; *lists (nullable) = number of lists.  Small N only. */
int orc_brute_force_lists(const orc_instance *in, int mode, long long *lists);
/* Optimum by enumerating left-justified start-time vectors; independent of
 * the schedule generation scheme.  Small N only. */
int orc_brute_force_starts(const orc_instance *in);

#ifdef __cplusplus
}
#endif
#endif
