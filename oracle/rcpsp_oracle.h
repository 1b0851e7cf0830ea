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
/* ---- Sec. 6.1: co-operating searches through a working set F ---------- */
typedef struct {
    int blocks;            /* B co-operating searches */
    int working_set;       /* |F| */
    int phi_max;           /* Phi_max: reads without improvement before diversification */
    int phi_steps;         /* Phi_steps: random feasible swaps of a diversification */
    int assign_fixed;      /* iterations per read; 0 = Eq. 8 */
    int words_per_block;   /* P: random words of each block, used cyclically */
    int fbi_every;         /* FBI on slots k with k % e == e-1; 0 = none (paper: 2) */
} orc_coop_params;

/* One exchange event of orc_coop_search (optional log). */
typedef struct {
    int iteration;         /* iterations every block had run; -1 = initial reads */
    int block;
    int kind;              /* 1 write, 2 read, 3 improved but the slot was better */
    int slot;
    int cmax;              /* write: C written; read: C of the block after the read */
    int assigned;          /* read: I_assigned */
    int diversified;       /* read: swaps applied */
    int phi;               /* slot's read count after the event */
    long long ic;          /* slot's iterations counter after the event */
} orc_coop_event;

/* Forward-backward improvement (Sec. 6, readings F1-F3) of the list W in
 * place with evaluator `mode`; returns the final C_max, *passes (nullable)
 * the passes that shortened it. */
int orc_fbi(const orc_instance *in, int mode, int *W, int *passes);
/* One FBI pass (F1-F2): the backward list of W's forward schedule decoded on
 * the reversed network (*T_out = its makespan T, S_back = the mirrored
 * starts T - tau_i - d_i, both nullable) and the forward list Wnext; returns
 * Wnext's forward makespan. */
int orc_fbi_pass(const orc_instance *in, int mode, const int *W, int *Wnext, int *T_out, int *S_back);
/* e^{-x} for x >= 0 in IEEE double, by the fixed recipe of reading C6. */
double orc_exp_neg(double x);
/* Eq. 8 (reading C6): iterations assigned to a read of slot k. */
int orc_assigned_iterations(int c_k, int c_star, long long ic_k, int i_block);
/* Diversification (reading C5): up to `steps` random feasible swaps of W;
 * words are taken cyclically from words[0..P-1] starting at *cursor, which
 * advances by one per swap.  Returns the swaps applied. */
int orc_diversify(const orc_instance *in, int *W, int delta, int steps, const unsigned *words,
                  int P, int *cursor);
/* B searches co-operating through |F| slots (Sec. 6.1, readings C1-C8).
 * slot_keys: NULL, or |F| pointers (each NULL or N keys) giving slot k's
 * initial order.  words: [B*P] (may be NULL when phi_steps == 0).  Result:
 * best slot / block list, iterations and evaluated summed over blocks.  log
 * (nullable) receives up to log_cap events, *log_len the number written. */
int orc_coop_search(const orc_instance *in, const orc_params *p, const orc_coop_params *cp,
                    const int *const *slot_keys, const unsigned *words, orc_result *res,
                    orc_coop_event *log, int log_cap, int *log_len);

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
