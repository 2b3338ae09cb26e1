/*
 * icd2s.h -- C ABI of the GB300 (sm_103a) IC-D2S hot path.
 *
 * IC-D2S (Abdollahi, Kamal, Pedram, ASP-DAC'25) minimises the QUBO objective
 * f(x) = x^T Q x over binary x for a symmetric integer Q (Eq. 1).  This
 * library runs the data-parallel part of its loop (Algorithm 2) on one GPU:
 * Tabu search (Algorithm 1), the control parameters (Eq. 6-8, Algorithm 3),
 * subQUBO selection and the emulated Ising machine (Eq. 4, Algorithm 4),
 * the write-back of accepted flips into exact int32 gain vectors, and the
 * mutation operator with its cosine rate schedule (Eq. 5).
 *
 * Conventions, for every entry point:
 *  - Return value: ICD2S_OK (0) or a negative ICD2S_ERR_* code; the message of
 *    the last failure on the calling thread is returned by icd2s_last_error().
 *  - Host pointers are read (or written) during the call only; the caller
 *    keeps ownership.
 *  - Device pointers ("_dev") are borrowed for the duration of the work the
 *    call enqueues on `stream`; they must stay valid until that work is done.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Calls that return host data synchronise that stream.
 *  - Handles are not thread-safe: one thread at a time per handle.
 *  - All energies are exact int64; gains are exact int32 (|g| <= 128 + 256 (n - 1)).
 *  - Limits: 1 <= n <= 16384, entries of Q are int8, 1 <= replicas <= 4096,
 *    subQUBO size 1..256, sweeps 1..16384.  Violations return ICD2S_ERR_RANGE /
 *    ICD2S_ERR_ARG.
 *  - Random numbers are Philox4x32-10 (Salmon et al., SC'11) keyed by the
 *    64-bit seed; every draw is a pure function of (seed, counter), so
 *    results do not depend on launch geometry or scheduling.
 */
#ifndef ICD2S_H
#define ICD2S_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ICD2S_OK 0
#define ICD2S_ERR_ARG (-1)        /* bad argument (null pointer, size mismatch, ...) */
#define ICD2S_ERR_ASYMMETRIC (-2) /* Q is not symmetric */
#define ICD2S_ERR_RANGE (-3)      /* a size is beyond the supported limits */
#define ICD2S_ERR_OOM (-4)        /* device allocation failed */
#define ICD2S_ERR_CUDA (-5)       /* a CUDA call failed; see icd2s_last_error() */
#define ICD2S_ERR_TIMEOUT (-6)    /* a bounded device-side wait gave up */
#define ICD2S_ERR_INVARIANT (-7)  /* tracked gains/energies differ from a recompute */
#define ICD2S_ERR_STATE (-8)      /* call made in the wrong order (e.g. mutate before select) */

typedef struct icd2s_qubo icd2s_qubo;   /* device copy of Q and its per-instance data */
typedef struct icd2s_state icd2s_state; /* z solutions (replicas) with gains and energies */
typedef struct icd2s_mlp icd2s_mlp;     /* proposal network of the learned selection */

/* Solver parameters (Algorithm 2; defaults from Table 1 via icd2s_default_params). */
typedef struct icd2s_params {
    int32_t z;          /* solutions (replicas) in S */
    int32_t K;          /* subQUBOs per solution per Ising-machine call (multi-IM fabric) */
    int32_t m_min;      /* subQUBO size range; m_min == m_max for the plain method */
    int32_t m_max;
    int32_t m_init;     /* block size of Call_IM_Solution_Set (0: m_max) */
    int32_t alpha;      /* Tabu iterations per call (Algorithm 1) */
    int32_t c;          /* Tabu tenure increment, 1 <= c <= n */
    int32_t sweeps;     /* anneal sweeps per subQUBO */
    double T_max;       /* cosine temperature schedule of the emulated Ising machine */
    double T_min;
    int64_t w1, w2, w3; /* aggregation weights, Q16 fixed point (65536 = 1.0), |w| <= 2^24 */
    int32_t mut_mode;   /* 0: rate r_t of Eq. 5; 1: constant rate mut_rate */
    double mut_rate;
    int32_t patience;   /* stop after this many iterations without a new best (<= 0: off) */
    int32_t max_iters;  /* hard cap on outer iterations */
    int32_t use_graph;  /* 1: icd2s_step / icd2s_run replay one captured CUDA graph per outer
                           iteration (re-captured when parameters or tuning change); the
                           iteration number and mutation rate are then read from device memory.
                           Results are identical; per-phase timing and traces are not available. */
    int32_t refresh_every; /* > 0: icd2s_run recomputes all gains and energies on the tensor cores
                              every this many iterations and fails with ICD2S_ERR_INVARIANT if
                              they differ from the tracked ones (see icd2s_refresh) */
    int32_t select_mode;   /* subset S' of Algorithm 4: 0 = the highest A (the paper's rule);
                              1 = the highest score of the proposal network attached with
                              icd2s_state_set_mlp (learned selection); 2 = learned on even
                              replicas, the paper's rule on odd ones.  A always ranks the
                              mutation candidates. */
    int32_t stop_at_target;/* 1: icd2s_run / icd2s_state_run stop as soon as the best energy is
                              <= target_E and report the device time to reach it */
    int64_t target_E;
    int32_t im_mode;       /* Ising machine: 0 = the cosine-schedule annealer; 1 = exact (every
                              assignment of the subQUBO is tried; m_max, m_init <= 24) */
    int32_t ablation;      /* the simplified versions of Section 4 (Fig. 23): 0 = the method;
                              1 = No_IM (no Ising-machine call, neither in Call_IM_Solution_Set nor
                              in the main loop, where the mutation then ranges over all variables); 2 = No_SM (no control parameters: subsets
                              and mutation candidates ranked by a random key
                              Philox(ctr = (j / 4, 7 << 24, p, t)).word[j mod 4] >> 1, and each
                              candidate flips with probability 1/2).  Needs select_mode 0. */
    int32_t aspiration;    /* 1: Tabu search with the aspiration criterion the text of Section 2.4
                              describes and Algorithm 1 omits (reading S4): a tabu move is also
                              admissible when it would beat the best objective visited so far; a
                              variable moved while tabu keeps c more iterations of tabu memory, and
                              when every move is tabu the unmasked arg-min is taken */
    int32_t im_order;      /* K > 1 subQUBOs per solution (Algorithm 4 on a multi-IM fabric): 0 =
                              each built from the solution before the call and the flips merged
                              (Jacobi, reading S16); 1 = one after the other, each built from the
                              solution the earlier ones left (Gauss-Seidel, the order Section 3
                              gives Call_IM_Solution_Set) */
    int32_t t_start;       /* icd2s_state_run: 0 = a fresh run (Call_IM_Solution_Set, best reset);
                              t > 0 = resume at outer iteration t on a state restored from a
                              checkpoint (icd2s_state_restore): no initial pass, the state's best
                              solution and stale-iteration count carry on; t <= max_iters */
    int32_t reserved[1];
} icd2s_params;

/* Per-call anneal parameters (the emulated Ising machine). */
typedef struct icd2s_anneal_params {
    int32_t sweeps;
    double T_max, T_min;
    uint32_t iter;      /* iteration number mixed into the Philox counter */
    int32_t per_replica;/* subQUBOs per replica: subQUBO s belongs to replica s / per_replica */
} icd2s_anneal_params;

/* Per-call selection parameters (control parameters + top-A choice). */
typedef struct icd2s_select_params {
    int64_t w1, w2, w3; /* Q16 weights of Algorithm 3 */
    int32_t K;          /* groups (subQUBOs) per replica */
    int32_t m_min, m_max;
    uint32_t iter;      /* iteration number (drives uneven sizes) */
} icd2s_select_params;

typedef struct icd2s_mutate_params {
    int32_t mut_mode;   /* 0: Eq. 5 rate at iteration `iter`; 1: constant mut_rate */
    double mut_rate;
    uint32_t iter;
} icd2s_mutate_params;

typedef struct icd2s_stats {
    int32_t iters;           /* outer iterations completed, counted from iteration 0 (a resumed
                                run's count includes the iterations before its checkpoint) */
    int64_t best_E;          /* best energy found */
    int64_t init_best_E;     /* best energy after Call_IM_Solution_Set (resumed: at the resume) */
    int64_t anneal_attempts; /* single-flip attempts made by the emulated Ising machine */
    int64_t tabu_moves;      /* Tabu iterations summed over solutions (this call) */
    double device_ms;        /* device time of the loop (CUDA events) */
    double ttt_ms;           /* stop_at_target: device time from the start of the run (initial
                                pass included) to the end of the iteration that reached the
                                target; -1 if it was not reached */
    int32_t hit_iter;        /* iterations completed when the target was reached (0: by the
                                initial pass; -1: not reached) */
} icd2s_stats;

/* Training parameters of the proposal network (icd2s_mlp_train). */
typedef struct icd2s_train_params {
    int32_t steps;       /* Adam steps */
    int32_t batch;       /* rows per step; >= rows: every row, in order (full batch) */
    float lr, beta1, beta2, eps;   /* Adam (Kingma & Ba, ICLR'15) */
    float pos_weight;    /* weight of the y = 1 term of the loss */
    int32_t reserved[3];
} icd2s_train_params;

/* Message of the last failure on this thread ("" if none).  Never NULL. */
const char* icd2s_last_error(void);

/* ABI version (major * 100 + minor). */
int32_t icd2s_version(void);

/* Table 1 defaults for a problem of size n: z = 4, c = n / 150 clamped to
 * [2, n], alpha = 5 n, w = (1, 1, 0.5), IM size 50 (Section 4.1), K = 1,
 * 256 sweeps, T_max = 100, T_min = 1, Eq. 5 mutation rate, patience 30. */
int icd2s_default_params(int32_t n, icd2s_params* out);

/* --- Problem ---------------------------------------------------------------
 * Copies the row-major n x n int8 matrix Q_host (Eq. 1) to the device.
 * Q must be symmetric (ICD2S_ERR_ASYMMETRIC otherwise).  Also computes the
 * diagonal, the normalised weight effect eta_j = sum_i |Q_ij| (Eq. 6) and the
 * gain bound, and, for an instance whose gain bound needs the Tabu keys on
 * parity labels, Q relabeled with the even-diagonal variables first (n x ld
 * more bytes of device memory; ICD2S_ERR_OOM if they cannot be had). */
int icd2s_qubo_create(const int8_t* Q_host, int32_t n, icd2s_qubo** out);
int icd2s_qubo_destroy(icd2s_qubo* q);
int icd2s_qubo_size(const icd2s_qubo* q, int32_t* n_out);
/* The largest gain magnitude of the instance over every x, computed once at
 * creation: max_j max(|Q_jj - 2 N_j|, |Q_jj + 2 P_j|), with P_j and N_j the
 * sums of the positive and of the negative off-diagonal entries of column j
 * in magnitude (g_j = (1 - 2x_j)(Q_jj + 2 sum_{i != j} Q_ij x_i), Section 2.4;
 * the bound is attained by some x).  The Tabu search uses it to decide
 * whether a move fits a 32-bit key. */
int icd2s_qubo_gain_bound(const icd2s_qubo* q, int64_t* bound_out);

/* Eq. 1 for `count` binary rows x_dev[count][n] (dense, row stride n, values
 * 0/1) into E_dev[count] (int64).  Enqueued on `stream`. */
int icd2s_energy(icd2s_qubo* q, const uint8_t* x_dev, int32_t count, int64_t* E_dev, void* stream);

/* --- Solutions -------------------------------------------------------------
 * z = `replicas` random solutions (Generate_Initial_Solution_Set, Algorithm 2)
 * drawn from Philox with `seed`; their gains and energies are computed. */
int icd2s_state_create(icd2s_qubo* q, int32_t replicas, uint64_t seed, icd2s_state** out);
int icd2s_state_destroy(icd2s_state* st);

/* A replica shard: replicas replica_base .. replica_base + replicas - 1 of a
 * solution set of replicas_total, for running one problem over several GPUs
 * (one shard per GPU).  Every random draw of the method (the initial
 * solutions, the subQUBO sizes, the annealer's and the mutation's streams,
 * the No_SM ranking) is keyed by the global replica index, so the shards
 * together make exactly the solution set that icd2s_state_create(q,
 * replicas_total, seed) makes.  The replicas interact only through gamma
 * (Eq. 8: column sums over all z solutions) and the best solution
 * (Algorithm 2): a shard steps with icd2s_step_shard_begin / _finish (the
 * caller adds up the shards' column counts in between) and reports its best
 * with icd2s_get_best_info.  icd2s_step, icd2s_run and icd2s_select_subqubos
 * return ICD2S_ERR_STATE on a shard with replicas < replicas_total; params
 * take z = replicas_total.  ERR_ARG if the shard lies outside the set. */
int icd2s_state_create_shard(icd2s_qubo* q, int32_t replicas, int32_t replica_base, int32_t replicas_total,
                             uint64_t seed, icd2s_state** out);

/* Replaces the solutions with x[replicas][n] (0/1; on the host when
 * x_is_device == 0, else on the device) and recomputes gains and energies. */
int icd2s_state_load(icd2s_state* st, const uint8_t* x, int32_t x_is_device, void* stream);

/* Copies the solutions, gains and energies to host arrays x[replicas][n],
 * g[replicas][n], E[replicas]; any pointer may be NULL.  Synchronises. */
int icd2s_get_state(icd2s_state* st, uint8_t* x, int32_t* g, int64_t* E);

/* Best solution seen by icd2s_best_update / icd2s_step (host copies). */
int icd2s_get_best(icd2s_state* st, uint8_t* x_best, int64_t* E_best);

/* The best solution's energy, its global replica index and when it was
 * reached: stamp = 3 t + k + 1 for the k-th best update (after the Tabu
 * search, the Ising machine, the mutation) of iteration t, 0 for
 * icd2s_best_update; replica = stamp = -1 before any update.  Across replica
 * shards the method's best (Algorithm 2, the lowest energy, first reached,
 * lowest replica at that update) is the shard best with the smallest
 * (E, stamp, replica).  Synchronises. */
int icd2s_get_best_info(icd2s_state* st, int64_t* E_best, int32_t* replica, int32_t* stamp);

/* --- Checkpoint and resume (no counterpart in the paper) ---------------------
 * A checkpoint holds what the later outer iterations read from a state: the
 * solutions (gains and energies are recomputed from them on restore), the
 * best solution and energy, the count of iterations without a new best, the
 * selection hit counts of the learned selection, the Philox seed and the next
 * iteration number t_next.  Every random number of iteration t is Philox of
 * (seed, t, slot, tag), so a state restored from a checkpoint taken after
 * iteration t_next - 1 and stepped from t_next on (icd2s_step, or
 * icd2s_state_run with t_start = t_next) gives the uninterrupted run's
 * solutions bit for bit.  Not included: the tuning (results do not depend on
 * it), the improvement log (a resumed run starts a new one) and the attached
 * network (icd2s_mlp_get_weights / icd2s_mlp_set_weights).
 *
 * Format (byte offsets, little-endian): 0 magic "ICD2SCKP"; 8 uint32 version
 * 1; 12 int32 n; 16 int32 replicas; 20 int32 t_next; 24 uint64 seed; 32 int64
 * best energy; 40 int32 stale iterations; 44 uint32 0; 48 uint64 payload bytes
 * P = 5 replicas n + n; 56 uint64 0; 64 payload: x [replicas][n] uint8, best x
 * [n] uint8, hit counts [replicas][n] int32; 64 + P: uint64 FNV-1a (64-bit) of
 * bytes 0 .. 64 + P - 1.  Total 72 + P bytes. */

/* Writes the checkpoint of `st` into buf[cap] (host memory) and its size to
 * *bytes (may be NULL).  buf == NULL: only the size.  ICD2S_ERR_RANGE if cap
 * is too small; ICD2S_ERR_ARG if t_next < 0.  Synchronises the device. */
int icd2s_state_save(icd2s_state* st, int32_t t_next, void* buf, size_t cap, size_t* bytes);

/* Checks a checkpoint without a state (host only, no CUDA call) and returns
 * its n, replicas, t_next and seed (each pointer may be NULL).
 * ICD2S_ERR_ARG: too short, wrong magic or version, sizes that disagree with
 * n and replicas, or entries of x that are not 0/1; ICD2S_ERR_INVARIANT: the
 * checksum differs (a corrupted checkpoint). */
int icd2s_checkpoint_info(const void* buf, size_t bytes, int32_t* n, int32_t* replicas, int32_t* t_next,
                          uint64_t* seed);

/* Replaces everything a checkpoint holds in `st` (whose n and replicas must
 * equal the checkpoint's: ICD2S_ERR_ARG otherwise), including its seed, and
 * recomputes gains and energies; *t_next (may be NULL) receives the iteration
 * to continue with.  The checks of icd2s_checkpoint_info come first: a bad
 * checkpoint leaves the state unchanged.  Synchronises the device. */
int icd2s_state_restore(icd2s_state* st, const void* buf, size_t bytes, int32_t* t_next);

/* --- The steps of one outer iteration (Algorithm 2) ------------------------ */

/* Algorithm 1 on every solution: alpha iterations of the non-tabu argmin move
 * with tenure c; each solution is replaced by the best one it visited.
 * Toggle counts T and final tabu memory C are kept for the control
 * parameters and can be read with icd2s_get_tabu. */
int icd2s_tabu(icd2s_state* st, int32_t alpha, int32_t c, void* stream);
int icd2s_get_tabu(icd2s_state* st, int32_t* T, int32_t* C);
/* icd2s_tabu with the aspiration criterion (see icd2s_params.aspiration). */
int icd2s_tabu_aspiration(icd2s_state* st, int32_t alpha, int32_t c, void* stream);

/* Control parameters and selection: gamma (Eq. 8) over the replicas, Delta
 * (Eq. 7) from the last Tabu toggle counts, A = w1 eta + w2 gamma - w3 Delta
 * (Algorithm 3, Q16), then per replica the K groups of the highest-A
 * variables (ranked by A desc, index asc), each listed in ascending index
 * order.  Writes idx_dev[sum of sizes] and off_dev[replicas * K + 1]
 * (group s = (p, k) is idx_dev[off_dev[s] .. off_dev[s+1])); both buffers
 * must hold replicas * K * m_max + 1 entries.  The selection and A are kept
 * for icd2s_mutate. */
int icd2s_select_subqubos(icd2s_state* st, const icd2s_select_params* sp, int32_t* idx_dev,
                          int32_t* off_dev, void* stream);

/* Copies A[replicas][n], gamma[n] and Delta[replicas][n] (Q16) of the last
 * selection to the host; any pointer may be NULL.  Synchronises. */
int icd2s_get_control(icd2s_state* st, int32_t* A, int32_t* gamma, int32_t* delta);

/* The emulated Ising machine (Eq. 4, Algorithm 4): for each of `count`
 * subQUBOs (indices idx_dev[off_dev[s] .. off_dev[s+1]), ascending, disjoint
 * within a replica), stage Q[S,S] and the boundary-biased diagonal, then run
 * `sweeps` single-flip Metropolis sweeps on the cosine temperature schedule.
 * All subQUBOs read the solutions as they were before the call.  Writes the
 * flip mask flips_dev[replicas][n] (1 = flipped; cleared by the call) and the
 * subQUBO energy changes dE_dev[count] (may be NULL).  Solutions are not
 * modified; apply the mask with icd2s_apply_flips_update_gains. */
int icd2s_anneal_subqubos_batch(icd2s_state* st, const int32_t* idx_dev, const int32_t* off_dev,
                                int32_t count, const icd2s_anneal_params* ap, uint8_t* flips_dev,
                                int64_t* dE_dev, void* stream);

/* Exact Ising machine for small subQUBOs (the "precise solution" of a
 * subQUBO, Section 3): for each of `count` subQUBOs (as for
 * icd2s_anneal_subqubos_batch; sizes 1..24), the assignment of its variables
 * that minimises the Eq. 4 objective with the other variables fixed, all 2^m
 * assignments tried (Gray-code order, one warp per subQUBO); ties go to the
 * smallest assignment read as sum_a y_a 2^a (position a = the a-th listed
 * variable).  Writes the changed variables to flips_dev[replicas][n]
 * (cleared by the call) and the objective change dE_dev[count] (<= 0; may be
 * NULL).  Solutions are not modified.  ICD2S_ERR_RANGE for a size above 24. */
int icd2s_exact_subqubos_batch(icd2s_state* st, const int32_t* idx_dev, const int32_t* off_dev,
                               int32_t count, int32_t per_replica, uint8_t* flips_dev, int64_t* dE_dev,
                               void* stream);

/* Flips every variable marked in flips_dev[replicas][n] and updates the
 * int32 gains g_i = (1 - 2 x_i)(Q_ii + 2 sum_{j != i} Q_ij x_j) and int64
 * energies exactly (streams the rows of Q of the flipped variables). */
int icd2s_apply_flips_update_gains(icd2s_state* st, const uint8_t* flips_dev, void* stream);

/* Mutation: per replica, the floor((n - |S'|) r) variables outside the last
 * selection S' with the highest A flip with probability given by A
 * normalised over the replica (min-max), then gains and energies are
 * updated.  r is Eq. 5 at mp->iter or a constant.  flips_dev[replicas][n]
 * receives the mutation mask when not NULL. */
int icd2s_mutate(icd2s_state* st, const icd2s_mutate_params* mp, uint8_t* flips_dev, void* stream);

/* Folds the current solutions into the best one (strictly lower energy,
 * lowest replica on ties). */
int icd2s_best_update(icd2s_state* st, void* stream);

/* Dense refresh: recomputes every gain g_i = (1 - 2x_i)(Q_ii + 2 sum_{j!=i} Q_ij x_j)
 * and energy (Eq. 1) of all replicas from scratch as H = Q X^T on the tensor
 * cores (tcgen05, BF16 operands, FP32 accumulation: exact for int8 Q and binary
 * x, since every partial sum is an integer below 2^24), and compares them with
 * the incrementally tracked values.  mismatches (host, may be NULL) receives
 * the number of differing entries and synchronises `stream`; rebuild != 0
 * replaces the tracked values with the recomputed ones (after checking,
 * synchronously, that the recompute completed).  ICD2S_ERR_TIMEOUT if a
 * bounded device-side wait of the tensor-core pipeline gave up (reported when
 * mismatches or rebuild is given); the tracked values are then left alone and
 * the state stays usable. */
int icd2s_refresh(icd2s_state* st, int32_t rebuild, int32_t* mismatches, void* stream);

/* Call_IM_Solution_Set (Algorithm 2): for each replica, floor(n / m_init)
 * disjoint blocks of m_init consecutive variables are annealed (or solved
 * exactly, im_mode 1) and written back one after the other (each sees the
 * previous ones' result).  With p->K > 1 Ising machines per solution and
 * p->im_order 0, K consecutive blocks are solved at once, each from the
 * solution before its group (Section 3: several IMs address several
 * subQUBOs concurrently). */
int icd2s_initial_pass(icd2s_state* st, const icd2s_params* p, void* stream);

/* One whole outer iteration t of Algorithm 2 on the device: Tabu, control
 * parameters, selection, Ising machine, write-back, mutation, best update.
 * Enqueued on `stream`; no host synchronisation. */
int icd2s_step(icd2s_state* st, const icd2s_params* p, int32_t t, void* stream);

/* One Ising-machine round (Algorithm 2's IM step alone): control parameters
 * and selection of the K subQUBOs per replica (Algorithm 3-4, Eq. 6-8, with
 * Delta from the last Tabu search's toggle counts), the batched anneal of all
 * replicas * K subQUBOs in one launch (Eq. 4; uneven sizes through the
 * persistent queue kernel) and the exact write-back of the flips into x, g
 * and E.  Iteration number t keys the random streams.  Enqueued on `stream`;
 * no host synchronisation.  A dense workload's drift check alternates rounds
 * with icd2s_refresh. */
int icd2s_im_round(icd2s_state* st, const icd2s_params* p, int32_t t, void* stream);

/* Outer iteration t on a replica shard, in two calls enqueued on `stream`.
 * _begin runs the Tabu search (Algorithm 1), the best update after it, the
 * learned selection's features and scores, and writes the shard's column
 * counts counts_dev[j] = sum over its replicas of x_pj (int32 [n], device).
 * The caller adds the counts of every shard (an allreduce) and passes the
 * totals to _finish, which takes gamma from them (Eq. 8 over all
 * replicas_total solutions) and runs the rest of the iteration: control
 * parameters and selection (Algorithm 3-4), Ising machine, write-back,
 * mutation (Eq. 5) and the best updates.  On a whole set (replicas ==
 * replicas_total) begin + finish with its own counts is icd2s_step. */
int icd2s_step_shard_begin(icd2s_state* st, const icd2s_params* p, int32_t t, int32_t* counts_dev, void* stream);
int icd2s_step_shard_finish(icd2s_state* st, const icd2s_params* p, int32_t t, const int32_t* counts_dev,
                            void* stream);

/* icd2s_step with host buffers: loads x_in[replicas][n] (if not NULL) into
 * the state, runs iteration t, and copies the solutions to x_out (if not
 * NULL) and energies to E_out[replicas] (if not NULL).  Synchronises. */
int icd2s_step_host(icd2s_state* st, const icd2s_params* p, int32_t t, const uint8_t* x_in,
                    uint8_t* x_out, int64_t* E_out, void* stream);

/* The whole method (Algorithm 2) from a fresh random set: returns the best
 * solution x_out[n] and its energy.  trace (optional, max_iters * (3 z + 1)
 * int64): per iteration the energies of all solutions after the Tabu
 * search, after the Ising-machine step and after the mutation, then the best
 * energy.  S_out (optional, z * n): the final solutions. */
int icd2s_run(icd2s_qubo* q, const icd2s_params* p, uint64_t seed, uint8_t* x_out, int64_t* E_out,
              icd2s_stats* stats, int64_t* trace, uint8_t* S_out);

/* icd2s_run on an existing state (its current solutions, its attached
 * proposal network and improvement log, its tuning): Call_IM_Solution_Set,
 * then outer iterations t = 0, 1, ... until max_iters, patience or the
 * target.  The state's best solution is reset to its current solutions
 * first.  Outputs as for icd2s_run. */
int icd2s_state_run(icd2s_state* st, const icd2s_params* p, uint8_t* x_out, int64_t* E_out,
                    icd2s_stats* stats, int64_t* trace, uint8_t* S_out);

/* --- Learned selection (an addition to the paper's method) -------------------
 * A proposal network scores every variable of every replica at selection
 * time from six features (reading of the method's data-driven choice of S'):
 *   f0 = x_i, f1 = g_i / (max_j |g_j| + 1), f2 = T_i / alpha, f3 = C_i / c,
 *   f4 = H_i / (t + 1), f5 = eta_hat_i / 2^16,
 * with g the gains after the Tabu search, T/C its toggle counts and final
 * tabu memory, H the selection hit counts (Ising-machine calls that included
 * variable i before iteration t) and eta_hat Eq. 6 normalised (Q16).  Each
 * quotient is the correctly rounded float quotient.  Network: 6 -> 64 ReLU ->
 * 64 ReLU -> 1, parameters flat as W1[64][6], b1[64], W2[64][64], b2[64],
 * w3[64], b3 (4673 floats; row o = weights into unit o).  It computes with the
 * BF16 roundings (nearest even) of float32 master weights, in float, one
 * fused multiply-add per product, units and inputs in increasing order.
 * S' = the highest scores (index ascending on ties; the score's IEEE bit
 * pattern orders -0 below +0). */
#define ICD2S_MLP_PARAMS 4673

/* New network with weights uniform in +-sqrt(6 / (fan_in + fan_out))
 * (Philox with `seed`), zero biases, Adam moments zero. */
int icd2s_mlp_create(uint64_t seed, icd2s_mlp** out);
int icd2s_mlp_destroy(icd2s_mlp* m);
/* Replaces the master weights (host, 4673 floats; must be finite) and
 * resets Adam. */
int icd2s_mlp_set_weights(icd2s_mlp* m, const float* W_host);
/* Host copies of the master weights and of the BF16 weights widened to
 * float (either may be NULL).  Synchronises. */
int icd2s_mlp_get_weights(icd2s_mlp* m, float* master_host, float* bf16_host);
/* Scores of the rows F_dev[rows][6] into score_dev[rows]. */
int icd2s_mlp_score(icd2s_mlp* m, const float* F_dev, int64_t rows, float* score_dev, void* stream);
/* Mean loss over all rows, l = pos_weight y softplus(-s) + (1 - y) softplus(s),
 * into loss_dev[1] and its gradient with respect to the (BF16) weights into
 * grad_dev[4673] (either may be NULL).  y_dev[rows] holds 0/1 labels.  The
 * sums are taken in a fixed order: the result does not depend on scheduling. */
int icd2s_mlp_grad(icd2s_mlp* m, const float* F_dev, const uint8_t* y_dev, int64_t rows, float pos_weight,
                   float* grad_dev, float* loss_dev, void* stream);
/* tp->steps Adam steps on mini-batches of the rows (see icd2s_train_params;
 * a batch smaller than rows draws its rows with Philox from the network's
 * seed and its running step count).  loss_host[tp->steps] (may be NULL)
 * receives each step's mean batch loss; synchronises `stream` then. */
int icd2s_mlp_train(icd2s_mlp* m, const float* F_dev, const uint8_t* y_dev, int64_t rows,
                    const icd2s_train_params* tp, float* loss_host, void* stream);

/* Where the network's gradient (icd2s_mlp_grad, icd2s_mlp_train) runs: 0 =
 * the CUDA cores in FP32 (the default), 1 = its three 64-wide contractions
 * (the layer-2 forward, the W2 gradient and the backward through W2) on the
 * tensor cores, mma.sync BF16 x BF16 -> FP32, with the activations rounded
 * to BF16 for the products; layer 1, the loss and the bias and W1 sums stay
 * FP32.  Both are deterministic.  Scores (icd2s_mlp_score, the learned
 * selection) are always FP32. */
int icd2s_mlp_set_tensor_cores(icd2s_mlp* m, int32_t enable);

/* Attaches a network to a state for select_mode 1/2 (NULL detaches).  The
 * state borrows it: it must outlive the state's use of it. */
int icd2s_state_set_mlp(icd2s_state* st, icd2s_mlp* m);
/* Features F_host[replicas][n][6] and scores score_host[replicas][n] of the
 * last step that computed them (learned mode or logging on); either may be
 * NULL.  Synchronises. */
int icd2s_get_features(icd2s_state* st, float* F_host, float* score_host);
/* Selection hit counts H_host[replicas][n] (reset by state_create/load). */
int icd2s_get_hits(icd2s_state* st, int32_t* H_host);

/* Improvement log (training data for the network, reading S22): with a
 * capacity > 0, every outer iteration that lowers the best energy appends one
 * entry: the features (at that iteration's selection time) of the replica
 * whose solution became the best, and labels y_i = 1 where the new best
 * solution differs from the best solution at the previous entry (at the
 * start of logging for the first one).  A ring buffer of `capacity` entries
 * of n rows; capacity 0 turns logging off and frees it. */
int icd2s_log_enable(icd2s_state* st, int32_t capacity);
/* entries: appended since enabling (may exceed capacity); capacity. */
int icd2s_log_info(icd2s_state* st, int32_t* entries, int32_t* capacity);
/* Copies the min(entries, capacity) stored entries in slot order (entry e is
 * in slot e mod capacity): F_out[count][n][6], y_out[count][n],
 * replica_out[count] (any may be NULL), to host memory or, with
 * out_is_device, to device memory.  Synchronises `stream`. */
int icd2s_log_copy(icd2s_state* st, float* F_out, uint8_t* y_out, int32_t* replica_out, int32_t out_is_device,
                   void* stream);

/* Per-phase device timing of icd2s_step.  When enabled, each step records
 * CUDA events on its stream around its phases; icd2s_get_phase_ms waits for
 * the last step and writes ICD2S_PHASES durations in milliseconds:
 * [0] Tabu search, [1] control parameters + selection, [2] Ising machine
 * (anneal), [3] write-back of the anneal flips, [4] mutation decision,
 * [5] write-back of the mutation flips, [6] the last best-solution update. */
#define ICD2S_PHASES 7
int icd2s_set_timing(icd2s_state* st, int32_t enable);
int icd2s_get_phase_ms(icd2s_state* st, double* ms);
/* With timing enabled: duration (ms) of the tensor-core kernel of the last
 * icd2s_refresh. */
int icd2s_get_refresh_ms(icd2s_state* st, double* ms);
/* With timing enabled: duration (ms) of the write-back kernel (without the
 * mask compaction) of the last icd2s_apply_flips_update_gains. */
int icd2s_get_apply_ms(icd2s_state* st, double* ms);

/* Kernel variants used by a state (launch configuration only: every variant
 * computes the same results bit for bit).  tabu_variant indexes the Tabu
 * kernel's (variables per thread, block size) builds, -1 = default;
 * anneal_warps_per_cta = subQUBOs per CTA of the Ising-machine kernel,
 * 0 = default.  The Tabu search packs a move into one 32-bit key (one
 * reduction per warp and per block) when every gain of the instance fits
 * beside the index: gain bound + 1 < 2^(30 - b), b = bits of n (see
 * icd2s_qubo_gain_bound); with one CTA per replica, where that fails by one
 * bit, on Q relabeled with the even-diagonal variables first, b = bits of the
 * larger class (made once at icd2s_qubo_create, n ld bytes beside Q);
 * tabu_wide_keys = 1 keeps the two-reduction 64-bit keys anyway.  tabu_rows
 * = 2 makes (once per instance, 2 n ld bytes beside Q) and uses the rows of Q
 * negated as well, so a move reads its row already multiplied by (1 - 2x_i);
 * not for instances with entries -128.  0 and 1 apply the sign per variable
 * (the default: as fast or faster on the measured sizes). */
typedef struct icd2s_tuning {
    int32_t tabu_variant;
    int32_t anneal_warps_per_cta;
    int32_t refresh_bn;       /* tensor-core refresh: replicas per tile (128 or 256; 0 = default) */
    int32_t refresh_splits;   /* tensor-core refresh: kinds 1 and 4, persistent CTAs (0 = one
                                 per SM); kind 3, K splits (0 = about one CTA per SM) */
    int32_t tabu_wide_keys;   /* 0 = compact Tabu keys where they apply, 1 = never */
    int32_t tabu_rows;        /* 0 = default (plain rows), 1 = plain rows, 2 = signed row pairs */
    int32_t anneal_scheme;    /* sweep of the Ising-machine kernel (every scheme gives the same
                                 trajectory): 0 = default (4), 1 = rounds of decisions, 2 =
                                 position by position, 3 = position by position with the next
                                 test taken for both outcomes, 4 = per sweep either 1 or 3,
                                 whichever the previous sweep's accepts predict cheaper */
    int32_t refresh_kind;     /* tensor-core refresh: 1 = a BF16 copy of Q, persistent over
                                 the SMs with tiles of 128 rows of Q (0 = default: 1); 4 = the
                                 same with tiles of 256 rows; 2 is not a valid value
                                 (ICD2S_ERR_ARG); 3 = int8 Q read as bytes
                                 and converted to BF16 in shared memory (no copy of Q:
                                 2 n ld bytes less device memory, 0.049 against 0.041 ms at
                                 n = 7000, R = 256) */
    int32_t tabu_cluster;     /* Tabu search: CTAs per replica, 1, 2 or 4 (a thread-block
                                 cluster; each CTA holds a slice of the variables and the
                                 per-move arg-min is exchanged through distributed shared
                                 memory); 0 = default: 4 where n >= 8192 and 4 x replicas
                                 <= SMs, else 1.  Results are the same for every value. */
} icd2s_tuning;
int icd2s_set_tuning(icd2s_state* st, const icd2s_tuning* t);
int icd2s_get_tuning(icd2s_state* st, icd2s_tuning* t);

/* Autotuner: times every Tabu variant that fits n (with plain rows, and with
 * signed rows where a state of the instance has asked for them through
 * tabu_rows = 2, which makes them) and every anneal CTA size
 * on this state with the parameters p (each trial restores the solutions it
 * changed), keeps the fastest for the state, and returns the choice in
 * `chosen` (may be NULL).  Synchronises `stream`. */
int icd2s_autotune(icd2s_state* st, const icd2s_params* p, icd2s_tuning* chosen, void* stream);

/* Number of kernel launches the library has made in this process. */
int icd2s_kernel_launches(uint64_t* count);

/* Testing aid for the error paths: after `count` more device allocations of
 * the library succeed, every later one fails as out of memory (the call that
 * needed it returns ICD2S_ERR_OOM) until a count < 0 switches the hook off
 * (the default).  Process-wide.  A handle stays usable after such a failure:
 * buffers that belong together are made all or none, and a later call makes
 * what is missing. */
int icd2s_debug_fail_allocations_after(int32_t count);

/* Fault injection for tests of the refresh's failure detection: the next
 * `launches` tensor-core refreshes of this state issue no operand loads and
 * bound every pipeline wait by wait_us microseconds (1..2000000), so their
 * waits time out, the kernel raises its error flag, releases its tensor
 * memory and returns, and icd2s_refresh returns ICD2S_ERR_TIMEOUT.  Later
 * refreshes run normally (waits bounded by 2 s).  launches = 0 disarms. */
int icd2s_debug_refresh_stall(icd2s_state* st, int32_t launches, int32_t wait_us);

/* Flip write-back that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code
 * whose device memory is owned and handed out by someone else (a host
 * framework with a fixed budget, a plugin inside another allocator) or that
 * must not allocate once running.  It does what
 * icd2s_apply_flips_update_gains does, on buffers the caller owns:
 *   Q_dev      int8 [n][ld]        the symmetric QUBO matrix, row stride ld
 *                                  (ld % 4 == 0, n <= ld; padding bytes unread
 *                                  for the result), 4-byte aligned
 *   flips_dev  uint8 [replicas][n] 1 = flip this variable
 *   x_dev      uint8 [replicas][ld] solutions, updated in place (4-byte aligned;
 *                                  columns n .. ld-1 are left as they are)
 *   g_dev      int32 [replicas][ld] exact gains of x_dev, updated in place
 *                                  (16-byte aligned; columns n .. ld-1 left as they are)
 *   E_dev      int64 [replicas]    energies of x_dev, updated in place
 * Its scratch (flip lists, per-replica counters, the diagonal of Q) is one
 * static device array of about 4.3 MB that every GPU loading the library
 * holds until the process exits; limits: 1 <= n <= 16384, replicas <= 4096,
 * replicas * ld <= 1048576 -- larger sizes return ICD2S_ERR_RANGE.  A call
 * made outside stream capture looks up the array's device address in the
 * current context of the current device and caches it; a call inside a
 * capture uses the cached address.  So make the first call on a device, and
 * the first after a device reset or a change of context, outside any
 * capture (a captured first call returns ICD2S_ERR_CUDA).  All calls
 * share the array: calls whose GPU work overlaps race and must be ordered by
 * the caller.  No device memory is allocated or freed. */
int icd2s_apply_flips_static(const int8_t* Q_dev, int32_t n, int32_t ld, int32_t replicas,
                             const uint8_t* flips_dev, uint8_t* x_dev, int32_t* g_dev, int64_t* E_dev,
                             void* stream);

/* Host copies of the library's tables, for checking: BETA[sweeps] (Q24
 * inverse temperatures of the cosine schedule) and NLOG[4096] (Q24 -ln). */
int icd2s_tables(int32_t sweeps, double T_max, double T_min, uint32_t* beta, uint32_t* nlog);

#ifdef __cplusplus
}
#endif
#endif /* ICD2S_H */
