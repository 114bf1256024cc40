/*
 * pg.h - C ABI of the GB300 parity-game solver (libpg.so).
 *
 * Greedy all-switches strategy improvement with best responses computed by
 * one-player strategy improvement, after Fearnley, "Efficient Parallel
 * Strategy Improvement for Parity Games" (arXiv 1705.02313).
 *
 * Conventions shared by every entry point:
 *  - Games are CSR int32: offsets[n+1] (offsets[0] = 0, non-decreasing,
 *    offsets[n] = m), targets[m] in [0, n), owner[n] (0 = Even, 1 = Odd),
 *    pri[n] >= 0. Every vertex has at least one out-edge (Section 2: no
 *    terminal vertices). Pairwise distinct priorities (the random workloads'
 *    permuted priorities) are ranked by the nearest-greater forest; a game
 *    whose priorities repeat runs in count-vector mode (below), which needs
 *    at most 5 distinct priorities after preprocessing and fewer than 2^24
 *    vertices, else PG_EUNSUPPORTED.
 *  - mem_kind says where caller arrays live: PG_MEM_HOST (pageable or pinned
 *    host memory) or PG_MEM_DEVICE (device memory of the context's GPU).
 *    Caller arrays are read or written during the call only and never
 *    retained. All work is ordered on the context's stream; every call
 *    returns after its results are complete (host or device).
 *  - Vertex ids in every input and output are the caller's original ids. The
 *    admissibility preprocessing (Section 3, "The algorithm": dummy Even
 *    vertices) adds k dummy vertices internally; they are reported only
 *    through pg_game_info / pg_game_dummies and the dummy_sigma arrays.
 *  - Every call returns a pg_status. No call aborts the process; on failure
 *    pg_last_error() gives a message. Games are library-owned handles freed
 *    with pg_game_free.
 *
 * Valuation encoding (Section 3, "Valuations"): with distinct priorities a
 * finite valuation Val(v) is the set of vertices on the play from v to the
 * sink, so the library reports, per vertex,
 *   val_class  1 = TOP (infinite play), 0 = finite;
 *   val_depth  number of vertices on the play before the sink (v and dummies
 *              included), -1 for TOP;
 *   val_rank   position of Val(v) in the total order of Section 3 among all
 *              finite valuations of the game (dummies included) together with
 *              the empty valuation of the sink, counted from 0; INT32_MAX for
 *              TOP.
 * Together with the strategies these determine every count vector exactly.
 *
 * Count-vector mode (games whose priorities repeat, as the verification games
 * the paper measures: Section 6, Table 1): the preprocessing gives every
 * dummy priority 0 and adds 2 to every original priority (so the dummies add
 * one priority, not k). A finite valuation is the count vector L(p) of
 * Section 3 over the d distinct priorities of G' (pg_game_levels lists them
 * in ascending order); val_counts receives it as n rows of d counts (zeros
 * for TOP); val_rank is -1 in this mode (equal valuations exist); val_class
 * and val_depth are as above. Batches and servers take distinct priorities
 * only.
 */
#ifndef PG_H
#define PG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pg_status;

#define PG_OK 0
#define PG_EINVAL 1          /* malformed arguments or CSR */
#define PG_ENOMEM 2          /* device or host allocation failed */
#define PG_ETIMEOUT 3        /* iteration cap reached (Lemma 2 bounds the inner loop) */
#define PG_ENOTADMISSIBLE 4  /* an odd cycle was met: sigma is not admissible (Section 3) */
#define PG_ECUDA 5           /* a CUDA runtime error */
#define PG_EUNSUPPORTED 6    /* input outside what this version handles */

#define PG_MEM_HOST 0
#define PG_MEM_DEVICE 1

typedef struct pg_ctx pg_ctx;
typedef struct pg_game pg_game;

/* Solution of a game (Algorithm 1, Section 4). Every pointer is caller-owned
 * and sized n (the original vertex count) unless stated; a NULL pointer skips
 * that output. Theorem 1: W_Even is the set of TOP vertices under the final
 * sigma. */
typedef struct {
    uint8_t *win;        /* 0 = Even wins, 1 = Odd wins (Section 2, winning sets) */
    int32_t *sigma;      /* Even's final strategy; -1 = the sink, -1 for Odd vertices */
    int32_t *tau;        /* Odd's best response to sigma; -1 for Even vertices */
    int8_t *val_class;   /* see the valuation encoding above */
    int32_t *val_depth;
    int32_t *val_rank;
    int8_t *dummy_sigma; /* k entries: 1 if dummy j moves on to its vertex, 0 if to the sink */
    int32_t mem_kind;    /* where the arrays above live */
    int64_t major;       /* out: outer iterations that switched Even's strategy */
    int64_t inner;       /* out: valuations computed (total inner iterations) */
    int32_t *val_counts; /* count-vector mode only: n x d counts (row per vertex); ignored otherwise */
} pg_result;

/* Options of pg_solve; pass NULL for the defaults. */
typedef struct {
    const int32_t *sigma_init;     /* nullable warm start: Even strategy (-1 = sink), n entries */
    const int32_t *tau_init;       /* nullable warm start: Odd strategy, n entries */
    const int8_t *dummy_sigma_init;/* nullable: k entries, as in pg_result */
    int32_t mem_kind;              /* where the warm-start arrays live */
    int64_t max_inner;             /* cap on valuations computed; 0 = 64 * (n' + 64) */
    int32_t reset_tau;             /* 1: SI-Reset (Section 6): after every Even switch the inner loop starts
                                      again from the initial Odd strategy (the first edge of each list of G')
                                      instead of the last best response; same major iterations, more inner */
} pg_solve_opts;

/* Valuation of one profile. Caller-owned arrays of n entries; NULL skips. */
typedef struct {
    int8_t *val_class;
    int32_t *val_depth;
    int32_t *val_rank;
    int32_t *dom;        /* TOP vertices: largest priority on the cycle reached; -1 if finite */
    int32_t mem_kind;
    int32_t *val_counts; /* count-vector mode only: n x d counts (row per vertex); ignored otherwise */
} pg_valuation;

/* Context: one GPU, one stream. device is the CUDA ordinal. pg_ctx_create
 * loads the tuning table named by PG_TUNING_FILE, if set (pg_load_tuning). */
pg_status pg_ctx_create(pg_ctx **out, int device);
/* The device's name (as the CUDA runtime reports it) into buf (cap bytes,
 * NUL-terminated, truncated to fit); used to find a device's tuning table. */
pg_status pg_device_name(int device, char *buf, int32_t cap);
void pg_ctx_destroy(pg_ctx *ctx);

/* Orders all later work of ctx on stream (a cudaStream_t, e.g. a torch
 * stream's handle); NULL selects the legacy default stream. */
pg_status pg_set_stream(pg_ctx *ctx, void *stream);

/* Message describing the last failure on ctx (never NULL). */
const char *pg_last_error(const pg_ctx *ctx);

/* Loads a game (Section 2) into library-owned device memory, validates it,
 * and runs the admissibility preprocessing of Section 3 (dummy Even vertices
 * in Odd's Even-free trap) and the internal relabelling. Returns PG_EINVAL
 * for a malformed CSR (bad offsets, a vertex without edges, a target out of
 * range, an owner other than 0/1, a negative priority, sizes beyond 2^30
 * vertices or 2^31-1 edges after preprocessing). Repeated priorities load in
 * count-vector mode (Section 5 with the count vectors of Section 3); such a
 * game returns PG_EUNSUPPORTED only beyond that mode's limits: more than 5
 * distinct priorities after preprocessing, or count digits (one per priority,
 * one bit wider than the bit length of that priority's number of vertices)
 * totalling more than 126 bits (5 priorities of 8M vertices each take 120). */
pg_status pg_load_csr(pg_ctx *ctx, int32_t n, int64_t m, const int32_t *offsets, const int32_t *targets,
                      const uint8_t *owner, const int32_t *pri, int32_t mem_kind, pg_game **out);

/* Frees a game (NULL is ignored). Waits for the work of every stream on the game's device (as cudaFree would),
 * then returns the game's memory to the pool of pg_release_cached_memory. */
void pg_game_free(pg_game *game);

/* Sizes of a loaded game: original n and m, dummies k (any pointer may be NULL). */
pg_status pg_game_info(const pg_game *game, int32_t *n, int64_t *m, int32_t *k);

/* Counters of the last valuation on game (instrumentation): walks that ran
 * out of direct steps and were finished by pointer jumping, the jumping
 * rounds, finite vertices, vertices reaching an odd cycle, parents ranked
 * by one block, parents ranked by the id-ordered scan, and the switches of
 * the last switching pass; deep = 1 if it took the ruling-set path
 * (pg_set_tuning), with its rulers and its pointer-jumping rounds over the
 * g-forest and over the rulers. */
typedef struct {
    int32_t n_pending, jump_rounds, n_fin, n_odd, n_big, n_huge, n_switch;
    int32_t deep, n_rulers, deep_rounds, rs_rounds;
} pg_counters;
pg_status pg_game_counters(const pg_game *game, pg_counters *out);

/* Count-vector mode: *d receives the number of distinct priorities of G'
 * (0 for a game with distinct priorities) and level_pri (nullable, d <= 5
 * entries) their values in G' (original priority + 2; 0 for the dummies), in
 * ascending order: column l of val_counts counts level_pri[l]. */
pg_status pg_game_levels(const pg_game *game, int32_t *d, int32_t *level_pri);

/* The vertex each dummy guards: out[j] = w for dummy j (k entries, host memory). */
pg_status pg_game_dummies(const pg_game *game, int32_t *out);

/* Full solve: Algorithm 1 (Section 4) from sigma_init (every Even vertex to
 * the sink, Section 3) and tau = the first edge of each list, or from the warm
 * start in opts. Switching takes a successor only when strictly better and
 * breaks ties by the lowest edge-list position, the sink first for Even.
 * Returns PG_ETIMEOUT if the cap on valuations is reached (results then hold
 * the last profile) and PG_ENOTADMISSIBLE if a warm start is not admissible. */
pg_status pg_solve(pg_game *game, const pg_solve_opts *opts, pg_result *out);

/* Best response to sigma (Section 4, one-player strategy improvement): the
 * inner loop of Algorithm 1 only. sigma: n entries (-1 = sink; ignored for Odd
 * vertices), dummy_sigma: k entries or NULL (all dummies to the sink, as in
 * sigma_init), tau_inout: n entries or NULL; on entry the starting Odd
 * strategy (NULL = first edges), on exit the best response. sigma must be
 * admissible; an odd cycle met on the way returns PG_ENOTADMISSIBLE.
 * iters_out (nullable, host) receives the number of valuations computed.
 * All of sigma, dummy_sigma and tau_inout use mem_kind. */
pg_status pg_best_response(pg_game *game, const int32_t *sigma, const int8_t *dummy_sigma, int32_t *tau_inout,
                           int32_t mem_kind, pg_valuation *out, int64_t *iters_out);

/* Valuation of any profile (Section 3; the pseudoforest of Section 5): class,
 * depth and rank per vertex, and for TOP vertices the dominant priority of the
 * cycle reached. An odd cycle is reported through dom (odd value) and the
 * call returns PG_ENOTADMISSIBLE after filling the outputs. */
pg_status pg_valuate(pg_game *game, const int32_t *sigma, const int8_t *dummy_sigma, const int32_t *tau,
                     int32_t mem_kind, pg_valuation *out);

/* Device time per kernel class, accumulated over calls since pg_reset_stats
 * (times only while timing is enabled; launch counts always). name is the
 * class (walk, jump, chain1, parents, big_parents, sink_scan, chain2,
 * switch_odd, switch_even); calls counts timed event pairs, launches counts
 * kernels. out has room for cap entries (host memory); count receives the
 * number of classes. The paper reports wall-clock time only (Section 6); this
 * breakdown has no counterpart there. */
typedef struct {
    char name[24];
    double ms;
    int64_t launches;
    int64_t calls;
} pg_kernel_stat;
pg_status pg_kernel_stats(const pg_game *game, pg_kernel_stat *out, int32_t cap, int32_t *count);
pg_status pg_reset_stats(pg_game *game);

/* Number of kernels launched through ctx since it was created. */
pg_status pg_launch_count(const pg_ctx *ctx, int64_t *out);

/* Results of a batch (pg_solve_batch). Per-vertex arrays are packed like the
 * inputs (game i's vertices at vtx_base[i] .. vtx_base[i+1]) and hold that
 * game's local vertex ids; NULL skips an output. dummy_sigma is packed by game
 * with dummy_base (ngames + 1 entries, host) telling where each game's dummies
 * start. major, inner and status are host arrays of ngames entries (each
 * nullable); status is PG_OK, PG_ETIMEOUT or PG_ENOTADMISSIBLE per game. */
typedef struct {
    uint8_t *win;
    int32_t *sigma;
    int32_t *tau;
    int8_t *val_class;
    int32_t *val_depth;
    int32_t *val_rank;
    int8_t *dummy_sigma;
    int32_t mem_kind;      /* where the per-vertex and dummy arrays live */
    int64_t *major;        /* host, ngames */
    int64_t *inner;        /* host, ngames */
    int32_t *status;       /* host, ngames */
    int64_t *dummy_base;   /* host, ngames + 1, out */
    int64_t iterations;    /* out: lockstep iterations run for the whole batch */
    double load_ms, pack_ms, loop_ms; /* out: wall time loading the games, packing them, and in the loop */
} pg_result_batch;

/* Solves many games together (Algorithm 1, Section 4, for each): all games
 * share one packed id space on the device, every pass runs once over all of
 * them, and each game keeps its own loop state, so each result is exactly the
 * one pg_solve gives for that game alone. Inputs are packed: game i has
 * vertices vtx_base[i] .. vtx_base[i+1] of owner and pri, edges
 * edge_base[i] .. edge_base[i+1] of targets (local vertex ids of the game),
 * and n_i + 1 local CSR offsets starting at offsets[vtx_base[i] + i].
 * vtx_base and edge_base are host arrays of ngames + 1 entries starting at 0;
 * the other inputs use mem_kind. Each game is validated and preprocessed as in
 * pg_load_csr (same errors); the batch may hold up to 2^30 vertices after
 * preprocessing and any number of edges. max_inner caps the lockstep
 * iterations (0 = 64 * (largest game + 64)). Returns PG_ETIMEOUT or
 * PG_ENOTADMISSIBLE if any game ended that way (results are still written). */
pg_status pg_solve_batch(pg_ctx *ctx, int32_t ngames, const int64_t *vtx_base, const int64_t *edge_base,
                         const int32_t *offsets, const int32_t *targets, const uint8_t *owner, const int32_t *pri,
                         int32_t mem_kind, int64_t max_inner, pg_result_batch *out);

/* ---- Serving: continuous batching of a stream of games ----------------------
 *
 * A server owns one CUDA stream on one device, a worker thread and a packed
 * batch allocated once at its capacity. pg_server_submit copies a game into a
 * FIFO queue and returns at once. Between rounds the worker retires finished
 * games and admits queued ones in arrival order while they fit the capacity
 * (vertices after preprocessing plus one sink slot each, edges, games); a
 * round runs Algorithm 1 (Section 4) over all resident games for at most
 * round_iters iterations. Each game keeps its strategies and loop state on
 * the device across rounds, so its result is exactly the one pg_solve gives
 * for it alone, whatever else is resident. The paper has no counterpart (it
 * solves one game at a time). */
typedef struct pg_server pg_server;

typedef struct {
    int64_t max_vertices;  /* capacity in ids (G' vertices + 1 per game); 0 = from free device memory */
    int64_t max_edges;     /* capacity in G' edges; 0 = from free device memory */
    int32_t max_games;     /* resident games; 0 = 4096 */
    int32_t round_iters;   /* iterations per round (admission points); 0 = 8 */
    int64_t max_inner;     /* per-game iteration cap; 0 = 64 (largest resident n' + 64) */
    int32_t wide_offsets;  /* 1: the resident layout keeps 64-bit edge offsets at any size (as
                              pg_set_wide_offsets); 0: only when it holds 2^31 or more edges */
} pg_server_opts;

/* One finished game, as reported by pg_server_poll. */
typedef struct {
    uint64_t tag;       /* the caller's tag from pg_server_submit */
    int32_t status;     /* PG_OK, PG_ETIMEOUT, PG_ENOTADMISSIBLE, or the load error (PG_EINVAL, PG_EUNSUPPORTED,
                           PG_ENOMEM when the game alone exceeds the capacity) */
    int32_t n;          /* original vertices */
    int32_t k;          /* dummies */
    int64_t major, inner;
    double queue_us;    /* submission to admission */
    double latency_us;  /* submission to result */
} pg_served;

typedef struct {
    int64_t submitted, admitted, completed, queued;
    int64_t admitted_while_busy;  /* games admitted while other games were resident */
    int64_t rounds, iterations, max_resident;
    int64_t capacity_vertices, capacity_edges;
    double loop_ms, repack_ms, collect_ms;  /* worker wall time in rounds, in repacking, in writing results */
} pg_server_stats;

/* Creates a server on device; opts may be NULL (defaults). */
pg_status pg_server_create(int device, const pg_server_opts *opts, pg_server **out);
/* Stops the worker (games in flight are abandoned) and frees everything. */
void pg_server_destroy(pg_server *server);
/* Queues a game given by host arrays (layout as pg_load_csr); the arrays are
 * copied before the call returns. tag must not be in use by a queued,
 * resident or unfetched game (PG_EINVAL). Validation happens at admission:
 * an invalid game finishes with the load error as its status. */
pg_status pg_server_submit(pg_server *server, int32_t n, int64_t m, const int32_t *offsets, const int32_t *targets,
                           const uint8_t *owner, const int32_t *pri, uint64_t tag);
/* Reports up to max finished games in completion order, waiting up to
 * timeout_ms for the first one; *count receives the number written. Returns
 * the server's error (PG_ECUDA ...) if its worker failed and nothing is left
 * to report. */
pg_status pg_server_poll(pg_server *server, pg_served *out, int32_t max, int32_t timeout_ms, int32_t *count);
/* Copies a reported game's results into caller host arrays (each may be
 * NULL; layouts as in pg_result, n entries, dummy_sigma k entries) and
 * releases them. PG_EINVAL for an unknown or not yet reported tag. */
pg_status pg_server_fetch(pg_server *server, uint64_t tag, uint8_t *win, int32_t *sigma, int32_t *tau,
                          int8_t *val_class, int32_t *val_depth, int32_t *val_rank, int8_t *dummy_sigma);
pg_status pg_server_get_stats(pg_server *server, pg_server_stats *out);
/* The message of the worker's failure, or "no error". */
const char *pg_server_error(pg_server *server);

/* Bellman-Ford best response (Section 4, "Computing Best Responses"), the
 * paper's comparison point for one-player strategy improvement (Table 2):
 * shortest paths to the sink under the order of Section 3, computed by Jacobi
 * rounds over all vertices until no value changes. Count-vector mode only
 * (repeated priorities; PG_EUNSUPPORTED otherwise). Arguments as in
 * pg_best_response, except that tau_out is output only (nullable; Odd's
 * choice: the first edge of least value). *rounds_out (nullable) receives the
 * rounds run. The valuation written to out is that of (sigma, tau_out): the
 * best-response values, equal to pg_best_response's. PG_ENOTADMISSIBLE when
 * the values keep decreasing past n + 2 rounds (sigma not admissible). */
pg_status pg_best_response_bf(pg_game *game, const int32_t *sigma, const int8_t *dummy_sigma, int32_t *tau_out,
                              int32_t mem_kind, pg_valuation *out, int64_t *rounds_out);

/* Valuation of one successor function without allocating any memory. The
 * paper has no counterpart: this entry point exists for callers that cannot
 * have this library allocate device memory for them, for example a host
 * framework that reserves the device's memory up front and owns every
 * allocation, or a latency-bound loop that must not call cudaMalloc (which can
 * synchronise the device) while it runs. Instead of per-game buffers it uses
 * one fixed array compiled into the library (about 19 MB of device memory,
 * held by every GPU that loads the library until the process exits).
 *
 * Input, all device pointers owned by the caller:
 *   n     vertex count, 1 <= n <= 262,144 (2^18); larger n returns PG_EUNSUPPORTED
 *         without touching the device;
 *   succ  n entries: the successor of each vertex under a profile, or n for the sink;
 *   odd   n entries: 1 if the vertex's priority is odd, 0 if even.
 * Vertex ids must already be priority ranks (vertex v has the v-th smallest of n
 * distinct priorities); pg_valuate relabels games this way internally.
 * Output, device pointers owned by the caller (each may be NULL): val_class,
 * val_depth and val_rank with the meaning given at the top of this file; ranks
 * are positions among the finite valuations of these n vertices and the sink.
 * stream: a cudaStream_t (NULL = the legacy default stream). The call enqueues
 * its work on the stream and then waits for the stream once, to read its error
 * words; it returns after its work is complete.
 *
 * Returns PG_OK, PG_ENOTADMISSIBLE if a play reaches a cycle whose largest
 * priority is odd (outputs are still filled), PG_EINVAL for a NULL input or a
 * successor outside [0, n] (outputs are then unspecified), PG_ECUDA for a CUDA
 * error. No message is recorded.
 *
 * Set-up: every call looks up the fixed array's device address on the current
 * device (a lookup, no allocation); the first call on a device also computes
 * the cooperative launch size and keeps it. All calls share the array and it
 * keeps the last call's contents (each call clears what must start at zero),
 * so calls that overlap on the GPU, from any thread or stream, race:
 * serialise them. */
pg_status pg_valuate_static(int32_t n, const int32_t *succ, const uint8_t *odd, int8_t *val_class,
                            int32_t *val_depth, int32_t *val_rank, void *stream);

/* Per-phase device time of the last pg_solve / pg_best_response / pg_valuate
 * on game, in milliseconds, measured with CUDA events on the context's stream
 * when timing is enabled (pg_set_timing). Each pointer may be NULL. */
pg_status pg_set_timing(pg_ctx *ctx, int32_t enable);
pg_status pg_last_timing(const pg_game *game, double *total_ms, double *valuation_ms, double *switch_ms,
                         int64_t *valuations);

/* How the iteration loop of pg_solve / pg_best_response / pg_solve_batch runs.
 * With graphs enabled (the default) the whole loop is one CUDA graph launch: a
 * conditional WHILE node repeats one iteration (valuation, switching passes,
 * per-game bookkeeping) until no game is active, with no host synchronisation
 * between iterations; the graph is built on first use per game and kept with
 * it. With graphs disabled, or when timing is enabled, or if the CUDA runtime
 * refuses to build the graph, the host launches each iteration and
 * synchronises once per iteration. Both give identical results. The paper has
 * no counterpart (it concerns launching work on the device only). */
pg_status pg_set_graphs(pg_ctx *ctx, int32_t enable);
/* Work partitioning of the valuation (the paper has no counterpart; results
 * never depend on it):
 *   deep_cut      a g-chain walk longer than this (the play rises that many
 *                 times), or pointer jumping that needs more rounds than its
 *                 cap, sends the call to the ruling-set path: the Euler tour of
 *                 the nearest-greater forest ranked by a sparse ruling set
 *                 (Section 5's list ranking), work linear in n whatever the
 *                 forest's depth; default 64;
 *   ruler_bits    the ruling set takes about one list element in 2^ruler_bits
 *                 as a ruler (1..16); default 5;
 *   walk_cap      steps of a direct nearest-greater walk before pointer
 *                 jumping takes over (16, 32, 64 or 128); default 64;
 *   switch_block  threads per block of the switching passes that compare
 *                 valuations (128, 256 or 512); default 256;
 *   loop_ranks    1: loop iterations rank every valuation (pg_set_loop_ranks).
 * pg_set_tuning sets the context's values (zero fields keep the current
 * ones); PG_EINVAL for a value outside the ranges above. */
typedef struct {
    int32_t deep_cut;
    int32_t ruler_bits;
    int32_t walk_cap;
    int32_t switch_block;
    int32_t loop_ranks;
} pg_tuning;
pg_status pg_set_tuning(pg_ctx *ctx, const pg_tuning *t);
pg_status pg_get_tuning(const pg_ctx *ctx, pg_tuning *t);

/* A table of partitionings by size, as the autotuner
 * (paper_1705_02313_gb300/tune.py) writes it: each call on a game (or batch,
 * or server layout) of n ids uses the first entry with n <= max_ids (entries
 * by increasing max_ids; zero fields take the defaults above), else the
 * context's values. count = 0 clears the table. pg_load_tuning reads the table
 * from a text file, one entry per line: "max_ids deep_cut ruler_bits walk_cap
 * switch_block loop_ranks" ('#' starts a comment line). pg_ctx_create loads the
 * file named by the environment variable PG_TUNING_FILE when it is set (a file
 * that cannot be read or parsed leaves the table empty). */
typedef struct {
    int64_t max_ids;
    pg_tuning t;
} pg_tuning_entry;
pg_status pg_set_tuning_table(pg_ctx *ctx, const pg_tuning_entry *entries, int32_t count);
pg_status pg_load_tuning(pg_ctx *ctx, const char *path);

/* Edge offsets of the packed layout of pg_solve_batch: 32-bit while the batch
 * holds fewer than 2^31 edges, 64-bit beyond. enable = 1 takes 64-bit offsets
 * at any size (the layout of the largest batches, e.g. to check it on small
 * ones); results are identical. The paper has no counterpart. */
pg_status pg_set_wide_offsets(pg_ctx *ctx, int32_t enable);

/* What each iteration of the loops of pg_solve / pg_best_response /
 * pg_solve_batch / the server computes for switching (distinct priorities;
 * count-vector games always rank). By default (enable = 0) an iteration builds
 * the nearest-greater forest of the profile (Section 5's pseudoforest) and the
 * class of every vertex, and the switching passes compare the valuations of
 * two successors by walking their chains in that forest to their lowest
 * common ancestor: the larger of the two vertices passed last decides by the
 * parity of its priority (the order of Section 3). The exact ranks, depths and
 * classes of the outputs come from one full valuation after the loop. With
 * enable = 1 every iteration ranks all valuations (the full valuation of
 * pg_valuate) and switches by rank. Both give identical results; the first
 * does less work per iteration. */
pg_status pg_set_loop_ranks(pg_ctx *ctx, int32_t enable);

/* graph: 1 if the last loop on game ran as a graph, else 0; iterations: the
 * valuations it computed (each may be NULL). */
pg_status pg_last_loop(const pg_game *game, int32_t *graph, int64_t *iterations);

/* Device memory of games (loads, scratch, batches, servers) comes from one
 * stream-ordered pool per device. Freed game memory stays cached in the pool,
 * up to a quarter of the device's memory, so that loading the next game
 * reuses it instead of mapping new memory. This call waits for the device and
 * returns everything the pool caches on `device` to the driver (for example
 * before other code in the process allocates large buffers); memory of live
 * games is untouched. PG_ECUDA if the device cannot be used. The paper has no
 * counterpart (memory management of the implementation only). */
pg_status pg_release_cached_memory(int device);

#ifdef __cplusplus
}
#endif

#endif /* PG_H */
