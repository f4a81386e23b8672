/*
 * qap.h - C-ABI of the GB300 swap-neighbourhood QAP search library.
 *
 * The library evaluates, selects and applies pairwise-exchange moves for the
 * quadratic assignment problem, the inner loop shared by best-improvement
 * 2opt and tabu search in Novoa & Qasem, "GPU-accelerated Parallel Solutions
 * to the Quadratic Assignment Problem":
 *
 *   cost   Section 2.1, Eq. 1:  cost(p) = sum_i sum_j F[i][j] * D[p[i]][p[j]]
 *   delta  Section 4.1, Eq. 2:  change of cost when units r < s exchange
 *          locations (with the diagonal term the printed formula omits)
 *   2opt   Section 4.1: move to the best neighbour until none improves
 *   tabu   Sections 4.3-4.4: best admissible neighbour (not tabu, or
 *          aspiring below the best cost), tabu tenure drawn from a range,
 *          early stop when no move is admissible
 *   walks  Sections 4.2, 4.4: many independent searches from random starts;
 *          the caller takes the minimum over walks.
 *
 * Conventions
 *   - p[u] is the location (0-based) of unit u.  The paper's pi (unit at a
 *     location) is the inverse permutation; costs are identical.
 *   - F and D are n x n, row-major.  F is the flow between units, D the
 *     distance between locations.
 *   - A move (r, s), r < s, swaps p[r] and p[s].  Ties between equal deltas
 *     go to the lexicographically lowest (r, s).
 *   - Walk k of a call draws its random numbers with Philox4x32-10 under
 *     key = seed and counter (walk id, stream, draw / 4, 0), where walk id =
 *     walk_base + k; stream 0 is the Fisher-Yates start permutation (draw
 *     n-1-i picks j in [0, i] for position i, as (x * (i+1)) >> 32), stream 1
 *     the tabu tenures (draw (it-1)/period, or it-1 when period == 0).
 *     Results therefore do not depend on launch shape, grid size, or what
 *     else runs on the GPU.
 *   - Tabu iterations are numbered from 1.  Move (r, s) is tabu at iteration
 *     it while tabu_until[r][s] > it; applying it at iteration it sets
 *     tabu_until[r][s] = it + t, t = tmin + (x * (tmax - tmin + 1)) >> 32.
 *     With aspiration on, a tabu move is admissible if cost + delta < best.
 *   - The per-walk trajectory hash is FNV-1a/64 over the applied moves:
 *     h = 14695981039346656037; per move h ^= (r << 16 | s); h *= 1099511628211.
 *
 * Arithmetic is exact integer arithmetic for any int64 F and D whose bound
 * B = (n^2 + 8n + 32) * max|F| * max|D| is below 2^62 (else QAP_EOVERFLOW).
 * Deltas are int32 when B is at most 2^31 - 2 and the instance is on a
 * narrow element path, else int64 (also when QAP_FORCE_INT64 is given).
 * Element paths, chosen per instance (per batch: the widest any instance
 * needs):
 *   int8 F, int8 D    every difference of two F entries and of two D
 *                     entries fits a byte, and the deltas are int32;
 *   int16 F, int8 D   F fits int16, D fits int8, and 2 n max|F| max|D| is
 *                     below 2^31 (the dot products of phase X sum in 32 bits);
 *   int64 F, int64 D  every other instance: int64 storage and arithmetic, F
 *                     read from global memory, P in shared memory while it
 *                     fits and in a per-CTA device workspace otherwise.
 *
 * Errors: every entry point returns a qap_status; on error nothing has been
 * written to the outputs unless stated otherwise.  A CUDA error is returned
 * as QAP_ECUDA and the CUDA error string is kept for qap_last_error().
 * Entry points are thread-safe for distinct contexts; one context must not
 * be used by two host threads at once.
 */
#ifndef QAP_H
#define QAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qap_ctx qap_ctx;  /* opaque: device copies of F and D */

typedef enum {
  QAP_OK = 0,
  QAP_EINVAL = 1,        /* invalid argument (n < 2, bad permutation, ...)      */
  QAP_EOVERFLOW = 2,     /* the bound B does not fit the int64 path (>= 2^62),
                            or a frequency penalty does not fit the deltas      */
  QAP_ENOMEM = 3,        /* device or host allocation failed                   */
  QAP_ECUDA = 4,         /* a CUDA runtime call failed; see qap_last_error()   */
  QAP_ETIMEOUT = 5,      /* a bounded wait ran out (serving loop)              */
  QAP_EUNSUPPORTED = 6   /* outside what the kernels hold: n > 256, a thread
                            count too small for n, or a form the entry point
                            does not offer (see qap_last_error())             */
} qap_status;

/* Tabu tenure rule: t drawn uniformly from [tmin, tmax]; a new t every
 * `period` iterations (at it = 1, period + 1, ...), or for every applied move
 * when period == 0 (the paper's rule, Section 4.3). */
typedef struct {
  int32_t tmin;
  int32_t tmax;
  int32_t period;
} qap_tenure;

#define QAP_FORCE_INT64 1u   /* qap_create flag: keep deltas in int64 */

/* Launch forms of a search. */
#define QAP_LAUNCH_PERSISTENT 0  /* one launch; CTAs loop over walks          */
#define QAP_LAUNCH_PLAIN 1       /* one launch per walk (comparison form)     */

/* Tabu criteria.  Applying move (r, s) at iteration it with tenure t marks
 * something "until it + t"; a mark m forbids while m > it.
 *   QAP_TABU_PAIR      the paper's Tabuarr (Section 4.3): move (r, s) itself
 *                      is forbidden.
 *   QAP_TABU_UNIT_LOC  Taillard's robust tabu search (1991), the elementary
 *                      search Section 4.3 follows: units r and s may not
 *                      return to the locations they leave; a move (u, v) is
 *                      forbidden when both u and v would return to a
 *                      location they are barred from.
 *   QAP_TABU_UNIT      Zhu et al.'s unit marking (Section 3.1): units r and s
 *                      are marked; a move is forbidden when either of its
 *                      units is marked. */
#define QAP_TABU_PAIR 0
#define QAP_TABU_UNIT_LOC 1
#define QAP_TABU_UNIT 2

/* How phase X (Section 4.4: the deltas of the pairs touching the move,
 * recomputed by Eq. 2) gets its dot products (qap_search_params.phase_x):
 *   QAP_PHASE_X_AUTO  the n x n products M[x][k] = F[x].P[k] + F^T[x].P^T[k]
 *                     kept in shared memory and brought up to date by a
 *                     rank-2 update per move, where they apply: int8 or
 *                     int16 flow storage, plans of at most 24 pairs per
 *                     thread (12 at 1024 threads; 26 at 512 threads with int16
 *                     flows), and an M that fits shared
 *                     memory (and still lets two walks share an SM where the
 *                     plan was taken for that), if need be without the
 *                     transposed copies of F and P (their entries then read
 *                     from columns); elsewhere dot products;
 *   QAP_PHASE_X_DOTS  dot products over the rows of F and P at every move.
 * Both give the same walks; qap_plan reports which one runs. */
#define QAP_PHASE_X_AUTO 0
#define QAP_PHASE_X_DOTS 1

typedef struct {
  int32_t n;
  int32_t delta_bytes;     /* 4 (int32 path) or 8 (int64 path)              */
  int32_t sym_flow;        /* F == F^T                                      */
  int32_t sym_dist;        /* D == D^T                                      */
  int64_t bound;           /* B above                                       */
  int32_t flow_bytes;      /* bytes per stored F element on the device: 1,
                              2, or 8 on the int64 element path            */
  int32_t dist_bytes;      /* bytes per stored D and P element: 1 or 8      */
} qap_ctx_info;

/* Create a context for one instance.
 *   F, D   host pointers to n*n int64 values, row-major, any sign.  Copied;
 *          the caller may free them when the call returns.  The element path
 *          and the delta width follow from the values (see above).
 *   n      2 <= n <= 256.  Up to n = 181 a walk keeps its deltas in
 *          registers; beyond, in a workspace in device memory (allocated by
 *          the library on first use), with F in shared or global memory.
 *   flags  0 or QAP_FORCE_INT64.
 *   out    receives the context (NULL on error).
 * Uses the CUDA device current at the call for all later calls.
 * Errors: QAP_EINVAL (null pointer, n < 2), QAP_EUNSUPPORTED, QAP_EOVERFLOW,
 * QAP_ENOMEM, QAP_ECUDA. */
qap_status qap_create(const int64_t* F, const int64_t* D, int32_t n, uint32_t flags,
                      qap_ctx** out);

/* Release a context and its device memory.  NULL is ignored. */
void qap_destroy(qap_ctx* ctx);

/* Describe a context.  Errors: QAP_EINVAL on null pointers. */
qap_status qap_info(const qap_ctx* ctx, qap_ctx_info* out);

/* Text for a status code (static storage). */
const char* qap_strerror(qap_status s);

/* Detail of the last QAP_ECUDA on this host thread (static per thread). */
const char* qap_last_error(void);

/* Eq. 1 for `count` permutations on the GPU.
 *   p     host pointer, count x n int32, row k a permutation of 0..n-1.
 *   cost  host pointer, count int64 outputs.
 * Errors: QAP_EINVAL (count < 0, null pointers, a row that is not a
 * permutation; nothing is computed), QAP_ENOMEM, QAP_ECUDA. */
qap_status qap_cost(qap_ctx* ctx, int32_t count, const int32_t* p, int64_t* cost);

/* Parameters of a search call. */
typedef struct {
  int32_t starts;          /* number of walks W >= 1                         */
  uint32_t walk_base;      /* walk k uses walk id walk_base + k              */
  int32_t descend;         /* 1: 2opt to a local minimum before tabu         */
  int32_t max_descent;     /* cap on 2opt moves; < 0 means 2^20 (a 2opt
                              descent ends long before on real instances) */
  int32_t iters;           /* tabu iterations, >= 0                          */
  qap_tenure tenure;       /* used when iters > 0: 1 <= tmin <= tmax         */
  int32_t aspiration;      /* 0 or 1                                         */
  uint64_t seed;           /* Philox key                                     */
  int32_t launch;          /* QAP_LAUNCH_PERSISTENT or QAP_LAUNCH_PLAIN      */
  int32_t threads_per_walk;/* 0 = automatic: the fewest threads holding n
                              with at most 8 pairs per thread, or 512 with
                              any; with starts >= 2 x SMs also 256 with any
                              (two walks per SM).  Else 128, 256, 512 or
                              1024 (n > 181 always uses 1024)                */
  int32_t tenure_per_n;    /* 1: tenure.tmin, tmax, period are hundredths of
                              each instance's n:
                              tmin' = max(1, floor(tmin n / 100)),
                              tmax' = max(tmin', ceil(tmax n / 100)),
                              period' = floor(period n / 100);
                              e.g. (10, 33, 0) is the paper's [0.1n, 0.33n]
                              drawn per move; 0: absolute                    */
  int32_t criterion;       /* QAP_TABU_PAIR (default), _UNIT_LOC or _UNIT    */
  int32_t freq_penalty;    /* lambda >= 0: frequency-based diversification,
                              the long-term memory Section 7 proposes.  A
                              non-improving move (delta >= 0) is ranked by
                              delta + lambda * (times the walk applied it in
                              its tabu phase); improving moves by delta.
                              Aspiration and the cost use the plain delta.
                              0 = off.  With int32 deltas the context's
                              bound B + lambda * iters must stay below 2^31
                              - 1, else QAP_EOVERFLOW (create the context
                              with QAP_FORCE_INT64).  criterion != PAIR or
                              lambda > 0 use a per-CTA device workspace of
                              (2 n^2 + n) int32 (not available to
                              qap_batch_search_noalloc: QAP_EUNSUPPORTED).
                              The serving loop picks int64 deltas itself
                              when the penalty needs them.                   */
  int32_t phase_x;         /* QAP_PHASE_X_AUTO (default) or _DOTS          */
} qap_search_params;

/* Per-walk outputs; every pointer may be NULL except best_cost.  For
 * qap_search they are host pointers, for qap_search_async device pointers.
 *   best_p        W x n  best permutation of the walk
 *   best_cost     W      its cost
 *   final_cost    W      cost of the walk's last solution
 *   best_iter     W      tabu iteration that reached best_cost (0 = before
 *                        the tabu phase)
 *   iters_done    W      tabu iterations that applied a move
 *   status        W      0 = completed, 1 = stopped early: no admissible move
 *   descent_moves W      moves applied by the 2opt phase
 *   hash          W      trajectory hash of the tabu phase
 *   descent_hash  W      trajectory hash of the 2opt phase
 *   freq          W x m x m  the frequency memory of Section 4.3: entry
 *                        [s][r] (r < s, lower triangle) counts how often the
 *                        tabu phase applied move (r, s); every other entry
 *                        is 0.  m = n for one instance, p_stride for a batch.
 *                        Not produced by the serving loop. */
typedef struct {
  int32_t* best_p;
  int64_t* best_cost;
  int64_t* final_cost;
  int32_t* best_iter;
  int32_t* iters_done;
  int32_t* status;
  int32_t* descent_moves;
  uint64_t* hash;
  uint64_t* descent_hash;
  int32_t* freq;
} qap_walk_outputs;

/* Run W independent walks of one instance; host buffers, blocking.
 *   starts  host pointer, W x n start permutations, or NULL to draw them
 *           (stream 0 of each walk).
 * Host<->device copies of starts and outputs are part of the call.
 * Errors: QAP_EINVAL (bad parameters or a start that is not a permutation;
 * nothing is run), QAP_EUNSUPPORTED (threads_per_walk too small for n),
 * QAP_ENOMEM, QAP_ECUDA. */
qap_status qap_search(qap_ctx* ctx, const qap_search_params* params, const int32_t* starts,
                      const qap_walk_outputs* out);

/* Stream-ordered form of qap_search: device pointers, no synchronisation.
 *   d_starts device pointer (W x n) or NULL.  Not validated: rows must be
 *            permutations of 0..n-1.
 *   out      device pointers, valid until the stream reaches the end of the
 *            call's work.
 *   stream   a cudaStream_t (NULL = legacy default stream).
 * Kernel launches only; capturable into a CUDA graph once a search with the
 * same n, starts, threads_per_walk and delta width has run outside capture.
 * Errors: QAP_EINVAL, QAP_EUNSUPPORTED, QAP_ECUDA (launch errors only). */
qap_status qap_search_async(qap_ctx* ctx, const qap_search_params* params,
                            const int32_t* d_starts, const qap_walk_outputs* out,
                            void* stream);

/* Launch shape a search would use.  Errors: as qap_search_async. */
typedef struct {
  int32_t threads_per_walk;
  int32_t pairs_per_thread;  /* register slots per thread                 */
  int32_t smem_bytes;        /* dynamic shared memory per CTA             */
  int32_t grid;              /* CTAs of the persistent launch             */
  int32_t ctas_per_sm;
  int32_t sms;
  int32_t classes;           /* launches of a batch search (size classes);
                                1 for one instance                          */
  int32_t products;          /* phase X: 0 by dot products; 1 from products
                                kept in shared memory (int8 or int16 flows,
                                when they fit); 2 the same without the
                                transposed copies of F and P, whose entries
                                are then read from columns (where M fits
                                only so)                                    */
  int32_t workspace;         /* 1: deltas and marks in the device workspace */
} qap_plan_info;
qap_status qap_plan(qap_ctx* ctx, const qap_search_params* params, qap_plan_info* out);

/* Convenience forms named after the two heuristics (host buffers, blocking).
 * qap_2opt: W walks of best-improvement 2opt to a local minimum from random
 *   starts; iters_done receives the number of moves of each walk.
 * qap_tabu: W walks of tabu search for `iters` iterations from random starts;
 *   status receives 0/1 as in qap_walk_outputs.
 * best_p (W x n) and best_cost (W) are required, the rest may be NULL. */
qap_status qap_2opt(qap_ctx* ctx, int32_t starts, uint64_t seed, int32_t max_iters,
                    int32_t* best_p, int64_t* best_cost, int32_t* iters_done);
qap_status qap_tabu(qap_ctx* ctx, int32_t starts, int32_t iters, qap_tenure tenure,
                    int32_t aspiration, uint64_t seed, int32_t* best_p, int64_t* best_cost,
                    int32_t* best_iter, int32_t* status);

/* The host's reduction over walks (Sections 4.2 and 4.4: each walk returns
 * its best solution, the minimum is taken on the CPU): for each of `groups`
 * consecutive groups of `walks` entries of best_cost (host pointer, groups x
 * walks), the index within the group of the lowest cost, ties to the lowest
 * walk index, into index[groups] (host).  groups = 1 for one instance; the
 * instance count for a batch search (rows i * starts + k).  Runs on the
 * host; no GPU call.  Errors: QAP_EINVAL on null pointers, walks < 1 or
 * groups < 0. */
qap_status qap_best_walks(const int64_t* best_cost, int32_t groups, int32_t walks,
                          int32_t* index);

/* ------------------------------------------------------------------------
 * Many instances of uneven n in one persistent launch (the walks of every
 * instance are independent searches, Sections 4.2 and 4.4).  CTAs take
 * (instance, walk) items from a device counter, largest n first, and reload
 * the instance into shared memory when it changes.  Walk k of every instance
 * uses walk id walk_base + k, so each instance's results equal a qap_search
 * of that instance alone.
 * ------------------------------------------------------------------------ */
typedef struct qap_batch qap_batch;  /* opaque: device copies of all instances */

/* Create a batch.
 *   count  number of instances, >= 1.
 *   F, D   host arrays of `count` host pointers; instance i is n[i] x n[i]
 *          int64, row-major, ranges as for qap_create.  Copied.
 *   n      host array of `count` sizes, 2 <= n[i] <= 256.
 *   flags  0 or QAP_FORCE_INT64.  One delta width serves the whole batch:
 *          int64 if any instance needs it.
 * Errors: as qap_create, for the first instance that fails. */
qap_status qap_batch_create(int32_t count, const int64_t* const* F, const int64_t* const* D,
                            const int32_t* n, uint32_t flags, qap_batch** out);
void qap_batch_destroy(qap_batch* b);

/* Instance count, largest n and delta width (4 or 8) of a batch; any output
 * pointer may be NULL. */
qap_status qap_batch_info(const qap_batch* b, int32_t* count, int32_t* nmax,
                          int32_t* delta_bytes);

/* Launch shape of a batch search.  Each instance takes the plan its own n
 * would get alone in a launch of the batch's total walks (or the plan the
 * autotuner kept); instances with the same plan form a size class with one
 * persistent launch, and the classes run concurrently on internal streams
 * forked from and joined back into the caller's stream.  Reports the class
 * of the largest n and the number of classes. */
qap_status qap_batch_plan(qap_batch* b, const qap_search_params* params, qap_plan_info* out);

/* Result of the autotuner for one size class of the rule. */
typedef struct {
  int32_t nmin, nmax;        /* n range of the class's instances             */
  int32_t instances;
  int32_t candidates;        /* plans timed                                  */
  int32_t threads_per_walk;  /* the plan kept                                */
  int32_t pairs_per_thread;
  int32_t workspace;         /* 1: deltas and marks in the device workspace  */
  int32_t products;          /* as in qap_plan_info                         */
  float trial_ms;            /* its trial time                               */
  float rule_ms;             /* the rule's plan's trial time                 */
} qap_tune_result;

/* Autotune the launch plans of a batch for searches like `params`.  For each
 * size class of the rule (instances sharing the rule's plan), every compiled
 * plan that holds the class's largest n is timed on the class's own
 * instances: each thread count with the fewest slots that fit (with int8
 * flows also in its products form, which keeps the n x n dot products of
 * phase X in shared memory and updates them per move), and the workspace
 * plan that keeps the deltas and tabu marks in L2/HBM instead of registers
 * and shared memory.  The trial runs params->starts walks of
 * `trial_iters` iterations; the fastest plan is kept for the class, and
 * later searches with threads_per_walk = 0 use the kept plans (classes are
 * regrouped by them).  Results are unchanged: every plan computes the same
 * walks.  params->threads_per_walk must be 0 and launch persistent.
 *   results   up to max_results per-class reports (may be NULL when 0)
 *   nresults  receives the number of classes (may be NULL)
 * Synchronous; not capturable.  Errors: QAP_EINVAL, QAP_EOVERFLOW,
 * QAP_ENOMEM, QAP_ECUDA. */
qap_status qap_batch_autotune(qap_batch* b, const qap_search_params* params,
                              int32_t trial_iters, qap_tune_result* results,
                              int32_t max_results, int32_t* nresults);

/* One size class of a batch search: the instances that share a launch plan
 * and the persistent launch that runs their walks. */
typedef struct {
  int32_t nmin, nmax;        /* n range of the class's instances             */
  int32_t instances;
  int32_t walks;             /* walks of the launch (instances x starts)     */
  int32_t threads_per_walk;
  int32_t pairs_per_thread;
  int32_t products;          /* as in qap_plan_info                         */
  int32_t workspace;         /* 1: deltas and marks in the device workspace  */
  int32_t grid;              /* CTAs of the launch                           */
  int32_t ctas_per_sm;
  int32_t smem_bytes;        /* dynamic shared memory per CTA                */
  int32_t delta_bytes;       /* 4 or 8, as for the whole batch               */
  int32_t flow_bytes;        /* bytes per stored F element                   */
  int32_t dist_bytes;        /* bytes per stored D and P element             */
  float last_ms;             /* device time of the class's kernel in the
                                last search made with timing on (CUDA events
                                on the stream the kernel ran on), else -1   */
} qap_class_info;

/* Timing of the classes' kernels: with on = 1, each later search of the
 * batch records a CUDA event before and after each class's kernel launch, on
 * the stream the launch uses; qap_batch_classes reports the elapsed time.
 * Off (0) by default; a search with timing on should not be captured in a
 * CUDA graph.  Errors: QAP_EINVAL. */
qap_status qap_batch_set_timing(qap_batch* b, int32_t on);

/* The size classes a search like `params` runs (plans them if needed, as
 * qap_batch_plan does): up to max_out entries into out (may be NULL when
 * 0), the number of classes into *count (may be NULL), and the class index
 * of every instance into inst_class[count of the batch] (may be NULL).
 * last_ms waits for the last timed launch of the class to finish.
 * Errors: QAP_EINVAL, QAP_EUNSUPPORTED, QAP_ECUDA. */
qap_status qap_batch_classes(qap_batch* b, const qap_search_params* params,
                             qap_class_info* out, int32_t max_out, int32_t* count,
                             int32_t* inst_class);

/* Run params->starts walks of every instance.  Output row i * starts + k
 * holds walk k of instance i; best_p rows hold p_stride >= max n elements
 * (the first n[i] are the permutation).  params->launch must be
 * QAP_LAUNCH_PERSISTENT.
 * qap_batch_search: host outputs, blocking.
 * qap_batch_search_async: device outputs, stream-ordered (per size class a
 *   counter reset and one kernel launch, on internal streams forked from
 *   `stream` by an event and joined back into it).  The first call for a
 *   given (starts, thread count, rule tables on or off) writes device
 *   tables synchronously and must not be captured in a CUDA graph; later
 *   calls can be.
 * Errors: QAP_EINVAL, QAP_EUNSUPPORTED, QAP_ENOMEM, QAP_ECUDA. */
qap_status qap_batch_search(qap_batch* b, const qap_search_params* params,
                            const qap_walk_outputs* out, int32_t p_stride);
qap_status qap_batch_search_async(qap_batch* b, const qap_search_params* params,
                                  const qap_walk_outputs* out, int32_t p_stride, void* stream);

/* ------------------------------------------------------------------------
 * Serving loop: continuous batching of solve requests (each request is a
 * multi-walk search of its own instance, Sections 4.2 and 4.4).  A worker
 * thread admits queued requests in arrival order as soon as a slot (a CUDA
 * stream) is free and the device arena has room for the request's
 * instance, outputs and workspace; admitted requests run on the device at
 * the same time.  The arena is allocated once at creation, so serving does
 * no cudaMalloc or cudaFree.  A request's results depend only on its own
 * instance and parameters (walk ids 0..starts-1 of its seed), never on what
 * else is running.
 * ------------------------------------------------------------------------ */
typedef struct qap_server qap_server;

typedef struct {
  int32_t slots;      /* requests on the device at once, 1..128             */
  int32_t reserved;   /* must be 0                                          */
  int64_t mem_bytes;  /* device arena for admitted requests, >= 1 MiB       */
} qap_server_config;

typedef struct {
  double queued_us;   /* submit -> admission                                */
  double device_us;   /* admission -> results on the host                   */
  double total_us;    /* submit -> results on the host                      */
  double kernel_start_us;  /* the request's search kernel on the device clock
                              (CUDA events on its stream), microseconds from
                              the server's creation; -1 if not measured     */
  double kernel_end_us;
} qap_request_times;

typedef struct {
  int64_t submitted, completed, pending, in_flight;
  int64_t arena_bytes, arena_used;
  int64_t peak_in_flight;  /* most requests admitted at once so far        */
} qap_server_stats;

/* Start a server on the current device.  Errors: QAP_EINVAL, QAP_ENOMEM,
 * QAP_ECUDA. */
qap_status qap_server_create(const qap_server_config* cfg, qap_server** out);

/* Queue one request.  F, D (host, n x n int64) are copied before return;
 * params->launch must be QAP_LAUNCH_PERSISTENT.  *ticket identifies the
 * request for qap_server_wait.  Errors: as qap_create and qap_search, and
 * QAP_ENOMEM when the request can never fit the arena. */
qap_status qap_server_submit(qap_server* s, const int64_t* F, const int64_t* D, int32_t n,
                             uint32_t flags, const qap_search_params* params,
                             uint64_t* ticket);

/* Wait at most timeout_ms for a request.  On completion its results are
 * written to `out` (host pointers, rows as for qap_search, NULL fields
 * skipped), its times to `times` (may be NULL), and the ticket is released.
 * Returns QAP_ETIMEOUT (ticket kept) if it has not completed in time,
 * QAP_EINVAL for an unknown ticket, or the request's own error. */
qap_status qap_server_wait(qap_server* s, uint64_t ticket, int32_t timeout_ms,
                           const qap_walk_outputs* out, qap_request_times* times);

/* Counters of a server. */
qap_status qap_server_get_stats(qap_server* s, qap_server_stats* out);

/* Finish every queued and running request, then free the server. */
void qap_server_destroy(qap_server* s);

/* ------------------------------------------------------------------------
 * Batch search that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when
 * they search, for example a host runtime whose own allocator owns all
 * device memory, or code on a latency-critical path where a cudaMalloc (and
 * the device-wide synchronisation it can cause) is not allowed.
 *
 * Same arguments, results and errors as qap_batch_search_async (device
 * outputs, stream-ordered kernel launch), but the work-queue counter, the
 * instance table and the item lists live in one static device array of
 * about 1 MiB compiled into the library, held by every GPU that loads the
 * library until the process exits.  The call performs no cudaMalloc or
 * cudaFree and no other device allocation, and its host-side bookkeeping
 * uses fixed-size static tables (no heap allocation either).  It makes the
 * batch's device current for its own work and gives the caller's current
 * device back on return.
 *
 * Limits: at most 4096 instances and at most 65536 walks in total
 * (count x params->starts); larger calls return QAP_EINVAL and
 * qap_last_error() says which limit was exceeded.
 *
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress; make that first call before any stream capture.
 * Every call reuses the same array and leaves its tables in it: the call
 * rewrites the tables and zeroes the counter before its kernel starts, so
 * two calls whose kernels overlap on the GPU race on the array; order them
 * on one stream or synchronise between them.  The call copies its tables
 * from static host memory, so it may wait until the stream reaches them.
 * For the same reason it returns QAP_EUNSUPPORTED, and launches nothing,
 * while `stream` is being captured: a captured copy would read host tables
 * that later calls overwrite. */
qap_status qap_batch_search_noalloc(qap_batch* b, const qap_search_params* params,
                                    const qap_walk_outputs* out, int32_t p_stride, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QAP_H */
