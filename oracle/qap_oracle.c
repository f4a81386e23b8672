/*
 * Plain, slow CPU oracle for the swap-neighbourhood QAP search
 * (Novoa & Qasem, "GPU-accelerated Parallel Solutions to the Quadratic
 * Assignment Problem").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  The GPU library never
 * links, calls or includes it, and this file includes nothing of the GPU
 * library: the two share no kernels, headers, helpers or tables.
 *
 * Conventions (readings of the paper; each is listed in the design notes):
 *   - p[u] is the LOCATION of unit u, 0-based.  The paper's pi_i (unit at
 *     location i, Section 2.1) is the inverse permutation; the cost is the
 *     same sum written over units instead of locations.
 *   - F is the flow between units, D the distance between locations, both
 *     n x n row-major int64.  cost(p) = sum_ij F[i][j] * D[p[i]][p[j]]
 *     (Section 2.1, Eq. 1).
 *   - A move (r, s), r < s, exchanges the locations of units r and s.  The
 *     neighbourhood is all n(n-1)/2 such moves, enumerated in lexicographic
 *     order (Section 4.1, Fig. 1: "systematic" enumeration).
 *   - Ties between equal deltas go to the lexicographically lowest (r, s).
 *
 * Everything here is scalar int64 with explicit overflow checks; any
 * overflow sets *err (the oracle never silently wraps).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "qap_oracle.h"

/* ------------------------------------------------------------------------ */
/* Overflow-checked int64 helpers                                            */
/* ------------------------------------------------------------------------ */

static inline int64_t chk_mul(int64_t a, int64_t b, int *err) {
  int64_t r;
  if (__builtin_mul_overflow(a, b, &r)) { *err = ORC_EOVERFLOW; return 0; }
  return r;
}
static inline int64_t chk_add(int64_t a, int64_t b, int *err) {
  int64_t r;
  if (__builtin_add_overflow(a, b, &r)) { *err = ORC_EOVERFLOW; return 0; }
  return r;
}
static inline int64_t chk_sub(int64_t a, int64_t b, int *err) {
  int64_t r;
  if (__builtin_sub_overflow(a, b, &r)) { *err = ORC_EOVERFLOW; return 0; }
  return r;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  The paper only says that walks use different  */
/* random seeds (Sections 4.2, 4.4); this counter-based generator is the    */
/* reading chosen so that every walk's draws are reproducible by index.     */
/* ------------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {             /* key schedule: add the Weyl constants */
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Draw number idx of stream `stream` of walk `walk` under key `seed`:
 * counter = (walk, stream, idx / 4, 0), word idx % 4 of the output block. */
uint32_t orc_draw(uint64_t seed, uint32_t walk, uint32_t stream, uint32_t idx) {
  uint32_t ctr[4] = {walk, stream, idx >> 2, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[idx & 3u];
}

/* Uniform integer in [0, m) from a 32-bit draw by multiply-shift. */
uint32_t orc_bounded(uint32_t x, uint32_t m) {
  return (uint32_t)(((uint64_t)x * (uint64_t)m) >> 32);
}

/* Random initial solution of a walk (Sections 4.2 and 4.4 draw one random
 * permutation per walk).  Fisher-Yates: start from the identity, and for
 * i = n-1 down to 1 swap p[i] with p[j], j uniform in [0, i], using draw
 * number n-1-i of stream 0. */
void orc_start_perm(uint64_t seed, uint32_t walk, int n, int32_t *p) {
  for (int i = 0; i < n; ++i) p[i] = i;
  for (int i = n - 1; i >= 1; --i) {
    uint32_t x = orc_draw(seed, walk, ORC_STREAM_START, (uint32_t)(n - 1 - i));
    int j = (int)orc_bounded(x, (uint32_t)(i + 1));
    int32_t t = p[i]; p[i] = p[j]; p[j] = t;
  }
}

/* Tenure of the tabu list (Section 4.3, dynamic tabu list size): a random
 * integer t in [tmin, tmax].  With period > 0 a new t is drawn at
 * iterations it where (it - 1) % period == 0 (draw number (it-1)/period);
 * with period == 0 a new t is drawn for every applied move (draw it-1),
 * which is the paper's own rule. */
int32_t orc_tenure(const orc_tenure_t *tn, uint64_t seed, uint32_t walk, int32_t it) {
  uint32_t k = tn->period > 0 ? (uint32_t)((it - 1) / tn->period) : (uint32_t)(it - 1);
  uint32_t x = orc_draw(seed, walk, ORC_STREAM_TENURE, k);
  return tn->tmin + (int32_t)orc_bounded(x, (uint32_t)(tn->tmax - tn->tmin + 1));
}

/* FNV-1a, 64-bit, over the applied moves: h ^= (r << 16 | s); h *= prime.
 * An observation device for comparing whole trajectories, not part of the
 * method. */
uint64_t orc_hash_init(void) { return 14695981039346656037ull; }
uint64_t orc_hash_move(uint64_t h, int r, int s) {
  h ^= (uint64_t)(((uint32_t)r << 16) | (uint32_t)s);
  return h * 1099511628211ull;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 and Eq. 2                                                           */
/* ------------------------------------------------------------------------ */

/* Section 2.1, Eq. 1, written over units: sum_i sum_j F[i][j] D[p[i]][p[j]]. */
int64_t orc_cost(const int64_t *F, const int64_t *D, int n, const int32_t *p, int *err) {
  int64_t z = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      z = chk_add(z, chk_mul(F[(size_t)i * n + j],
                             D[(size_t)p[i] * n + p[j]], err), err);
  return z;
}

/* Section 4.1, Eq. 2 (the Burkard-Rendl delta), restated for exchanging the
 * locations of units r and s, with P[a][b] = D[p[a]][p[b]]:
 *
 *   delta = sum_{k != r,s} [ (F[r][k]-F[s][k]) (P[s][k]-P[r][k])
 *                          + (F[k][r]-F[k][s]) (P[k][s]-P[k][r]) ]
 *         + (F[r][s]-F[s][r]) (P[s][r]-P[r][s])
 *         + (F[r][r]-F[s][s]) (P[s][s]-P[r][r])
 *
 * The last (diagonal) term is absent from the printed Eq. 2, which is exact
 * only when the diagonals of F or D are constant; it is included here so
 * that delta == cost(after) - cost(before) for every instance. */
int64_t orc_delta(const int64_t *F, const int64_t *D, int n, const int32_t *p,
                  int r, int s, int *err) {
#define Fx(a, b) F[(size_t)(a) * n + (b)]
#define Px(a, b) D[(size_t)p[a] * n + p[b]]
  int64_t d = 0;
  for (int k = 0; k < n; ++k) {
    if (k == r || k == s) continue;
    int64_t t1 = chk_mul(chk_sub(Fx(r, k), Fx(s, k), err),
                         chk_sub(Px(s, k), Px(r, k), err), err);
    int64_t t2 = chk_mul(chk_sub(Fx(k, r), Fx(k, s), err),
                         chk_sub(Px(k, s), Px(k, r), err), err);
    d = chk_add(d, chk_add(t1, t2, err), err);
  }
  d = chk_add(d, chk_mul(chk_sub(Fx(r, s), Fx(s, r), err),
                         chk_sub(Px(s, r), Px(r, s), err), err), err);
  d = chk_add(d, chk_mul(chk_sub(Fx(r, r), Fx(s, s), err),
                         chk_sub(Px(s, s), Px(r, r), err), err), err);
  return d;
#undef Fx
#undef Px
}

/* ------------------------------------------------------------------------ */
/* The delta table of a walk                                                 */
/*                                                                           */
/* ORC_REF  : every delta recomputed from Eq. 2 at every iteration (the      */
/*            definition, O(n^3) per iteration).                             */
/* ORC_FAST : after a move (r, s), deltas of pairs (u, v) disjoint from      */
/*            {r, s} are updated in O(1) (Taillard's update, which the paper */
/*            cites for its tabu search in Section 4.3 without printing it), */
/*            and the 2(n-2) pairs that touch r or s are recomputed from     */
/*            Eq. 2.  Derivation: for (u, v) disjoint from {r, s}, only the  */
/*            k = r and k = s terms of Eq. 2 change, and they combine to     */
/*              (a_u - a_v)(b_u - b_v) + (c_u - c_v)(e_u - e_v)              */
/*            with a_x = F[r][x]-F[s][x], b_x = P'[s][x]-P'[r][x],           */
/*                 c_x = F[x][r]-F[x][s], e_x = P'[x][s]-P'[x][r],           */
/*            P' being the permuted distances after the move.                */
/*            The pair (r, s) itself becomes -delta(r, s).                   */
/* ORC_CHECK: ORC_FAST, and after every update the whole table is compared   */
/*            with a fresh Eq. 2 evaluation; a mismatch sets ORC_EMISMATCH.  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n;
  int64_t *dl;  /* n*n, entry [r*n+s] for r < s */
} delta_table;

static void table_fill(delta_table *t, const int64_t *F, const int64_t *D,
                       const int32_t *p, int *err) {
  int n = t->n;
  for (int r = 0; r < n; ++r)
    for (int s = r + 1; s < n; ++s)
      t->dl[(size_t)r * n + s] = orc_delta(F, D, n, p, r, s, err);
}

/* Called with p already holding the solution AFTER move (r, s). */
static void table_update(delta_table *t, const int64_t *F, const int64_t *D,
                         const int32_t *p, int r, int s, int mode, int *err) {
  int n = t->n;
  if (mode == ORC_REF) { table_fill(t, F, D, p, err); return; }
  int64_t *a = malloc(sizeof(int64_t) * 4 * (size_t)n);
  int64_t *b = a + n, *c = a + 2 * n, *e = a + 3 * n;
  for (int x = 0; x < n; ++x) {
    a[x] = F[(size_t)r * n + x] - F[(size_t)s * n + x];
    b[x] = D[(size_t)p[s] * n + p[x]] - D[(size_t)p[r] * n + p[x]];
    c[x] = F[(size_t)x * n + r] - F[(size_t)x * n + s];
    e[x] = D[(size_t)p[x] * n + p[s]] - D[(size_t)p[x] * n + p[r]];
  }
  for (int u = 0; u < n; ++u) {
    for (int v = u + 1; v < n; ++v) {
      int64_t *slot = &t->dl[(size_t)u * n + v];
      if (u == r && v == s) {
        *slot = -*slot;
      } else if (u == r || u == s || v == r || v == s) {
        *slot = orc_delta(F, D, n, p, u, v, err);
      } else {
        int64_t d1 = chk_mul(chk_sub(a[u], a[v], err), chk_sub(b[u], b[v], err), err);
        int64_t d2 = chk_mul(chk_sub(c[u], c[v], err), chk_sub(e[u], e[v], err), err);
        *slot = chk_add(*slot, chk_add(d1, d2, err), err);
      }
    }
  }
  free(a);
  if (mode == ORC_CHECK) {
    for (int u = 0; u < n; ++u)
      for (int v = u + 1; v < n; ++v)
        if (t->dl[(size_t)u * n + v] != orc_delta(F, D, n, p, u, v, err))
          *err = ORC_EMISMATCH;
  }
}

static void apply_swap(int32_t *p, int r, int s) {
  int32_t t = p[r]; p[r] = p[s]; p[s] = t;
}

/* ------------------------------------------------------------------------ */
/* Best-improvement 2opt (Section 4.1): evaluate every pairwise exchange,    */
/* move to the lowest-cost neighbour.  The paper runs a fixed iteration      */
/* count that it never states; the reading taken here stops at a local       */
/* minimum (no neighbour with a negative delta) or after max_iters moves     */
/* (max_iters < 0: no cap).                                                  */
/* ------------------------------------------------------------------------ */

int orc_2opt(const int64_t *F, const int64_t *D, int n, int32_t *p,
             int32_t max_iters, int mode, int32_t *moves, int32_t moves_cap,
             orc_walk_result *res) {
  int err = ORC_OK;
  delta_table t = {n, calloc((size_t)n * n, sizeof(int64_t))};
  int64_t cur = orc_cost(F, D, n, p, &err);
  uint64_t h = orc_hash_init();
  int32_t it = 0;
  table_fill(&t, F, D, p, &err);
  for (;;) {
    if (max_iters >= 0 && it >= max_iters) break;
    int br = -1, bs = -1;
    int64_t bd = 0;
    for (int r = 0; r < n; ++r)
      for (int s = r + 1; s < n; ++s) {
        int64_t d = t.dl[(size_t)r * n + s];
        if (br < 0 || d < bd) { br = r; bs = s; bd = d; }
      }
    if (br < 0 || bd >= 0) break;          /* local minimum */
    apply_swap(p, br, bs);
    cur = chk_add(cur, bd, &err);
    h = orc_hash_move(h, br, bs);
    if (moves && it < moves_cap) { moves[2 * it] = br; moves[2 * it + 1] = bs; }
    ++it;
    table_update(&t, F, D, p, br, bs, mode, &err);
    if (err) break;
  }
  free(t.dl);
  res->best_cost = cur;
  res->final_cost = cur;
  res->best_iter = it;
  res->iters_done = it;
  res->status = 0;
  res->hash = h;
  return err;
}

/* ------------------------------------------------------------------------ */
/* Tabu search (Sections 4.3, 4.4).  Iterations are numbered from 1.         */
/* Per iteration:                                                            */
/*   1. evaluate every pairwise exchange (Eq. 2);                            */
/*   2. a move is admissible if it is not tabu under the chosen criterion    */
/*      (below) or, with aspiration on, if it leads to a cost strictly below */
/*      the best cost so far;                                                */
/*   3. take the admissible move of lowest score, ties to the lowest (r, s)  */
/*      (the paper's "next lowest cost" loop over forbidden moves selects    */
/*      exactly this).  The score is the delta itself; with a frequency      */
/*      penalty lambda > 0 a non-improving move (delta >= 0) scores          */
/*      delta + lambda * (times the move was applied so far);               */
/*   4. if no move is admissible the walk stops early (status 1);            */
/*   5. apply it with a tenure t from the tenure rule, mark it tabu under    */
/*      the criterion, count the exchange in the frequency memory (lower     */
/*      triangle of Tabuarr) and keep the solution if its cost is strictly   */
/*      below the best.                                                      */
/*                                                                           */
/* Tabu criteria (every mark is "until iteration it + t"; a mark m forbids   */
/* while m > it):                                                            */
/*   ORC_TABU_PAIR      the paper's Tabuarr (Section 4.3): the applied move  */
/*                      (r, s) itself is forbidden;                          */
/*   ORC_TABU_UNIT_LOC  Taillard's robust tabu search (1991, the elementary  */
/*                      search Section 4.3 follows): units r and s may not   */
/*                      return to the locations they leave; a move (u, v) is */
/*                      forbidden when BOTH u would return to a forbidden    */
/*                      location and v would;                                */
/*   ORC_TABU_UNIT      Zhu et al.'s unit marking (Section 3.1): units r and */
/*                      s are marked; a move is forbidden when EITHER of its */
/*                      units is marked.                                     */
/* The frequency penalty is the long-term frequency-based memory Section 7   */
/* proposes as future work, in the usual form of a penalty on non-improving  */
/* moves (Glover & Laguna, cited in Section 4.3).                            */
/* ------------------------------------------------------------------------ */

static int move_is_tabu(int crit, int n, const int32_t *p, int u, int v, int32_t it,
                        const int32_t *pair_until, const int32_t *loc_until,
                        const int32_t *unit_until) {
  if (crit == ORC_TABU_PAIR) return pair_until[(size_t)u * n + v] > it;
  if (crit == ORC_TABU_UNIT_LOC)  /* u would move to p[v], v to p[u] */
    return loc_until[(size_t)u * n + p[v]] > it && loc_until[(size_t)v * n + p[u]] > it;
  return unit_until[u] > it || unit_until[v] > it;
}

int orc_tabu(const int64_t *F, const int64_t *D, int n, int32_t *p,
             int32_t iters, const orc_tenure_t *tn, int aspiration,
             const orc_rules_t *rules, uint64_t seed, uint32_t walk, int mode,
             int32_t *best_p, int32_t *freq, int32_t *moves,
             orc_walk_result *res) {
  const int crit = rules ? rules->criterion : ORC_TABU_PAIR;
  const int64_t lambda = rules ? rules->penalty : 0;
  if (crit < ORC_TABU_PAIR || crit > ORC_TABU_UNIT || lambda < 0) return ORC_EINVAL;
  int err = ORC_OK;
  delta_table t = {n, calloc((size_t)n * n, sizeof(int64_t))};
  int32_t *pair_until = calloc((size_t)n * n, sizeof(int32_t)); /* [r][s], r < s  */
  int32_t *loc_until = calloc((size_t)n * n, sizeof(int32_t));  /* [unit][location] */
  int32_t *unit_until = calloc((size_t)n, sizeof(int32_t));     /* [unit]          */
  int32_t *applied = calloc((size_t)n * n, sizeof(int32_t));    /* [r][s], r < s  */
  int64_t cur = orc_cost(F, D, n, p, &err);
  int64_t best = cur;
  int32_t best_iter = 0, status = 0, done = 0;
  uint64_t h = orc_hash_init();
  memcpy(best_p, p, sizeof(int32_t) * (size_t)n);
  table_fill(&t, F, D, p, &err);
  for (int32_t it = 1; it <= iters && !err; ++it) {
    int br = -1, bs = -1;
    int64_t bd = 0, bscore = 0;
    for (int r = 0; r < n; ++r)
      for (int s = r + 1; s < n; ++s) {
        int64_t d = t.dl[(size_t)r * n + s];
        int not_tabu = !move_is_tabu(crit, n, p, r, s, it, pair_until, loc_until, unit_until);
        int aspires = aspiration && chk_add(cur, d, &err) < best;
        if (!(not_tabu || aspires)) continue;
        int64_t score = d;
        if (d >= 0) score = chk_add(d, chk_mul(lambda, applied[(size_t)r * n + s], &err), &err);
        if (br < 0 || score < bscore) { br = r; bs = s; bd = d; bscore = score; }
      }
    if (br < 0) { status = 1; break; }
    int32_t tenure = orc_tenure(tn, seed, walk, it);
    pair_until[(size_t)br * n + bs] = it + tenure;
    loc_until[(size_t)br * n + p[br]] = it + tenure;  /* the locations they leave */
    loc_until[(size_t)bs * n + p[bs]] = it + tenure;
    unit_until[br] = unit_until[bs] = it + tenure;
    applied[(size_t)br * n + bs] += 1;
    apply_swap(p, br, bs);
    cur = chk_add(cur, bd, &err);
    h = orc_hash_move(h, br, bs);
    if (moves) { moves[2 * (it - 1)] = br; moves[2 * (it - 1) + 1] = bs; }
    done = it;
    if (cur < best) {
      best = cur;
      best_iter = it;
      memcpy(best_p, p, sizeof(int32_t) * (size_t)n);
    }
    table_update(&t, F, D, p, br, bs, mode, &err);
  }
  if (freq) { /* lower triangle: [s][r] counts move (r, s) */
    memset(freq, 0, sizeof(int32_t) * (size_t)n * n);
    for (int r = 0; r < n; ++r)
      for (int s = r + 1; s < n; ++s) freq[(size_t)s * n + r] = applied[(size_t)r * n + s];
  }
  free(t.dl);
  free(pair_until);
  free(loc_until);
  free(unit_until);
  free(applied);
  res->best_cost = best;
  res->final_cost = cur;
  res->best_iter = best_iter;
  res->iters_done = done;
  res->status = status;
  res->hash = h;
  return err;
}

/* ------------------------------------------------------------------------ */
/* Many walks of one instance, one per OpenMP thread (the CPU counterpart    */
/* of the paper's one-search-per-GPU-thread layout, Sections 4.2 and 4.4).   */
/*                                                                           */
/* Walk w uses walk id walk_ids[w] for its random draws.  If starts is NULL  */
/* the initial solution is drawn by orc_start_perm, else row w of starts is  */
/* used.  descend: 1 = run 2opt to a local minimum before the tabu phase.   */
/* iters == 0 with descend == 1 gives plain 2opt.                            */
/* Outputs are per walk: best_p (walks x n), best_cost, final_cost,          */
/* best_iter, iters_done, status, hash; descent_moves (may be NULL).         */
/* Returns the first non-zero error of any walk.                             */
/* ------------------------------------------------------------------------ */

int orc_run_walks(const int64_t *F, const int64_t *D, int n, int32_t walks,
                  const uint32_t *walk_ids, const int32_t *starts,
                  int descend, int32_t max_descent, int32_t iters,
                  const orc_tenure_t *tn, int aspiration, const orc_rules_t *rules,
                  uint64_t seed, int mode, int threads,
                  int32_t *best_p, int64_t *best_cost, int64_t *final_cost,
                  int32_t *best_iter, int32_t *iters_done, int32_t *status,
                  uint64_t *hash, uint64_t *descent_hash, int32_t *descent_moves) {
  int first_err = ORC_OK;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int32_t w = 0; w < walks; ++w) {
    int32_t *p = malloc(sizeof(int32_t) * (size_t)n);
    uint32_t wid = walk_ids ? walk_ids[w] : (uint32_t)w;
    if (starts) memcpy(p, starts + (size_t)w * n, sizeof(int32_t) * (size_t)n);
    else orc_start_perm(seed, wid, n, p);
    orc_walk_result r2 = {0}, rt = {0};
    int err = ORC_OK;
    int32_t dmoves = 0;
    uint64_t dh = orc_hash_init();
    if (descend) {
      err = orc_2opt(F, D, n, p, max_descent, mode, NULL, 0, &r2);
      dmoves = r2.iters_done;
      dh = r2.hash;
    }
    if (!err && (iters > 0 || !descend)) {
      err = orc_tabu(F, D, n, p, iters, tn, aspiration, rules, seed, wid, mode,
                     best_p + (size_t)w * n, NULL, NULL, &rt);
    } else if (!err) {
      memcpy(best_p + (size_t)w * n, p, sizeof(int32_t) * (size_t)n);
      rt = r2;
      rt.best_iter = 0;
      rt.iters_done = 0;
      rt.hash = orc_hash_init();
    }
    best_cost[w] = rt.best_cost;
    if (final_cost) final_cost[w] = rt.final_cost;
    best_iter[w] = rt.best_iter;
    iters_done[w] = rt.iters_done;
    status[w] = rt.status;
    if (hash) hash[w] = rt.hash;
    if (descent_hash) descent_hash[w] = dh;
    if (descent_moves) descent_moves[w] = dmoves;
    if (err) {
#ifdef _OPENMP
#pragma omp critical
#endif
      { if (!first_err) first_err = err; }
    }
    free(p);
  }
  return first_err;
}

/* ------------------------------------------------------------------------ */
/* Exhaustive search over all n! permutations (n <= 10): the exact optimum,  */
/* lowest-cost permutation first met in lexicographic order of p.            */
/* ------------------------------------------------------------------------ */

int64_t orc_brute_force(const int64_t *F, const int64_t *D, int n, int32_t *best_p, int *err) {
  int32_t p[16];
  int64_t best = 0;
  int have = 0;
  if (n < 1 || n > 10) { *err = ORC_EINVAL; return 0; }
  /* lexicographic enumeration of p by the next-permutation step */
  for (int i = 0; i < n; ++i) p[i] = i;
  for (;;) {
    int64_t c = orc_cost(F, D, n, p, err);
    if (!have || c < best) {
      best = c; have = 1;
      memcpy(best_p, p, sizeof(int32_t) * (size_t)n);
    }
    int i = n - 2;
    while (i >= 0 && p[i] > p[i + 1]) --i;
    if (i < 0) break;
    int j = n - 1;
    while (p[j] < p[i]) --j;
    int32_t t = p[i]; p[i] = p[j]; p[j] = t;
    for (int a = i + 1, b = n - 1; a < b; ++a, --b) { t = p[a]; p[a] = p[b]; p[b] = t; }
  }
  return best;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
