/*
 * CPU oracle for the QAP swap-neighbourhood search (test infrastructure only;
 * see qap_oracle.c for the conventions and the passages each function
 * follows).
 */
#ifndef QAP_ORACLE_H
#define QAP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EOVERFLOW = 1, ORC_EINVAL = 2, ORC_EMISMATCH = 3 };
enum { ORC_REF = 0, ORC_FAST = 1, ORC_CHECK = 2 };
enum { ORC_STREAM_START = 0, ORC_STREAM_TENURE = 1 };

typedef struct { int32_t tmin, tmax, period; } orc_tenure_t;

/* Tabu criterion and frequency penalty of the tabu phase (see orc_tabu). */
enum { ORC_TABU_PAIR = 0, ORC_TABU_UNIT_LOC = 1, ORC_TABU_UNIT = 2 };
typedef struct { int32_t criterion; int32_t penalty; } orc_rules_t;

typedef struct {
  int64_t best_cost;
  int64_t final_cost;
  int32_t best_iter;
  int32_t iters_done;
  int32_t status;
  uint64_t hash;
} orc_walk_result;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t orc_draw(uint64_t seed, uint32_t walk, uint32_t stream, uint32_t idx);
uint32_t orc_bounded(uint32_t x, uint32_t m);
void orc_start_perm(uint64_t seed, uint32_t walk, int n, int32_t *p);
int32_t orc_tenure(const orc_tenure_t *tn, uint64_t seed, uint32_t walk, int32_t it);
uint64_t orc_hash_init(void);
uint64_t orc_hash_move(uint64_t h, int r, int s);

int64_t orc_cost(const int64_t *F, const int64_t *D, int n, const int32_t *p, int *err);
int64_t orc_delta(const int64_t *F, const int64_t *D, int n, const int32_t *p,
                  int r, int s, int *err);

int orc_2opt(const int64_t *F, const int64_t *D, int n, int32_t *p,
             int32_t max_iters, int mode, int32_t *moves, int32_t moves_cap,
             orc_walk_result *res);
int orc_tabu(const int64_t *F, const int64_t *D, int n, int32_t *p,
             int32_t iters, const orc_tenure_t *tn, int aspiration,
             const orc_rules_t *rules, uint64_t seed, uint32_t walk, int mode,
             int32_t *best_p, int32_t *freq, int32_t *moves,
             orc_walk_result *res);
int orc_run_walks(const int64_t *F, const int64_t *D, int n, int32_t walks,
                  const uint32_t *walk_ids, const int32_t *starts,
                  int descend, int32_t max_descent, int32_t iters,
                  const orc_tenure_t *tn, int aspiration, const orc_rules_t *rules,
                  uint64_t seed, int mode, int threads,
                  int32_t *best_p, int64_t *best_cost, int64_t *final_cost,
                  int32_t *best_iter, int32_t *iters_done, int32_t *status,
                  uint64_t *hash, uint64_t *descent_hash, int32_t *descent_moves);
int64_t orc_brute_force(const int64_t *F, const int64_t *D, int n, int32_t *best_p, int *err);
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
