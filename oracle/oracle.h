/* oracle.h — FP64 CPU reference for CFR+ (TEST INFRASTRUCTURE ONLY).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library. It is independent of the CUDA path: no shared code,
 * headers or helpers. The game arrives as plain arrays in the generator's
 * tabular form (node 0 is the root; children in action order).
 *
 * Slots: information set I owns slots off(I) .. off(I) + nact(I) - 1 where
 * off is the prefix sum of iset_nact in information-set id order.
 */
#ifndef CFR_ORACLE_H
#define CFR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_game {
  int64_t n_nodes;
  int64_t n_infosets;
  const int8_t *kind;         /* [N] 0 terminal, 1 chance, 2 player 1, 3 player 2 */
  const int32_t *infoset;     /* [N] */
  const int64_t *child_begin; /* [N+1] */
  const int32_t *child;       /* [E] */
  const double *chance_prob;  /* [E] */
  const double *payoff;       /* [N] payoff to player 1 */
  const int8_t *iset_player;  /* [I] 0 or 1 */
  const int32_t *iset_nact;   /* [I] */
} or_game;

enum { OR_CFR_PLUS = 0, OR_CFR = 1, OR_PCFR_PLUS = 2 };
enum { OR_SIMULTANEOUS = 0, OR_ALTERNATING = 1 };

/* Runs iterations t0+1 .. t0+T of CFR (rule OR_CFR_PLUS, OR_CFR or
 * OR_PCFR_PLUS) from the state (R, sbar), both [A] and updated in place.
 * Zero state and t0 = 0 is a fresh solve. Averaging weight w_t = t, or t^2
 * for PCFR+. PCFR+ (Section 3, "update rules"): the CFR+ regret update, and
 * the strategy is regret matching of R + pred, where pred [A] holds each
 * slot's last instantaneous regret (the prediction; zero at the start,
 * updated in place; required for OR_PCFR_PLUS, ignored otherwise). root_value (optional)
 * receives the chance-weighted root value of the last pass. Returns 0, or
 * < 0 on error. */
int or_cfr_run(const or_game *g, int64_t t0, int64_t T, int rule, int order, double *R, double *sbar,
               double *pred, double *root_value);

/* Average strategy: sbar normalised per information set, uniform if zero. */
void or_avg_strategy(const or_game *g, const double *sbar, double *out);

/* Regret-matching strategy of the cumulative regrets R (plus the prediction
 * pred [A] when it is not NULL: the PCFR+ strategy). */
void or_current_strategy(const or_game *g, const double *R, const double *pred, double *out);

/* Expected payoff to player 1 when both players follow sigma [A]. */
double or_expected_value(const or_game *g, const double *sigma);

/* Exact best-response values in player-1 units: br1 = max over player 1's
 * strategies against sigma's player 2, br2 = min over player 2's strategies
 * against sigma's player 1; value = u(sigma). Returns 0 or < 0. */
int or_best_response(const or_game *g, const double *sigma, double *br1, double *br2, double *value);

/* NashConv / 2 = (br1 - br2) / 2. */
double or_exploitability(const or_game *g, const double *sigma);

/* Best response of `player` (0 or 1) by enumerating all pure strategies
 * (refuses with -4 above max_strategies). Player 1 maximises, player 2
 * minimises player 1's payoff. */
int or_bruteforce_br(const or_game *g, const double *sigma, int player, int64_t max_strategies,
                     double *out);

#ifdef __cplusplus
}
#endif
#endif
