/* gamegen.h — seeded synthetic two-player zero-sum extensive-form games.
 *
 * Input generators only: this module builds game trees (structure, chance
 * probabilities, payoffs, information sets). It contains no CFR arithmetic and
 * is shared, as an input source, by the FP64 oracle and by the CUDA path.
 *
 * A game is returned in the tabular form of the paper's compiler input
 * (Appendix H, "Input representation"): per node its kind, acting player's
 * information set and ordered child list; per edge the chance probability; per
 * terminal the payoff to player 1; per information set its player and action
 * count. Node 0 is the root. Children are listed in action order.
 *
 * Ownership: every gg_* constructor returns a heap object owned by the caller
 * and released with gg_free(). On failure a constructor returns NULL and
 * gg_last_error() describes why.
 */
#ifndef GAMEGEN_H
#define GAMEGEN_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { GG_TERMINAL = 0, GG_CHANCE = 1, GG_P1 = 2, GG_P2 = 3 };

typedef struct gg_spec {
  int64_t n_nodes;       /* N */
  int64_t n_edges;       /* child_begin[N] (= N-1 for a tree) */
  int64_t n_infosets;    /* I */
  int8_t *kind;          /* [N] GG_TERMINAL / GG_CHANCE / GG_P1 / GG_P2 */
  int32_t *infoset;      /* [N] information set of a decision node, else -1 */
  int64_t *child_begin;  /* [N+1] offsets into child[] */
  int32_t *child;        /* [n_edges] child node ids in action order */
  double *chance_prob;   /* [n_edges] outcome probability under a chance parent, else 0 */
  double *payoff;        /* [N] payoff to player 1 at terminals, else 0 */
  int8_t *iset_player;   /* [I] 0 = player 1, 1 = player 2 */
  int32_t *iset_nact;    /* [I] number of actions */
  double pot;            /* normaliser for exploitability thresholds */
  /* Optional per-information-set feature metadata (card games only, else NULL):
   * iset_feat[I * GG_NFEAT] small integers describing the set (see gamegen.c). */
  int32_t *iset_feat;
} gg_spec;

#define GG_NFEAT 16

const char *gg_last_error(void);
void gg_free(gg_spec *g);

/* One-card poker: `ranks` distinct cards, one private card per player dealt
 * by a uniform chance root over ordered deals, one betting round with
 * check/bet, fold/call/raise, ante 1, bet 1, at most `cap` bets. ranks=3,
 * cap=1 is Kuhn poker. Nodes are in depth-first preorder. */
gg_spec *gg_tiny_card(int ranks, int cap);

/* Seeded random perfect-recall tree: `depth` node levels (leaves at depth
 * depth-1), branching uniform in {bmin..bmax} per chance node / per
 * information set, chance nodes with probability p_chance (Dirichlet(1)
 * outcome probabilities), player nodes grouped by their own sequence into
 * information sets of 1..max_group members, leaf payoffs U[-1,1].
 * Nodes are in breadth-first order. */
gg_spec *gg_random_tree(uint64_t seed, int depth, int bmin, int bmax,
                        double p_chance, int max_group);

/* Two-round card game: 8 ranks x 4 suits, two private cards each, one public
 * card between the rounds, bets raise to call + f*(pot after call) for f in
 * {1/2, 1} or all-in, at most `cap` bets per round, stacks of `stack` antes
 * behind an ante of 1 each. Showdown ranks three-card hands (trips > pair >
 * high card, kickers lexicographic, suits ignored, ties split).
 * `n_ranks`/`n_suits` shrink the deck for small test instances.
 * Nodes are in breadth-first order. */
gg_spec *gg_large_card(int n_ranks, int n_suits, int stack, int cap);

/* The same game restricted to every deal_stride-th deal of the root (deal
 * probabilities renormalised): a uniform sample of the full game's subtrees,
 * used to time the CPU reference on a bounded part of the workload. */
gg_spec *gg_large_card_sampled(int n_ranks, int n_suits, int stack, int cap, int deal_stride);

/* River-style endgame subgame: one betting round over a fixed one-card board,
 * K1 and K2 distinct two-card hands per player drawn from the 8x4 deck minus
 * the board, ranges Dirichlet(0.5), 2..4 pot-fraction bet sizes, cap 2 bets.
 * Deal probability is proportional to range1(h1) * range2(h2) over
 * non-overlapping hand pairs. Sizes are reject-sampled so that the edge count
 * lands near `target_edges`. Nodes are in breadth-first order. */
gg_spec *gg_endgame(uint64_t seed, int64_t target_edges);

/* Counter-based SplitMix64 stream shared by all generators:
 * gg_rand(seed, stream, i) is the i-th 64-bit word of stream `stream`. */
uint64_t gg_rand(uint64_t seed, uint64_t stream, uint64_t i);

#ifdef __cplusplus
}
#endif
#endif
