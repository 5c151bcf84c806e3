/* oracle.c — plain, slow, FP64 CPU reference for CFR+ (TEST INFRASTRUCTURE).
 *
 * This file is the oracle that the CUDA path is checked against. Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it; the product path never does. It shares no code, header, table or helper
 * with the CUDA path: it reads the game in the generator's tabular form
 * (plain arrays) and walks the tree recursively.
 *
 * Build: gcc -O2 -ffp-contract=off (no fused multiply-add, so every product
 * and sum rounds exactly as written).
 *
 * What it follows (paper sections / equations):
 *   - reach, counterfactual value, regret, regret matching: Section 3,
 *     eqs. (reach), (cfv), (regret), (rm); uniform strategy when the positive
 *     regrets sum to zero.
 *   - CFR+ clamps the cumulative regret at zero after each update (Section 3,
 *     the CFR+ paragraph); vanilla CFR skips the clamp.
 *   - simultaneous updates: both players update from one profile (Section 3).
 *   - linear averaging w_t = t, t = 1, 2, ... with the reach-weighted current
 *     strategy (eq. (rm), Algorithm 1's last line), accumulated in FP64
 *     (Proposition 4 and the paragraph after it).
 *   - the per-history regret term s * pi_{-i}(h) * (v(h.a) - v(h)) with v in
 *     player-1 units (eq. (instregret)); its sum over h in I is the standard
 *     counterfactual regret.
 *   - exploitability = NashConv / 2 by exact best response (eq.
 *     (exploitability)).
 *
 * Summation order: the walk is depth-first preorder. Every information set's
 * members sit at one depth, and for nodes of equal depth the depth-first
 * order equals the breadth-first (level, left-to-right) order, so the regret
 * and average sums of a set run over its members in ascending breadth-first
 * order, each term added as soon as its history's subtree returns.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXA 64

enum { T_TERM = 0, T_CHANCE = 1, T_P1 = 2, T_P2 = 3 };

typedef struct {
  const or_game *g;
  const int64_t *off;  /* slot offset of each information set */
  const double *sigma; /* current strategy, [A] */
  double *r;           /* instantaneous regret sums, [A] */
  double *m;           /* reach-weighted strategy sums, [A] */
  int update_mask;     /* bit p set: record terms of player p */
  int fail;
} walk_ctx;

/* Returns the chance-weighted player-1 value of the subtree at h, i.e. the
 * sum over terminals z below h of pi_c(z) * pi_1,2(h -> z) * u(z) (the value
 * the paper's backward recurrence returns, Proposition 1). pc is the chance
 * product of the path root..h in path order. */
static double walk(walk_ctx *w, int32_t h, double pi1, double pi2, double pc) {
  const or_game *g = w->g;
  const int k = g->kind[h];
  const int64_t b = g->child_begin[h], e = g->child_begin[h + 1];
  if (k == T_TERM) return pc * g->payoff[h];
  if (k == T_CHANCE) {
    double v = 0.0;
    for (int64_t q = b; q < e; ++q) v += walk(w, g->child[q], pi1, pi2, pc * g->chance_prob[q]);
    return v;
  }
  const int p = k - T_P2 + 1; /* 0 for player 1, 1 for player 2 */
  const int32_t I = g->infoset[h];
  const int64_t s0 = w->off[I];
  const int na = (int)(e - b);
  if (na > OR_MAXA) { w->fail = 1; return 0.0; }
  double vals[OR_MAXA];
  for (int a = 0; a < na; ++a) {
    const double sa = w->sigma[s0 + a];
    vals[a] = p == 0 ? walk(w, g->child[b + a], pi1 * sa, pi2, pc)
                     : walk(w, g->child[b + a], pi1, pi2 * sa, pc);
  }
  double v = 0.0;
  for (int a = 0; a < na; ++a) v += w->sigma[s0 + a] * vals[a];
  if (w->update_mask & (1 << p)) {
    const double sgn = p == 0 ? 1.0 : -1.0;   /* s(e): orient toward the actor */
    const double pi_opp = p == 0 ? pi2 : pi1; /* counterfactual reach (chance is in v) */
    const double pi_own = p == 0 ? pi1 : pi2;
    for (int a = 0; a < na; ++a) {
      w->r[s0 + a] += (sgn * pi_opp) * (vals[a] - v);
      w->m[s0 + a] += pi_own * w->sigma[s0 + a];
    }
  }
  return v;
}

static int64_t *slot_offsets(const or_game *g) {
  int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g->n_infosets + 1));
  if (!off) return NULL;
  off[0] = 0;
  for (int64_t i = 0; i < g->n_infosets; ++i) off[i + 1] = off[i] + g->iset_nact[i];
  return off;
}

/* Regret matching (eq. (rm)): sigma proportional to the positive part of R,
 * uniform when that part sums to zero. With a prediction (PCFR+), the
 * positive part of R + pred. */
static void regret_matching(const or_game *g, const int64_t *off, const double *R, const double *pred,
                            double *sigma, int player_mask) {
  for (int64_t I = 0; I < g->n_infosets; ++I) {
    if (!(player_mask & (1 << g->iset_player[I]))) continue;
    const int64_t s0 = off[I];
    const int na = g->iset_nact[I];
    double tot = 0.0;
    for (int a = 0; a < na; ++a) {
      const double x = pred ? R[s0 + a] + pred[s0 + a] : R[s0 + a];
      tot += x > 0.0 ? x : 0.0;
    }
    for (int a = 0; a < na; ++a) {
      const double x = pred ? R[s0 + a] + pred[s0 + a] : R[s0 + a];
      sigma[s0 + a] = tot > 0.0 ? (x > 0.0 ? x : 0.0) / tot : 1.0 / (double)na;
    }
  }
}

int or_cfr_run(const or_game *g, int64_t t0, int64_t T, int rule, int order, double *R, double *sbar,
               double *pred, double *root_value) {
  if (!g || T < 0 || !R || !sbar) return -1;
  if (rule == OR_PCFR_PLUS && !pred) return -1;
  const double *pr = rule == OR_PCFR_PLUS ? pred : NULL;
  int64_t *off = slot_offsets(g);
  if (!off) return -2;
  const int64_t A = off[g->n_infosets];
  double *sigma = (double *)malloc(sizeof(double) * (size_t)(A > 0 ? A : 1));
  double *r = (double *)malloc(sizeof(double) * (size_t)(A > 0 ? A : 1));
  double *m = (double *)malloc(sizeof(double) * (size_t)(A > 0 ? A : 1));
  if (!sigma || !r || !m) { free(off); free(sigma); free(r); free(m); return -2; }
  walk_ctx w;
  memset(&w, 0, sizeof w);
  w.g = g; w.off = off; w.sigma = sigma; w.r = r; w.m = m;
  int rc = 0;
  double v = 0.0;
  for (int64_t it = 1; it <= T && rc == 0; ++it) {
    /* averaging weight: linear w_t = t (CFR, CFR+); quadratic w_t = t^2 for
     * PCFR+ (the reading that reproduces the alternating Kuhn cell of the
     * convergence table) */
    const double tt = (double)(t0 + it);
    const double wt = rule == OR_PCFR_PLUS ? tt * tt : tt;
    const int halves = order == OR_ALTERNATING ? 2 : 1;
    for (int hlf = 0; hlf < halves; ++hlf) {
      const int mask = order == OR_ALTERNATING ? (1 << hlf) : 3;
      regret_matching(g, off, R, pr, sigma, 3);
      memset(r, 0, sizeof(double) * (size_t)A);
      memset(m, 0, sizeof(double) * (size_t)A);
      w.update_mask = mask;
      v = walk(&w, 0, 1.0, 1.0, 1.0);
      if (w.fail) { rc = -3; break; }
      for (int64_t I = 0; I < g->n_infosets; ++I) {
        if (!(mask & (1 << g->iset_player[I]))) continue;
        for (int64_t q = off[I]; q < off[I + 1]; ++q) {
          sbar[q] += wt * m[q]; /* average accumulates sigma^t before the clamp */
          const double nr = R[q] + r[q];
          R[q] = (rule == OR_CFR) ? nr : (nr > 0.0 ? nr : 0.0); /* CFR+ and PCFR+ clamp */
          if (rule == OR_PCFR_PLUS) pred[q] = r[q];               /* next prediction */
        }
      }
    }
  }
  if (root_value) *root_value = v;
  free(off); free(sigma); free(r); free(m);
  return rc;
}

void or_avg_strategy(const or_game *g, const double *sbar, double *out) {
  int64_t s0 = 0;
  for (int64_t I = 0; I < g->n_infosets; ++I) {
    const int na = g->iset_nact[I];
    double tot = 0.0;
    for (int a = 0; a < na; ++a) tot += sbar[s0 + a];
    for (int a = 0; a < na; ++a) out[s0 + a] = tot > 0.0 ? sbar[s0 + a] / tot : 1.0 / (double)na;
    s0 += na;
  }
}

void or_current_strategy(const or_game *g, const double *R, const double *pred, double *out) {
  int64_t *off = slot_offsets(g);
  if (!off) return;
  regret_matching(g, off, R, pred, out, 3);
  free(off);
}

/* ------------------------------------------------ evaluation (no folding) */
/* Expected payoff to player 1 when both play `sigma`: the plain recursive
 * definition with chance probabilities applied at chance nodes. */
static double ev_rec(const or_game *g, const int64_t *off, const double *sigma, int32_t h) {
  const int k = g->kind[h];
  const int64_t b = g->child_begin[h], e = g->child_begin[h + 1];
  if (k == T_TERM) return g->payoff[h];
  double v = 0.0;
  if (k == T_CHANCE) {
    for (int64_t q = b; q < e; ++q) v += g->chance_prob[q] * ev_rec(g, off, sigma, g->child[q]);
    return v;
  }
  const int64_t s0 = off[g->infoset[h]];
  for (int64_t q = b; q < e; ++q) v += sigma[s0 + (q - b)] * ev_rec(g, off, sigma, g->child[q]);
  return v;
}

double or_expected_value(const or_game *g, const double *sigma) {
  int64_t *off = slot_offsets(g);
  if (!off) return NAN;
  double v = ev_rec(g, off, sigma, 0);
  free(off);
  return v;
}

/* Exact best response by depth levels (members of a set share a depth).
 * For the responder i and each set I of i at depth d, Q(I,a) sums over the
 * members h (depth-first order) the reach of chance and the opponent under
 * sigma_bar times the continuation value of h.a, where deeper sets already
 * play their best action; the best action is the lowest-index maximiser
 * (player 1) or minimiser of player 1's payoff (player 2). */
int or_best_response(const or_game *g, const double *sbar_sigma, double *br1, double *br2,
                     double *value) {
  const int64_t N = g->n_nodes;
  int64_t *off = slot_offsets(g);
  int32_t *depth = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  int32_t *pre = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  double *cf = (double *)malloc(sizeof(double) * (size_t)N * 2); /* [v*2 + i]: reach of all but i */
  double *V = (double *)malloc(sizeof(double) * (size_t)N * 2);  /* [v*2 + i]: value for BR of i */
  if (!off || !depth || !pre || !stack || !cf || !V) {
    free(off); free(depth); free(pre); free(stack); free(cf); free(V);
    return -2;
  }
  const int64_t A = off[g->n_infosets];
  double *Q = (double *)calloc((size_t)(A > 0 ? A : 1), sizeof(double));
  int32_t *best = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n_infosets > 0 ? g->n_infosets : 1));
  if (!Q || !best) { free(off); free(depth); free(pre); free(stack); free(cf); free(V); free(Q); free(best); return -2; }
  /* preorder with explicit stack; children pushed in reverse to visit in order */
  int64_t sp = 0, np = 0;
  stack[sp++] = 0;
  depth[0] = 0;
  cf[0] = 1.0; cf[1] = 1.0;
  int32_t maxd = 0;
  while (sp > 0) {
    const int32_t h = stack[--sp];
    pre[np++] = h;
    if (depth[h] > maxd) maxd = depth[h];
    const int k = g->kind[h];
    const int64_t b = g->child_begin[h], e = g->child_begin[h + 1];
    for (int64_t q = e - 1; q >= b; --q) {
      const int32_t c = g->child[q];
      depth[c] = depth[h] + 1;
      double f0 = cf[2 * h], f1 = cf[2 * h + 1];
      if (k == T_CHANCE) { f0 *= g->chance_prob[q]; f1 *= g->chance_prob[q]; }
      else if (k == T_P1) { f1 *= sbar_sigma[off[g->infoset[h]] + (q - b)]; } /* P1 plays sigma_bar in P2's BR */
      else if (k == T_P2) { f0 *= sbar_sigma[off[g->infoset[h]] + (q - b)]; }
      cf[2 * c] = f0; cf[2 * c + 1] = f1;
      stack[sp++] = c;
    }
  }
  /* bucket preorder by depth (stable) */
  int64_t *dcount = (int64_t *)calloc((size_t)maxd + 2, sizeof(int64_t));
  int32_t *bydepth = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  if (!dcount || !bydepth) { free(off); free(depth); free(pre); free(stack); free(cf); free(V); free(Q); free(best); free(dcount); free(bydepth); return -2; }
  for (int64_t i = 0; i < N; ++i) dcount[depth[pre[i]] + 1]++;
  for (int32_t d = 0; d <= maxd; ++d) dcount[d + 1] += dcount[d];
  {
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)maxd + 1));
    for (int32_t d = 0; d <= maxd; ++d) fill[d] = dcount[d];
    for (int64_t i = 0; i < N; ++i) bydepth[fill[depth[pre[i]]]++] = pre[i];
    free(fill);
  }
  for (int resp = 0; resp < 2; ++resp) {
    const int kresp = resp == 0 ? T_P1 : T_P2;
    for (int32_t d = maxd; d >= 0; --d) {
      /* Q sums of the responder's sets at this depth */
      for (int64_t i = dcount[d]; i < dcount[d + 1]; ++i) {
        const int32_t h = bydepth[i];
        if (g->kind[h] != kresp) continue;
        const int64_t s0 = off[g->infoset[h]];
        const int64_t b = g->child_begin[h];
        const int na = g->iset_nact[g->infoset[h]];
        for (int a = 0; a < na; ++a) Q[s0 + a] += cf[2 * h + resp] * V[2 * g->child[b + a] + resp];
      }
      for (int64_t i = dcount[d]; i < dcount[d + 1]; ++i) {
        const int32_t h = bydepth[i];
        if (g->kind[h] != kresp) continue;
        const int32_t I = g->infoset[h];
        const int64_t s0 = off[I];
        int ba = 0;
        for (int a = 1; a < g->iset_nact[I]; ++a)
          if (resp == 0 ? Q[s0 + a] > Q[s0 + ba] : Q[s0 + a] < Q[s0 + ba]) ba = a;
        best[I] = ba;
      }
      for (int64_t i = dcount[d]; i < dcount[d + 1]; ++i) {
        const int32_t h = bydepth[i];
        const int k = g->kind[h];
        const int64_t b = g->child_begin[h], e = g->child_begin[h + 1];
        double v = 0.0;
        if (k == T_TERM) v = g->payoff[h];
        else if (k == T_CHANCE) for (int64_t q = b; q < e; ++q) v += g->chance_prob[q] * V[2 * g->child[q] + resp];
        else if (k == kresp) v = V[2 * g->child[b + best[g->infoset[h]]] + resp];
        else {
          const int64_t s0 = off[g->infoset[h]];
          for (int64_t q = b; q < e; ++q) v += sbar_sigma[s0 + (q - b)] * V[2 * g->child[q] + resp];
        }
        V[2 * h + resp] = v;
      }
    }
  }
  if (br1) *br1 = V[0];
  if (br2) *br2 = V[1];
  if (value) *value = ev_rec(g, off, sbar_sigma, 0);
  free(off); free(depth); free(pre); free(stack); free(cf); free(V); free(Q); free(best);
  free(dcount); free(bydepth);
  return 0;
}

double or_exploitability(const or_game *g, const double *sbar_sigma) {
  double b1 = 0.0, b2 = 0.0;
  if (or_best_response(g, sbar_sigma, &b1, &b2, NULL) != 0) return NAN;
  return 0.5 * (b1 - b2);
}

/* ---------------------------------------------- brute-force best response */
/* Value of a pure strategy of the responder (choice[I] per own set) against
 * sigma for the other player. */
static double pure_rec(const or_game *g, const int64_t *off, const double *sigma, const int32_t *choice,
                       int kresp, int32_t h) {
  const int k = g->kind[h];
  const int64_t b = g->child_begin[h], e = g->child_begin[h + 1];
  if (k == T_TERM) return g->payoff[h];
  if (k == kresp) return pure_rec(g, off, sigma, choice, kresp, g->child[b + choice[g->infoset[h]]]);
  double v = 0.0;
  if (k == T_CHANCE) {
    for (int64_t q = b; q < e; ++q) v += g->chance_prob[q] * pure_rec(g, off, sigma, choice, kresp, g->child[q]);
    return v;
  }
  const int64_t s0 = off[g->infoset[h]];
  for (int64_t q = b; q < e; ++q) v += sigma[s0 + (q - b)] * pure_rec(g, off, sigma, choice, kresp, g->child[q]);
  return v;
}

int or_bruteforce_br(const or_game *g, const double *sigma, int player, int64_t max_strategies,
                     double *out) {
  int64_t *off = slot_offsets(g);
  int32_t *choice = (int32_t *)calloc((size_t)(g->n_infosets > 0 ? g->n_infosets : 1), sizeof(int32_t));
  if (!off || !choice) { free(off); free(choice); return -2; }
  double count = 1.0;
  for (int64_t I = 0; I < g->n_infosets; ++I)
    if (g->iset_player[I] == player) count *= g->iset_nact[I];
  if (count > (double)max_strategies) { free(off); free(choice); return -4; }
  const int kresp = player == 0 ? T_P1 : T_P2;
  double bestv = player == 0 ? -INFINITY : INFINITY;
  for (;;) {
    const double v = pure_rec(g, off, sigma, choice, kresp, 0);
    if (player == 0 ? v > bestv : v < bestv) bestv = v;
    /* next pure strategy: mixed-radix increment over the responder's sets */
    int64_t I = 0;
    for (; I < g->n_infosets; ++I) {
      if (g->iset_player[I] != player) continue;
      if (++choice[I] < g->iset_nact[I]) break;
      choice[I] = 0;
    }
    if (I == g->n_infosets) break;
  }
  *out = bestv;
  free(off); free(choice);
  return 0;
}
