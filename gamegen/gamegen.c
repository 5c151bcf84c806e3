/* gamegen.c — seeded synthetic games (see gamegen.h). Input generation only:
 * no CFR arithmetic lives here. */
#include "gamegen.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static __thread char g_err[512];
static void set_err(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}
const char *gg_last_error(void) { return g_err; }

/* ---------------------------------------------------------------- RNG ---- */
static inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
uint64_t gg_rand(uint64_t seed, uint64_t stream, uint64_t i) {
  return splitmix64(splitmix64(seed ^ splitmix64(stream + 0x632BE59BD9B4E019ull)) + i);
}
static inline double u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }
/* open interval (0,1) for logarithms */
static inline double u01_open(uint64_t r) { return ((double)(r >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

/* --------------------------------------------------------- allocation ---- */
void gg_free(gg_spec *g) {
  if (!g) return;
  free(g->kind); free(g->infoset); free(g->child_begin); free(g->child);
  free(g->chance_prob); free(g->payoff); free(g->iset_player); free(g->iset_nact);
  free(g->iset_feat);
  free(g);
}

static gg_spec *spec_alloc(int64_t n, int64_t e, int64_t ni, int with_feat) {
  gg_spec *g = (gg_spec *)calloc(1, sizeof(gg_spec));
  if (!g) { set_err("out of host memory"); return NULL; }
  g->n_nodes = n; g->n_edges = e; g->n_infosets = ni;
  g->kind = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
  g->infoset = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  g->child_begin = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  g->child = (int32_t *)malloc(sizeof(int32_t) * (size_t)(e > 0 ? e : 1));
  g->chance_prob = (double *)calloc((size_t)(e > 0 ? e : 1), sizeof(double));
  g->payoff = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  g->iset_player = (int8_t *)malloc((size_t)(ni > 0 ? ni : 1));
  g->iset_nact = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ni > 0 ? ni : 1));
  if (with_feat) {
    g->iset_feat = (int32_t *)malloc(sizeof(int32_t) * (size_t)GG_NFEAT * (size_t)(ni > 0 ? ni : 1));
    if (g->iset_feat)
      for (int64_t i = 0; i < ni * GG_NFEAT; ++i) g->iset_feat[i] = -1;
  }
  if (!g->kind || !g->infoset || !g->child_begin || !g->child || !g->chance_prob ||
      !g->payoff || !g->iset_player || !g->iset_nact || (with_feat && !g->iset_feat)) {
    gg_free(g);
    set_err("out of host memory for a game of %lld nodes", (long long)n);
    return NULL;
  }
  return g;
}

/* Growable builder for depth-first generation. */
typedef struct {
  int64_t n, ncap, e, ecap, ni, nicap;
  gg_spec *g;
} builder;

static int grow(void **p, size_t elem, int64_t *cap, int64_t need) {
  if (need <= *cap) return 1;
  int64_t nc = *cap ? *cap : 64;
  while (nc < need) nc *= 2;
  void *q = realloc(*p, elem * (size_t)nc);
  if (!q) return 0;
  *p = q;
  *cap = nc;
  return 1;
}

static int b_init(builder *b) {
  memset(b, 0, sizeof *b);
  b->g = (gg_spec *)calloc(1, sizeof(gg_spec));
  return b->g != NULL;
}

/* New node with `nch` children whose ids are filled later via b_set_child. */
static int64_t b_node(builder *b, int kind, int32_t iset, double payoff, int nch) {
  gg_spec *g = b->g;
  int64_t nc = b->ncap, ec = b->ecap;
  if (!grow((void **)&g->kind, 1, &nc, b->n + 2)) return -1;
  nc = b->ncap;
  if (!grow((void **)&g->infoset, 4, &nc, b->n + 2)) return -1;
  nc = b->ncap;
  if (!grow((void **)&g->payoff, 8, &nc, b->n + 2)) return -1;
  nc = b->ncap;
  if (!grow((void **)&g->child_begin, 8, &nc, b->n + 2)) return -1;
  b->ncap = nc;
  if (!grow((void **)&g->child, 4, &ec, b->e + nch)) return -1;
  ec = b->ecap;
  if (!grow((void **)&g->chance_prob, 8, &ec, b->e + nch)) return -1;
  b->ecap = ec;
  int64_t id = b->n++;
  g->kind[id] = (int8_t)kind;
  g->infoset[id] = iset;
  g->payoff[id] = payoff;
  g->child_begin[id] = b->e;
  for (int a = 0; a < nch; ++a) { g->child[b->e + a] = -1; g->chance_prob[b->e + a] = 0.0; }
  b->e += nch;
  g->child_begin[b->n] = b->e;
  return id;
}

static int b_iset(builder *b, int player, int nact) {
  gg_spec *g = b->g;
  int64_t c = b->nicap;
  if (!grow((void **)&g->iset_player, 1, &c, b->ni + 1)) return -1;
  c = b->nicap;
  if (!grow((void **)&g->iset_nact, 4, &c, b->ni + 1)) return -1;
  c = b->nicap;
  if (!grow((void **)&g->iset_feat, 4 * GG_NFEAT, &c, b->ni + 1)) return -1;
  b->nicap = c;
  g->iset_player[b->ni] = (int8_t)player;
  g->iset_nact[b->ni] = nact;
  for (int f = 0; f < GG_NFEAT; ++f) g->iset_feat[b->ni * GG_NFEAT + f] = -1;
  return (int)b->ni++;
}

static gg_spec *b_finish(builder *b) {
  gg_spec *g = b->g;
  g->n_nodes = b->n;
  g->n_edges = b->e;
  g->n_infosets = b->ni;
  if (!g->iset_player) { g->iset_player = (int8_t *)malloc(1); g->iset_nact = (int32_t *)malloc(4); g->iset_feat = (int32_t *)malloc(4 * GG_NFEAT); }
  return g;
}

/* ------------------------------------------------------ one-card poker ---- */
/* Betting state of the single round: number of bets so far, whether the
 * actor faces a bet, and whether player 1 opened with a check. History ids
 * index the (actor, betting sequence) pairs so that infoset = (card, hist). */
typedef struct {
  builder *b;
  int ranks, cap;
  int c1, c2;
  int32_t *iset_of; /* [hist * ranks + card] */
  int nhist_cap;
  int hist_counter;
  int fail;
} tiny_ctx;

/* contributions: each player put ante 1 plus `put[i]` bet units. */
static int64_t tiny_bet(tiny_ctx *t, int actor, int bets, int facing, int put1, int put2, int hist,
                        int *next_hist) {
  builder *b = t->b;
  const int card = actor == 0 ? t->c1 : t->c2;
  int nact = facing ? (bets < t->cap ? 3 : 2) : 2;
  int32_t *slot = &t->iset_of[hist * t->ranks + card];
  if (*slot < 0) {
    *slot = b_iset(b, actor, nact);
    if (*slot < 0) { t->fail = 1; return -1; }
    b->g->iset_feat[(int64_t)*slot * GG_NFEAT + 0] = actor;
    b->g->iset_feat[(int64_t)*slot * GG_NFEAT + 1] = card;
    b->g->iset_feat[(int64_t)*slot * GG_NFEAT + 5] = nact;
    b->g->iset_feat[(int64_t)*slot * GG_NFEAT + 6] = hist;
  }
  int64_t me = b_node(b, actor == 0 ? GG_P1 : GG_P2, *slot, 0.0, nact);
  if (me < 0) { t->fail = 1; return -1; }
  const int win = (t->c1 > t->c2) ? 1 : -1; /* player 1's showdown sign */
  for (int a = 0; a < nact; ++a) {
    int64_t ch;
    int h_child = (*next_hist)++;
    if (!facing) {
      if (a == 0) { /* check */
        if (actor == 1) { /* check-check: showdown for the antes */
          ch = b_node(b, GG_TERMINAL, -1, (double)win * 1.0, 0);
        } else {
          ch = tiny_bet(t, 1, bets, 0, put1, put2, h_child, next_hist);
        }
      } else { /* bet one unit */
        int p1 = put1, p2 = put2;
        if (actor == 0) p1 = bets + 1; else p2 = bets + 1;
        ch = tiny_bet(t, 1 - actor, bets + 1, 1, p1, p2, h_child, next_hist);
      }
    } else {
      if (a == 0) { /* fold: the folder loses its own contribution */
        double own = 1.0 + (actor == 0 ? put1 : put2);
        ch = b_node(b, GG_TERMINAL, -1, actor == 0 ? -own : own, 0);
      } else if (a == 1) { /* call: showdown for ante + bets matched */
        ch = b_node(b, GG_TERMINAL, -1, (double)win * (1.0 + bets), 0);
      } else { /* raise one unit over the current bet */
        int p1 = put1, p2 = put2;
        if (actor == 0) p1 = bets + 1; else p2 = bets + 1;
        ch = tiny_bet(t, 1 - actor, bets + 1, 1, p1, p2, h_child, next_hist);
      }
    }
    if (ch < 0) { t->fail = 1; return -1; }
    b->g->child[b->g->child_begin[me] + a] = (int32_t)ch;
  }
  return me;
}

gg_spec *gg_tiny_card(int ranks, int cap) {
  if (ranks < 2 || ranks > 64 || cap < 1 || cap > 8) {
    set_err("gg_tiny_card: need 2 <= ranks <= 64 and 1 <= cap <= 8");
    return NULL;
  }
  builder b;
  if (!b_init(&b)) { set_err("out of host memory"); return NULL; }
  const int ndeal = ranks * (ranks - 1);
  tiny_ctx t;
  memset(&t, 0, sizeof t);
  t.b = &b; t.ranks = ranks; t.cap = cap;
  t.nhist_cap = 4096;
  t.iset_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)t.nhist_cap * (size_t)ranks);
  if (!t.iset_of) { gg_free(b_finish(&b)); set_err("out of host memory"); return NULL; }
  for (int i = 0; i < t.nhist_cap * ranks; ++i) t.iset_of[i] = -1;
  int64_t root = b_node(&b, GG_CHANCE, -1, 0.0, ndeal);
  int k = 0;
  for (int c1 = 0; c1 < ranks; ++c1)
    for (int c2 = 0; c2 < ranks; ++c2) {
      if (c1 == c2) continue;
      t.c1 = c1; t.c2 = c2;
      int next_hist = 1; /* history ids are the betting-tree preorder, equal for every deal */
      int64_t ch = tiny_bet(&t, 0, 0, 0, 0, 0, 0, &next_hist);
      if (t.fail || ch < 0 || next_hist > t.nhist_cap) {
        free(t.iset_of); gg_free(b_finish(&b));
        set_err("gg_tiny_card: generation failed (history table or memory)");
        return NULL;
      }
      b.g->child[b.g->child_begin[root] + k] = (int32_t)ch;
      b.g->chance_prob[b.g->child_begin[root] + k] = 1.0 / (double)ndeal;
      ++k;
    }
  free(t.iset_of);
  gg_spec *g = b_finish(&b);
  g->pot = 2.0;
  return g;
}

/* ------------------------------------------------------ random trees ---- */
enum { RS_KIND = 1, RS_PLAYER, RS_HASH, RS_CHUNK, RS_NACT, RS_NCHANCE, RS_DIRICHLET, RS_PAYOFF };

typedef struct { int64_t key; uint64_t h; int32_t idx; int8_t player; } rt_item;
static int rt_cmp(const void *pa, const void *pb) {
  const rt_item *a = (const rt_item *)pa, *b = (const rt_item *)pb;
  if (a->player != b->player) return a->player < b->player ? -1 : 1;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->h != b->h) return a->h < b->h ? -1 : 1;
  return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

gg_spec *gg_random_tree(uint64_t seed, int depth, int bmin, int bmax, double p_chance, int max_group) {
  if (depth < 1 || depth > 24 || bmin < 1 || bmax < bmin || bmax > 16 || max_group < 1 ||
      p_chance < 0.0 || p_chance > 1.0) {
    set_err("gg_random_tree: bad parameters");
    return NULL;
  }
  /* grow level by level; node ids are breadth-first */
  int64_t ncap = 1024, n = 1, e = 0, ni = 0, nicap = 1024;
  int8_t *kind = (int8_t *)malloc((size_t)ncap);
  int32_t *iset = (int32_t *)malloc(4 * (size_t)ncap);
  double *pay = (double *)malloc(8 * (size_t)ncap);
  double *cprob = (double *)malloc(8 * (size_t)ncap); /* probability of the edge into node */
  int64_t *key1 = (int64_t *)malloc(8 * (size_t)ncap); /* last own slot of player 1 (-1 none) */
  int64_t *key2 = (int64_t *)malloc(8 * (size_t)ncap);
  int32_t *nch = (int32_t *)malloc(4 * (size_t)ncap);
  int8_t *ipl = (int8_t *)malloc((size_t)nicap);
  int32_t *ina = (int32_t *)malloc(4 * (size_t)nicap);
  int64_t *islot = (int64_t *)malloc(8 * (size_t)nicap);
  int64_t nslots = 0;
  int ok = kind && iset && pay && cprob && key1 && key2 && nch && ipl && ina && islot;
  if (ok) { key1[0] = -1; key2[0] = -1; cprob[0] = 0.0; }
  int64_t lo = 0, hi = 1;
  rt_item *items = NULL;
  for (int d = 0; ok && d < depth; ++d) {
    const int leaf = (d == depth - 1);
    int64_t m = hi - lo;
    items = (rt_item *)realloc(items, sizeof(rt_item) * (size_t)(m > 0 ? m : 1));
    if (!items) { ok = 0; break; }
    int64_t np = 0;
    for (int64_t v = lo; v < hi; ++v) {
      pay[v] = 0.0;
      iset[v] = -1;
      nch[v] = 0;
      if (leaf) {
        kind[v] = GG_TERMINAL;
        pay[v] = 2.0 * u01(gg_rand(seed, RS_PAYOFF, (uint64_t)v)) - 1.0;
        continue;
      }
      if (u01(gg_rand(seed, RS_KIND, (uint64_t)v)) < p_chance) {
        kind[v] = GG_CHANCE;
        nch[v] = bmin + (int)(gg_rand(seed, RS_NCHANCE, (uint64_t)v) % (uint64_t)(bmax - bmin + 1));
      } else {
        int p = (int)(gg_rand(seed, RS_PLAYER, (uint64_t)v) & 1);
        kind[v] = (int8_t)(p == 0 ? GG_P1 : GG_P2);
        items[np].player = (int8_t)p;
        items[np].key = p == 0 ? key1[v] : key2[v];
        items[np].h = gg_rand(seed, RS_HASH, (uint64_t)v);
        items[np].idx = (int32_t)(v - lo);
        ++np;
      }
    }
    /* group player nodes by (player, own sequence), order by a seeded hash,
     * cut into chunks of 1..max_group members, one information set each */
    qsort(items, (size_t)np, sizeof(rt_item), rt_cmp);
    for (int64_t s = 0; s < np;) {
      int64_t t = s;
      while (t < np && items[t].player == items[s].player && items[t].key == items[s].key) ++t;
      for (int64_t c = s; c < t;) {
        int64_t sz = 1 + (int64_t)(gg_rand(seed, RS_CHUNK, (uint64_t)ni) % (uint64_t)max_group);
        if (c + sz > t) sz = t - c;
        if (ni + 1 > nicap) {
          nicap *= 2;
          ipl = (int8_t *)realloc(ipl, (size_t)nicap);
          ina = (int32_t *)realloc(ina, 4 * (size_t)nicap);
          islot = (int64_t *)realloc(islot, 8 * (size_t)nicap);
          if (!ipl || !ina || !islot) { ok = 0; break; }
        }
        ipl[ni] = items[s].player;
        ina[ni] = bmin + (int)(gg_rand(seed, RS_NACT, (uint64_t)ni) % (uint64_t)(bmax - bmin + 1));
        islot[ni] = nslots;
        nslots += ina[ni];
        for (int64_t q = c; q < c + sz; ++q) {
          int64_t v = lo + items[q].idx;
          iset[v] = (int32_t)ni;
          nch[v] = ina[ni];
        }
        ++ni;
        c += sz;
      }
      if (!ok) break;
      s = t;
    }
    if (!ok || leaf) break;
    /* children, breadth-first */
    int64_t total = 0;
    for (int64_t v = lo; v < hi; ++v) total += nch[v];
    if (hi + total > ncap) {
      while (hi + total > ncap) ncap *= 2;
      kind = (int8_t *)realloc(kind, (size_t)ncap);
      iset = (int32_t *)realloc(iset, 4 * (size_t)ncap);
      pay = (double *)realloc(pay, 8 * (size_t)ncap);
      cprob = (double *)realloc(cprob, 8 * (size_t)ncap);
      key1 = (int64_t *)realloc(key1, 8 * (size_t)ncap);
      key2 = (int64_t *)realloc(key2, 8 * (size_t)ncap);
      nch = (int32_t *)realloc(nch, 4 * (size_t)ncap);
      if (!kind || !iset || !pay || !cprob || !key1 || !key2 || !nch) { ok = 0; break; }
    }
    int64_t c = hi;
    for (int64_t v = lo; v < hi; ++v) {
      double esum = 0.0;
      for (int a = 0; a < nch[v]; ++a, ++c) {
        key1[c] = key1[v];
        key2[c] = key2[v];
        cprob[c] = 0.0;
        if (kind[v] == GG_CHANCE) {
          double ex = -log(u01_open(gg_rand(seed, RS_DIRICHLET, (uint64_t)c)));
          cprob[c] = ex;
          esum += ex;
        } else if (kind[v] == GG_P1) {
          key1[c] = islot[iset[v]] + a;
        } else {
          key2[c] = islot[iset[v]] + a;
        }
      }
      if (kind[v] == GG_CHANCE)
        for (int64_t q = c - nch[v]; q < c; ++q) cprob[q] /= esum;
    }
    n = hi + total;
    lo = hi;
    hi = n;
    (void)e;
  }
  free(items);
  if (!ok) {
    free(kind); free(iset); free(pay); free(cprob); free(key1); free(key2); free(nch);
    free(ipl); free(ina); free(islot);
    set_err("gg_random_tree: out of host memory");
    return NULL;
  }
  gg_spec *g = (gg_spec *)calloc(1, sizeof(gg_spec));
  g->n_nodes = n;
  g->n_edges = n - 1;
  g->n_infosets = ni;
  g->kind = kind;
  g->infoset = iset;
  g->payoff = pay;
  g->iset_player = ipl;
  g->iset_nact = ina;
  g->iset_feat = NULL;
  g->child_begin = (int64_t *)malloc(8 * (size_t)(n + 1));
  g->child = (int32_t *)malloc(4 * (size_t)(n > 1 ? n - 1 : 1));
  g->chance_prob = (double *)malloc(8 * (size_t)(n > 1 ? n - 1 : 1));
  if (!g->child_begin || !g->child || !g->chance_prob) {
    free(key1); free(key2); free(nch); free(islot); free(cprob);
    gg_free(g);
    set_err("gg_random_tree: out of host memory");
    return NULL;
  }
  int64_t cur = 0;
  for (int64_t v = 0; v < n; ++v) { g->child_begin[v] = cur; cur += nch[v]; }
  g->child_begin[n] = cur;
  for (int64_t q = 0; q + 1 < n; ++q) { g->child[q] = (int32_t)(q + 1); g->chance_prob[q] = cprob[q + 1]; }
  free(key1); free(key2); free(nch); free(islot); free(cprob);
  g->pot = 1.0;
  return g;
}


/* --------------------------------------------- card games (public trees) ---- */
/* Three-card showdown value: trips > pair > high card, kickers lexicographic,
 * suits ignored. Larger is better. */
static int rank3(int r0, int r1, int r2) {
  int a = r0, b = r1, c = r2, t;
  if (a < b) { t = a; a = b; b = t; }
  if (b < c) { t = b; b = c; c = t; }
  if (a < b) { t = a; a = b; b = t; }
  if (a == c) return 2 * 4096 + a;
  if (a == b) return 1 * 4096 + a * 64 + c;
  if (b == c) return 1 * 4096 + b * 64 + a;
  return a * 256 + b * 16 + c;
}

/* A node of the public (betting + board) tree that every deal shares. */
typedef struct {
  int8_t kind;      /* GG_*; a chance node deals the board card */
  int8_t term;      /* terminal: 0 player 1 folded, 1 player 2 folded, 2 showdown */
  int8_t round;     /* 0 or 1 */
  int8_t nch;
  int8_t nhist;
  int8_t hist[8];   /* action codes of the current round: 0 check, 2 call, 3+i i-th bet size */
  int32_t kid0;     /* offset into kids[] */
  int32_t level;    /* depth below the deal node (0 = first decision) */
  int32_t pos;      /* breadth-first index within its level */
  int32_t bet_id;   /* betting state, equal for every board outcome */
  int32_t oidx;     /* board outcome index, -1 before the board */
  double c1, c2;    /* contributions (ante included) */
} pnode;

typedef struct {
  pnode *p;
  int64_t n, cap;
  int32_t *kids;
  int64_t nk, kcap;
  double maxc;      /* 1 + stack */
  int cap_bets;
  int n_out;        /* board outcomes (0: single round, showdown at round end) */
  const double *fr; /* bet fractions */
  int nfr;
  int fail;
} ptree;

static int32_t pt_new(ptree *t, int kind, int nch) {
  if (!grow((void **)&t->p, sizeof(pnode), &t->cap, t->n + 1)) { t->fail = 1; return -1; }
  if (!grow((void **)&t->kids, 4, &t->kcap, t->nk + nch)) { t->fail = 1; return -1; }
  pnode *P = &t->p[t->n];
  memset(P, 0, sizeof *P);
  P->kind = (int8_t)kind;
  P->nch = (int8_t)nch;
  P->kid0 = (int32_t)t->nk;
  P->oidx = -1;
  P->bet_id = -1;
  for (int i = 0; i < 8; ++i) P->hist[i] = -1;
  t->nk += nch;
  return (int32_t)t->n++;
}

static int dbl_cmp(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return x < y ? -1 : x > y;
}

static int32_t pt_bet(ptree *t, int round, double c1, double c2, int actor, int bets, int nchecks,
                      int oidx, const int8_t *hist, int nhist, int32_t *seq);

/* End of a betting round with both contributions equal. */
static int32_t pt_round_end(ptree *t, int round, double c1, double c2, int oidx, int32_t *seq) {
  if (round == 0 && t->n_out > 0) {
    int32_t me = pt_new(t, GG_CHANCE, t->n_out);
    if (me < 0) return -1;
    t->p[me].round = 0; t->p[me].c1 = c1; t->p[me].c2 = c2; t->p[me].bet_id = (*seq)++;
    const int allin = (c1 >= t->maxc || c2 >= t->maxc);
    const int32_t seq0 = *seq;
    int32_t seq_end = seq0;
    for (int o = 0; o < t->n_out; ++o) {
      int32_t s = seq0; /* every board outcome replays the same bet ids */
      int32_t ch;
      if (allin) {
        ch = pt_new(t, GG_TERMINAL, 0);
        if (ch < 0) return -1;
        t->p[ch].term = 2; t->p[ch].round = 1; t->p[ch].c1 = c1; t->p[ch].c2 = c2;
        t->p[ch].oidx = o; t->p[ch].bet_id = s++;
      } else {
        ch = pt_bet(t, 1, c1, c2, 0, 0, 0, o, NULL, 0, &s);
        if (ch < 0) return -1;
      }
      t->kids[t->p[me].kid0 + o] = ch;
      seq_end = s;
    }
    *seq = seq_end;
    return me;
  }
  int32_t me = pt_new(t, GG_TERMINAL, 0);
  if (me < 0) return -1;
  t->p[me].term = 2; t->p[me].round = (int8_t)round; t->p[me].c1 = c1; t->p[me].c2 = c2;
  t->p[me].oidx = oidx; t->p[me].bet_id = (*seq)++;
  return me;
}

static int32_t pt_bet(ptree *t, int round, double c1, double c2, int actor, int bets, int nchecks,
                      int oidx, const int8_t *hist, int nhist, int32_t *seq) {
  const double cme = actor == 0 ? c1 : c2, cop = actor == 0 ? c2 : c1;
  const double to_call = cop - cme;
  /* actions: check | fold, call; then bet/raise sizes ascending, all-in last */
  int code[24];
  double amt[24];
  int na = 0;
  if (to_call > 0) { code[na] = 1; amt[na++] = 0; code[na] = 2; amt[na++] = 0; }
  else { code[na] = 0; amt[na++] = 0; }
  if (bets < t->cap_bets && t->maxc > cop) {
    double cand[20];
    int nc = 0;
    const double potc = 2.0 * cop; /* pot once the actor has called */
    for (int f = 0; f < t->nfr && nc < 19; ++f) {
      double x = cop + t->fr[f] * potc;
      if (x < t->maxc && x > cop) cand[nc++] = x;
    }
    cand[nc++] = t->maxc;
    qsort(cand, (size_t)nc, sizeof(double), dbl_cmp);
    int k = 0;
    for (int i = 0; i < nc; ++i) {
      if (i > 0 && cand[i] == cand[i - 1]) continue;
      code[na] = 3 + k++;
      amt[na++] = cand[i];
    }
  }
  int32_t me = pt_new(t, actor == 0 ? GG_P1 : GG_P2, na);
  if (me < 0) return -1;
  {
    pnode *P = &t->p[me];
    P->round = (int8_t)round; P->c1 = c1; P->c2 = c2; P->oidx = oidx; P->bet_id = (*seq)++;
    P->nhist = (int8_t)(nhist < 8 ? nhist : 8);
    for (int i = 0; i < P->nhist; ++i) P->hist[i] = hist[i];
  }
  for (int a = 0; a < na; ++a) {
    int8_t h2[8];
    int nh2 = nhist < 8 ? nhist + 1 : 8;
    for (int i = 0; i < 8; ++i) h2[i] = (hist && i < nhist) ? hist[i] : -1;
    if (nhist < 8) h2[nhist] = (int8_t)code[a];
    int32_t ch;
    if (code[a] == 0) { /* check */
      if (nchecks == 1) ch = pt_round_end(t, round, c1, c2, oidx, seq);
      else ch = pt_bet(t, round, c1, c2, 1 - actor, bets, 1, oidx, h2, nh2, seq);
    } else if (code[a] == 1) { /* fold */
      ch = pt_new(t, GG_TERMINAL, 0);
      if (ch < 0) return -1;
      t->p[ch].term = (int8_t)actor; t->p[ch].round = (int8_t)round;
      t->p[ch].c1 = c1; t->p[ch].c2 = c2; t->p[ch].oidx = oidx; t->p[ch].bet_id = (*seq)++;
    } else if (code[a] == 2) { /* call */
      ch = pt_round_end(t, round, actor == 0 ? cop : c1, actor == 0 ? c2 : cop, oidx, seq);
    } else { /* bet or raise to amt[a] */
      ch = pt_bet(t, round, actor == 0 ? amt[a] : c1, actor == 0 ? c2 : amt[a], 1 - actor,
                  bets + 1, 0, oidx, h2, nh2, seq);
    }
    if (ch < 0) return -1;
    t->kids[t->p[me].kid0 + a] = ch;
  }
  return me;
}

/* Breadth-first levels of the public tree: fills level/pos and returns the
 * public node ids per level (order[level_off[l] .. level_off[l+1])). */
static int pt_levels(ptree *t, int32_t **order_out, int64_t **level_off_out, int *nlev_out) {
  int32_t *order = (int32_t *)malloc(4 * (size_t)t->n);
  int64_t *loff = (int64_t *)malloc(8 * (size_t)(t->n + 2));
  if (!order || !loff) { free(order); free(loff); return 0; }
  int64_t head = 0, tail = 0;
  order[tail++] = 0;
  t->p[0].level = 0;
  int nlev = 0;
  loff[0] = 0;
  int cur = 0;
  while (head < tail) {
    int32_t v = order[head];
    if (t->p[v].level != cur) { loff[++nlev] = head; cur = t->p[v].level; }
    t->p[v].pos = (int32_t)(head - loff[nlev]);
    ++head;
    for (int a = 0; a < t->p[v].nch; ++a) {
      int32_t c = t->kids[t->p[v].kid0 + a];
      t->p[c].level = t->p[v].level + 1;
      order[tail++] = c;
    }
  }
  loff[++nlev] = head;
  *order_out = order;
  *level_off_out = loff;
  *nlev_out = nlev;
  return 1;
}

/* Builds the full game: a chance root over `ndeal` deals (probabilities
 * deal_p), each followed by a copy of the public tree. Node ids are
 * breadth-first: level L >= 1 holds deal-major blocks of the public level
 * L-1. Information sets: one block per (player, bet state) of size
 * n_priv(round) where the private index comes from priv_of(deal, player,
 * board outcome). */
typedef struct {
  int ncards, nranks, nsuits;
  int nhands;
  int hand_a[2048], hand_b[2048];
  int64_t ndeal;
  int32_t *deal_h1, *deal_h2;   /* hand index per deal (into hand_a/b) */
  double *deal_p;
  int board_fixed;              /* single-round games: the fixed board card */
  int32_t *pair_idx;            /* [hand * ncards + card] compact (hand, board) id or -1 */
  int npairs;
  int npriv_p[2];               /* private states per player before the board */
  int32_t priv_of_hand[2048];   /* hand index -> position in its player's list */
  int32_t hand_of_priv[2][2048];
} deck_ctx;

static int card_rank(const deck_ctx *d, int c) { return c / d->nsuits; }

static int deal_board(const deck_ctx *d, int64_t k, int o) {
  if (o < 0) return d->board_fixed;
  const int a1 = d->hand_a[d->deal_h1[k]], b1 = d->hand_b[d->deal_h1[k]];
  const int a2 = d->hand_a[d->deal_h2[k]], b2 = d->hand_b[d->deal_h2[k]];
  int seen = 0;
  for (int c = 0; c < d->ncards; ++c) {
    if (c == a1 || c == b1 || c == a2 || c == b2) continue;
    if (seen == o) return c;
    ++seen;
  }
  return -1;
}

static gg_spec *build_card_game(ptree *t, deck_ctx *d, double pot, int with_board_chance) {
  int32_t *order = NULL;
  int64_t *loff = NULL;
  int nlev = 0;
  if (!pt_levels(t, &order, &loff, &nlev)) { set_err("out of host memory"); return NULL; }
  /* bet ids -> infoset block bases */
  int32_t nbet = 0;
  for (int64_t v = 0; v < t->n; ++v) if (t->p[v].bet_id + 1 > nbet) nbet = t->p[v].bet_id + 1;
  int64_t *base = (int64_t *)malloc(8 * (size_t)(nbet > 0 ? nbet : 1));
  int32_t *rep = (int32_t *)malloc(4 * (size_t)(nbet > 0 ? nbet : 1));
  if (!base || !rep) { free(order); free(loff); free(base); free(rep); set_err("out of host memory"); return NULL; }
  for (int32_t b = 0; b < nbet; ++b) { base[b] = -1; rep[b] = -1; }
  int64_t ni = 0;
  for (int64_t q = 0; q < t->n; ++q) { /* preorder of public ids */
    const pnode *P = &t->p[q];
    if (P->kind != GG_P1 && P->kind != GG_P2) continue;
    if (base[P->bet_id] >= 0) continue;
    base[P->bet_id] = ni;
    rep[P->bet_id] = (int32_t)q;
    const int pl = P->kind == GG_P1 ? 0 : 1;
    const int npriv = (P->round == 1 && with_board_chance) ? d->npairs : d->npriv_p[pl];
    ni += npriv;
  }
  /* node counts */
  int64_t N = 1;
  for (int l = 0; l < nlev; ++l) N += d->ndeal * (loff[l + 1] - loff[l]);
  if (N >= (int64_t)2147483647) { free(order); free(loff); free(base); free(rep); set_err("game too large for 32-bit node ids"); return NULL; }
  gg_spec *g = spec_alloc(N, N - 1, ni, 1);
  if (!g) { free(order); free(loff); free(base); free(rep); return NULL; }
  /* information-set metadata; compact (hand, board) ids decoded by table */
  int32_t *pair_hand = NULL, *pair_card = NULL;
  if (with_board_chance) {
    pair_hand = (int32_t *)malloc(4 * (size_t)(d->npairs > 0 ? d->npairs : 1));
    pair_card = (int32_t *)malloc(4 * (size_t)(d->npairs > 0 ? d->npairs : 1));
    if (!pair_hand || !pair_card) {
      free(pair_hand); free(pair_card); free(order); free(loff); free(base); free(rep); gg_free(g);
      set_err("out of host memory");
      return NULL;
    }
    for (int hh = 0; hh < d->nhands; ++hh)
      for (int c = 0; c < d->ncards; ++c) {
        const int32_t j = d->pair_idx[hh * d->ncards + c];
        if (j >= 0) { pair_hand[j] = hh; pair_card[j] = c; }
      }
  }
  for (int32_t b = 0; b < nbet; ++b) {
    if (base[b] < 0) continue;
    const pnode *P = &t->p[rep[b]];
    const int pl = P->kind == GG_P1 ? 0 : 1;
    const int npriv = (P->round == 1 && with_board_chance) ? d->npairs : d->npriv_p[pl];
    for (int j = 0; j < npriv; ++j) {
      const int64_t I = base[b] + j;
      g->iset_player[I] = (int8_t)(P->kind == GG_P1 ? 0 : 1);
      g->iset_nact[I] = P->nch;
      int32_t *f = &g->iset_feat[I * GG_NFEAT];
      int h, board = d->board_fixed;
      if (P->round == 1 && with_board_chance) { /* decode the compact (hand, board) id */
        h = pair_hand[j];
        board = pair_card[j];
      } else {
        h = d->hand_of_priv[pl][j];
      }
      f[0] = P->kind == GG_P1 ? 0 : 1;
      f[1] = d->hand_a[h];
      f[2] = d->hand_b[h];
      f[3] = board;
      f[4] = P->round;
      f[5] = P->nch;
      for (int i = 0; i < 8; ++i) f[6 + i] = P->hist[i];
      f[14] = (int32_t)(P->c1 * 2.0 + 0.5);
      f[15] = (int32_t)(P->c2 * 2.0 + 0.5);
    }
  }
  /* root */
  int64_t cur_child = 0;
  g->kind[0] = GG_CHANCE; g->infoset[0] = -1; g->payoff[0] = 0.0;
  g->child_begin[0] = 0;
  for (int64_t k = 0; k < d->ndeal; ++k) { g->child[k] = (int32_t)(1 + k); g->chance_prob[k] = d->deal_p[k]; }
  cur_child = d->ndeal;
  int64_t id = 1;
  int64_t next_level_base = 1 + d->ndeal * (loff[1] - loff[0]);
  for (int l = 0; l < nlev; ++l) {
    const int64_t H = loff[l + 1] - loff[l];
    const int64_t Hn = (l + 1 < nlev) ? loff[l + 2] - loff[l + 1] : 0;
    for (int64_t k = 0; k < d->ndeal; ++k) {
      const int h1 = d->deal_h1[k], h2 = d->deal_h2[k];
      for (int64_t j = 0; j < H; ++j, ++id) {
        const pnode *P = &t->p[order[loff[l] + j]];
        g->kind[id] = P->kind;
        g->infoset[id] = -1;
        g->payoff[id] = 0.0;
        g->child_begin[id] = cur_child;
        if (P->kind == GG_TERMINAL) {
          double u;
          if (P->term == 0) u = -P->c1;
          else if (P->term == 1) u = P->c2;
          else {
            const int bc = deal_board(d, k, P->oidx);
            const int s1 = rank3(card_rank(d, d->hand_a[h1]), card_rank(d, d->hand_b[h1]), card_rank(d, bc));
            const int s2 = rank3(card_rank(d, d->hand_a[h2]), card_rank(d, d->hand_b[h2]), card_rank(d, bc));
            u = s1 > s2 ? P->c2 : (s1 < s2 ? -P->c1 : 0.0);
          }
          g->payoff[id] = u;
          continue;
        }
        /* children: consecutive ids in the next level, deal-major */
        const int64_t first = next_level_base + k * Hn + t->p[t->kids[P->kid0]].pos;
        for (int a = 0; a < P->nch; ++a) {
          g->child[cur_child + a] = (int32_t)(first + a);
          g->chance_prob[cur_child + a] = P->kind == GG_CHANCE ? 1.0 / (double)t->n_out : 0.0;
        }
        cur_child += P->nch;
        if (P->kind == GG_P1 || P->kind == GG_P2) {
          const int hand = P->kind == GG_P1 ? h1 : h2;
          int64_t j2 = d->priv_of_hand[hand];
          if (P->round == 1 && with_board_chance)
            j2 = d->pair_idx[hand * d->ncards + deal_board(d, k, P->oidx)];
          g->infoset[id] = (int32_t)(base[P->bet_id] + j2);
        }
      }
    }
    next_level_base += d->ndeal * Hn;
  }
  g->child_begin[N] = cur_child;
  free(order); free(loff); free(base); free(rep); free(pair_hand); free(pair_card);
  g->pot = pot;
  /* a subsample of the deals can leave information sets without members:
   * drop them and renumber the rest in order */
  {
    int32_t *remap = (int32_t *)malloc(4 * (size_t)(ni > 0 ? ni : 1));
    if (!remap) { gg_free(g); set_err("out of host memory"); return NULL; }
    for (int64_t i = 0; i < ni; ++i) remap[i] = -1;
    for (int64_t v = 0; v < N; ++v) if (g->infoset[v] >= 0) remap[g->infoset[v]] = 0;
    int64_t m = 0;
    for (int64_t i = 0; i < ni; ++i) {
      if (remap[i] < 0) continue;
      remap[i] = (int32_t)m;
      g->iset_player[m] = g->iset_player[i];
      g->iset_nact[m] = g->iset_nact[i];
      for (int f = 0; f < GG_NFEAT; ++f) g->iset_feat[m * GG_NFEAT + f] = g->iset_feat[i * GG_NFEAT + f];
      ++m;
    }
    if (m != ni) {
      for (int64_t v = 0; v < N; ++v) if (g->infoset[v] >= 0) g->infoset[v] = remap[g->infoset[v]];
      g->n_infosets = m;
    }
    free(remap);
  }
  return g;
}

static void deck_init(deck_ctx *d, int nranks, int nsuits) {
  memset(d, 0, sizeof *d);
  d->nranks = nranks; d->nsuits = nsuits; d->ncards = nranks * nsuits;
  d->board_fixed = -1;
}

static void deck_free(deck_ctx *d) {
  free(d->deal_h1); free(d->deal_h2); free(d->deal_p); free(d->pair_idx);
}

gg_spec *gg_large_card(int n_ranks, int n_suits, int stack, int cap) {
  return gg_large_card_sampled(n_ranks, n_suits, stack, cap, 1);
}

gg_spec *gg_large_card_sampled(int n_ranks, int n_suits, int stack, int cap, int deal_stride) {
  if (deal_stride < 1 || n_ranks < 1 || n_suits < 1 || n_ranks * n_suits < 5 || n_ranks * n_suits > 64 || stack < 1 ||
      stack > 1000 || cap < 1 || cap > 8) {
    set_err("gg_large_card: bad parameters");
    return NULL;
  }
  deck_ctx d;
  deck_init(&d, n_ranks, n_suits);
  for (int a = 0; a < d.ncards; ++a)
    for (int b = a + 1; b < d.ncards; ++b) { d.hand_a[d.nhands] = a; d.hand_b[d.nhands] = b; ++d.nhands; }
  const int64_t per = (int64_t)(d.ncards - 2) * (d.ncards - 3) / 2;
  d.ndeal = (int64_t)d.nhands * per;
  d.deal_h1 = (int32_t *)malloc(4 * (size_t)d.ndeal);
  d.deal_h2 = (int32_t *)malloc(4 * (size_t)d.ndeal);
  d.deal_p = (double *)malloc(8 * (size_t)d.ndeal);
  d.pair_idx = (int32_t *)malloc(4 * (size_t)d.nhands * (size_t)d.ncards);
  if (!d.deal_h1 || !d.deal_h2 || !d.deal_p || !d.pair_idx) { deck_free(&d); set_err("out of host memory"); return NULL; }
  int64_t k = 0;
  for (int h1 = 0; h1 < d.nhands; ++h1)
    for (int h2 = 0; h2 < d.nhands; ++h2) {
      if (d.hand_a[h2] == d.hand_a[h1] || d.hand_a[h2] == d.hand_b[h1] || d.hand_b[h2] == d.hand_a[h1] ||
          d.hand_b[h2] == d.hand_b[h1])
        continue;
      d.deal_h1[k] = h1; d.deal_h2[k] = h2; d.deal_p[k] = 1.0 / (double)d.ndeal; ++k;
    }
  if (deal_stride > 1) { /* uniform subsample of the deals (every deal_stride-th) */
    int64_t m = 0;
    for (int64_t q = 0; q < d.ndeal; q += deal_stride) { d.deal_h1[m] = d.deal_h1[q]; d.deal_h2[m] = d.deal_h2[q]; ++m; }
    d.ndeal = m;
    for (int64_t q = 0; q < m; ++q) d.deal_p[q] = 1.0 / (double)m;
  }
  for (int h = 0; h < d.nhands; ++h)
    for (int c = 0; c < d.ncards; ++c) {
      int in = (c == d.hand_a[h] || c == d.hand_b[h]);
      d.pair_idx[h * d.ncards + c] = in ? -1 : d.npairs++;
    }
  d.npriv_p[0] = d.npriv_p[1] = d.nhands;
  for (int h = 0; h < d.nhands; ++h) { d.priv_of_hand[h] = h; d.hand_of_priv[0][h] = h; d.hand_of_priv[1][h] = h; }
  static const double fr[2] = {0.5, 1.0};
  ptree t;
  memset(&t, 0, sizeof t);
  t.maxc = 1.0 + stack; t.cap_bets = cap; t.n_out = d.ncards - 4; t.fr = fr; t.nfr = 2;
  int32_t seq = 0;
  pt_bet(&t, 0, 1.0, 1.0, 0, 0, 0, -1, NULL, 0, &seq);
  if (t.fail) { free(t.p); free(t.kids); deck_free(&d); set_err("out of host memory"); return NULL; }
  gg_spec *g = build_card_game(&t, &d, 2.0, 1);
  free(t.p); free(t.kids); deck_free(&d);
  return g;
}

/* size of one deal's betting tree for a single-round game */
static int64_t endgame_tree_size(const double *fr, int nfr, double maxc, int cap) {
  ptree t;
  memset(&t, 0, sizeof t);
  t.maxc = maxc; t.cap_bets = cap; t.n_out = 0; t.fr = fr; t.nfr = nfr;
  int32_t seq = 0;
  pt_bet(&t, 0, 1.0, 1.0, 0, 0, 0, -1, NULL, 0, &seq);
  int64_t n = t.fail ? -1 : t.n;
  free(t.p); free(t.kids);
  return n;
}

enum { ES_TARGET = 101, ES_MENU, ES_K, ES_BOARD, ES_HANDS, ES_RANGE };

gg_spec *gg_endgame(uint64_t seed, int64_t target_edges) {
  static const double menu[6] = {0.25, 0.5, 0.75, 1.0, 1.5, 2.0};
  if (target_edges <= 0) {
    /* log-uniform target in [1e3, 1e6] */
    double u = u01(gg_rand(seed, ES_TARGET, 0));
    target_edges = (int64_t)exp(log(1e3) + u * (log(1e6) - log(1e3)));
  }
  const double maxc = 1.0 + 8.0; /* stacks of 8 antes behind */
  const int cap = 2;
  double fr[4];
  int nfr = 2 + (int)(gg_rand(seed, ES_MENU, 0) % 3);
  { /* choose nfr distinct fractions from the menu */
    int used[6] = {0};
    for (int i = 0; i < nfr; ++i) {
      int j = (int)(gg_rand(seed, ES_MENU, 1 + (uint64_t)i) % 6);
      while (used[j]) j = (j + 1) % 6;
      used[j] = 1;
    }
    int m = 0;
    for (int j = 0; j < 6; ++j) if (used[j]) fr[m++] = menu[j];
  }
  const int64_t T = endgame_tree_size(fr, nfr, maxc, cap);
  if (T <= 0) { set_err("gg_endgame: out of host memory"); return NULL; }
  /* hands per player so that K1*K2*0.85*T ~ target */
  int K1 = 10 + (int)(gg_rand(seed, ES_K, 0) % 191);
  double k2f = (double)target_edges / ((double)T * (double)K1 * 0.85);
  if (k2f < 10.0) {
    K1 = (int)ceil((double)target_edges / ((double)T * 10.0 * 0.85));
    if (K1 < 10) K1 = 10;
    if (K1 > 200) K1 = 200;
    k2f = (double)target_edges / ((double)T * (double)K1 * 0.85);
  }
  int K2 = (int)(k2f + 0.5);
  if (K2 < 10) K2 = 10;
  if (K2 > 200) K2 = 200;
  deck_ctx d;
  deck_init(&d, 8, 4);
  d.board_fixed = (int)(gg_rand(seed, ES_BOARD, 0) % (uint64_t)d.ncards);
  /* all hands avoiding the board, then a seeded choice of K1 and K2 of them */
  int allA[512], allB[512], nall = 0;
  for (int a = 0; a < d.ncards; ++a)
    for (int b = a + 1; b < d.ncards; ++b)
      if (a != d.board_fixed && b != d.board_fixed) { allA[nall] = a; allB[nall] = b; ++nall; }
  int H1[200], H2[200];
  double r1[200], r2[200];
  for (int p = 0; p < 2; ++p) {
    int K = p == 0 ? K1 : K2;
    int *H = p == 0 ? H1 : H2;
    double *r = p == 0 ? r1 : r2;
    int idx[512];
    for (int i = 0; i < nall; ++i) idx[i] = i;
    for (int i = 0; i < K; ++i) { /* partial Fisher-Yates */
      int j = i + (int)(gg_rand(seed, ES_HANDS + 10 * (uint64_t)p, (uint64_t)i) % (uint64_t)(nall - i));
      int tmp = idx[i]; idx[i] = idx[j]; idx[j] = tmp;
    }
    /* sort the chosen hands by card order for a canonical layout */
    for (int i = 0; i < K; ++i)
      for (int j = i + 1; j < K; ++j)
        if (idx[j] < idx[i]) { int tmp = idx[i]; idx[i] = idx[j]; idx[j] = tmp; }
    double s = 0.0;
    for (int i = 0; i < K; ++i) {
      H[i] = idx[i];
      /* Dirichlet(0.5): Gamma(0.5) = 0.5 * chi^2_1 = 0.5 * z^2 */
      double u1 = u01_open(gg_rand(seed, ES_RANGE + 10 * (uint64_t)p, 2 * (uint64_t)i));
      double u2 = u01_open(gg_rand(seed, ES_RANGE + 10 * (uint64_t)p, 2 * (uint64_t)i + 1));
      double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
      r[i] = 0.5 * z * z + 1e-12;
      s += r[i];
    }
    for (int i = 0; i < K; ++i) r[i] /= s;
  }
  d.nhands = 0;
  for (int i = 0; i < K1; ++i) { d.hand_a[d.nhands] = allA[H1[i]]; d.hand_b[d.nhands] = allB[H1[i]]; ++d.nhands; }
  const int off2 = d.nhands;
  for (int i = 0; i < K2; ++i) { d.hand_a[d.nhands] = allA[H2[i]]; d.hand_b[d.nhands] = allB[H2[i]]; ++d.nhands; }
  d.npriv_p[0] = K1; d.npriv_p[1] = K2;
  for (int i = 0; i < K1; ++i) { d.priv_of_hand[i] = i; d.hand_of_priv[0][i] = i; }
  for (int i = 0; i < K2; ++i) { d.priv_of_hand[off2 + i] = i; d.hand_of_priv[1][i] = off2 + i; }
  d.ndeal = 0;
  d.deal_h1 = (int32_t *)malloc(4 * (size_t)K1 * (size_t)K2);
  d.deal_h2 = (int32_t *)malloc(4 * (size_t)K1 * (size_t)K2);
  d.deal_p = (double *)malloc(8 * (size_t)K1 * (size_t)K2);
  if (!d.deal_h1 || !d.deal_h2 || !d.deal_p) { deck_free(&d); set_err("out of host memory"); return NULL; }
  double ptot = 0.0;
  for (int i = 0; i < K1; ++i)
    for (int j = 0; j < K2; ++j) {
      const int a1 = d.hand_a[i], b1 = d.hand_b[i], a2 = d.hand_a[off2 + j], b2 = d.hand_b[off2 + j];
      if (a1 == a2 || a1 == b2 || b1 == a2 || b1 == b2) continue;
      d.deal_h1[d.ndeal] = i; d.deal_h2[d.ndeal] = off2 + j;
      d.deal_p[d.ndeal] = r1[i] * r2[j];
      ptot += d.deal_p[d.ndeal];
      ++d.ndeal;
    }
  if (d.ndeal == 0) { deck_free(&d); set_err("gg_endgame: no compatible deals"); return NULL; }
  for (int64_t k = 0; k < d.ndeal; ++k) d.deal_p[k] /= ptot;
  ptree t;
  memset(&t, 0, sizeof t);
  t.maxc = maxc; t.cap_bets = cap; t.n_out = 0; t.fr = fr; t.nfr = nfr;
  int32_t seq = 0;
  pt_bet(&t, 0, 1.0, 1.0, 0, 0, 0, -1, NULL, 0, &seq);
  if (t.fail) { free(t.p); free(t.kids); deck_free(&d); set_err("out of host memory"); return NULL; }
  gg_spec *g = build_card_game(&t, &d, 2.0, 0);
  free(t.p); free(t.kids); deck_free(&d);
  return g;
}
