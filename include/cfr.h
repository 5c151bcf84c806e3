/* cfr.h — C ABI of the GB300 CFR+ library (libcfr.so).
 *
 * One CFR+ iteration (simultaneous updates, regret matching+, linear
 * averaging) over a two-player zero-sum game compiled once into static flat
 * arrays (the paper's Section 4 and Algorithm 1): a depth-level forward pass
 * of both players' reach (dual-lane buffer, eq. (lanes)), terminal utilities
 * with chance folded in at compile time (eq. (template), Proposition 1), a
 * depth-level backward pass of counterfactual values as deterministic
 * segmented sums with no float atomics (eq. (opbwd)), and the per-information
 * -set regret update, regret matching and average accumulation (eqs.
 * (instregret), (regret), (rm), the CFR+ clamp).
 *
 * Conventions
 *  - Every function returns CFR_OK (0) or a negative CFR_ERR_* code and never
 *    throws or aborts; cfr_last_error() describes the last failure of the
 *    calling thread.
 *  - Device memory is owned by the caller: cfr_plan() reports the bytes one
 *    solver needs, the caller allocates them (e.g. a PyTorch uint8 tensor)
 *    and hands them to cfr_bind(). The library sub-allocates inside that
 *    arena and never frees it. The caller keeps it alive until cfr_destroy()
 *    or the next cfr_bind().
 *  - Streams are plain cudaStream_t values passed as void*; NULL means the
 *    legacy default stream. Kernels are enqueued asynchronously unless a
 *    function says it synchronises.
 *  - Host arrays passed in are read during the call only (the library copies
 *    what it keeps). Slot-indexed vectors use the spec's order: information
 *    set I owns slots off(I) .. off(I)+nact(I)-1, off = prefix sum of nact in
 *    information-set id order.
 */
#ifndef CFR_H
#define CFR_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CFR_OK = 0,
  CFR_ERR_ARG = -1,          /* null pointer, bad size or bad option */
  CFR_ERR_INVALID_SPEC = -2, /* the game fails a structural check (Algorithm "Compile", step 1) */
  CFR_ERR_NOT_BOUND = -3,    /* the call needs device memory: call cfr_bind first */
  CFR_ERR_REBOUND = -4,      /* reserved: cfr_bind drops a captured graph, so no call returns it */
  CFR_ERR_ARENA_SMALL = -5,  /* the arena is smaller than cfr_plan reported */
  CFR_ERR_TIMEOUT = -6,      /* a grid barrier of the persistent kernel gave up waiting */
  CFR_ERR_DEVICE = -7,       /* a CUDA call failed (message in cfr_last_error) */
  CFR_ERR_HOST_MEMORY = -8,  /* host allocation failed */
  CFR_ERR_UNSUPPORTED = -9   /* option not available for this game */
};

/* Node kinds of the input game. */
enum { CFR_TERMINAL = 0, CFR_CHANCE = 1, CFR_PLAYER1 = 2, CFR_PLAYER2 = 3 };

/* The input game in the paper's tabular form (Appendix H, "Input
 * representation"): node 0 is the root; children listed in action order.
 * All arrays are host memory owned by the caller. */
typedef struct cfr_game_spec {
  int64_t n_nodes;            /* N >= 1, N < 2^31 */
  int64_t n_infosets;         /* I >= 0 */
  const int8_t *kind;         /* [N] CFR_TERMINAL / CFR_CHANCE / CFR_PLAYER1 / CFR_PLAYER2 */
  const int32_t *infoset;     /* [N] acting player's information set (decision nodes), else -1 */
  const int64_t *child_begin; /* [N+1] offsets into child[]; child_begin[N] = number of edges */
  const int32_t *child;       /* [E] child ids in action order */
  const double *chance_prob;  /* [E] outcome probability below chance nodes (others ignored) */
  const double *payoff;       /* [N] payoff to player 1 at terminals (others ignored) */
  const int8_t *iset_player;  /* [I] 0 = player 1, 1 = player 2 */
  const int32_t *iset_nact;   /* [I] actions of each set, 1 .. 64 */
} cfr_game_spec;

enum { CFR_P64 = 0, CFR_P32 = 1 };
enum { CFR_EXEC_AUTO = 0, CFR_EXEC_LEVELS = 1, CFR_EXEC_GRAPH = 2, CFR_EXEC_PERSISTENT = 3 };
enum { CFR_RULE_CFR_PLUS = 0, CFR_RULE_CFR = 1, CFR_RULE_PCFR_PLUS = 2 };
enum { CFR_ORDER_SIMULTANEOUS = 0, CFR_ORDER_ALTERNATING = 1 };
enum { CFR_REACH_MEMBERS = 0, CFR_REACH_BFS = 1, CFR_REACH_SLOTS = 2 };
enum { CFR_TILES_AUTO = 0, CFR_TILES_OFF = 1, CFR_TILES_ON = 2 };
enum { CFR_OVERLAP_AUTO = 0, CFR_OVERLAP_OFF = 1, CFR_OVERLAP_ON = 2 };

typedef struct cfr_options {
  /* CFR_P64: every value in FP64 (the parity mode). CFR_P32: reach, values,
   * strategy and per-history terms in FP32; cumulative regret, average
   * strategy and best-response sums in FP64 (Proposition 4). */
  int precision;
  /* CFR_EXEC_LEVELS: per-level kernels launched eagerly; CFR_EXEC_GRAPH: the
   * same kernels captured once into a CUDA graph and replayed (Section 4.3);
   * CFR_EXEC_PERSISTENT: one kernel per cfr_iterate call with a grid-wide
   * barrier between depth levels; CFR_EXEC_AUTO picks by game size: the
   * persistent form up to 768 nodes in CFR_P32 and 350 in CFR_P64 (where
   * it was measured faster than graph replay), the graph form above. */
  int exec_form;
  /* Update rule (Section 3, update rules): CFR_RULE_CFR_PLUS (regret clamped
   * at zero, linear averaging w_t = t), CFR_RULE_CFR (no clamp, linear
   * averaging) or CFR_RULE_PCFR_PLUS (clamp; the next strategy matches
   * R + r, the iteration's instantaneous regret as the prediction; quadratic
   * averaging w_t = t^2). */
  int rule;
  int lanes_per_set;   /* 0 = by mean set size (see cfr_autotune); else 1, 2, 4, 8, 16 or 32 lanes per set,
                          or 256 = one thread block per set in the per-level kernels (sets of at most 8
                          actions; the persistent kernel then uses 32), or 512 = the streaming backward
                          (CFR_P32 in member order, sets of at most 8 actions): each depth's sets go in
                          chunks whose reach, child values, member slots, set descriptors, strategy,
                          regrets and averages are staged in shared memory by bulk asynchronous copies,
                          and its narrow chance nodes in chunks of their children's values (depths
                          where a group of sets exceeds one 48 KiB stage keep the default; the
                          form pays only for long sets, and cfr_autotune tries it where sets have at least
                          32 members on average) */
  int persistent_ctas; /* 0 = co-resident maximum; else a cap on the persistent grid */
  int64_t barrier_spin_limit; /* 0 = default; polls before a grid barrier reports CFR_ERR_TIMEOUT */
  /* CFR_ORDER_SIMULTANEOUS: both players' regrets from one strategy profile;
   * CFR_ORDER_ALTERNATING: each iteration is two half-iterations (forward and
   * backward pass each), the first updating player 1's sets, the second
   * player 2's with player 1's new strategy; each half accumulates only its
   * player's average (Section 3; Section 4.2 runs the body twice). */
  int order;
  /* Order of the internal nodes' reach (a layout choice; results are
   * bitwise the same). CFR_REACH_MEMBERS (default): depth by depth, the
   * members of the depth's information sets in set order, then the depth's
   * chance nodes; the backward pass reads each set's reach as one run and
   * needs no rank table, and the forward pass pulls (every internal node
   * reads its parent's reach). CFR_REACH_BFS: breadth-first, and
   * CFR_REACH_SLOTS: the order of the nodes' places in their parents' value
   * blocks, taken member by member (the value blocks themselves are
   * action-major, see cfr_export_array 19-20); in both a parent's
   * internal children have consecutive ranks and the forward pass pushes
   * (every parent writes its children's reach). */
  int reach_order;
  /* Member order only: tiles of kTileSets consecutive information sets of
   * equal size store their members' reach interleaved (member k of the
   * tile's set j at tile base + k * kTileSets + j), so that a run of
   * children in one set pulls from a compact block of parents when the
   * parents' sets are tiled the same way (the two players' views of the
   * same private-card pairs); lane groups at tiled depths take at most 8
   * lanes. CFR_TILES_AUTO (default): tile the depths with at least 8192
   * sets where tiles hold at least half the members; CFR_TILES_ON: every
   * depth where tiles hold at least half the members (small games served
   * in batches); CFR_TILES_OFF: none. */
  int member_tiles;
  /* CFR_OVERLAP_ON: the per-level kernels of an iteration are launched
   * with programmatic dependent launch: each kernel first waits for the
   * previous launch to complete (so every read sees every earlier write),
   * but its launch and block scheduling overlap the previous kernel's tail
   * (and the FP32 streaming backward copies its first inputs before that
   * wait). CFR_OVERLAP_OFF: plain stream order. CFR_OVERLAP_AUTO (default):
   * on in CFR_P32, off in CFR_P64 (measured on one GB300: the FP64 card
   * game takes 8.5 ms per iteration without it and 10.4 ms with it; FP32
   * gains 1-2%). Results are bitwise the same. */
  int launch_overlap;
  /* Graph form: iterations recorded into one CUDA graph (the paper's
   * alternative-execution table records 1, 10 and 100); 0 or 1 = one.
   * cfr_iterate(n) replays the k-iteration graph n / k times and a
   * one-iteration graph for the rest (both captured on first use); the
   * device counter makes the results bitwise those of one iteration per
   * graph. At most 1000. */
  int graph_iters;
} cfr_options;

typedef struct cfr_counts {
  int64_t n_nodes, n_edges, n_infosets, n_slots;
  int64_t n_internal, n_decision, n_chance, n_terminal;
  int64_t depth_blocks;       /* D: number of distinct parent depths (eq. (blocks)) */
  int64_t max_actions;
  int64_t algo_bytes_per_iter; /* algorithmic HBM bytes of one iteration: every array element the
                                  layout needs, touched once (the per-launch sums of cfr_level_bytes;
                                  twice that under alternating updates) */
  int64_t upload_bytes;       /* host-to-device bytes cfr_bind copies */
  int64_t iteration;          /* t: iterations completed since bind/reset */
  int exec_form;              /* resolved execution form */
  int lanes_per_set;          /* resolved lanes per information set */
  int64_t graph_kernels;      /* kernel nodes in the captured one-iteration graph (0 until captured) */
  int64_t graph_k_kernels;    /* kernel nodes in the captured graph_iters-iteration graph (0 until captured) */
} cfr_counts;

typedef struct cfr_handle cfr_handle;

/* Compiles the game (Algorithm "Compile", steps 1-8): validation,
 * breadth-first numbering (parent before child, siblings contiguous in action
 * order), depth blocks, chance folding into the values template, slot and
 * member index emission. Host only; no device memory is touched.
 * opt may be NULL (P32, AUTO, CFR+). On success *out owns the result. */
int cfr_compile(const cfr_game_spec *spec, const cfr_options *opt, cfr_handle **out);

/* Sizes of the compiled game in the paper's counts (Section 4.1 and
 * Algorithm "Compile", steps 2-5: nodes, edges, information sets, slots, and
 * D, the number of depth blocks of eq. (blocks)), the iteration counter t
 * (Section 4.3) and the resolved options. Host only; never fails on a valid
 * handle. */
int cfr_get_counts(const cfr_handle *h, cfr_counts *out);

/* The memory plan (Algorithm "Compile", step 8, and the memory-plan table
 * of Appendix H): the device bytes one solver needs, sized from the game's
 * counts and the precision: the compiled index arrays, the values template,
 * the per-iteration buffers (reach lanes, values, strategy), the FP64
 * accumulators (regrets, average-strategy sum) and the best-response
 * scratch, each 256-byte aligned. Host only. Unlike the paper, the plan is
 * binding, not an indicator: cfr_bind refuses a smaller arena. */
int cfr_plan(const cfr_handle *h, size_t *device_bytes);

/* Binds the caller's device arena (>= cfr_plan bytes, 256-byte aligned;
 * else CFR_ERR_ARENA_SMALL or CFR_ERR_ARG) and lays the memory plan out in it
 * (the buffers of the memory-plan table, Appendix H), uploads the compiled
 * arrays and the values template, and initialises the state (R = 0,
 * average = 0, uniform strategy, t = 0). Synchronises `stream`. Section 4.3
 * refuses to replay a captured graph whose buffers moved; here binding
 * again re-uploads and drops any captured graph, so the next cfr_iterate
 * captures against the new arena and a stale replay cannot happen. */
int cfr_bind(cfr_handle *h, void *device_arena, size_t bytes, void *stream);

/* Runs n iterations t+1 .. t+n of the compiled iteration (Algorithm 1:
 * forward reach, terminal values, backward values with the fused regret and
 * average update, regret matching), asynchronously on `stream`, in the
 * execution form the options chose: per-level launches, one CUDA graph of an
 * iteration replayed n times (Section 4.3; captured on the first call), or
 * one persistent kernel. The weight w_t of the average comes from a device
 * counter the iteration itself advances (Section 4.3), so n = 0 is a no-op
 * and split calls give bitwise the same state as one call. CFR_ERR_NOT_BOUND
 * before cfr_bind. If capturing the graph fails, the call warns once on
 * stderr and runs the same kernels in the same order as per-level launches
 * from then on (Section 4.3): the results are bitwise the same. */
int cfr_iterate(cfr_handle *h, int64_t n, void *stream);

/* Waits for `stream` (the synchronisation point of Section 4.3's
 * asynchronous replay) and reports a device-side failure of earlier calls:
 * CFR_ERR_TIMEOUT if a grid barrier of the persistent kernel gave up (the
 * state is then undefined until cfr_reset). */
int cfr_synchronize(cfr_handle *h, void *stream);

/* Average strategy (eq. (rm): the linear-weighted sum normalised per set,
 * uniform where it is zero), [A] doubles in spec slot order. out is a device
 * pointer if out_on_device, else host memory (then the call synchronises). */
int cfr_avg_strategy(cfr_handle *h, double *out, int out_on_device, void *stream);

/* Current strategy sigma^{t+1} (regret matching of the cumulative regret),
 * same layout and synchronisation rules as cfr_avg_strategy. */
int cfr_current_strategy(cfr_handle *h, double *out, int out_on_device, void *stream);

/* Exploitability of the average strategy, NashConv/2 by exact best response
 * (eq. (exploitability)), on the GPU with FP64 sums. out_br (optional, [3])
 * receives (br1, br2, u) in player-1 units: player 1's best-response value,
 * player 2's best-response value, and the value of the average profile.
 * Synchronises `stream`. */
int cfr_exploitability(cfr_handle *h, double *out_expl, double *out_br, void *stream);

/* reset() of Appendix H ("Mutable and immutable fields") and the lifecycle
 * table: zeroes regrets, averages and t and restores the uniform strategy, in
 * place; no buffer moves, so a captured graph stays valid and the next
 * cfr_iterate runs from iteration one. Asynchronous on `stream`.
 * CFR_ERR_NOT_BOUND before cfr_bind. */
int cfr_reset(cfr_handle *h, void *stream);

/* set_payoffs of Appendix H ("Mutable and immutable fields") and the
 * lifecycle table: rewrites the terminal payoffs (payoff[N] in spec node
 * order, host; finite at terminals, else CFR_ERR_ARG) into the values
 * template (eq. (template)) from the retained chance products; no
 * recompilation. Solver state is kept. Synchronises `stream`. */
int cfr_set_payoffs(cfr_handle *h, const double *payoff, void *stream);

/* Rewrites the root's chance distribution, the other input Appendix H
 * marks mutable without recompilation: prob[n] (host doubles, the root's
 * outcomes in the spec's order; n must equal the root's child count; each
 * finite and >= 0). The root must be a chance node (else
 * CFR_ERR_UNSUPPORTED). The chance products below the root are recomputed in
 * path order from the retained edge probabilities, so the template is
 * bitwise the one a fresh compile with these probabilities produces. Works
 * before cfr_bind (host only; bind uploads it); after bind it also rewrites
 * the device template and synchronises `stream`. Solver state (R, avg, t)
 * is kept: call cfr_reset to start a new solve. Ranges over private hands
 * compose into it: prob[k] = r1[hand1(k)] * r2[hand2(k)] / Z for a deal
 * root. */
int cfr_set_root_chance(cfr_handle *h, const double *prob, int64_t n, void *stream);

/* Copies the solver state out / in (the accumulators of the memory-plan
 * table and the iteration counter that Section 4.3 carries across split
 * solver calls), host arrays in spec slot order: R[A] and avg[A]
 * (un-normalised strategy sums) as doubles, and t. Both synchronise
 * `stream`; set_state recomputes the current strategy by regret matching
 * (eq. (rm)). Under
 * PCFR+ the prediction is not part of the state: cfr_set_state restarts it
 * at zero (the next strategy is regret matching of R alone). */
int cfr_get_state(cfr_handle *h, double *R, double *avg, int64_t *t, void *stream);
int cfr_set_state(cfr_handle *h, const double *R, const double *avg, int64_t t, void *stream);

/* Host copies of the compiled index arrays that index emission produced
 * (Algorithm "Compile", step 7, in this library's layout; Section 4.1), for
 * bit-exact checks against an independent flattener. Host only.
 * which: 0 child_begin[N+1], 1 node_slot[N], 2 level_begin[D+2],
 * 3 iset_slot[I+1], 4 iset_mem[I+1], 5 mem_node[N_dec], 6 chance_list
 * (chance nodes with at most 1024 children), 7 level_chance[D+1],
 * 8 level_iset[2D+1] (per level: player-1 sets then player-2 sets), 9 new id
 * of each spec node [N], 10 template values [N] (doubles, node order),
 * 11 spec slot of each compiled slot [A], 12 lanes per set of each depth (a
 * runtime choice), 13 int_slot, 14 int_mask (bit pattern), 15 int_cirank
 * [N_int each: the pushing forward's internal-node records; empty in
 * member order], 16 big_irank (empty in member order), 17 mem_irank
 * [N_dec], 18 level_int[D+1], 19 vslot[N] (value slot of each node; the
 * root's is N-1), 20 iset_vb[I] (first slot of the block holding set I's
 * members' children, action-major: child a of member k at iset_vb[I] +
 * a * M + k - first member, M members), 21 mem_vs[N_dec] (value slot of each member),
 * 22 ch_vb, 23 ch_nch, 24 ch_vs (per chance node of list 6: first child
 * slot, child count, own slot), 25 wide_vb, 26 wide_nch, 27 wide_vs (the
 * same for chance nodes with more than 1024 children), 28 template values
 * in value-slot order [N] (doubles), 29 int_edge[2 N_int] (member order:
 * per internal node in rank order, its parent's rank and the slot word of
 * its edge, -1 under a chance node; the root's pair is -1, -1), 30
 * iset_rank[2 I] (member order: rank of each set's first member and the
 * stride of its members' ranks, 4 inside a tile), 31 level_tiled[D],
 * 32 set descriptors of the streaming FP32 backward [8 I] (per set: first
 * slot, actions, first member, members, first child value slot, reach rank
 * of member 0, rank stride, flags: bits 0-2 the sets of the group it starts
 * (1, 4 for a tile, 0 inside one), bit 8 player 2), 33 its chunks [16 per
 * chunk: sets I0, I1, then the staged element ranges (start, count) of
 * reach ranks, child value slots, members and slots, widened to 16-byte
 * boundaries, then the kind (0 sets; 1 chance: I0, I1 are narrow chance
 * nodes, the ranges their children's value slots and their entries of the
 * chance arrays, reach and slot ranges 0); 5 unused; each depth's set
 * chunks come first], 34 first chunk of each depth [D+1], 35 per depth
 * whether it can stream [D] (all empty unless FP32 in member order with sets
 * of at most 8 actions), 36 blocks of each depth's pulling forward launch
 * [D] (member order: one wave, the blocks all SMs hold at once, or fewer
 * where the depth needs fewer; set by cfr_bind; 0 before the first bind and
 * for the deepest depth).
 * Integer arrays are int32. *count receives the element count; out may be
 * NULL to query it. */
int cfr_export_array(const cfr_handle *h, int which, void *out, int64_t capacity, int64_t *count);

/* Autotuner for the thread-to-work mapping: for every depth it times the
 * backward launch with each supported number of lanes per information set
 * (1, 2, 4, 8, 16, 32, and 256 = one block per set when sets have at most 8
 * actions, and 512 = the streaming backward at depths that can stream;
 * `reps` launches each; 512 only where sets have at least 32 members on
 * average) and keeps the fastest; in the
 * persistent form it also times whole persistent iterations per lane count.
 * Trial launches overwrite the solver state, so the call ends by resetting it
 * (as cfr_reset) and dropping a captured graph. The chosen counts are
 * exported as array 12. In the FP32 mode the lane count fixes the shape of
 * the member reductions, so a different choice changes the last bits of the
 * iterates; pin it with cfr_options.lanes_per_set for bitwise repeatability
 * across processes. Synchronises `stream`. */
int cfr_autotune(cfr_handle *h, int reps, void *stream);

/* The launch floor of one iteration (no counterpart in the paper's API; its
 * Section 4.3 discusses the graph-launch floor): the mean time of one
 * iteration's launch structure with no work in it, over n iterations.
 * graph_ms: a CUDA graph of the same launches as the per-level form (2D,
 * or 2D - 1 in member order, whose deepest depth has no forward launch;
 * twice that under alternating updates) with the same grid sizes
 * (depth-first forward, then backward), each an empty kernel. persistent_ms: one
 * cooperative launch of an empty kernel with the persistent form's grid and
 * its 2D (4D) grid barriers per iteration (bounded
 * waits: CFR_ERR_TIMEOUT if one gives up). The handle must be bound; solver
 * state is untouched. Synchronises `stream`. */
int cfr_launch_floor(cfr_handle *h, int64_t n, void *stream, double *graph_ms, double *persistent_ms);

/* Chance sums per information set from the chance products the compiler
 * folded (Algorithm "Compile", step 6): mass[I] = the sum over the set's
 * members h of pi_c(h), and, when root_w is given, wsum[I] = the sum of
 * pi_c(h) * root_w[the root outcome above h] (root_w has one weight per
 * outcome of a chance root, in the spec's order; CFR_ERR_UNSUPPORTED if the
 * root is not a chance node). Members are added in ascending compiled id.
 * Host arrays, spec set order; host only. Used for the learned warm start's
 * features (a set's weight in its range, its equity against the opponent's
 * range); no counterpart in the paper's API. */
int cfr_set_chance_sums(const cfr_handle *h, const double *root_w, double *mass, double *wsum);

/* Page-locks (pin != 0) or releases (pin == 0) the host memory that
 * cfr_bind and the lifecycle calls copy to the device (the compiled arrays
 * and the value template, owned by the handle), so those copies run at the
 * pinned host-to-device rate. No counterpart in the paper's API. Ranges the
 * driver reports as already page-locked (a page shared with another pinned
 * range) stay as they are. cfr_destroy releases what is still pinned.
 * Returns CFR_ERR_DEVICE if the driver refuses. */
int cfr_pin_host(cfr_handle *h, int pin);

/* Batched solves (many independent games in one launch). Every handle must
 * be bound (each to its own arena) and use the same precision, with sets of
 * at most 8 actions. One CTA of `threads` threads (256 or 1024; 0 = 256)
 * runs all iterations of one instance with `lanes` lanes per information set
 * (2, 4, 8 or 32; 0 = 4); cfr_batch_iterate can instead give every instance
 * a thread-block cluster of `cluster` CTAs (2, 4 or 8) that share its work
 * and meet at the hardware cluster barrier between depths (for large
 * instances). A solve's result depends only on its own data and on
 * (threads, lanes, cluster): it is bitwise the same alone and in any mix.
 * table_dev: caller-owned device buffer of at least cfr_batch_table_bytes(n)
 * bytes (16-byte aligned) for the instance descriptors; it must stay
 * untouched until the launch completes. */
size_t cfr_batch_table_bytes(int n);

/* Runs iters[i] iterations of instance i (iters may be NULL: every
 * instance runs n_iter), asynchronously on `stream`. cluster: CTAs per
 * instance (0 or 1 = one CTA; 2, 4 or 8 = a thread-block cluster). */
int cfr_batch_iterate(cfr_handle *const *handles, int n, const int64_t *iters, int64_t n_iter, void *table_dev,
                      size_t table_bytes, int threads, int lanes, int cluster, void *stream);

/* Exploitability of every instance's average strategy in one launch; out
 * (host, [4n]) receives per instance (NashConv/2, br1, br2, u). Synchronises
 * `stream`. */
int cfr_batch_exploitability(cfr_handle *const *handles, int n, double *out, void *table_dev, size_t table_bytes,
                             int threads, int lanes, void *stream);

/* Algorithmic device bytes of depth level d (0 <= d < D) for the forward
 * kernel and the backward kernel of one iteration: every array element the
 * layout needs, touched once. With T the bytes of the compute type (4 or 8)
 * and member-order reach, the launch of depth d < D-1 that fills depth d+1
 * moves 8 per internal child (edge record) + 2T per internal parent and per
 * internal child (reach read and written) + T per slot of depth d (sigma);
 * the backward of depth d moves 12 per set (slot and member ranges, value
 * block) + (32 + 2T) per slot (R and the average read and written in FP64,
 * sigma read and written) + (4 + 3T) per member (value slot, reach lanes,
 * value written) + (12 + T) per chance node + T per child value read. The
 * other reach orders read an internal rank per member (4 more) and push
 * records (12 per internal parent, 4 per long child list entry). Host only.
 * The paper counts the same kind of bytes-moved lower bound (Appendix
 * "Kernel-Level Profile"). */
int cfr_level_bytes(const cfr_handle *h, int level, int64_t *fwd_bytes, int64_t *bwd_bytes);

/* Measurement: runs ONE iteration (t -> t+1) as per-level launches on
 * `stream` with a CUDA event pair around every launch, and writes each
 * launch's device time in milliseconds: fwd_ms[d] and bwd_ms[d] for
 * d = 0 .. D-1 (host arrays of D doubles; under alternating updates the two
 * halves' times of a depth are added). Synchronises `stream`. */
int cfr_profile_iteration(cfr_handle *h, double *fwd_ms, double *bwd_ms, void *stream);

/* Allocation-free variant of cfr_iterate, for callers that cannot allocate
 * device memory while they run iterations: a serving loop whose device
 * memory is carved out once at start-up (an allocation inside the loop could
 * fail or stall the other solves sharing the GPU), or a host program that
 * embeds the library without owning the device allocator. The paper has no
 * counterpart to this entry point.
 * It runs n iterations with the persistent kernel, exactly as the
 * CFR_EXEC_PERSISTENT form does (same grid, same lane groups: the state it
 * leaves is bitwise that form's), but takes the per-iteration scratch (reach
 * lanes, node values, wide-node partial sums, grid-barrier words) from one
 * static 12 MiB device array compiled into the library (held on every GPU
 * that loads the library, until the process exits) instead of the arena.
 * The arena bound with cfr_bind still holds the inputs and outputs: the
 * compiled game and the solver state (regrets, average, strategy, t).
 * No cudaMalloc, cudaFree or other allocating call is made. The first call on
 * a device resolves the array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it for the life of the process; make that
 * first call before any stream capture. The kept address is void after a
 * cudaDeviceReset (or any teardown of the device's primary context): do not
 * call this entry point after one.
 * Limits: games whose scratch exceeds the array are rejected with
 * CFR_ERR_ARG; the scratch is both reach lanes of every internal node and
 * every node's value, at most 24 bytes per node in FP64 and 12 in FP32
 * (about 524,000 and 1,048,000 nodes for any tree shape). Every call
 * re-initialises the part of the array it uses (values from the template,
 * root reach, counters and barrier words at zero).
 * All calls share the one array, so calls that overlap on the GPU (other
 * streams, other threads, other handles) race: serialise them. Synchronises
 * `stream`; a barrier timeout returns CFR_ERR_TIMEOUT. */
int cfr_iterate_noalloc(cfr_handle *h, int64_t n, void *stream);

/* Fault-injection hooks for tests (no effect unless set; set on the host).
 * CFR_DEBUG_BARRIER_MISSING_ARRIVALS = k: the persistent kernel's grid
 * barriers wait for k blocks that do not exist, so every wait runs into its
 * spin limit (cfr_options.barrier_spin_limit) and the launch ends with
 * CFR_ERR_TIMEOUT reported by cfr_synchronize. Nothing faults or hangs: each
 * block stops after its bounded wait.
 * CFR_DEBUG_FAIL_GRAPH_CAPTURE = 1: the next graph capture of the graph form
 * is treated as refused after it ends (the captured graph is discarded), so
 * cfr_iterate takes the capture-failure path of Section 4.3: one warning on
 * stderr per handle, then per-level launches of the same kernels in the same
 * order.
 * CFR_DEBUG_STREAM_STALL = 1 (a bound handle; cleared by cfr_reset): the
 * streaming backward's copy warp issues no copies beyond each CTA's first
 * chunks, so the compute threads' and the update warp's waits for the next
 * chunk run out (about a second each) and cfr_synchronize reports
 * CFR_ERR_TIMEOUT. Nothing faults or hangs: every wait is bounded. */
enum { CFR_DEBUG_BARRIER_MISSING_ARRIVALS = 1, CFR_DEBUG_FAIL_GRAPH_CAPTURE = 2, CFR_DEBUG_STREAM_STALL = 3 };
int cfr_debug_set(cfr_handle *h, int key, int64_t value);

/* Message of the calling thread's last failure (thread-local, valid until
 * that thread's next failing call). No counterpart in the paper. */
const char *cfr_last_error(void);
/* Releases the handle's host memory, its captured graph and its page-locked
 * ranges; the caller's arena is not freed. NULL is ignored. No counterpart in
 * the paper. */
void cfr_destroy(cfr_handle *h);

#ifdef __cplusplus
}
#endif
#endif
