// compiled.h — host-side compiled game (output of the compiler, input of the
// runtime). Plain C++; no CUDA types so the compiler builds with any C++17
// compiler.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cfr.h"

namespace cfr {

// Bit 30 of node_slot marks a player-2 decision node; the low 30 bits hold
// the first slot of the node's information set. Chance and terminal nodes
// hold -1.
constexpr int32_t kSlotP2Bit = 1 << 30;
constexpr int32_t kSlotMask = kSlotP2Bit - 1;
constexpr int kMaxActions = 64;
// Chance nodes with more than kWide children ("wide", e.g. a deal root) are
// handled by chunks of kWideChunk children instead of one thread.
constexpr int kWide = 1024;
constexpr int kWideChunk = 2048;
constexpr uint32_t kBigNode = 0x80000000u;  // int_mask flag: children listed in big_irank

// Member order: sets per reach tile, and the number of sets a depth needs
// before it is tiled by default (tiled depths run lane groups of at most
// 32 / kTileSets lanes, so they need many sets to fill the GPU).
constexpr int32_t kTileSets = 4;
constexpr int64_t kTileMinSets = 8192;

struct Compiled {
  int64_t N = 0, E = 0, I = 0, A = 0, D = 0;
  int64_t n_dec = 0, n_chance = 0, n_term = 0, n_int = 0, max_act = 0;
  // Breadth-first node numbering: parent before child, siblings contiguous
  // in action order. Node h's children are child_begin[h] .. child_begin[h+1]-1.
  std::vector<int32_t> child_begin;  // [N+1]
  std::vector<int32_t> node_slot;    // [N]
  std::vector<int32_t> level_begin;  // [D+2]: nodes of depth d are level_begin[d] .. level_begin[d+1]-1
  // Information sets in compiled order: by depth, player 1 before player 2,
  // then by the smallest value slot among the set's members (first member on
  // ties; see compile_game). Slots are contiguous per set in that order.
  std::vector<int32_t> iset_slot;    // [I+1]
  std::vector<int32_t> iset_mem;     // [I+1] offsets into mem_node
  std::vector<int32_t> mem_node;     // [n_dec] members, ascending node id per set
  std::vector<int32_t> mem_cb;       // [n_dec] first child of each member (member order)
  std::vector<int32_t> level_iset;   // [2D+1]: depth d: P1 sets [2d, 2d+1), P2 sets [2d+1, 2d+2)
  std::vector<int32_t> chance_list;  // [n_chance - n_wide] chance nodes with <= kWide children, ascending id
  std::vector<int32_t> level_chance; // [D+1]
  std::vector<int32_t> wide_list;    // [n_wide] chance nodes with > kWide children, ascending id
  std::vector<int32_t> level_wide;   // [D+1]
  std::vector<int32_t> wide_chunk;   // [n_wide+1] prefix of chunk counts (kWideChunk children each)
  int64_t n_wide = 0;
  // Compact index space of the internal nodes (reach lives only there:
  // terminal reach is never read). Internal node h has rank int_rank(h) =
  // number of internal nodes before it; the internal nodes of depth d are
  // ranks level_int[d] .. level_int[d+1]-1. Per internal node (rank order):
  //   int_slot  = node_slot (set's first slot | player-2 bit, or -1 for chance)
  //   int_mask  = bit a set if child a is internal (nodes with <= 31 children),
  //               or kBigNode for nodes with more children
  //   int_cirank= rank of the first internal child (mask nodes; the others
  //               follow it), or the offset of [nch, rank of child 0, rank of
  //               child 1, ...] in big_irank (-1 for terminal children)
  std::vector<int32_t> level_int;    // [D+1]
  std::vector<int32_t> int_slot;     // [n_int]
  std::vector<uint32_t> int_mask;    // [n_int]
  std::vector<int32_t> int_cirank;   // [n_int]
  std::vector<int32_t> big_irank;    // [...]
  // member order only (the push records above and wide_irank stay empty):
  //   int_edge  = [2 n_int] per internal node (rank order): its parent's rank
  //               (root -1) and the slot word of the edge from the parent
  //               (parent's slot word + action), or -1 under a chance node
  std::vector<int32_t> int_edge;
  //   iset_rank = [2 I] per set: rank of its member 0 and the rank stride of
  //               its members (kTileSets inside a tile, else 1)
  //   level_tiled = [D] 1 if depth d's sets are tiled
  std::vector<int32_t> iset_rank;
  std::vector<int32_t> level_tiled;
  std::vector<int32_t> mem_irank;    // [n_dec] internal rank of each member
  std::vector<int32_t> wide_irank;   // [n_wide] internal rank of each wide node
  // Value slots. The value of node h lives in slot vslot[h] of the value
  // array (not at h): the children of the members of one information set
  // fill one block of slots, action-major (child a of every member in member
  // order, then action a + 1: child a of member k at block + a * M + k - m0),
  // the children of one chance node another. Blocks go by parent depth;
  // within a depth the sets' blocks (set order) come before the chance
  // nodes' (node order). The root takes the last slot, N-1. A set's backward
  // pass therefore reads its members' children as one contiguous run (and
  // each action's as a run of its own); each node writes its own value to
  // the one slot its parent reads. Action-major keeps the children that
  // are written (decision and chance nodes) apart from those that are not
  // (terminals, which keep their template value), and puts the writes of
  // the sets of one tile (neighbouring members of the parent set) into
  // neighbouring words.
  std::vector<int32_t> vslot;        // [N]
  std::vector<int32_t> iset_vb;      // [I] first slot of set I's block
  std::vector<int32_t> mem_vs;       // [n_dec] own value slot of each member (member order)
  std::vector<int32_t> ch_vb, ch_nch, ch_vs;        // [narrow chance nodes] block, children, own slot
  std::vector<int32_t> wide_vb, wide_nch, wide_vs;  // [n_wide] the same for wide chance nodes
  std::vector<double> tmpl_vs;       // [N] the values template in slot order
  std::vector<double> pc;            // [N] chance product root..h (retained for set_payoffs)
  std::vector<double> edge_p;        // [N] probability of the chance edge into h (1 below decision nodes and at the root)
  std::vector<double> u;             // [N] payoff to player 1 at terminals, 0 elsewhere
  std::vector<double> tmpl;          // [N] pi_c(z) * u(z) at terminals, else 0 (eq. (template))
  std::vector<int32_t> new_of_spec;  // [N] compiled id of each spec node
  std::vector<int32_t> spec_of_new;  // [N]
  std::vector<int32_t> spec_slot_of; // [A] spec slot of each compiled slot
  std::vector<int32_t> level_max_members; // [D] largest information set per depth
  std::vector<double> level_mean_members; // [D]
  std::vector<int64_t> level_pull_parents; // [D] member order: distinct parents of depth d + 1's internal nodes
  std::vector<int32_t> spec_set_of;  // [I] the spec's id of each compiled set
};

// Returns CFR_OK or CFR_ERR_INVALID_SPEC / CFR_ERR_HOST_MEMORY with a message.
int compile_game(const cfr_game_spec &spec, Compiled &out, std::string &err, int reach_order = CFR_REACH_MEMBERS,
                 int member_tiles = CFR_TILES_AUTO);

// Chance folding from the retained edge probabilities and payoffs: the
// products root..h in path order (pc), the template pi_c(z) u(z) (eq.
// (template)) in node order and in value-slot order. The same arithmetic as
// the compile pass, so a rewritten input gives bitwise the template of a
// fresh compile.
void fold_chance(Compiled &c);

// Algorithmic device bytes of one iteration: each array element touched the
// minimum number of times the layout allows, i.e. the sum over depths of the
// forward and backward launch models (per internal child an 8-byte edge
// record and both reach lanes written, per internal parent its reach read,
// per slot sigma read; per set 12 bytes of ranges, per slot R and the
// average read and written in FP64 plus sigma read and written, per member
// its value slot, reach and value written, per chance node its ranges and
// value, per child its value read).
int64_t algo_bytes_per_iter(const Compiled &c, int precision);

}  // namespace cfr
