// compile.cpp — host game compiler (the paper's Algorithm "Compile", steps
// 1-8, Appendix H): validation, slot prefix sums, breadth-first node arrays,
// depth blocks (eq. (blocks)), chance folding into the values template
// (eq. (template)) and index emission. Differences from the paper's layout:
// edges are implicit (siblings are contiguous, so node h's children are
// child_begin[h] .. child_begin[h+1]-1 and edge e leads to node e+1), indices
// are int32, and information-set members are listed per set (member CSR) so
// that the regret update is a per-set segmented reduction instead of a
// scatter.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "compiled.h"

namespace cfr {

static int fail(std::string &err, const std::string &msg) {
  err = msg;
  return CFR_ERR_INVALID_SPEC;
}

int compile_game(const cfr_game_spec &s, Compiled &c, std::string &err, int reach_order, int member_tiles) {
  try {
    const int64_t N = s.n_nodes, I = s.n_infosets;
    if (N < 1 || N >= (int64_t(1) << 31) - 2) return fail(err, "n_nodes must be in [1, 2^31-2)");
    if (I < 0 || I >= (int64_t(1) << 30)) return fail(err, "n_infosets out of range");
    if (!s.kind || !s.infoset || !s.child_begin || (!s.child && s.child_begin[N] > 0) || !s.payoff ||
        (I > 0 && (!s.iset_player || !s.iset_nact)))
      return fail(err, "null array in game spec");
    const int64_t E = s.child_begin[N];
    if (s.child_begin[0] != 0 || E != N - 1) return fail(err, "child_begin must start at 0 and end at n_nodes-1 (a tree)");
    if (E > 0 && !s.chance_prob) {
      // probabilities are only needed below chance nodes
      for (int64_t v = 0; v < N; ++v)
        if (s.kind[v] == CFR_CHANCE) return fail(err, "chance_prob is null but the game has chance nodes");
    }
    // ---- step 1: structural checks
    int64_t A = 0;
    std::vector<int64_t> spec_off(I + 1, 0);
    for (int64_t i = 0; i < I; ++i) {
      if (s.iset_player[i] != 0 && s.iset_player[i] != 1) return fail(err, "iset_player must be 0 or 1");
      if (s.iset_nact[i] < 1 || s.iset_nact[i] > kMaxActions) return fail(err, "iset_nact must be in [1, 64]");
      spec_off[i + 1] = spec_off[i] + s.iset_nact[i];
    }
    A = spec_off[I];
    if (A >= (int64_t(1) << 30)) return fail(err, "too many slots (>= 2^30)");
    for (int64_t v = 0; v < N; ++v) {
      const int k = s.kind[v];
      const int64_t nch = s.child_begin[v + 1] - s.child_begin[v];
      if (nch < 0) return fail(err, "child_begin must be non-decreasing");
      if (k == CFR_TERMINAL) {
        if (nch != 0) return fail(err, "terminal node with children");
        if (!std::isfinite(s.payoff[v])) return fail(err, "non-finite payoff");
      } else if (k == CFR_CHANCE) {
        if (nch < 1) return fail(err, "chance node without children");
        double sum = 0.0;
        for (int64_t q = s.child_begin[v]; q < s.child_begin[v + 1]; ++q) {
          const double p = s.chance_prob[q];
          if (!(p >= 0.0) || !std::isfinite(p)) return fail(err, "chance probability must be finite and >= 0");
          sum += p;
        }
        if (std::fabs(sum - 1.0) > 1e-6) return fail(err, "chance probabilities of a node must sum to 1");
      } else if (k == CFR_PLAYER1 || k == CFR_PLAYER2) {
        const int32_t is = s.infoset[v];
        if (is < 0 || is >= I) return fail(err, "decision node with an information set out of range");
        if (s.iset_player[is] != k - CFR_PLAYER1) return fail(err, "information set owned by another player");
        if (s.iset_nact[is] != nch) return fail(err, "member's child count differs from its set's action count");
      } else {
        return fail(err, "unknown node kind");
      }
    }
    // ---- step 3: breadth-first numbering (parents before children, siblings contiguous)
    c.N = N; c.E = E; c.I = I; c.A = A;
    c.new_of_spec.assign(N, -1);
    c.spec_of_new.assign(N, -1);
    std::vector<int32_t> depth(N, 0);
    c.new_of_spec[0] = 0;
    c.spec_of_new[0] = 0;
    int64_t head = 0, tail = 1;
    while (head < tail) {
      const int32_t sv = c.spec_of_new[head];
      for (int64_t q = s.child_begin[sv]; q < s.child_begin[sv + 1]; ++q) {
        const int32_t ch = s.child[q];
        if (ch <= 0 || ch >= N) return fail(err, "child id out of range (or the root listed as a child)");
        if (c.new_of_spec[ch] >= 0) return fail(err, "node with two parents: not a tree");
        c.new_of_spec[ch] = (int32_t)tail;
        c.spec_of_new[tail] = ch;
        depth[tail] = depth[head] + 1;
        ++tail;
      }
      ++head;
    }
    if (tail != N) return fail(err, "nodes unreachable from the root");
    // ---- step 5: depth schedule
    const int32_t maxd = depth[N - 1];
    int64_t D = 0;
    {
      int32_t maxd_int = -1;
      for (int64_t h = 0; h < N; ++h) {
        const int32_t sv = c.spec_of_new[h];
        if (s.child_begin[sv + 1] > s.child_begin[sv]) maxd_int = std::max(maxd_int, depth[h]);
      }
      D = maxd_int + 1;  // number of parent depths (every depth below the deepest parent has one)
    }
    c.D = D;
    c.level_begin.assign(D + 2, (int32_t)N);
    c.level_begin[0] = 0;
    for (int64_t h = N - 1; h >= 0; --h)
      if (depth[h] <= D) c.level_begin[depth[h]] = (int32_t)h;
    for (int64_t d = D; d >= 0; --d)  // depths with no node (impossible in a tree) stay consistent
      if (c.level_begin[d] > c.level_begin[d + 1]) c.level_begin[d] = c.level_begin[d + 1];
    (void)maxd;
    // ---- node arrays and chance folding
    c.child_begin.assign(N + 1, 0);
    c.node_slot.assign(N, -1);
    c.pc.assign(N, 0.0);
    c.tmpl.assign(N, 0.0);
    c.edge_p.assign(N, 1.0);
    c.u.assign(N, 0.0);
    c.pc[0] = 1.0;
    int64_t next = 1;
    c.n_dec = c.n_chance = c.n_term = c.n_int = 0;
    c.max_act = 0;
    for (int64_t h = 0; h < N; ++h) {
      const int32_t sv = c.spec_of_new[h];
      const int k = s.kind[sv];
      const int64_t b = s.child_begin[sv], e = s.child_begin[sv + 1];
      c.child_begin[h] = (int32_t)next;
      if (e > b && c.new_of_spec[s.child[b]] != next) return fail(err, "internal: children not contiguous");
      next += e - b;
      if (k == CFR_TERMINAL) {
        ++c.n_term;
        c.u[h] = s.payoff[sv];
        c.tmpl[h] = c.pc[h] * c.u[h];  // values template, eq. (template)
        continue;
      }
      ++c.n_int;
      if (k != CFR_CHANCE) c.max_act = std::max<int64_t>(c.max_act, e - b);
      for (int64_t q = b; q < e; ++q) {
        const int32_t ch = c.new_of_spec[s.child[q]];
        if (k == CFR_CHANCE) c.edge_p[ch] = s.chance_prob[q];
        c.pc[ch] = (k == CFR_CHANCE) ? c.pc[h] * c.edge_p[ch] : c.pc[h];
      }
      if (k == CFR_CHANCE) ++c.n_chance; else ++c.n_dec;
    }
    c.child_begin[N] = (int32_t)next;
    // ---- information sets and value slots, depth by depth. The sets of
    // depth d go player 1 first, then player 2, each group ordered by the
    // smallest value slot among a set's members: sets whose members pass
    // their values into the same parent blocks come together, so the sets
    // processed at the same time fill whole blocks. The members' children
    // then take the next value slots (set by set, members in ascending id,
    // children in action order), followed by the children of depth d's
    // chance nodes (node order). The root's slot is N - 1.
    std::vector<int32_t> first(I, -1), cid_of_spec(I, -1);
    std::vector<int64_t> smb(I + 1, 0);
    std::vector<int32_t> enc;  // spec sets in order of their first member
    enc.reserve(I);
    for (int64_t h = 0; h < N; ++h) {
      const int32_t sv = c.spec_of_new[h];
      const int k = s.kind[sv];
      if (k != CFR_PLAYER1 && k != CFR_PLAYER2) continue;
      const int32_t is = s.infoset[sv];
      if (first[is] < 0) { first[is] = (int32_t)h; enc.push_back(is); }
      else if (depth[first[is]] != depth[h])
        return fail(err, "information set with members at different depths");
      smb[is + 1]++;
    }
    if ((int64_t)enc.size() != I) return fail(err, "information set without members");
    for (int64_t is = 0; is < I; ++is) smb[is + 1] += smb[is];
    std::vector<int32_t> smem(c.n_dec);  // members of each spec set, ascending node id
    {
      std::vector<int64_t> fill(smb.begin(), smb.end() - 1);
      for (int64_t h = 0; h < N; ++h) {
        const int k = s.kind[c.spec_of_new[h]];
        if (k == CFR_PLAYER1 || k == CFR_PLAYER2) smem[fill[s.infoset[c.spec_of_new[h]]]++] = (int32_t)h;
      }
    }
    c.level_iset.assign(2 * D + 1, 0);
    c.vslot.assign(N, -1);
    c.vslot[0] = (int32_t)(N - 1);
    c.iset_vb.assign(I, 0);
    // the value-slot reach order ranks internal nodes by their block position
    // taken member-major (member, then action), so that a parent's internal
    // children stay consecutive for the pushing forward
    std::vector<int64_t> slot_key(N, (int64_t)N - 1);
    {
      std::vector<int32_t> order;
      order.reserve(I);
      std::vector<std::pair<int64_t, int32_t>> keyed;
      int64_t next = 0;
      size_t i = 0;
      for (int64_t d = 0; d < D; ++d) {
        size_t j = i;
        while (j < enc.size() && depth[first[enc[j]]] == d) ++j;
        for (int pl = 0; pl < 2; ++pl) {
          c.level_iset[2 * d + pl] = (int32_t)order.size();
          keyed.clear();
          for (size_t q = i; q < j; ++q) {
            const int32_t is = enc[q];
            if (s.iset_player[is] != pl) continue;
            int64_t key = N;
            for (int64_t m = smb[is]; m < smb[is + 1]; ++m) key = std::min<int64_t>(key, c.vslot[smem[m]]);
            keyed.emplace_back(key * (int64_t)I + (int64_t)(q - i), is);  // ties: first-member order
          }
          std::sort(keyed.begin(), keyed.end());
          for (const auto &kv : keyed) order.push_back(kv.second);
        }
        for (size_t q = c.level_iset[2 * d]; q < order.size(); ++q) {  // value slots of depth d + 1
          const int32_t is = order[q];
          c.iset_vb[q] = (int32_t)next;
          // action-major: the children of action a of all members, in member order, then action a + 1
          const int32_t na = s.iset_nact[is];
          for (int64_t m = smb[is]; m < smb[is + 1]; ++m)
            for (int32_t a = 0; a < na; ++a) slot_key[c.child_begin[smem[m]] + a] = next + (m - smb[is]) * na + a;
          for (int32_t a = 0; a < na; ++a)
            for (int64_t m = smb[is]; m < smb[is + 1]; ++m) c.vslot[c.child_begin[smem[m]] + a] = (int32_t)next++;
        }
        for (int64_t h = c.level_begin[d]; h < c.level_begin[d + 1]; ++h) {
          if (s.kind[c.spec_of_new[h]] != CFR_CHANCE) continue;
          for (int32_t x = c.child_begin[h]; x < c.child_begin[h + 1]; ++x) {
            slot_key[x] = next;
            c.vslot[x] = (int32_t)next++;
          }
        }
        i = j;
      }
      c.level_iset[2 * D] = (int32_t)order.size();
      if (i != enc.size()) return fail(err, "internal: information set below the deepest parent");
      if (next != N - 1) return fail(err, "internal error: value slots do not cover the tree");
      for (size_t q = 0; q < order.size(); ++q) cid_of_spec[order[q]] = (int32_t)q;
      c.spec_set_of.assign(order.begin(), order.end());
      c.iset_slot.assign(I + 1, 0);
      c.spec_slot_of.assign(A, 0);
      for (int64_t q = 0; q < I; ++q) {
        const int32_t sp = order[q];
        c.iset_slot[q + 1] = c.iset_slot[q] + s.iset_nact[sp];
        for (int a = 0; a < s.iset_nact[sp]; ++a) c.spec_slot_of[c.iset_slot[q] + a] = (int32_t)(spec_off[sp] + a);
      }
    }
    // member lists (counting sort by compiled set, ascending node id)
    c.iset_mem.assign(I + 1, 0);
    for (int64_t h = 0; h < N; ++h) {
      const int32_t sv = c.spec_of_new[h];
      const int k = s.kind[sv];
      if (k == CFR_PLAYER1 || k == CFR_PLAYER2) c.iset_mem[cid_of_spec[s.infoset[sv]] + 1]++;
    }
    for (int64_t q = 0; q < I; ++q) c.iset_mem[q + 1] += c.iset_mem[q];
    c.mem_node.assign(c.n_dec, 0);
    {
      std::vector<int32_t> fill(c.iset_mem.begin(), c.iset_mem.end() - 1);
      for (int64_t h = 0; h < N; ++h) {
        const int32_t sv = c.spec_of_new[h];
        const int k = s.kind[sv];
        if (k != CFR_PLAYER1 && k != CFR_PLAYER2) continue;
        const int32_t cid = cid_of_spec[s.infoset[sv]];
        c.mem_node[fill[cid]++] = (int32_t)h;
        c.node_slot[h] = c.iset_slot[cid] | (k == CFR_PLAYER2 ? kSlotP2Bit : 0);
      }
    }
    c.mem_cb.resize(c.n_dec);
    for (int64_t k = 0; k < c.n_dec; ++k) c.mem_cb[k] = c.child_begin[c.mem_node[k]];
    // chance nodes per depth (narrow ones per thread, wide ones by chunks)
    c.chance_list.clear();
    c.chance_list.reserve(c.n_chance);
    c.wide_list.clear();
    c.level_chance.assign(D + 1, 0);
    c.level_wide.assign(D + 1, 0);
    c.wide_chunk.assign(1, 0);
    for (int64_t d = 0; d < D; ++d) {
      c.level_chance[d] = (int32_t)c.chance_list.size();
      c.level_wide[d] = (int32_t)c.wide_list.size();
      for (int64_t h = c.level_begin[d]; h < c.level_begin[d + 1]; ++h) {
        if (s.kind[c.spec_of_new[h]] != CFR_CHANCE) continue;
        const int64_t nch = c.child_begin[h + 1] - c.child_begin[h];
        if (nch > kWide) {
          c.wide_list.push_back((int32_t)h);
          c.wide_chunk.push_back(c.wide_chunk.back() + (int32_t)((nch + kWideChunk - 1) / kWideChunk));
        } else {
          c.chance_list.push_back((int32_t)h);
        }
      }
    }
    c.level_chance[D] = (int32_t)c.chance_list.size();
    c.level_wide[D] = (int32_t)c.wide_list.size();
    c.n_wide = (int64_t)c.wide_list.size();
    // compact internal-node index space. Member order (the default; depth by
    // depth: the members of the depth's sets in set order, then the depth's
    // chance nodes in the order they are pulled from): the backward reads
    // every set's reach as one run and
    // needs no rank table (member k of depth d has rank k + a per-depth
    // offset); the forward pulls, each internal node reading its parent's
    // reach through int_edge. Breadth-first order: the forward reads parents
    // and writes children as two streams. Value-slot order (the root, then
    // depth by depth in parents' block order): the members of the sets
    // processed together have neighbouring ranks. In both a parent's internal
    // children have consecutive ranks and the forward pushes each parent's
    // reach to them.
    {
      std::vector<int32_t> rank(N, -1);
      int32_t r = 0;
      const bool members = reach_order == CFR_REACH_MEMBERS;
      if (members) {
        // A depth's chance nodes go in the order the next depth's internal
        // nodes (its members in set order, then its chance nodes) first pull
        // from them, so that a run of children reads neighbouring parents;
        // chance nodes without internal children follow in node order.
        // Found bottom-up.
        std::vector<int32_t> parent(N, -1);
        for (int64_t h = 0; h < N; ++h)
          for (int32_t x = c.child_begin[h]; x < c.child_begin[h + 1]; ++x) parent[x] = (int32_t)h;
        auto is_chance_int = [&](int32_t h) { return c.node_slot[h] < 0 && c.child_begin[h + 1] > c.child_begin[h]; };
        std::vector<std::vector<int32_t>> chance_at(D);
        std::vector<char> placed(N, 0);
        for (int64_t d = D - 1; d >= 0; --d) {
          std::vector<int32_t> &L = chance_at[d];
          auto pull = [&](int32_t x) {
            const int32_t p = parent[x];
            if (p >= 0 && is_chance_int(p) && !placed[p]) { placed[p] = 1; L.push_back(p); }
          };
          if (d + 1 < D) {
            const int32_t i0 = c.level_iset[2 * d + 2], i1 = c.level_iset[2 * d + 4];
            for (int32_t k = c.iset_mem[i0]; k < c.iset_mem[i1]; ++k) pull(c.mem_node[k]);
            for (int32_t x : chance_at[d + 1]) pull(x);
          }
          for (int32_t h = c.level_begin[d]; h < c.level_begin[d + 1]; ++h)
            if (is_chance_int(h) && !placed[h]) { placed[h] = 1; L.push_back(h); }
        }
        // Tiles: kTileSets consecutive sets of one player and one size;
        // member k of the tile's set j has rank base + k * kTileSets + j.
        c.iset_rank.assign(2 * (size_t)c.I, 0);
        c.level_tiled.assign(D, 0);
        for (int64_t d = 0; d < D; ++d) {
          const int32_t i0 = c.level_iset[2 * d], i1 = c.level_iset[2 * d + 2];
          auto size = [&](int32_t I) { return c.iset_mem[I + 1] - c.iset_mem[I]; };
          auto tile_at = [&](int32_t I, int32_t end) {  // a tile starts at set I
            if (I + kTileSets > end) return false;
            for (int32_t j = 1; j < kTileSets; ++j)
              if (size(I + j) != size(I)) return false;
            return true;
          };
          bool tiled = false;
          if (member_tiles != CFR_TILES_OFF && (member_tiles == CFR_TILES_ON || i1 - i0 >= kTileMinSets)) {
            int64_t in_tiles = 0;
            for (int pl = 0; pl < 2; ++pl) {
              const int32_t b = c.level_iset[2 * d + pl], e = c.level_iset[2 * d + pl + 1];
              for (int32_t I = b; I < e;)
                if (tile_at(I, e)) { in_tiles += (int64_t)kTileSets * size(I); I += kTileSets; } else ++I;
            }
            tiled = 2 * in_tiles >= (int64_t)(c.iset_mem[i1] - c.iset_mem[i0]) && in_tiles > 0;
          }
          c.level_tiled[d] = tiled ? 1 : 0;
          for (int pl = 0; pl < 2; ++pl) {
            const int32_t b = c.level_iset[2 * d + pl], e = c.level_iset[2 * d + pl + 1];
            for (int32_t I = b; I < e;) {
              if (tiled && tile_at(I, e)) {
                for (int32_t j = 0; j < kTileSets; ++j) {
                  c.iset_rank[2 * (size_t)(I + j)] = r + j;
                  c.iset_rank[2 * (size_t)(I + j) + 1] = kTileSets;
                  for (int32_t k = 0; k < size(I); ++k) rank[c.mem_node[c.iset_mem[I + j] + k]] = r + k * kTileSets + j;
                }
                r += kTileSets * size(I);
                I += kTileSets;
              } else {
                c.iset_rank[2 * (size_t)I] = r;
                c.iset_rank[2 * (size_t)I + 1] = 1;
                for (int32_t k = c.iset_mem[I]; k < c.iset_mem[I + 1]; ++k) rank[c.mem_node[k]] = r++;
                ++I;
              }
            }
          }
          for (int32_t h : chance_at[d]) rank[h] = r++;
        }
      } else if (reach_order == CFR_REACH_SLOTS) {
        if (N > 0 && c.child_begin[1] > c.child_begin[0]) rank[0] = r++;
        std::vector<int32_t> node_of_slot(N > 0 ? N - 1 : 0);
        for (int64_t h = 1; h < N; ++h) node_of_slot[slot_key[h]] = (int32_t)h;
        for (int64_t q = 0; q + 1 < N; ++q) {
          const int32_t h = node_of_slot[q];
          if (c.child_begin[h + 1] > c.child_begin[h]) rank[h] = r++;
        }
      } else {
        for (int64_t h = 0; h < N; ++h)
          if (c.child_begin[h + 1] > c.child_begin[h]) rank[h] = r++;
      }
      c.level_int.assign(D + 1, 0);
      for (int64_t h = 0; h < N; ++h)  // internal nodes sit at depths < D
        if (rank[h] >= 0 && depth[h] < D) c.level_int[depth[h] + 1]++;
      for (int64_t d = 0; d < D; ++d) c.level_int[d + 1] += c.level_int[d];
      c.int_slot.clear();
      c.int_mask.clear();
      c.int_cirank.clear();
      c.big_irank.clear();
      c.int_edge.clear();
      c.wide_irank.clear();
      if (!members) {
        c.iset_rank.clear();
        c.level_tiled.assign(D, 0);
      }
      if (members) {  // each internal node's parent rank and the slot word of its edge
        c.int_edge.assign(2 * (size_t)r, -1);
        for (int64_t h = 0; h < N; ++h) {
          const int32_t q = rank[h];
          if (q < 0) continue;
          for (int32_t a = 0; a < c.child_begin[h + 1] - c.child_begin[h]; ++a) {
            const int32_t k = rank[c.child_begin[h] + a];
            if (k < 0) continue;
            c.int_edge[2 * (size_t)k] = q;
            c.int_edge[2 * (size_t)k + 1] = c.node_slot[h] < 0 ? -1 : c.node_slot[h] + a;
          }
        }
        // the parents whose reach the pull of depth d reads: those with an
        // internal child (a parent with terminal children only is not read)
        std::vector<char> seen(r, 0);
        c.level_pull_parents.assign(D, 0);
        for (int64_t d = 0; d + 1 < D; ++d)
          for (int32_t k = c.level_int[d + 1]; k < c.level_int[d + 2]; ++k) {
            const int32_t q = c.int_edge[2 * (size_t)k];
            if (q >= 0 && !seen[q]) {
              seen[q] = 1;
              ++c.level_pull_parents[d];
            }
          }
      } else {  // each internal node's record for the forward that pushes
        c.int_slot.resize(r);
        c.int_mask.resize(r);
        c.int_cirank.resize(r);
        for (int64_t h = 0; h < N; ++h) {
          const int32_t q = rank[h];
          if (q < 0) continue;
          const int32_t cb = c.child_begin[h], ce = c.child_begin[h + 1];
          const int32_t nch = ce - cb;
          c.int_slot[q] = c.node_slot[h];
          if (nch <= 31) {
            uint32_t mask = 0;
            int32_t first = 0;
            bool got = false;
            for (int32_t a = 0; a < nch; ++a)
              if (rank[cb + a] >= 0) {
                mask |= 1u << a;
                if (!got) { first = rank[cb + a]; got = true; }
              }
            c.int_mask[q] = mask;
            c.int_cirank[q] = first;
          } else {
            c.int_mask[q] = kBigNode;
            c.int_cirank[q] = (int32_t)c.big_irank.size();
            c.big_irank.push_back(nch);
            for (int32_t a = 0; a < nch; ++a) c.big_irank.push_back(rank[cb + a]);
          }
        }
        c.wide_irank.resize(c.n_wide);
        for (int64_t w = 0; w < c.n_wide; ++w) c.wide_irank[w] = rank[c.wide_list[w]];
        if ((int64_t)c.big_irank.size() >= (int64_t(1) << 31)) return fail(err, "too many children of large nodes");
      }
      c.mem_irank.resize(c.n_dec);
      for (int64_t k = 0; k < c.n_dec; ++k) c.mem_irank[k] = rank[c.mem_node[k]];
    }
    // arrays read through the value slots (laid out with the set order above)
    {
      c.mem_vs.resize(c.n_dec);
      for (int64_t k = 0; k < c.n_dec; ++k) c.mem_vs[k] = c.vslot[c.mem_node[k]];
      const size_t nn = c.chance_list.size();
      c.ch_vb.resize(nn);
      c.ch_nch.resize(nn);
      c.ch_vs.resize(nn);
      for (size_t i = 0; i < nn; ++i) {
        const int32_t h = c.chance_list[i];
        c.ch_vb[i] = c.vslot[c.child_begin[h]];
        c.ch_nch[i] = c.child_begin[h + 1] - c.child_begin[h];
        c.ch_vs[i] = c.vslot[h];
      }
      c.wide_vb.resize(c.n_wide);
      c.wide_nch.resize(c.n_wide);
      c.wide_vs.resize(c.n_wide);
      for (int64_t i = 0; i < c.n_wide; ++i) {
        const int32_t h = c.wide_list[i];
        c.wide_vb[i] = c.vslot[c.child_begin[h]];
        c.wide_nch[i] = c.child_begin[h + 1] - c.child_begin[h];
        c.wide_vs[i] = c.vslot[h];
      }
      c.tmpl_vs.assign(N, 0.0);
      for (int64_t h = 0; h < N; ++h) c.tmpl_vs[c.vslot[h]] = c.tmpl[h];
    }
    // per-depth member statistics (used to size the per-set lane groups)
    c.level_max_members.assign(D, 0);
    c.level_mean_members.assign(D, 0.0);
    for (int64_t d = 0; d < D; ++d) {
      const int32_t i0 = c.level_iset[2 * d], i1 = c.level_iset[2 * d + 2];
      int64_t tot = 0;
      for (int32_t q = i0; q < i1; ++q) {
        const int32_t m = c.iset_mem[q + 1] - c.iset_mem[q];
        c.level_max_members[d] = std::max(c.level_max_members[d], m);
        tot += m;
      }
      c.level_mean_members[d] = i1 > i0 ? (double)tot / (double)(i1 - i0) : 0.0;
    }
    return CFR_OK;
  } catch (const std::bad_alloc &) {
    err = "out of host memory while compiling";
    return CFR_ERR_HOST_MEMORY;
  }
}

void fold_chance(Compiled &c) {
  const int64_t N = c.N;
  if (N == 0) return;
  c.pc[0] = 1.0;
  for (int64_t h = 0; h < N; ++h) {
    const int32_t cb = c.child_begin[h], ce = c.child_begin[h + 1];
    if (cb == ce) {  // terminal
      c.tmpl[h] = c.pc[h] * c.u[h];
      c.tmpl_vs[c.vslot[h]] = c.tmpl[h];
      continue;
    }
    const bool chance = c.node_slot[h] < 0;
    for (int32_t ch = cb; ch < ce; ++ch) c.pc[ch] = chance ? c.pc[h] * c.edge_p[ch] : c.pc[h];
  }
}

int64_t algo_bytes_per_iter(const Compiled &c, int precision) {
  // Forward: every internal node's record (slot word, child mask, first
  // internal child: 12 B) and its two reach lanes read, every internal
  // child's reach lanes written, the strategy read once. Backward: per set
  // its slot, member and value-block offsets (12 B); per slot R and the
  // average read and written (FP64) and the strategy read and written; per
  // member its value slot and internal rank (8 B), its reach lanes read and
  // its value written; per chance node its block, child count and value slot
  // (12 B) and its value written; every edge's child value read once.
  // Member order: the forward reads every internal node's edge (parent rank
  // and slot word, 8 B) instead of the 12-byte records, and each parent's
  // reach and strategy once (the deepest depth's nodes and sets are nobody's
  // parents: no launch reads them); the backward reads no member rank.
  // A chance root's sum is not done in an iteration (nothing reads it).
  const int64_t T = precision == CFR_P64 ? 8 : 4;
  const int64_t int_kids = c.n_int > 0 ? c.n_int - 1 : 0;  // every internal node but the root
  const bool chance_root = c.N > 1 && c.node_slot[0] < 0;
  const int64_t root_sum = chance_root ? (12 + T) + T * (c.child_begin[1] - c.child_begin[0]) : 0;
  if (!c.int_edge.empty()) {
    int64_t parents = 0;  // reach the pulls read: every internal node with an internal child
    for (int64_t x : c.level_pull_parents) parents += x;
    const int64_t last_slots =
        c.D > 0 ? c.iset_slot[c.level_iset[2 * c.D]] - c.iset_slot[c.level_iset[2 * (c.D - 1)]] : 0;
    return 8 * int_kids + 2 * T * parents + 2 * T * int_kids + T * (c.A - last_slots) + 12 * c.I +
           (32 + 2 * T) * c.A + (4 + 3 * T) * c.n_dec + (12 + T) * c.n_chance + T * c.E - root_sum;
  }
  return 12 * c.n_int + 2 * T * c.n_int + 2 * T * int_kids + 4 * (int64_t)c.big_irank.size() + 12 * c.I +
         (32 + 3 * T) * c.A + (8 + 3 * T) * c.n_dec + (12 + T) * c.n_chance + T * c.E - root_sum;
}

}  // namespace cfr
