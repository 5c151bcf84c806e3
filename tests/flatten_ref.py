"""Independent re-derivation of the compiled arrays from a GameSpec (tests only).

Written from the definitions, not from the C++ compiler: breadth-first
numbering (the paper's compile pass: parents before children, siblings in
action order), depth blocks = distinct parent depths (eq. (blocks)),
information sets ordered by depth, then player, then the smallest value slot
among their members (first member on ties), slots contiguous in that order,
members ascending, chance product along the path and the values template
pi_c(z) u(z) (eq. (template)), value slots laid out depth by depth.
"""
from collections import deque

import numpy as np

TERMINAL, CHANCE, P1, P2 = 0, 1, 2, 3
P2BIT = 1 << 30
WIDE = 1024
WIDE_CHUNK = 2048


MEMBERS, BFS, SLOTS = 0, 1, 2  # internal-rank orders
TILES_AUTO, TILES_OFF, TILES_ON = 0, 1, 2
TILE, TILE_MIN_SETS = 4, 8192


def flatten(g, reach_order=MEMBERS, member_tiles=TILES_AUTO):
    """Internal ranks: MEMBERS, depth by depth the members of the depth's
    sets in member order (interleaved within tiles of TILE equal-size sets
    at tiled depths), then its chance nodes; BFS, breadth-first; SLOTS, the
    root, then by (depth, value slot)."""
    N = g.n_nodes
    order = []
    depth_of = {}
    q = deque([(0, 0)])
    while q:
        v, d = q.popleft()
        order.append(v)
        depth_of[v] = d
        for c in g.child[g.child_begin[v]:g.child_begin[v + 1]]:
            q.append((int(c), d + 1))
    new = np.empty(N, dtype=np.int64)
    new[np.array(order)] = np.arange(N)
    depth = np.array([depth_of[v] for v in order])
    nch = np.array([g.child_begin[v + 1] - g.child_begin[v] for v in order])
    child_begin = np.concatenate([[1], 1 + np.cumsum(nch)]).astype(np.int32)
    internal = nch > 0
    D = int(depth[internal].max()) + 1 if internal.any() else 0
    level_begin = np.array([int(np.searchsorted(depth, d)) for d in range(D + 1)] + [N], dtype=np.int32)
    kinds = np.array([g.kind[v] for v in order])
    # information sets and value slots, depth by depth: the sets of a depth
    # go player 1 first, then player 2, each group by the smallest value slot
    # among its members (ties: first member); then the children of those
    # sets' members take the next value slots (set, member, action order),
    # then the children of the depth's chance nodes (node order); the root's
    # value goes last
    child_begin_l = child_begin.tolist()
    first, mem_of = {}, {}
    for h, v in enumerate(order):
        if kinds[h] in (P1, P2):
            first.setdefault(int(g.infoset[v]), h)
            mem_of.setdefault(int(g.infoset[v]), []).append(h)
    by_first = sorted(first, key=lambda s: first[s])
    vslot = np.full(N, -1, dtype=np.int64)
    vslot[0] = N - 1
    slot_key = np.full(N, N - 1, dtype=np.int64)  # member-major block position (value-slot reach order)
    sets, vb_of = [], {}
    nxt = 0
    for d in range(D):
        here = [s_ for s_ in by_first if depth[first[s_]] == d]
        start = len(sets)
        for p in (0, 1):
            grp = [s_ for s_ in here if int(g.iset_player[s_]) == p]
            sets.extend(sorted(grp, key=lambda s_: (min(vslot[h] for h in mem_of[s_]), first[s_])))
        for s_ in sets[start:]:  # action-major: child a of every member, then a + 1
            vb_of[s_] = nxt
            na = int(g.iset_nact[s_])
            for i_, h in enumerate(mem_of[s_]):
                for a in range(na):
                    slot_key[child_begin_l[h] + a] = nxt + i_ * na + a  # member-major position
            for a in range(na):
                for h in mem_of[s_]:
                    vslot[child_begin_l[h] + a] = nxt
                    nxt += 1
        for h in range(level_begin[d], level_begin[d + 1]):
            if kinds[h] == CHANCE:
                for x in range(child_begin_l[h], child_begin_l[h + 1]):
                    slot_key[x] = nxt
                    vslot[x] = nxt
                    nxt += 1
    assert nxt == N - 1 or N == 1
    cid = {s: i for i, s in enumerate(sets)}
    nact = np.array([g.iset_nact[s] for s in sets], dtype=np.int64)
    iset_slot = np.concatenate([[0], np.cumsum(nact)]).astype(np.int32)
    spec_off = g.slot_offsets()
    spec_slot_of = np.concatenate([np.arange(spec_off[s], spec_off[s + 1]) for s in sets]).astype(np.int32) \
        if sets else np.zeros(0, np.int32)
    members = [[] for _ in sets]
    node_slot = np.full(N, -1, dtype=np.int32)
    for h, v in enumerate(order):
        if kinds[h] in (P1, P2):
            c = cid[int(g.infoset[v])]
            members[c].append(h)
            node_slot[h] = iset_slot[c] | (P2BIT if kinds[h] == P2 else 0)
    iset_mem = np.concatenate([[0], np.cumsum([len(m) for m in members])]).astype(np.int32)
    mem_node = np.array([h for m in members for h in m], dtype=np.int32)
    level_iset = [0]
    for d in range(D):
        for p in (0, 1):
            level_iset.append(sum(1 for s in sets if depth[first[s]] < d or
                                  (depth[first[s]] == d and int(g.iset_player[s]) <= p)))
    level_iset = np.array(level_iset, dtype=np.int32)
    chance_list, wide_list, level_chance, level_wide = [], [], [], []
    for d in range(D):
        level_chance.append(len(chance_list))
        level_wide.append(len(wide_list))
        for h in range(level_begin[d], level_begin[d + 1]):
            if kinds[h] == CHANCE:
                (wide_list if nch[h] > WIDE else chance_list).append(h)
    level_chance.append(len(chance_list))
    level_wide.append(len(wide_list))
    # chance product along the path, then the template
    pc = np.zeros(N)
    pc[0] = 1.0
    tmpl = np.zeros(N)
    for h, v in enumerate(order):
        b, e = g.child_begin[v], g.child_begin[v + 1]
        for q_, c in zip(range(b, e), g.child[b:e]):
            pc[new[c]] = pc[h] * g.chance_prob[q_] if kinds[h] == CHANCE else pc[h]
        if kinds[h] == TERMINAL:
            tmpl[h] = pc[h] * g.payoff[v]
    # compact space of internal nodes (reach lives only there): breadth-first,
    # or the root then by (depth, value slot)
    internal = nch > 0
    rank = np.full(N, -1, dtype=np.int64)
    int_nodes = np.nonzero(internal)[0].tolist()
    if reach_order == SLOTS:
        int_nodes = sorted(int_nodes, key=lambda h: (depth[h], slot_key[h]))
    elif reach_order == MEMBERS:
        # per depth: the members in member order, then the chance nodes in the
        # order the next depth's internal nodes first pull from them (those
        # with no internal child after, in node order), found bottom-up
        parent = np.full(N, -1, dtype=np.int64)
        for h in range(N):
            parent[child_begin[h]:child_begin[h + 1]] = h
        members_at = [[int(x) for x in mem_node[iset_mem[level_iset[2 * d]]:iset_mem[level_iset[2 * d + 2]]]]
                      for d in range(D)]
        chance_at = [[] for _ in range(D)]
        placed = set()
        for d in reversed(range(D)):
            below = members_at[d + 1] + chance_at[d + 1] if d + 1 < D else []
            for x in below:
                p = int(parent[x])
                if p >= 0 and kinds[p] == CHANCE and p not in placed:
                    placed.add(p)
                    chance_at[d].append(p)
            for h in range(level_begin[d], level_begin[d + 1]):
                if kinds[h] == CHANCE and internal[h] and h not in placed:
                    placed.add(h)
                    chance_at[d].append(h)
        # tiles: TILE consecutive sets of one player and one size; member k of
        # the tile's set j at tile base + k * TILE + j
        iset_rank = np.zeros(2 * len(sets), dtype=np.int32)
        level_tiled = np.zeros(D, dtype=np.int32)
        size = lambda s_: int(iset_mem[s_ + 1] - iset_mem[s_])
        tile_at = lambda s_, e: s_ + TILE <= e and all(size(s_ + j) == size(s_) for j in range(1, TILE))
        r = 0
        for d in range(D):
            ranges = [(int(level_iset[2 * d + pl]), int(level_iset[2 * d + pl + 1])) for pl in (0, 1)]
            tiled = False
            if member_tiles != TILES_OFF and (member_tiles == TILES_ON
                                              or level_iset[2 * d + 2] - level_iset[2 * d] >= TILE_MIN_SETS):
                in_tiles = 0
                for b, e in ranges:
                    s_ = b
                    while s_ < e:
                        if tile_at(s_, e):
                            in_tiles += TILE * size(s_)
                            s_ += TILE
                        else:
                            s_ += 1
                tiled = in_tiles > 0 and 2 * in_tiles >= len(members_at[d])
            level_tiled[d] = int(tiled)
            for b, e in ranges:
                s_ = b
                while s_ < e:
                    if tiled and tile_at(s_, e):
                        for j in range(TILE):
                            iset_rank[2 * (s_ + j)], iset_rank[2 * (s_ + j) + 1] = r + j, TILE
                            for k in range(size(s_)):
                                rank[mem_node[iset_mem[s_ + j] + k]] = r + k * TILE + j
                        r += TILE * size(s_)
                        s_ += TILE
                    else:
                        iset_rank[2 * s_], iset_rank[2 * s_ + 1] = r, 1
                        for k in range(size(s_)):
                            rank[mem_node[iset_mem[s_] + k]] = r + k
                        r += size(s_)
                        s_ += 1
            for h in chance_at[d]:
                rank[h] = r
                r += 1
        int_nodes = sorted(int_nodes, key=lambda h: rank[h])
    if reach_order != MEMBERS:
        rank[int_nodes] = np.arange(len(int_nodes))
        iset_rank = np.zeros(0, dtype=np.int32)
        level_tiled = np.zeros(D, dtype=np.int32)
    level_int = np.array([int(internal[:level_begin[d]].sum()) for d in range(D + 1)], dtype=np.int32)
    int_slot, int_mask, int_cirank, big, int_edge, wide_irank = [], [], [], [], [], []
    if reach_order == MEMBERS:  # each internal node's parent rank and edge slot word (the forward pulls)
        int_edge = [-1] * (2 * len(int_nodes))
        for h in int_nodes:
            for a in range(child_begin[h + 1] - child_begin[h]):
                k = int(rank[child_begin[h] + a])
                if k >= 0:
                    int_edge[2 * k] = int(rank[h])
                    int_edge[2 * k + 1] = -1 if node_slot[h] < 0 else int(node_slot[h]) + a
    else:  # each internal node's record (the forward pushes)
        for h in int_nodes:  # records in rank order
            cb, ce = child_begin[h], child_begin[h + 1]
            kids = rank[cb:ce]
            int_slot.append(node_slot[h])
            if ce - cb <= 31:
                m = 0
                for a, r in enumerate(kids):
                    if r >= 0:
                        m |= 1 << a
                int_mask.append(m)
                firsts = [r for r in kids if r >= 0]
                int_cirank.append(firsts[0] if firsts else 0)
            else:
                int_mask.append(1 << 31)
                int_cirank.append(len(big))
                big.append(ce - cb)
                big.extend(int(r) for r in kids)
        wide_irank = [int(rank[h]) for h in wide_list]
    mem_irank = rank[mem_node] if len(mem_node) else np.zeros(0, np.int64)
    iset_vb = np.array([vb_of[s_] for s_ in sets], dtype=np.int64)
    tmpl_vs = np.zeros(N)
    tmpl_vs[vslot] = tmpl

    def chance_arrays(lst):
        lst = np.array(lst, dtype=np.int64)
        if len(lst) == 0:
            z = np.zeros(0, np.int32)
            return z, z, z
        return (vslot[child_begin[lst]].astype(np.int32), (child_begin[lst + 1] - child_begin[lst]).astype(np.int32),
                vslot[lst].astype(np.int32))
    ch_vb, ch_nch, ch_vs = chance_arrays(chance_list)
    wide_vb, wide_nch, wide_vs = chance_arrays(wide_list)
    return {
        "vslot": vslot.astype(np.int32), "iset_vb": iset_vb.astype(np.int32),
        "mem_vs": (vslot[mem_node] if len(mem_node) else np.zeros(0, np.int64)).astype(np.int32),
        "ch_vb": ch_vb, "ch_nch": ch_nch, "ch_vs": ch_vs, "wide_vb": wide_vb, "wide_nch": wide_nch,
        "wide_vs": wide_vs, "tmpl_vs": tmpl_vs,
        "int_slot": np.array(int_slot, dtype=np.int32), "int_mask": np.array(int_mask, dtype=np.uint32).view(np.int32),
        "int_cirank": np.array(int_cirank, dtype=np.int32), "big_irank": np.array(big, dtype=np.int32),
        "int_edge": np.array(int_edge, dtype=np.int32), "wide_irank": np.array(wide_irank, dtype=np.int32),
        "iset_rank": iset_rank, "level_tiled": level_tiled,
        "mem_irank": mem_irank.astype(np.int32), "level_int": level_int,
        "child_begin": child_begin, "node_slot": node_slot, "level_begin": level_begin,
        "iset_slot": iset_slot, "iset_mem": iset_mem, "mem_node": mem_node,
        "chance_list": np.array(chance_list, dtype=np.int32), "level_chance": np.array(level_chance, dtype=np.int32),
        "level_iset": level_iset, "new_of_spec": new.astype(np.int32), "tmpl": tmpl, "spec_slot_of": spec_slot_of,
        "D": D, "wide_list": wide_list,
    }
