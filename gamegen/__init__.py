"""Seeded synthetic games: the input generators shared by the oracle and the
CUDA path.

This module only builds game trees (structure, chance probabilities, payoffs,
information sets) in the tabular form of the paper's compiler input
(Appendix H, "Input representation"); it holds none of the CFR arithmetic.
The heavy generators are C (``gamegen.c``), compiled to ``libgamegen.so`` by
``gamegen.build``; :class:`GameSpec` can also be filled by hand for toy games.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

TERMINAL, CHANCE, P1, P2 = 0, 1, 2, 3
NFEAT = 16

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libgamegen.so")


@dataclass
class GameSpec:
    """A two-player zero-sum extensive-form game in tabular form.

    kind[N] (int8): TERMINAL / CHANCE / P1 / P2.  infoset[N] (int32): the
    acting player's information set at decision nodes, else -1.
    child_begin[N+1] (int64) / child[E] (int32): children in action order.
    chance_prob[E] (float64): outcome probabilities below chance nodes.
    payoff[N] (float64): payoff to player 1 at terminals.
    iset_player[I] (int8, 0 or 1) and iset_nact[I] (int32).
    pot: the normaliser of exploitability thresholds.
    iset_feat[I, 16] (int32, optional): small integer features of each set.
    Node 0 is the root.
    """

    kind: np.ndarray
    infoset: np.ndarray
    child_begin: np.ndarray
    child: np.ndarray
    chance_prob: np.ndarray
    payoff: np.ndarray
    iset_player: np.ndarray
    iset_nact: np.ndarray
    pot: float = 1.0
    iset_feat: Optional[np.ndarray] = None
    _owner: object = field(default=None, repr=False, compare=False)

    @property
    def n_nodes(self) -> int:
        return int(self.kind.shape[0])

    @property
    def n_edges(self) -> int:
        return int(self.child.shape[0])

    @property
    def n_infosets(self) -> int:
        return int(self.iset_player.shape[0])

    @property
    def n_slots(self) -> int:
        return int(self.iset_nact.sum())

    def slot_offsets(self) -> np.ndarray:
        """First slot of every information set in spec order (prefix sum)."""
        off = np.zeros(self.n_infosets + 1, dtype=np.int64)
        np.cumsum(self.iset_nact, out=off[1:])
        return off


class _Owner:
    def __init__(self, lib, ptr):
        self._lib, self._ptr = lib, ptr

    def __del__(self):
        try:
            self._lib.gg_free(self._ptr)
        except Exception:
            pass


class _CSpec(ctypes.Structure):
    _fields_ = [
        ("n_nodes", ctypes.c_int64),
        ("n_edges", ctypes.c_int64),
        ("n_infosets", ctypes.c_int64),
        ("kind", ctypes.POINTER(ctypes.c_int8)),
        ("infoset", ctypes.POINTER(ctypes.c_int32)),
        ("child_begin", ctypes.POINTER(ctypes.c_int64)),
        ("child", ctypes.POINTER(ctypes.c_int32)),
        ("chance_prob", ctypes.POINTER(ctypes.c_double)),
        ("payoff", ctypes.POINTER(ctypes.c_double)),
        ("iset_player", ctypes.POINTER(ctypes.c_int8)),
        ("iset_nact", ctypes.POINTER(ctypes.c_int32)),
        ("pot", ctypes.c_double),
        ("iset_feat", ctypes.POINTER(ctypes.c_int32)),
    ]


_lib = None


def build(verbose: bool = False) -> str:
    """Compile ``libgamegen.so`` next to this file (plain gcc, no GPU)."""
    import subprocess

    src = os.path.join(_HERE, "gamegen.c")
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(
        os.path.join(_HERE, "gamegen.c")
    ):
        build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.POINTER(_CSpec)
    lib.gg_tiny_card.restype = P
    lib.gg_tiny_card.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.gg_random_tree.restype = P
    lib.gg_random_tree.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int]
    lib.gg_large_card.restype = P
    lib.gg_large_card.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.gg_large_card_sampled.restype = P
    lib.gg_large_card_sampled.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.gg_endgame.restype = P
    lib.gg_endgame.argtypes = [ctypes.c_uint64, ctypes.c_int64]
    lib.gg_free.argtypes = [P]
    lib.gg_free.restype = None
    lib.gg_last_error.restype = ctypes.c_char_p
    lib.gg_rand.restype = ctypes.c_uint64
    lib.gg_rand.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
    _lib = lib
    return lib


def _wrap(ptr) -> GameSpec:
    lib = _load()
    if not ptr:
        raise RuntimeError("gamegen: " + (lib.gg_last_error() or b"").decode())
    s = ptr.contents
    n, e, ni = s.n_nodes, s.n_edges, s.n_infosets

    def view(p, count, shape=None):
        if count == 0:
            return np.zeros(shape or (0,), dtype=np.ctypeslib.as_ctypes_type(p._type_) and None)
        a = np.ctypeslib.as_array(p, shape=(count,))
        return a.reshape(shape) if shape else a

    owner = _Owner(lib, ptr)
    feat = None
    if s.iset_feat and ni > 0:
        feat = np.ctypeslib.as_array(s.iset_feat, shape=(ni * NFEAT,)).reshape(ni, NFEAT)
    return GameSpec(
        kind=np.ctypeslib.as_array(s.kind, shape=(n,)),
        infoset=np.ctypeslib.as_array(s.infoset, shape=(n,)),
        child_begin=np.ctypeslib.as_array(s.child_begin, shape=(n + 1,)),
        child=np.ctypeslib.as_array(s.child, shape=(max(e, 0),)) if e > 0 else np.zeros(0, np.int32),
        chance_prob=np.ctypeslib.as_array(s.chance_prob, shape=(e,)) if e > 0 else np.zeros(0),
        payoff=np.ctypeslib.as_array(s.payoff, shape=(n,)),
        iset_player=np.ctypeslib.as_array(s.iset_player, shape=(ni,)) if ni > 0 else np.zeros(0, np.int8),
        iset_nact=np.ctypeslib.as_array(s.iset_nact, shape=(ni,)) if ni > 0 else np.zeros(0, np.int32),
        pot=float(s.pot),
        iset_feat=feat,
        _owner=owner,
    )


def spec_digest(g: GameSpec) -> str:
    """SHA-256 of a game spec's arrays (dtype and bytes, in field order) and
    its pot: the key under which stored expected values of a game are kept."""
    import hashlib

    h = hashlib.sha256()
    for name, dt in (("kind", np.int8), ("infoset", np.int32), ("child_begin", np.int64), ("child", np.int32),
                     ("chance_prob", np.float64), ("payoff", np.float64), ("iset_player", np.int8),
                     ("iset_nact", np.int32)):
        a = np.ascontiguousarray(getattr(g, name), dtype=dt)
        h.update(name.encode())
        h.update(str(a.shape[0]).encode())
        h.update(memoryview(a).cast("B"))
    h.update(repr(float(g.pot)).encode())
    return h.hexdigest()


def tiny_card(ranks: int = 5, cap: int = 2) -> GameSpec:
    """One-card poker (5 ranks, cap 2 bets: N=301, 30 infosets, 70 slots)."""
    return _wrap(_load().gg_tiny_card(ranks, cap))


def kuhn() -> GameSpec:
    """Kuhn poker: the one-card game with 3 ranks and one bet."""
    return tiny_card(3, 1)


def random_tree(seed: int, depth: int = 14, bmin: int = 2, bmax: int = 4, p_chance: float = 0.2,
                max_group: int = 16) -> GameSpec:
    """Seeded random perfect-recall tree (depth 14 gives about 2.4M edges)."""
    return _wrap(_load().gg_random_tree(seed, depth, bmin, bmax, p_chance, max_group))


def large_card(n_ranks: int = 8, n_suits: int = 4, stack: int = 2, cap: int = 3) -> GameSpec:
    """Two-round card game (8x4 deck, stack 2 antes: 264,306,001 nodes)."""
    return _wrap(_load().gg_large_card(n_ranks, n_suits, stack, cap))


def large_card_sampled(deal_stride: int, n_ranks: int = 8, n_suits: int = 4, stack: int = 2,
                       cap: int = 3) -> GameSpec:
    """The two-round card game on every deal_stride-th root deal (a uniform sample)."""
    return _wrap(_load().gg_large_card_sampled(n_ranks, n_suits, stack, cap, deal_stride))


def endgame(seed: int, target_edges: int = 0) -> GameSpec:
    """One-round endgame subgame; target_edges=0 draws it log-uniformly in [1e3, 1e6]."""
    return _wrap(_load().gg_endgame(seed, target_edges))


def leduc() -> GameSpec:
    """Leduc poker: six cards (three ranks, two suits), ante 1 each, one
    private card each (dealt to player 1, then to player 2), a betting round
    with bets of 2, a public card, a betting round with bets of 4; at most
    two bets per round, player 1 acts first in both; folding only facing a
    bet. A private card pairing the public card wins, else the higher rank;
    equal ranks split. Information sets hold the acting player's own card,
    the public card and the betting so far: 936 sets, 1,093 sequences per
    player, 9,457 nodes."""
    n_cards, rank = 6, [0, 0, 1, 1, 2, 2]
    nodes, isets, index = [], [], {}

    def new_node():
        nodes.append(None)
        return len(nodes) - 1

    def info_set(key, player, n_act):
        if key not in index:
            index[key] = len(isets)
            isets.append((player, n_act))
        return index[key]

    def showdown(c1, c2, pub, put):
        s1 = (int(rank[c1] == rank[pub]), rank[c1])
        s2 = (int(rank[c2] == rank[pub]), rank[c2])
        return float(put[1]) if s1 > s2 else (-float(put[0]) if s2 > s1 else 0.0)

    def bet_round(c1, c2, pub, rnd, hist, put, me, bets, checks):
        h = new_node()
        owe = put[1 - me] - put[me]
        acts = (["f"] if owe > 0 else []) + ["c"] + (["r"] if bets < 2 else [])
        key = (me, c1 if me == 0 else c2, pub, hist)
        kids = []
        for a in acts:
            if a == "f":  # the folder loses what it put in
                kids.append(len(nodes))
                nodes.append((TERMINAL, -1, [], None, -float(put[0]) if me == 0 else float(put[1])))
            elif a == "c":
                now = list(put)
                now[me] = put[1 - me]
                if owe > 0 or checks == 1:  # the round is over
                    if rnd == 0:
                        kids.append(public_card(c1, c2, hist + "c/", now))
                    else:
                        kids.append(len(nodes))
                        nodes.append((TERMINAL, -1, [], None, showdown(c1, c2, pub, now)))
                else:
                    kids.append(bet_round(c1, c2, pub, rnd, hist + "c", now, 1 - me, bets, checks + 1))
            else:
                now = list(put)
                now[me] = put[1 - me] + (2 if rnd == 0 else 4)
                kids.append(bet_round(c1, c2, pub, rnd, hist + "r", now, 1 - me, bets + 1, 0))
        nodes[h] = (P1 if me == 0 else P2, info_set(key, me, len(acts)), kids, None, 0.0)
        return h

    def public_card(c1, c2, hist, put):
        h = new_node()
        left = [c for c in range(n_cards) if c not in (c1, c2)]
        kids = [bet_round(c1, c2, p, 1, hist, put, 0, 0, 0) for p in left]
        nodes[h] = (CHANCE, -1, kids, [1.0 / len(left)] * len(left), 0.0)
        return h

    root = new_node()
    firsts = []
    for c1 in range(n_cards):
        h = new_node()
        seconds = [bet_round(c1, c2, -1, 0, "", [1, 1], 0, 0, 0) for c2 in range(n_cards) if c2 != c1]
        nodes[h] = (CHANCE, -1, seconds, [1.0 / (n_cards - 1)] * (n_cards - 1), 0.0)
        firsts.append(h)
    nodes[root] = (CHANCE, -1, firsts, [1.0 / n_cards] * n_cards, 0.0)
    return from_lists(nodes, isets, pot=2.0)


def rand_u64(seed: int, stream: int, i: int) -> int:
    """The counter-based SplitMix64 word every generator draws from."""
    return int(_load().gg_rand(seed, stream, i))


def from_lists(nodes, infosets, pot: float = 1.0) -> GameSpec:
    """Build a small spec by hand.

    nodes: list of (kind, infoset, [children], [chance probs] or None, payoff).
    infosets: list of (player, n_actions).
    """
    n = len(nodes)
    kind = np.array([x[0] for x in nodes], dtype=np.int8)
    iset = np.array([x[1] for x in nodes], dtype=np.int32)
    cb = np.zeros(n + 1, dtype=np.int64)
    ch, cp = [], []
    for i, x in enumerate(nodes):
        cb[i] = len(ch)
        ch.extend(x[2])
        probs = x[3] if x[3] is not None else [0.0] * len(x[2])
        cp.extend(probs)
    cb[n] = len(ch)
    return GameSpec(
        kind=kind,
        infoset=iset,
        child_begin=cb,
        child=np.array(ch, dtype=np.int32),
        chance_prob=np.array(cp, dtype=np.float64),
        payoff=np.array([float(x[4]) for x in nodes], dtype=np.float64),
        iset_player=np.array([p for p, _ in infosets], dtype=np.int8),
        iset_nact=np.array([a for _, a in infosets], dtype=np.int32),
        pot=pot,
    )


def permute_nodes(g: GameSpec, perm: np.ndarray) -> GameSpec:
    """Relabel node ids (new id of old node v is perm[v]); the root must stay 0.

    The game is unchanged; only the tabular order differs. Used to check that
    compilation does not depend on the input numbering.
    """
    perm = np.asarray(perm, dtype=np.int64)
    assert perm[0] == 0
    n = g.n_nodes
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    nch = np.diff(g.child_begin)
    new_nch = nch[inv]
    cb = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(new_nch, out=cb[1:])
    child = np.empty_like(g.child)
    cprob = np.empty_like(g.chance_prob)
    for new in range(n):
        old = inv[new]
        a, b = g.child_begin[old], g.child_begin[old + 1]
        child[cb[new]:cb[new + 1]] = perm[g.child[a:b]]
        cprob[cb[new]:cb[new + 1]] = g.chance_prob[a:b]
    return GameSpec(
        kind=g.kind[inv].copy(), infoset=g.infoset[inv].copy(), child_begin=cb, child=child,
        chance_prob=cprob, payoff=g.payoff[inv].copy(), iset_player=g.iset_player.copy(),
        iset_nact=g.iset_nact.copy(), pot=g.pot,
        iset_feat=None if g.iset_feat is None else g.iset_feat.copy(),
    )


def validate(g: GameSpec) -> None:
    """Structural checks of a spec (tree, infoset consistency, probabilities)."""
    n = g.n_nodes
    assert g.child_begin[0] == 0 and g.child_begin[-1] == g.n_edges
    nch = np.diff(g.child_begin)
    assert (nch >= 0).all()
    parents = np.zeros(n, dtype=np.int64)
    np.add.at(parents, g.child, 1)
    assert parents[0] == 0 and (parents[1:] == 1).all(), "not a tree"
    term = g.kind == TERMINAL
    assert (nch[term] == 0).all() and (nch[~term] > 0).all()
    dec = (g.kind == P1) | (g.kind == P2)
    assert (g.infoset[dec] >= 0).all() and (g.infoset[~dec] == -1).all()
    pl = (g.kind[dec] - P1).astype(np.int8)
    assert (g.iset_player[g.infoset[dec]] == pl).all()
    assert (g.iset_nact[g.infoset[dec]] == nch[dec]).all()
    seen = np.zeros(g.n_infosets, dtype=bool)
    seen[g.infoset[dec]] = True
    assert seen.all(), "information set without members"
    ch_nodes = np.nonzero(g.kind == CHANCE)[0]
    for v in ch_nodes[:100000]:
        p = g.chance_prob[g.child_begin[v]:g.child_begin[v + 1]]
        assert (p > 0).all() and abs(p.sum() - 1.0) < 1e-9
