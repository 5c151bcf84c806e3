"""Sequence-form linear program for the game value — TEST INFRASTRUCTURE.

Pins the oracle from outside CFR: for any strategy profile the best-response
values bracket the game value, br2 <= v* <= br1 (the value certificate of
the paper's Appendix E, eq. (valuecert)), and exploitability -> 0 must drive
u(sigma_bar) to v*.

Formulation (player-1 realization plan x, player-2 plan y, payoff matrix
A[s1, s2] = sum of pi_c(z) u(z) over terminals z whose last own sequences are
s1 and s2):  v* = max_x min_y x^T A y  subject to  E x = e, F y = f,
x, y >= 0.  Dualising the inner minimum gives one LP in (x, q):
maximise f^T q  s.t.  E x = e, x >= 0, F^T q - A^T x <= 0.
Solved with SciPy's HiGHS.
"""
from __future__ import annotations

import numpy as np
import scipy.optimize
import scipy.sparse as sp

TERMINAL, CHANCE, P1, P2 = 0, 1, 2, 3


def sequence_form(spec):
    """(E, e, F, f, A) of the game; sequence 0 is the empty sequence."""
    off = np.zeros(spec.n_infosets + 1, dtype=np.int64)
    np.cumsum(spec.iset_nact, out=off[1:])
    # per-player sequence ids: 1 + rank of the slot among the player's slots
    seq_id = np.full(int(off[-1]), -1, dtype=np.int64)
    nseq = [1, 1]
    for I in range(spec.n_infosets):
        p = int(spec.iset_player[I])
        for a in range(int(spec.iset_nact[I])):
            seq_id[off[I] + a] = nseq[p]
            nseq[p] += 1
    parent_seq = np.full(spec.n_infosets, -1, dtype=np.int64)
    rows = {0: ([], [], []), 1: ([], [], [])}
    Arow, Acol, Aval = [], [], []
    stack = [(0, 0, 0, 1.0)]  # node, last seq of p1, last seq of p2, chance product
    while stack:
        h, s1, s2, pc = stack.pop()
        k = int(spec.kind[h])
        b, e = int(spec.child_begin[h]), int(spec.child_begin[h + 1])
        if k == TERMINAL:
            Arow.append(s1)
            Acol.append(s2)
            Aval.append(pc * float(spec.payoff[h]))
            continue
        if k == CHANCE:
            for q in range(b, e):
                stack.append((int(spec.child[q]), s1, s2, pc * float(spec.chance_prob[q])))
            continue
        I = int(spec.infoset[h])
        p = k - P1
        own = s1 if p == 0 else s2
        if parent_seq[I] < 0:
            parent_seq[I] = own
        elif parent_seq[I] != own:
            raise ValueError("game does not have perfect recall")
        for a, q in enumerate(range(b, e)):
            sid = int(seq_id[off[I] + a])
            stack.append((int(spec.child[q]), sid if p == 0 else s1, sid if p == 1 else s2, pc))
    mats = []
    for p in (0, 1):
        r, c, v = [0], [0], [1.0]
        row = 1
        for I in range(spec.n_infosets):
            if int(spec.iset_player[I]) != p:
                continue
            r.append(row); c.append(int(parent_seq[I])); v.append(-1.0)
            for a in range(int(spec.iset_nact[I])):
                r.append(row); c.append(int(seq_id[off[I] + a])); v.append(1.0)
            row += 1
        M = sp.csr_matrix((v, (r, c)), shape=(row, nseq[p]))
        rhs = np.zeros(row)
        rhs[0] = 1.0
        mats.append((M, rhs))
    A = sp.csr_matrix((Aval, (Arow, Acol)), shape=(nseq[0], nseq[1]))
    (E, e), (F, f) = mats
    return E, e, F, f, A


def game_value(spec) -> float:
    """v* = max over player 1 of min over player 2 of the expected payoff."""
    E, e, F, f, A = sequence_form(spec)
    n1, m2 = E.shape[1], F.shape[0]
    c = np.concatenate([np.zeros(n1), -f])
    A_ub = sp.hstack([-A.T, F.T]).tocsr()
    b_ub = np.zeros(A_ub.shape[0])
    A_eq = sp.hstack([E, sp.csr_matrix((E.shape[0], m2))]).tocsr()
    bounds = [(0, None)] * n1 + [(None, None)] * m2
    res = scipy.optimize.linprog(c, A_ub=A_ub, b_ub=b_ub, A_eq=A_eq, b_eq=e, bounds=bounds,
                                 method="highs")
    if res.status != 0:
        raise RuntimeError("sequence-form LP failed: " + res.message)
    return float(-res.fun)
