"""Host side of the warm start (no GPU): the held-out games generated one at
a time are the games of the list, and the features of many games computed on
a thread pool equal the features computed one by one."""
import numpy as np

from paper_2609_11923_gb300 import warmstart as ws


def test_lazy_family_equals_the_list():
    seeds = list(range(20000, 20006))
    a = ws.endgame_family(seeds, 1e3, 1e5)
    b = list(ws.iter_endgame_family(iter(seeds), 1e3, 1e5))
    assert [g.n_edges for g in a] == [g.n_edges for g in b]
    for x, y in zip(a, b):
        assert np.array_equal(x.child, y.child) and np.array_equal(x.payoff, y.payoff)
        assert np.array_equal(x.chance_prob, y.chance_prob) and np.array_equal(x.infoset, y.infoset)


def test_features_are_per_game_and_order_free():
    from concurrent.futures import ThreadPoolExecutor

    games = ws.endgame_family(list(range(30000, 30008)), 1e3, 2e4)
    one = [ws.features(g, return_mass=True) for g in games]
    with ThreadPoolExecutor(4) as ex:
        many = list(ex.map(lambda g: ws.features(g, return_mass=True), games))
    for (x1, n1, m1), (x2, n2, m2) in zip(one, many):
        assert np.array_equal(x1, x2) and np.array_equal(n1, n2) and np.array_equal(m1, m2)
        assert x1.shape == (len(n1), ws.F_IN) and np.all(np.isfinite(x1))
        assert np.all(m1 > 0) and np.all(n1 >= 2)


def _chance_sums_by_definition(g, root_w):
    """Per spec set: the sum of its members' chance products (product of the
    chance probabilities on the path from the root), and of those times the
    weight of the root outcome above each member, by a plain walk."""
    N = g.n_nodes
    pc, owner = np.zeros(N), np.full(N, -1)
    pc[0] = 1.0
    stack = [0]
    while stack:
        h = stack.pop()
        for i, e in enumerate(range(g.child_begin[h], g.child_begin[h + 1])):
            c = int(g.child[e])
            pc[c] = pc[h] * (g.chance_prob[e] if g.kind[h] == 1 else 1.0)
            owner[c] = i if h == 0 else owner[h]
            stack.append(c)
    mass, wsum = np.zeros(g.n_infosets), np.zeros(g.n_infosets)
    for h in range(N):
        s = int(g.infoset[h])
        if s >= 0:
            mass[s] += pc[h]
            wsum[s] += pc[h] * root_w[owner[h]]
    return mass, wsum


def test_library_chance_sums_equal_the_definition():
    from paper_2609_11923_gb300 import cfr

    for g in ws.endgame_family([31000, 31001], 1e3, 2e4):
        n_root = int(g.child_begin[1] - g.child_begin[0])
        w = np.random.default_rng(0).uniform(0, 1, n_root)
        h = cfr.cfr_compile(g)
        try:
            mass, wsum = cfr.cfr_set_chance_sums(h, g.n_infosets, w)
        finally:
            cfr.cfr_destroy(h)
        m_ref, w_ref = _chance_sums_by_definition(g, w)
        np.testing.assert_allclose(mass, m_ref, rtol=1e-12, atol=0)
        np.testing.assert_allclose(wsum, w_ref, rtol=1e-12, atol=1e-300)
