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
