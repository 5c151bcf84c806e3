"""Learned warm start: the trained network gains over cold-start CFR+.

Small instance of the full pipeline: solve training endgames with the batched
kernels, train the MLP with the library's BF16 kernels, seed held-out solves
with R0 = kappa * pot * mass(I) * sigma_hat and compare the iterations to
1e-3 pot exploitability against cold starts on the same games (the cold
start stays the judge).
"""
import numpy as np
import pytest

from paper_2609_11923_gb300 import warmstart as ws

pytestmark = pytest.mark.gpu


def test_warm_start_needs_fewer_iterations_than_cold_start():
    train = ws.endgame_family(list(range(10000, 11200)), 1e3, 3e4)
    X, na, T = ws.make_dataset(train, iters=1000)
    net = ws.train(X, na, T, epochs=4)
    assert net.history[-1] < net.history[0]
    held = ws.endgame_family(list(range(20000, 20064)), 1e3, 3e4)
    cold, cold_fin, _ = ws.iterations_to_target(held, max_iters=3000)
    warm, warm_fin, _ = ws.iterations_to_target(held, init=[ws.warm_regrets(net, sp, 8.0) for sp in held],
                                                max_iters=3000)
    assert np.mean(warm) < np.mean(cold)
    assert warm_fin.mean() >= cold_fin.mean()


def test_features_are_finite_and_shaped():
    g = ws.endgame_family([5], 1e3, 1e4)[0]
    X, na = ws.features(g)
    assert X.shape == (g.n_infosets, ws.F_IN) and np.isfinite(X).all()
    assert (na == g.iset_nact).all()
    # private cards two-hot, equity in [0, 1] with exactly one bucket set
    assert (X[:, :32].sum(1) == 2).all()
    assert ((X[:, 172] >= 0) & (X[:, 172] <= 1)).all() and (X[:, 173:183].sum(1) == 1).all()
