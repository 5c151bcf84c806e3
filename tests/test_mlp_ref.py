"""The FP64 reference of the warm-start network, pinned by central finite
differences (no GPU)."""
import numpy as np

from oracle import mlp_ref


def test_reference_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    dims = [6, 5, 4, 3]
    W = [rng.standard_normal((a, b)) * 0.7 for a, b in zip(dims[:-1], dims[1:])]
    b = [rng.standard_normal(d) * 0.1 for d in dims[1:]]
    X = rng.standard_normal((7, dims[0]))
    nact = np.array([3, 2, 3, 1, 3, 2, 3])
    T = np.zeros((7, 3))
    for i in range(7):
        p = rng.random(nact[i])
        T[i, :nact[i]] = p / p.sum()
    w = rng.random(7) + 0.5
    loss, gW, gb = mlp_ref.loss_and_grads(W, b, X, nact, T, w)
    eps = 1e-6
    for params, grads in ((W, gW), (b, gb)):
        for P, G in zip(params, grads):
            it = np.nditer(P, flags=["multi_index"])
            for _ in it:
                i = it.multi_index
                old = P[i]
                P[i] = old + eps
                lp = mlp_ref.loss_and_grads(W, b, X, nact, T, w)[0]
                P[i] = old - eps
                lm = mlp_ref.loss_and_grads(W, b, X, nact, T, w)[0]
                P[i] = old
                assert abs((lp - lm) / (2 * eps) - G[i]) < 1e-7


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.0e38], dtype=np.float32)
    r = mlp_ref.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0  # halfway between 1 and 1+2^-7 rounds to even (1.0)
    assert r[2] == 1.0 + 2 ** -7
    assert r[3] == -2.5
