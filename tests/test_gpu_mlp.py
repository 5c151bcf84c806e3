"""Warm-start network kernels: BF16 tensor-core GEMM (all stride forms), the
network's gradients against the FP64 reference (tests/oracle), and training
that lowers the loss."""
import numpy as np
import pytest
import torch

from oracle import mlp_ref
from paper_2609_11923_gb300 import mlp as M

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k", [(100, 70, 50), (64, 64, 32), (257, 129, 300), (1, 8, 176)])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True)])
def test_gemm_matches_bf16_rounded_fp64_products(m, n, k, ta, tb):
    rng = np.random.default_rng(m * 7 + n + k)
    A = rng.standard_normal((k, m) if ta else (m, k)).astype(np.float32)
    B = rng.standard_normal((n, k) if tb else (k, n)).astype(np.float32)
    bias = rng.standard_normal(n).astype(np.float32)
    Ad, Bd, bd = (torch.tensor(x, device="cuda") for x in (A, B, bias))
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    sam, sak = (1, m) if ta else (k, 1)
    sbk, sbn = (1, k) if tb else (n, 1)
    s = int(torch.cuda.current_stream().cuda_stream)
    M._ck(M._lib.mlp_gemm(Ad.data_ptr(), 0, sam, sak, Bd.data_ptr(), 0, sbk, sbn, C.data_ptr(), None, n, m, n, k,
                          bd.data_ptr(), 1, 0, s))
    Aop = A.T if ta else A
    Bop = B.T if tb else B
    ref = np.maximum(mlp_ref.bf16_round(Aop) @ mlp_ref.bf16_round(Bop) + bias, 0.0)
    np.testing.assert_allclose(C.cpu().numpy(), ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())


def test_network_gradients_match_fp64_reference():
    rng = np.random.default_rng(0)
    B = 96
    X = rng.standard_normal((B, M.N_OUT * 22)).astype(np.float32)
    nact = rng.integers(1, M.N_OUT + 1, size=B).astype(np.int32)
    T = np.zeros((B, M.N_OUT), dtype=np.float32)
    for i in range(B):
        p = rng.random(nact[i])
        T[i, :nact[i]] = p / p.sum()
    net = M.MLP(X.shape[1], seed=3)
    loss = net.loss_and_grad(torch.tensor(X, device="cuda"), torch.tensor(nact, device="cuda"),
                             torch.tensor(T, device="cuda"))
    W, b = net.numpy_params()
    gW, gb = net.numpy_grads()
    rl, rW, rb = mlp_ref.loss_and_grads(W, b, X.astype(np.float64), nact, T.astype(np.float64), bf16=True)
    assert loss == pytest.approx(rl, rel=1e-4)
    # element by element: both sides round the same operands to BF16; what
    # is left is FP32 against FP64 accumulation and activations whose BF16
    # rounding flips on the last bit (2^-8 of one term), so each entry must
    # agree to 2% of itself or 0.5% of the tensor's largest entry
    for g, r in zip(gW + gb, rW + rb):
        np.testing.assert_allclose(g, r, rtol=2e-2, atol=5e-3 * np.abs(r).max())


def test_training_lowers_the_loss_on_a_fixed_task():
    rng = np.random.default_rng(1)
    n, F = 8192, M.N_OUT * 22
    X = rng.standard_normal((n, F)).astype(np.float32)
    Wt = rng.standard_normal((F, M.N_OUT)) * 0.5
    nact = np.full(n, 4, dtype=np.int32)
    z = X @ Wt
    z[:, 4:] = -np.inf
    T = np.exp(z - z.max(1, keepdims=True))
    T = (T / T.sum(1, keepdims=True)).astype(np.float32)
    from paper_2609_11923_gb300 import warmstart

    net = warmstart.train(np.pad(X, ((0, 0), (0, warmstart.F_IN - F))), nact, T, epochs=4, batch=1024, lr=3e-3)
    assert net.history[-1] < 0.6 * net.history[0]
