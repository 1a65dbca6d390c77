"""Pins of the oracle's closure network (15 -> 128 -> 128 -> 3, tanh-form GELU,
MSE, Adam) against torch's independent CPU implementation in float64:
outputs, loss and autograd gradients, and torch.optim.Adam steps."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


def _torch_net(P):
    W1 = torch.tensor(P[:1920].reshape(128, 15), dtype=torch.float64, requires_grad=True)
    b1 = torch.tensor(P[1920:2048], dtype=torch.float64, requires_grad=True)
    W2 = torch.tensor(P[2048:2048 + 16384].reshape(128, 128), dtype=torch.float64, requires_grad=True)
    b2 = torch.tensor(P[18432:18560], dtype=torch.float64, requires_grad=True)
    W3 = torch.tensor(P[18560:18944].reshape(3, 128), dtype=torch.float64, requires_grad=True)
    b3 = torch.tensor(P[18944:18947], dtype=torch.float64, requires_grad=True)
    return [W1, b1, W2, b2, W3, b3]


def _torch_loss(ps, X, T):
    W1, b1, W2, b2, W3, b3 = ps
    g = torch.nn.functional.gelu
    h = g(torch.as_tensor(X) @ W1.T + b1, approximate="tanh")
    h = g(h @ W2.T + b2, approximate="tanh")
    y = h @ W3.T + b3
    return ((y - torch.as_tensor(T)) ** 2).mean(), y


def _params(seed):
    rng = np.random.default_rng(seed)
    P = np.concatenate([rng.standard_normal(1920) / np.sqrt(15), 0.1 * rng.standard_normal(128),
                        rng.standard_normal(16384) / np.sqrt(128), 0.1 * rng.standard_normal(128),
                        rng.standard_normal(384) / np.sqrt(128), 0.1 * rng.standard_normal(3)])
    assert len(P) == oracle.MLP_NPARAM
    return P


def test_forward_and_gradients_match_torch_autograd():
    P = _params(1)
    rng = np.random.default_rng(2)
    X, T = rng.standard_normal((37, 15)), rng.standard_normal((37, 3))
    loss, y, g = oracle.mlp_forward_backward(P, X, T)
    ps = _torch_net(P)
    tl, ty = _torch_loss(ps, X, T)
    tl.backward()
    tg = np.concatenate([p.grad.numpy().ravel() for p in ps])
    assert loss == pytest.approx(tl.item(), rel=1e-12)
    assert np.allclose(y, ty.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert np.allclose(g, tg, rtol=1e-9, atol=1e-13)


def test_bf16_mode_rounds_but_stays_close():
    P = _params(3)
    rng = np.random.default_rng(4)
    X, T = rng.standard_normal((64, 15)), rng.standard_normal((64, 3))
    l64, _, g64 = oracle.mlp_forward_backward(P, X, T)
    lbf, _, gbf = oracle.mlp_forward_backward(P, X, T, bf16=True)
    assert lbf != l64 and abs(lbf / l64 - 1) < 2e-2
    assert np.linalg.norm(gbf - g64) < 3e-2 * np.linalg.norm(g64)


def test_adam_matches_torch():
    P = _params(5)
    rng = np.random.default_rng(6)
    X, T = rng.standard_normal((50, 15)), rng.standard_normal((50, 3))
    ps = _torch_net(P)
    opt = torch.optim.Adam(ps, lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m, v = np.zeros_like(P), np.zeros_like(P)
    Q = P.copy()
    for t in range(1, 4):
        _, _, g = oracle.mlp_forward_backward(Q, X, T)
        oracle.mlp_adam(Q, g, m, v, t)
        opt.zero_grad()
        tl, _ = _torch_loss(ps, X, T)
        tl.backward()
        opt.step()
    tp = np.concatenate([p.detach().numpy().ravel() for p in ps])
    assert np.allclose(Q, tp, rtol=1e-10, atol=1e-12)
