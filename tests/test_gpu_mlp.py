"""The closure network's GPU kernels (BF16 tensor-core forward/backward,
deterministic gradient reduction, Adam) against the CPU oracle network."""
import numpy as np
import pytest

import oracle
import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild

pytestmark = pytest.mark.gpu

GROUPS = {"W1": (0, 1920), "b1": (1920, 2048), "W2": (2048, 18432), "b2": (18432, 18560),
          "W3": (18560, 18944), "b3": (18944, 18947)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def _params(seed):
    rng = np.random.default_rng(seed)
    P = np.concatenate([rng.standard_normal(1920) / np.sqrt(15), 0.1 * rng.standard_normal(128),
                        rng.standard_normal(16384) / np.sqrt(128), 0.1 * rng.standard_normal(128),
                        rng.standard_normal(384) / np.sqrt(128), 0.1 * rng.standard_normal(3)])
    return P.astype(np.float32).astype(np.float64)


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 15)).astype(np.float32)
    T = np.stack([np.tanh(X[:, :5].sum(1)), np.sin(X[:, 5:10].sum(1)), X[:, 10:].mean(1) ** 2], 1)
    return X, T.astype(np.float32)


def test_gradients_match_the_oracle():
    import torch
    P = _params(11)
    X, T = _data(300, 12)          # 5 tiles of 64, the last one ragged
    m = pb.Mlp()
    m.set_params(P)
    loss, g = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    lo, _, go = oracle.mlp_forward_backward(P, X.astype(np.float64), T.astype(np.float64), bf16=True)
    assert abs(loss / lo - 1) < 1e-4
    for k, (a, b) in GROUPS.items():
        err = np.linalg.norm(g[a:b] - go[a:b]) / np.linalg.norm(go[a:b])
        assert err < 1e-2, (k, err)
    # and against the unrounded FP64 network: the BF16 rounding error
    _, _, g64 = oracle.mlp_forward_backward(P, X.astype(np.float64), T.astype(np.float64))
    assert np.linalg.norm(g - g64) < 5e-2 * np.linalg.norm(g64)


def test_forward_matches_the_oracle():
    import torch
    P = _params(13)
    X, T = _data(1000, 14)
    m = pb.Mlp()
    m.set_params(P)
    Y = m.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    _, yo, _ = oracle.mlp_forward_backward(P, X.astype(np.float64), T.astype(np.float64), bf16=True,
                                           want_grad=False)
    assert np.abs(Y - yo).max() < 2e-3 * np.abs(yo).max()


def test_gradients_are_deterministic_and_adam_steps_like_the_oracle():
    import torch
    P = _params(15)
    X, T = _data(512, 16)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    m = pb.Mlp()
    m.set_params(P)
    l1, g1 = m.grad(Xd, Td)
    l2, g2 = m.grad(Xd, Td)
    assert l1 == l2 and np.array_equal(g1, g2)
    m.train(Xd, Td, batch=512, steps=1, lr=1e-3)
    Pg = m.params().astype(np.float64)
    Q = P.copy()
    mo, vo = np.zeros_like(Q), np.zeros_like(Q)
    oracle.mlp_adam(Q, g1.astype(np.float64), mo, vo, 1)
    # first Adam step: every parameter moves by lr (sign of its gradient) up to eps effects
    big = np.abs(g1) > 1e-6
    assert np.allclose(Pg[big], Q[big], atol=2e-6)


def test_training_reduces_the_loss():
    import torch
    X, T = _data(16384, 17)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    m = pb.Mlp(seed=3)
    l0, _ = m.grad(Xd, Td)
    m.train(Xd, Td, batch=4096, steps=400, lr=2e-3)
    l1, _ = m.grad(Xd, Td)
    assert l1 < 0.3 * l0, (l0, l1)
