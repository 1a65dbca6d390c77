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


def _gelu_d(z):
    c = np.sqrt(2 / np.pi)
    th = np.tanh(c * (z + 0.044715 * z ** 3))
    return 0.5 * (1 + th) + 0.5 * z * (1 - th * th) * c * (1 + 3 * 0.044715 * z * z)


def _gradient_magnitudes(P, X, T):
    """Per parameter, the sum over samples of the magnitudes of the terms its gradient adds up,
    with magnitudes carried through the backward chain (|dy| |W3| |gelu'| ... ): the scale of
    the rounding error each gradient element can collect (a running error bound)."""
    W1, b1 = P[:1920].reshape(128, 15), P[1920:2048]
    W2, b2 = P[2048:18432].reshape(128, 128), P[18432:18560]
    W3, b3 = P[18560:18944].reshape(3, 128), P[18944:]
    z1 = X @ W1.T + b1
    c = np.sqrt(2 / np.pi)
    a1 = 0.5 * z1 * (1 + np.tanh(c * (z1 + 0.044715 * z1 ** 3)))
    z2 = a1 @ W2.T + b2
    a2 = 0.5 * z2 * (1 + np.tanh(c * (z2 + 0.044715 * z2 ** 3)))
    y = a2 @ W3.T + b3
    dy = np.abs(2 * (y - T) / y.size)
    m3 = dy.T @ np.abs(a2)
    d2 = (dy @ np.abs(W3)) * np.abs(_gelu_d(z2))
    m2 = d2.T @ np.abs(a1)
    d1 = (d2 @ np.abs(W2)) * np.abs(_gelu_d(z1))
    m1 = d1.T @ np.abs(X)
    return np.concatenate([m1.ravel(), d1.sum(0), m2.ravel(), d2.sum(0), m3.ravel(), dy.sum(0)])


# Element-wise bound of the GPU gradient against the oracle's (which rounds the same operands to
# BF16): |g - g_oracle| <= C_BF16 * 2^-8 * (sum of the magnitudes of the gradient's terms).
# 2^-8 is one BF16 unit in the last place relative to the value; the GPU's FP32 sums and its
# hardware tanh can move a BF16 rounding to the neighbouring value on either factor of a term,
# and the errors of the layers above propagate into the lower layers' terms.
C_BF16 = 0.25   # measured worst 0.09 (W2) on a GB300


def _check_gradients(n, pseed, dseed):
    import torch
    P = _params(pseed)
    X, T = _data(n, dseed)
    m = pb.Mlp()
    m.set_params(P)
    loss, g = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    X64, T64 = X.astype(np.float64), T.astype(np.float64)
    lo, _, go = oracle.mlp_forward_backward(P, X64, T64, bf16=True)
    assert abs(loss / lo - 1) < 1e-4
    mag = _gradient_magnitudes(P, X64, T64)
    ratio = np.abs(g - go) / (2.0 ** -8 * mag + 1e-30)
    worst = {k: float(ratio[a:b].max()) for k, (a, b) in GROUPS.items()}
    print(f"n={n}: gradient error / (2^-8 sum|terms|), worst per group:", worst)
    for k, (a, b) in GROUPS.items():
        assert worst[k] <= C_BF16, (k, worst[k], int(np.argmax(ratio[a:b])))
    # and against the unrounded FP64 network: the BF16 rounding error
    _, _, g64 = oracle.mlp_forward_backward(P, X64, T64)
    assert np.linalg.norm(g - g64) < 5e-2 * np.linalg.norm(g64)


def test_gradients_match_the_oracle_element_by_element():
    _check_gradients(300, 11, 12)          # 3 tiles of 128, the last one ragged


def test_gradients_accumulated_over_several_tiles_per_cta():
    # 313 tiles of 128 (the last holds 64 samples) on at most one CTA per SM: every CTA
    # accumulates the weight gradients of two or three tiles in tensor memory
    _check_gradients(40000, 21, 22)


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
