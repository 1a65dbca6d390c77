"""The bounded waits of the closure network's kernels run out cleanly.

A test hook arms a wait on an mbarrier on which nothing is ever issued (no bulk copy of
the weights for the training kernel, no MMA for one group of the tensor-core forward
kernel) and caps the polls at a few, so the wait gives up within microseconds with
nothing left in flight.  The call must return PIC_ETIMEOUT without touching the
parameters, the error must latch on the handle, and pic_mlp_set_params must clear it,
after which the network computes exactly what an untouched network computes.  No GPU
fault is involved: the wait simply finds its barrier incomplete."""
import numpy as np
import pytest

import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild

pytestmark = pytest.mark.gpu

PIC_ETIMEOUT = -6


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def _data(n, seed):
    import torch
    rng = np.random.default_rng(seed)
    X = torch.from_numpy(rng.standard_normal((n, 15)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.standard_normal((n, 3)).astype(np.float32)).cuda()
    return X, T


def test_training_weight_wait_gives_up_latches_and_clears():
    X, T = _data(700, 1)
    ref = pb.Mlp(seed=5)
    l_ref, g_ref = ref.grad(X, T)
    m = pb.Mlp(seed=5)
    P0 = m.params()
    m.test_hook(pb.MLP_HOOK_NO_WEIGHT_COPY, spin=4)
    with pytest.raises(pb.PicError) as e:
        m.train(X, T, batch=256, steps=2)
    assert e.value.code == PIC_ETIMEOUT
    assert np.array_equal(m.params(), P0)          # no Adam step was applied
    m.test_hook(0, 0)
    with pytest.raises(pb.PicError) as e:          # latched until the parameters are set again
        m.grad(X, T)
    assert e.value.code == PIC_ETIMEOUT
    m.set_params(P0)
    l1, g1 = m.grad(X, T)
    assert l1 == l_ref and np.array_equal(g1, g_ref)


def test_forward_mma_wait_gives_up_latches_and_clears():
    X, _ = _data(5000, 2)
    ref = pb.Mlp(seed=6)
    Y_ref = ref.forward(X).cpu().numpy()
    m = pb.Mlp(seed=6)
    P0 = m.params()
    m.test_hook(pb.MLP_HOOK_NO_FORWARD_MMA, spin=4)
    with pytest.raises(pb.PicError) as e:
        m.forward(X)
    assert e.value.code == PIC_ETIMEOUT
    m.test_hook(0, 0)
    with pytest.raises(pb.PicError) as e:
        m.forward(X)
    assert e.value.code == PIC_ETIMEOUT
    m.set_params(P0)
    assert np.array_equal(m.forward(X).cpu().numpy(), Y_ref)


def test_hook_arguments_are_checked():
    m = pb.Mlp(seed=1)
    with pytest.raises(pb.PicError):
        m.test_hook(1 << 5, 4)
    with pytest.raises(pb.PicError):
        m.test_hook(0, -1)
