"""The standalone periodic Poisson entry point (pic_field_periodic) on device
memory, bit-exact against the oracle's exact integer route, and the node
field formula E_j = (E_{j-1/2} + E_{j+1/2})/2 - E0."""
import numpy as np
import pytest

import oracle
import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


@pytest.mark.parametrize("N", [3, 97, 500, 16384, 30000, 65536])
def test_field_periodic_matches_oracle(N):
    import torch
    rng = np.random.default_rng(N)
    Qi = rng.integers(0, 2**46, N, dtype=np.int64)
    Qe = rng.integers(0, 2**46, N, dtype=np.int64)
    C = 1.602176634e-19 * 5e8 / (8.8541878128e-12 * 2.0**32)
    E0 = 600.0
    E, Eh = pb.field_periodic(torch.from_numpy(Qi).cuda(), torch.from_numpy(Qe).cuda(), C, E0)
    Eh_o = oracle.field_exact(Qi, Qe, C)
    assert np.array_equal(Eh.cpu().numpy(), Eh_o)
    E_o = 0.5 * (np.roll(Eh_o, 1) + Eh_o) + (-E0)
    assert np.array_equal(E.cpu().numpy(), E_o)


def test_field_periodic_rejects_bad_sizes():
    import torch
    q = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(pb.PicError):
        pb.field_periodic(q, q, 1.0, 0.0)
