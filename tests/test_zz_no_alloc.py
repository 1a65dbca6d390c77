"""pic_field_periodic_noalloc: the field solve for callers that must not
allocate device memory during a call (cudaFree idles the whole device, and
pooled-memory callers may not allocate behind their pool).  It must give the
result of pic_field_periodic bit for bit, on consecutive calls that share its
fixed scratch array, and reject sizes beyond that array.

Collected last on purpose: a run that stops at the first failure has run
every other test before this one."""
import numpy as np
import pytest

import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild

pytestmark = pytest.mark.gpu

C_UNIT = 1.602176634e-19 * 5e8 / (8.8541878128e-12 * 2.0**32)


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def _charges(N, seed):
    import torch
    rng = np.random.default_rng(seed)
    qi = torch.from_numpy(rng.integers(0, 2**46, N, dtype=np.int64)).cuda()
    qe = torch.from_numpy(rng.integers(0, 2**46, N, dtype=np.int64)).cuda()
    return qi, qe


def test_noalloc_matches_allocating_entry_on_consecutive_calls():
    import torch
    # two calls in a row, larger then smaller, so stale scratch from the first would show in the second
    for N, seed, E0 in ((65536, 1, 600.0), (16384, 2, -250.0), (501, 3, 0.0)):
        qi, qe = _charges(N, seed)
        E_ref, Eh_ref = pb.field_periodic(qi, qe, C_UNIT, E0)
        E = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        Eh = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        pb.field_periodic_noalloc(qi, qe, C_UNIT, E0, E, Eh)
        assert torch.equal(E, E_ref) and torch.equal(Eh, Eh_ref), N


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    q = torch.zeros(65537, dtype=torch.int64, device="cuda")
    out = torch.empty(65537, dtype=torch.float64, device="cuda")
    with pytest.raises(pb.PicError):
        pb.field_periodic_noalloc(q, q, C_UNIT, 0.0, out, out)


def test_noalloc_binding_rejects_outputs_the_kernel_would_overrun():
    import torch
    qi, qe = _charges(1000, 4)
    good = torch.empty(1000, dtype=torch.float64, device="cuda")
    for bad in (torch.empty(1000, dtype=torch.float32, device="cuda"),
                torch.empty(999, dtype=torch.float64, device="cuda"),
                torch.empty(2000, dtype=torch.float64, device="cuda")[::2]):
        with pytest.raises(ValueError):
            pb.field_periodic_noalloc(qi, qe, C_UNIT, 0.0, bad, good)
        with pytest.raises(ValueError):
            pb.field_periodic_noalloc(qi, qe, C_UNIT, 0.0, good, bad)
    with pytest.raises(ValueError):
        pb.field_periodic_noalloc(qi, qe[:999], C_UNIT, 0.0, good, good)
