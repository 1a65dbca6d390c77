"""Closure data (uniform-field swarms and self-consistent column windows,
produced by the GPU particle step) and the trained closure network."""
import numpy as np
import pytest

import paper_2202_03215_gb300 as pb
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import closure as cl
from paper_2202_03215_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


@pytest.fixture(scope="module")
def swarms():
    return cl.swarm_table([5.0, 10.0, 20.0, 40.0, 80.0], n=20000, relax=2000, windows=2, window=400)


def test_swarm_transport_trends(swarms):
    table, ps, mom = swarms
    eps = [s.mean_eps_eV for s in table]
    wd = [s.drift_mps for s in table]
    nu = [s.nu_iz for s in table]
    assert all(np.diff(eps) > 0) and all(np.diff(wd) > 0)      # heating and drift grow with E/N
    assert nu[-1] > nu[0] >= 0 and nu[-1] > 0
    # energy balance per electron in steady state: e E w = loss (eV/s), positive
    assert all(s.loss_eVps > 0 for s in table)


def test_samples_and_trained_network_beats_the_mean(swarms):
    import torch
    table, ps, mom = swarms
    Xs, Ts = cl.swarm_samples(ps, mom)
    p = w.config_neon_column(n_per_species=200_000, n_cells=512, L_m=0.06, sort_every=0, diag_every=10)
    Xc, Tc = cl.column_samples([p.with_(E0_Vpm=600.0, column=0), p.with_(E0_Vpm=900.0, column=1)],
                               steps=2000, window=200, warmup=500)
    assert Xc.shape[1] == 15 and Tc.shape[1] == 3 and len(Xc) == 2 * 10 * 512
    X, T = cl.normalise(np.concatenate([Xs, Xc]), np.concatenate([Ts, Tc]))
    rng = np.random.default_rng(0)
    idx = rng.permutation(len(X))
    cut = int(0.9 * len(X))
    tr, te = idx[:cut], idx[cut:]
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    m = pb.Mlp(seed=1)
    m.train(Xd[tr].contiguous(), Td[tr].contiguous(), batch=1024, steps=600, lr=2e-3)
    Y = m.forward(Xd[te].contiguous()).cpu().numpy()
    err = ((Y - T[te]) ** 2).mean()
    base = ((T[te] - T[tr].mean(0)) ** 2).mean()
    assert err < 0.5 * base, (err, base)
