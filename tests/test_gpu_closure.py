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


def test_network_gains_over_the_tabulated_closure():
    """What the trained network adds to the fluid model's closure without it.  The method
    without the network is the tabulated (two-term) closure of Sec. IV.A (eqs. 8-13): from the
    local density and temperature it gives the electron flux, the energy flux and the
    ionization frequency.  The particle model's moment windows of four neon columns (1 Torr,
    6, 7.5, 10.5 and 12 V/cm) train the network on that closure's residuals, and the column at
    9 V/cm is held out.  On the held-out column the tabulated closure alone predicts a zero
    residual.  The network's correction must remove most of the ionization residual (the
    particle model's ionization frequency departs systematically from the two-term table) and
    must not make the flux or the energy flux worse; at this size their residuals are mostly
    sampling noise (normalised errors 0.96 and 0.92 against 0.98 and 0.98 when written)."""
    import torch
    from paper_2202_03215_gb300 import screen as sc
    tab = sc.Table(sc.transport())
    T_range = (tab.Te[0], tab.Te[-1])
    base = w.config_neon_column(n_per_species=800_000, n_cells=512, L_m=0.06, sort_every=100, diag_every=10)
    fields = [600.0, 750.0, 900.0, 1050.0, 1200.0]
    held = 2
    params = [base.with_(E0_Vpm=E, column=k) for k, E in enumerate(fields)]
    mom, _ = cl.run_windows(params, warmup=2000, windows=6, window=3000)
    Xs, Ys, col = [], [], []
    for k, p in enumerate(params):
        mu = sc.mu_iN_neon(p.E0_Vpm / (cl.n_gas(p) * cl.TD))
        for m in mom[k]:
            X, Y = cl.residual_samples(m, p, tab, mu, T_range)
            Xs.append(X)
            Ys.append(Y)
            col.append(np.full(len(X), k))
    X, Y, col = np.concatenate(Xs), np.concatenate(Ys), np.concatenate(col)
    assert np.isfinite(X).all() and np.isfinite(Y).all()
    ts = np.maximum(np.std(Y, 0), 1e-30).astype(np.float32)
    Xn, Yn = (X / cl.FEATURE_SCALE).astype(np.float32), (Y / ts).astype(np.float32)
    tr, te = col != held, col == held
    perm = np.random.default_rng(0).permutation(np.nonzero(tr)[0])
    m = pb.Mlp(seed=3)
    m.train(torch.from_numpy(Xn[perm]).cuda(), torch.from_numpy(Yn[perm]).cuda(), batch=1024, steps=1500, lr=2e-3)
    Yh = m.forward(torch.from_numpy(Xn[te]).cuda()).cpu().numpy()
    mse_net = ((Yh - Yn[te]) ** 2).mean(0)
    mse_tab = (Yn[te] ** 2).mean(0)           # the tabulated closure alone: zero residual
    print("held-out residual MSE, network vs tabulated closure:", mse_net, mse_tab)
    assert mse_net[2] < 0.5 * mse_tab[2], (mse_net, mse_tab)      # ionization frequency
    assert mse_net[1] < mse_tab[1], (mse_net, mse_tab)            # energy flux
    assert mse_net[0] < mse_tab[0], (mse_net, mse_tab)            # electron flux
