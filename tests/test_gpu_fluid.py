"""The GPU fluid screen (pic_fluid_*) against the oracle's fluid step
(Sec. IV.A, eqs. 3-5, 8-9, 11, 17): FP32 on the device, FP64 in the oracle.
Tolerances: the implicit solves are well conditioned (diagonally dominant),
so one FP32 step agrees to a few 1e-6 relative; 1e-5 after one step,
1e-4 after 40 steps, spectral modes to 1e-5 of the mean density."""
import numpy as np
import pytest

import paper_2202_03215_gb300 as pb
from oracle import fluid as fl
from oracle import two_term as tt
from paper_2202_03215_gb300 import build as pbuild
from paper_2202_03215_gb300 import workloads as w

pytestmark = pytest.mark.gpu

N_GAS = 3.219e22


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


@pytest.fixture(scope="module")
def records():
    xo = [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in w.neon_xsecs() if x.kind <= 2]
    out = []
    for en in np.geomspace(2.0, 200.0, 28):
        r = tt.solve(xo, w.AMU_NE, en, eps_max=200.0, n=800)
        out.append(dict(EN_Td=en, mean_eps_eV=r["mean_eps"], muN=r["muN"], DN=r["DN"], mueN=r["mueN"],
                        DeN=r["DeN"], nu_izN=r["nu_izN"], lossN=r["loss_N"], powerN=r["power_N"],
                        alphaN=r["alphaN"]))
    return out


def columns():
    return [dict(L_m=0.05, N_gas_m3=N_GAS, mu_iN=1.1e22, Gamma_T=1.5e20, nu_w=2e4, n_cells=64),
            dict(L_m=0.30, N_gas_m3=0.5 * N_GAS, mu_iN=1.1e22, Gamma_T=3e20, nu_w=5e4, n_cells=512),
            dict(L_m=0.30, N_gas_m3=2 * N_GAS, mu_iN=1.1e22, Gamma_T=2e20, nu_w=1e4, n_cells=4096),
            dict(L_m=0.10, N_gas_m3=N_GAS, mu_iN=1.3e22, Gamma_T=2e20, nu_w=0.0, n_cells=1024, loss=pb.FLUID_LOSS_PAIR),
            dict(L_m=0.20, N_gas_m3=N_GAS, mu_iN=1.2e22, Gamma_T=2.5e20, nu_w=3e4, n_cells=2048)]


def initial(N, seed):
    rng = np.random.default_rng(seed)
    x = np.arange(N) / N
    n = 1e16 * (1 + 0.02 * np.sin(2 * np.pi * 3 * x + rng.random()) + 0.01 * np.sin(2 * np.pi * 7 * x))
    T = 5.0 + 0.4 * np.sin(2 * np.pi * 2 * x + rng.random()) + 0.1 * np.cos(2 * np.pi * 11 * x)
    return n, T


def oracle_col(c):
    return dict(L_m=c["L_m"], N_gas=c["N_gas_m3"], mu_iN=c["mu_iN"], Gamma_T=c["Gamma_T"], nu_w=c["nu_w"],
                pair=c.get("loss", 0) == pb.FLUID_LOSS_PAIR)


@pytest.mark.parametrize("steps,tol", [(1, 1e-5), (40, 1e-4)])
def test_fluid_steps_match_oracle(records, steps, tol):
    cols = columns()
    dt = 2e-8
    f = pb.Fluid(cols, records, n_T=128, dt_s=dt, diag_every=10, n_modes=8)
    tab = fl.make_table(records, 128)
    states = []
    for k, c in enumerate(cols):
        n, T = initial(c["n_cells"], k)
        f.set_state(k, n, T)
        states.append((n, T))
    f.step(steps)
    rec = f.modes()
    assert rec.shape == (steps // 10, len(cols), 9)
    for k, c in enumerate(cols):
        n, T = states[k]
        omodes = []
        for s in range(steps):
            n, T = fl.step(oracle_col(c), tab, n, T, dt)
            if (s + 1) % 10 == 0:
                omodes.append(np.concatenate([[n.mean()], fl.modes(n, 8)]))
        gn, gT = f.get_state(k)
        assert np.max(np.abs(gn / n - 1)) < tol, (k, np.max(np.abs(gn / n - 1)))
        assert np.max(np.abs(gT / T - 1)) < tol, (k, np.max(np.abs(gT / T - 1)))
        for s, om in enumerate(omodes):
            assert np.max(np.abs(rec[s, k] - om)) < 1e-5 * om[0].real + tol * np.abs(om).max()
    ms, launches = f.elapsed()
    assert ms > 0 and launches >= 1
    f.close()


def test_fluid_features_match_oracle(records):
    import torch
    cols = columns()
    f = pb.Fluid(cols, records, n_T=128, dt_s=2e-8)
    tab = fl.make_table(records, 128)
    for k, c in enumerate(cols):
        f.set_state(k, *initial(c["n_cells"], k + 10))
    X = f.features().cpu().numpy()
    off = f.offsets
    for k, c in enumerate(cols):
        ox = fl.features(oracle_col(c), tab, *initial(c["n_cells"], k + 10))
        gx = X[off[k]:off[k + 1]]
        scale = np.abs(ox).max(axis=0)
        assert np.max(np.abs(gx - ox) / scale) < 1e-4, k
    f.close()


def test_fluid_corrections_match_oracle(records):
    import torch
    cols = columns()
    dt = 2e-8
    f = pb.Fluid(cols, records, n_T=128, dt_s=dt)
    tab = fl.make_table(records, 128)
    rng = np.random.default_rng(3)
    total = int(f.offsets[-1])
    corr = np.stack([2e3 * rng.standard_normal(total), 1e4 * rng.standard_normal(total),
                     5e3 * rng.standard_normal(total)], 1).astype(np.float32)
    f.set_corrections(torch.from_numpy(corr).cuda())
    for k, c in enumerate(cols):
        f.set_state(k, *initial(c["n_cells"], k + 20))
    f.step(5)
    for k, c in enumerate(cols):
        n, T = initial(c["n_cells"], k + 20)
        ck = corr[f.offsets[k]:f.offsets[k + 1]].astype(np.float64).T
        for _ in range(5):
            n, T = fl.step(oracle_col(c), tab, n, T, dt, corr=ck)
        gn, gT = f.get_state(k)
        # white-noise corrections make the explicit flux differences the largest right-hand-side
        # terms; FP32 rounds relative to them: the multi-step tolerance applies
        assert np.max(np.abs(gn / n - 1)) < 1e-4, k
        assert np.max(np.abs(gT / T - 1)) < 1e-4, k
    f.close()


@pytest.mark.parametrize("stencil", [1, 4])
def test_fluid_network_closure_matches_oracle(records, stencil):
    import torch
    from oracle import mlp_forward_backward
    cols = columns()[:2] + columns()[3:]
    dt, period = 2e-8, 4
    fs = np.array([1.0] * 5 + [10.0] * 5 + [50.0] * 5, dtype=np.float32)
    ts = np.array([1e3, 1e4, 1e3], dtype=np.float32)
    net = pb.Mlp(seed=5)
    f = pb.Fluid(cols, records, n_T=128, dt_s=dt)
    bound = 0.05                       # active: the random network's dnu exceeds 5% of nu_i in places
    f.set_closure(net, period, fs, ts, nu_bound=bound, stencil=stencil)
    for k, c in enumerate(cols):
        f.set_state(k, *initial(c["n_cells"], k + 30))
    f.step(2 * period)
    P = net.params().astype(np.float64)
    tab = fl.make_table(records, 128)
    for k, c in enumerate(cols):
        n, T = initial(c["n_cells"], k + 30)
        for _ in range(2):
            X = fl.features(oracle_col(c), tab, n, T, step=stencil) / fs
            Y = mlp_forward_backward(P, X, np.zeros((len(X), 3)), bf16=True, want_grad=False)[1]
            ck = (Y * ts).T
            for _ in range(period):
                nu = fl.coefficients(oracle_col(c), tab, T)["nu_i"]
                cb = ck.copy()
                cb[2] = np.clip(cb[2], -bound * nu, bound * nu)
                n, T = fl.step(oracle_col(c), tab, n, T, dt, corr=cb)
        gn, gT = f.get_state(k)
        assert np.max(np.abs(gn / n - 1)) < 1e-4, k
        assert np.max(np.abs(gT / T - 1)) < 1e-4, k
    _, launches = f.elapsed()
    assert launches == 2 + 2 * 2   # features + forward, then (chunk + forward) per period
    f.close()


def test_fluid_rejects_bad_columns(records):
    bad = dict(columns()[0], n_cells=100)
    with pytest.raises(pb.PicError):
        pb.Fluid([bad], records)
