#!/usr/bin/env python
"""Throughput of the PIC-MCC step on GB300: pushed particle-steps per second.

Workload: the periodic neon column, 1 Torr, 300 K, L = 0.30 m, 16384 cells,
2e7 electrons + 2e7 ions, dt = 4e-11 s, ions subcycled x10, particle state
int32 cell + FP32 offset/velocity (float4), FP64 field; synthetic analytic
neon-like cross sections stand in for the LXCat data.  A step is one pass of
the whole hot path: electron gather/push/collisions/deposit, the ion step on
every 10th step, births and paired removals, and the Poisson solve.  A pushed
particle-step counts every electron every step and every ion on its push steps.

python bench.py [--gpus N --steps K --warmup W] prints one JSON line.
--impl reference times the CPU oracle (the reference arm) instead.
Multi-GPU runs are independent replicas, one column per rank (no collective
in the data path); value = particle-steps of all ranks / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "particle-steps/s and % HBM roofline on 1 GB300 vs CPU oracle; batched vs serial"
UNIT = "particle-steps/s"
BYTES_PER_PUSH = 48  # float4 state read + write (32 B) + id read (8 B) + int32 cell read + write (8 B)
WORKLOAD = ("neon periodic column, 1 Torr 300 K, L=0.30 m, R=0.01 m, I=1 mA (field and density from eq. 2), "
            "16384 cells, 2e7 electrons + 2e7 ions, dt=4e-11 s, ions subcycled x10, PAIR losses, int32 cell + "
            "FP32 offset/velocity, FP64 Poisson")


def column_params(w, n_per_species: int, seed: int = 1, column: int = 0):
    """The neon column of the throughput workload: R = 1 cm carrying I = 1 mA; pic_init
    resolves the homogeneous field E0 and density n0 of eq. 2."""
    return w.config_neon_column(n_per_species=n_per_species, seed=seed, column=column, drive=w.DRIVE_RI,
                                I_A=1e-3)


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """Hash of the particle-step sources with comments and blank space removed (a comment edit
    does not change the kernel the traffic figure was taken on)."""
    import re
    h = hashlib.sha256()
    for f in ("pic_kernels.cu", "pic_device.cuh", "pic_internal.cuh"):
        src = (ROOT / "paper_2202_03215_gb300" / "csrc" / f).read_text()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(n_e: int):
    """DRAM bytes per launch of the electron step from the committed ncu summary,
    scaled to n_e electrons; None if the kernel changed since it was taken."""
    f = ROOT / "profiles" / "k_push_electron_neon_traffic.json"
    if not f.exists():
        return None
    d = json.loads(f.read_text())
    if d.get("source_sha") != kernel_source_hash():
        return None
    return float(d["dram_bytes_per_electron"]) * n_e


class Clocks:
    """SM clock and throttle reasons during the timed region, by read-only NVML queries from a
    sampling thread (every millisecond, plus one sample as it starts and one as it stops, so
    that even a few-millisecond window has samples); nvidia-smi sampling where NVML cannot be
    loaded."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.p = None
        self.nvml = self._nvml_handle(index)
        if self.nvml is not None:
            import threading
            self.stop_ev = threading.Event()
            self._sample()
            self.th = threading.Thread(target=self._loop, daemon=True)
            self.th.start()
            return
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def _nvml_handle(self, index: int):
        import ctypes as C
        try:
            L = C.CDLL("libnvidia-ml.so.1")
            if L.nvmlInit_v2() != 0:
                return None
            cnt = C.c_uint(0)
            if L.nvmlDeviceGetCount_v2(C.byref(cnt)) != 0 or cnt.value == 0:
                return None
            want = None
            try:
                import torch
                want = str(torch.cuda.get_device_properties(index).uuid).lower()
            except Exception:
                pass
            pick = None
            for i in range(cnt.value):
                h = C.c_void_p()
                if L.nvmlDeviceGetHandleByIndex_v2(i, C.byref(h)) != 0:
                    continue
                buf = C.create_string_buffer(96)
                if L.nvmlDeviceGetUUID(h, buf, 96) == 0 and want and want in buf.value.decode().lower():
                    pick = h
                    break
            if pick is None:
                h = C.c_void_p()
                if L.nvmlDeviceGetHandleByIndex_v2(index if cnt.value > index else 0, C.byref(h)) != 0:
                    return None
                pick = h
            reasons = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                L.nvmlDeviceGetCurrentClocksThrottleReasons
            self._L, self._reasons = L, reasons
            mx = C.c_uint(0)
            self.max_mhz = float(mx.value) if L.nvmlDeviceGetMaxClockInfo(pick, 1, C.byref(mx)) == 0 else None
            return pick
        except (OSError, AttributeError):
            return None

    def _sample(self):
        import ctypes as C
        mhz, r, mw = C.c_uint(0), C.c_ulonglong(0), C.c_uint(0)
        ok = self._L.nvmlDeviceGetClockInfo(self.nvml, 1, C.byref(mhz)) == 0
        self._reasons(self.nvml, C.byref(r))
        self._L.nvmlDeviceGetPowerUsage(self.nvml, C.byref(mw))
        if ok:
            self.rows.append((float(mhz.value), int(r.value), mw.value / 1e3))

    def _loop(self):
        while not self.stop_ev.wait(0.001):
            self._sample()

    def stop(self):
        if self.nvml is not None:
            self.stop_ev.set()
            self.th.join(5)
            self._sample()
            sm = [r[0] for r in self.rows]
            reasons = sorted({name for r in self.rows for bit, name in self.REASONS.items() if r[1] & bit})
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(self.rows), "source": "nvml",
                    "power_w_max": max(r[2] for r in self.rows) if self.rows else None}
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in Path(self.f.name).read_text().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi"}


def pushed_steps(s0: int, k: int, n_e: int, n_i: int, sub: int) -> int:
    ion_steps = sum(1 for s in range(s0, s0 + k) if sub > 0 and s % sub == 0)
    return k * n_e + ion_steps * n_i


def oracle_rate(n_per_species: int, steps: int, warmup: int = 1, seed: int = 1):
    """The CPU oracle as it stands (FP32-storage build, one thread) on a sample of the workload:
    (pushed particle-steps, seconds) of `steps` timed steps."""
    import oracle
    from paper_2202_03215_gb300 import workloads as w
    p = column_params(w, n_per_species, seed=seed)
    o = oracle.Oracle(p)                       # resolves eq. 2 with the oracle's own two-term solve
    o.step(warmup)
    s0 = o.stats()["step"]
    t = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t
    return pushed_steps(s0, steps, n_per_species, n_per_species, p.ion_subcycle), dt


def _oracle_worker(a):
    return oracle_rate(*a)


def oracle_rate_cores(n_per_species: int, steps: int, warmup: int = 1, procs: int | None = None):
    """The oracle on every host core: one process per core (spawned, so that no process is forked
    from one that has touched the GPU), each stepping its own sample of the column with its own
    seed.  Rate = the units of all processes / the longest process's timed seconds."""
    import multiprocessing as mp
    procs = procs or len(os.sched_getaffinity(0)) or 1
    if procs == 1:
        units, dt = oracle_rate(n_per_species, steps, warmup)
        return units / dt, dt, 1
    # one thread per process: the numerical libraries of each child stay single-threaded
    threads = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in threads}
    os.environ.update({k: "1" for k in threads})
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_worker, [(n_per_species, steps, warmup, 1 + k) for k in range(procs)])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    units = sum(u for u, _ in res)
    secs = max(d for _, d in res)
    return units / secs, secs, procs


def batched_vs_serial(pb, w, torch, steps: int, warmup: int, n_columns: int = 64):
    """The 64-column sweep (uneven L, p, I, particles; argon and neon) advanced as one
    batch (one launch per phase for all columns, graph-replayed ion cycles) and as 64
    lone columns stepped one after another on the same GPU."""
    cols = w.config_batch_sweep(n_columns=n_columns)
    sub = cols[0].ion_subcycle
    b = pb.Batch(cols)
    tuning = b.tune()                       # the autotuner's steps (it times candidate schedules)
    _, mult_e, mult_i = b.schedule()
    b.step(warmup)
    s0 = b.columns[0].stats()["step"]
    units = sum(pushed_steps(s0, steps, c.n_e0, c.n_i0, sub) for c in cols)
    ext = torch.cuda.ExternalStream(b.stream())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ext)
    b.step(steps)
    e1.record(ext)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    b.set_timing(True)
    b.kernel_times()                        # the counts so far (all steps since the batch was made)
    b.step(sub)
    launches = sum(v[1] for v in b.kernel_times().values())
    b.set_timing(False)
    b.close()
    lone = [pb.Column(c) for c in cols]
    for c in lone:
        c.step(warmup + 3)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for c in lone:
        c.step(steps)
    torch.cuda.synchronize()
    t_serial = time.perf_counter() - t
    for c in lone:
        c.close()
    return {"columns": n_columns, "steps": steps, "pushed_particle_steps": units,
            "batched": units / t_batch, "serial": units / t_serial, "unit": UNIT,
            "speedup": t_serial / t_batch, "launches_per_ion_cycle": launches,
            "schedule": {"tuning_steps": tuning, "ctas_per_sm_electrons": mult_e, "ctas_per_sm_ions": mult_i},
            "workload": "64 columns, seed 42: L 0.05-0.40 m, p 0.3-3 Torr, I 0.1-5 mA, 1e5-5e6 particles "
                        "per species, 2048-16384 cells, Ar/Ne alternating, dt 5e-12 s, MIXED"}


def bf16_peak():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return float(json.loads(p.read_text())["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


MLP_FWD_FLOP = 2 * (15 * 128 + 128 * 128 + 128 * 3)   # 37,376 per sample


def bounded_leg(pb, w, torch, steps: int = 1000, warmup: int = 200):
    """The bounded column of Sec. V (Fig. 18 conditions): neon 1 Torr, cathode-anode gap 15 cm,
    1000 cells, 5000 particles per cell and species, 270 V through 10 Ohm m^2, cathode emission
    10 A/m^2, loss frequency 1e6 s^-1."""
    p = w.Params(gas_mass_amu=w.AMU_NE, L_m=0.15, n_cells=1000, xsec=w.neon_xsecs(), dt_s=4e-11,
                 n_e0=5_000_000, n_i0=5_000_000, n0_m3=1e15, Te0_eV=2.0, drive=w.DRIVE_CIRCUIT, U_src=270.0,
                 E0_Vpm=1400.0,
                 R_ext_ohm_m2=10.0, loss_mode=w.LOSS_RADIAL, nu_w=1e6, flags=w.FLAG_BOUNDED, J_emit_Am2=10.0,
                 T_emit_eV=0.2, precision=w.MIXED, sort_every=250, eps_max_e_eV=200.0, capacity=8_000_000)
    col = pb.Column(p)
    col.step(warmup)
    st0 = col.stats()
    ext = torch.cuda.ExternalStream(col.stream())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ext)
    col.step(steps)
    e1.record(ext)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = col.stats()
    col.close()
    units = pushed_steps(st0["step"], steps, (st0["n_e"] + st["n_e"]) // 2, (st0["n_i"] + st["n_i"]) // 2,
                         p.ion_subcycle)
    return {"workload": "bounded neon column, 1 Torr, gap 0.15 m, 1000 cells, 5e6 + 5e6 particles, U = 270 V, "
                        "R = 10 Ohm m^2, J_emit = 10 A/m^2, nu_w = 1e6 s^-1, dt = 4e-11 s, MIXED",
            "steps": steps, "ms_per_step": ms / steps, "value": units / (ms / 1e3), "unit": UNIT,
            "n_e": st["n_e"], "n_i": st["n_i"], "V_D": st["E0"] * p.L_m,
            "absorbed_e": [a - b for a, b in zip(st["absorbed_e"], st0["absorbed_e"])],
            "absorbed_i": [a - b for a, b in zip(st["absorbed_i"], st0["absorbed_i"])],
            "emitted": st["emitted"] - st0["emitted"]}


def eepf_leg(pb, w, torch, n: int = 20_000_000, steps: int = 200, diag_every: int = 10):
    """Cost of the EEPF histogram (Sec. III.C) on the throughput column: the same diagnostic steps
    (moments every diag_every steps) with and without the 64 x 200 energy histogram."""
    p = column_params(w, n).with_(diag_every=diag_every)
    col = pb.Column(p)
    col.step(diag_every)
    ext = torch.cuda.ExternalStream(col.stream())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    snap = col.get_state()
    for on in (False, True):
        col.set_state(snap)
        if on:
            col.eepf_config(64, 200, 50.0)
        torch.cuda.synchronize()
        e0.record(ext)
        col.step(steps)
        e1.record(ext)
        torch.cuda.synchronize()
        out["ms_per_step_eepf" if on else "ms_per_step"] = e0.elapsed_time(e1) / steps
    c, ns = col.eepf()
    col.close()
    extra = (out["ms_per_step_eepf"] - out["ms_per_step"]) * diag_every
    return {"particles_per_species": n, "steps": steps, "diag_every": diag_every, "bins": [64, 201],
            "samples": ns, "counted": int(c.sum()), **out, "ms_per_sample_extra": extra}


def fluid_screen_leg(pb, torch, steps: int = 1000, warmup: int = 20, closure_steps: int = 200):
    """The fluid screen of a 32 x 32 grid of (pR, I/R) for neon columns (R = 1 cm, L = 0.30 m,
    4096 cells, FP32): homogeneous states from eq. 2 with seeded 1e-3 noise, pair losses, one batch.
    Timed with the handle's CUDA events; then the same screen with the closure network attached
    (random weights, ionization correction bounded to +-50 %, features -> network every 10 steps)."""
    from paper_2202_03215_gb300 import screen as sc
    recs = sc.transport()
    tab = sc.Table(recs)
    states = [sc.homogeneous_R(tab, pr, ir) for pr in np.geomspace(0.3, 3.0, 32) for ir in np.geomspace(0.01, 1.0, 32)]
    states = [h for h in states if np.isfinite(h.T0)]
    cols = sc.fluid_columns(states, 0.30, 4096)
    f = pb.Fluid(cols, recs, n_T=128, dt_s=2e-9, diag_every=50, n_modes=64)
    for k, h in enumerate(states):
        f.set_state(k, *sc.initial_state(4096, h, 100 + k))
    f.step(warmup)
    f.step(steps)
    ms, launches = f.elapsed()
    rec = f.modes()
    cells = len(cols) * 4096
    lin = [sc.linear(tab, h) for h in states]
    net = pb.Mlp(seed=3)
    ts = np.array([0.0, 0.0, 1e5], np.float32)
    f.set_closure(net, 10, np.array([1.0] * 5 + [10.0] * 5 + [50.0] * 5, np.float32), ts, 0.5)
    f.step(closure_steps)
    ms_c, launches_c = f.elapsed()
    f.close()
    net.close()
    inf_samples = cells * (closure_steps // 10 + 1)
    return {"columns": len(cols), "cells_per_column": 4096, "steps": steps,
            "column_steps_per_s": len(cols) * steps / (ms / 1e3), "cell_steps_per_s": cells * steps / (ms / 1e3),
            "ms_per_step": ms / steps, "launches": launches, "records": int(rec.shape[0]),
            "unstable_by_linear_theory": int(sum(1 for l in lin if l["unstable"])),
            "closure": {"steps": closure_steps, "period": 10, "ms_per_step": ms_c / closure_steps,
                        "launches": launches_c, "network_samples": inf_samples},
            "workload": "neon, R=1 cm, L=0.30 m, 4096 cells, pR 0.3-3 Torr cm x I/R 0.01-1 A/m (32x32 log grid), "
                        "homogeneous states from eq. 2, pair losses, dt=2e-9 s, FP32 (state as FP32 pairs), "
                        "spectral record every 50 steps"}


def closure_training_leg(pb, torch, n: int = 1 << 20, batch: int = 8192, steps: int = 300, warmup: int = 20,
                         big_steps: int = 100):
    """Adam training of the closure network on the GPU (BF16 operands, FP32 accumulation):
    forward + backward + deterministic gradient reduction + Adam per batch."""
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn((n, 15), device="cuda", generator=g)
    T = torch.randn((n, 3), device="cuda", generator=g)
    net = pb.Mlp(seed=9)
    net.train(X, T, batch=batch, steps=warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    net.train(X, T, batch=batch, steps=steps)
    e1.record()
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3
    sps = batch * steps / s
    tflops = 3 * MLP_FWD_FLOP * sps / 1e12
    peak, kind = bf16_peak()
    net.forward(X[:batch])
    torch.cuda.synchronize()
    e0.record()
    Yf = net.forward(X)
    e1.record()
    torch.cuda.synchronize()
    sf = e0.elapsed_time(e1) / 1e3
    # the same kernels with 64x the samples per Adam step (at most the data set): every SM holds
    # several tiles, and the step's fixed costs (partials, reduction, launches) are shared
    big = min(64 * batch, n)
    net.train(X, T, batch=big, steps=5)
    torch.cuda.synchronize()
    e0.record()
    net.train(X, T, batch=big, steps=big_steps)
    e1.record()
    torch.cuda.synchronize()
    sb = big * big_steps / (e0.elapsed_time(e1) / 1e3)
    return {"batch": batch, "steps": steps, "samples_per_s": sps, "tflops": tflops,
            "frac_of_bf16_peak": tflops / peak, "peak_tflops": peak, "peak_kind": kind,
            "flop_per_sample": 3 * MLP_FWD_FLOP,
            "large_batch": {"batch": big, "steps": big_steps, "samples_per_s": sb,
                            "tflops": 3 * MLP_FWD_FLOP * sb / 1e12,
                            "frac_of_bf16_peak": 3 * MLP_FWD_FLOP * sb / 1e12 / peak},
            "forward": {"samples": n, "samples_per_s": n / sf, "tflops": MLP_FWD_FLOP * n / sf / 1e12}}


def timed_steps(col, torch, steps: int):
    """Device milliseconds of `steps` steps on the column's stream (CUDA events)."""
    ext = torch.cuda.ExternalStream(col.stream())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ext)
    col.step(steps)
    e1.record(ext)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def fp64_form_leg(pb, w, torch, n: int, steps: int = 300, warmup: int = 10):
    """The throughput column in the plain FP64 form (32-byte double records): the same steps as
    the precision form, and the electron step's fraction of the HBM bandwidth at 80 B per
    electron (double record read + write, int32 cell read + write, id read)."""
    p = column_params(w, n).with_(precision=w.FP64)
    col = pb.Column(p)
    col.step(warmup)
    st0 = col.stats()
    ms = timed_steps(col, torch, steps)
    col.set_timing(True)
    col.kernel_times()
    timed_steps(col, torch, steps)
    kt = col.kernel_times()
    col.close()
    units = pushed_steps(st0["step"], steps, st0["n_e"], st0["n_i"], p.ion_subcycle)
    push_ms, push_n = kt["push_e"]
    avg = push_ms / max(1, push_n) / 1e3
    peak, kind = peaks()
    return {"value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "electron_step_us": avg * 1e6, "bytes_per_electron": 80,
            "electron_step_frac_of_hbm": 80 * st0["n_e"] / avg / 1e9 / peak, "peak_kind": kind,
            "workload": "the throughput column with FP64 particle records"}


def small_column_leg(pb, w, torch, steps: int = 2000, warmup: int = 20):
    """The argon parity column (1 Torr, L = 5 cm, 500 cells, 1e5 + 1e5 particles, FP64, 20 V,
    dt = 2e-11 s): microseconds per step with the ion cycles replayed as CUDA graphs.  8.8 MB
    of state stay in L2, so the step is bound by launch latency, not by HBM."""
    p = w.config_argon_small()
    col = pb.Column(p)
    col.step(warmup)
    st0 = col.stats()
    ms = timed_steps(col, torch, steps)
    col.close()
    units = pushed_steps(st0["step"], steps, st0["n_e"], st0["n_i"], p.ion_subcycle)
    return {"us_per_step": ms * 1e3 / steps, "steps": steps, "value": units / (ms / 1e3), "unit": UNIT,
            "workload": "argon 1 Torr, L=0.05 m, 500 cells, 1e5 + 1e5 particles, FP64, V=20 V, dt=2e-11 s"}


def replica_params(w, rank: int, n_per_species: int):
    """The column of rank `rank` in a multi-GPU run: an independent replica of the neon column
    (its own seed and RNG column index), no data shared between ranks."""
    return column_params(w, n_per_species, seed=1 + rank, column=rank)


def aggregate(dist, torch, seconds: float, units: int, device: str = "cuda"):
    """Whole-job figures of a timed region: the slowest rank's time and the units of all ranks
    (identity without a process group)."""
    if dist is None:
        return seconds, units
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    # each step one oracle step of a sample of the workload on every host core, sized so that K
    # steps take about two minutes
    n = int(min(2_000_000, max(100_000, 120.0 * 2.5e7 / max(1, args.steps) / 1.1)))
    rate, dt, cores = oracle_rate_cores(n, args.steps, warmup=min(args.warmup, 3))
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "sample": f"{n} electrons + {n} ions per step and process (same cells, dt, gas), "
                                 f"{cores} processes"},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} oracle steps of {n}+{n} particles in each of {cores} "
                                       f"processes (one per core), {dt:.1f} s"},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=20_000_000, help="particles per species")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-screen", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-eepf", action="store_true")
    ap.add_argument("--no-bounded", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-steady", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import paper_2202_03215_gb300 as pb
    from paper_2202_03215_gb300 import build as pbuild
    from paper_2202_03215_gb300 import workloads as w
    pbuild.build()
    # the CPU baseline runs before the first GPU call of this process (rank 0, N=1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_s = 2_000_000
        steps_s = 40
        rate, dt, cores = oracle_rate_cores(n_s, steps_s)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{steps_s} oracle steps (FP32-storage build) of {n_s} electrons + {n_s} ions on the "
                         f"same column in each of {cores} processes (one per core, own seeds), "
                         f"{dt:.1f} s per process"}

    p = replica_params(w, rank, args.n)
    col = pb.Column(p)
    col.step(args.warmup)
    st0 = col.stats()
    snap = col.get_state()          # the second pass below replays the same steps from here
    ext = torch.cuda.ExternalStream(col.stream())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # timed region: the library's own path (ion cycles replayed as CUDA graphs)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(torch.cuda.current_device()) if rank == 0 else None
    e0.record(ext)
    col.step(args.steps)
    e1.record(ext)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop() if clk else None
    ms = e0.elapsed_time(e1)
    st1 = col.stats()
    units = pushed_steps(st0["step"], args.steps, st0["n_e"], st0["n_i"], p.ion_subcycle)
    assert st1["n_e"] == st0["n_e"] and st1["step"] == st0["step"] + args.steps
    # the same steps again (state restored: bit-exact replay) with a CUDA event around every
    # kernel (no graphs): the kernel breakdown, the launch count and the electron step's
    # average launch time
    col.set_state(snap)
    del snap
    col.set_timing(True)
    col.kernel_times()
    torch.cuda.synchronize()
    e0.record(ext)
    col.step(args.steps)
    e1.record(ext)
    torch.cuda.synchronize()
    ms_inst = e0.elapsed_time(e1)
    kt = col.kernel_times()
    col.set_timing(False)
    assert col.stats()["step"] == st1["step"]
    launches = sum(v[1] for v in kt.values())
    # the step amortised over a whole sort cycle: sort_every x ion_subcycle steps hold every
    # electron sort and ion sort of the cycle in their proportion
    cyc = p.sort_every * p.ion_subcycle
    torch.cuda.synchronize()
    e0.record(ext)
    col.step(cyc)
    e1.record(ext)
    torch.cuda.synchronize()
    amort = {"ms_per_step": e0.elapsed_time(e1) / cyc, "steps": cyc,
             "sorts": {"electrons": cyc // p.sort_every, "ions": 1}}
    ms, units = aggregate(dist, torch, ms, units)
    value = units / (ms / 1e3)

    # roofline of the dominant kernel (electron step), live from the timed region
    push_ms, push_n = kt["push_e"]
    n_e = st0["n_e"]
    avg_s = push_ms / max(1, push_n) / 1e3
    achieved = BYTES_PER_PUSH * n_e / avg_s / 1e9
    peak, peak_kind = peaks()
    traffic = ncu_traffic(n_e)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "k_push<float,electrons>", "peak_kind": peak_kind,
            "algorithmic_bytes_per_launch": BYTES_PER_PUSH * n_e, "avg_launch_us": avg_s * 1e6,
            "share_of_step": push_ms / ms_inst, "timed_with": "CUDA events around every kernel, second pass"}

    # steady state: the column continued (untimed) to step 4000, by which its electrons have heated
    # from the initial 2 eV to their steady mean energy (more collision candidates, more births
    # than right after the start), then 1000 steps timed under graph replay, and the same steps
    # again from a snapshot with a CUDA event around every kernel
    steady = None
    if not args.no_steady:
        cur = col.stats()["step"]
        if cur < 4000:
            col.step(4000 - cur)
        st_s = col.stats()
        snap = col.get_state()
        torch.cuda.synchronize()
        e0.record(ext)
        col.step(1000)
        e1.record(ext)
        torch.cuda.synchronize()
        ms_s = e0.elapsed_time(e1)
        units_s = pushed_steps(st_s["step"], 1000, st_s["n_e"], st_s["n_i"], p.ion_subcycle)
        col.set_state(snap)
        del snap
        col.set_timing(True)
        col.kernel_times()
        col.step(1000)
        kt_s = col.kernel_times()
        col.set_timing(False)
        avg_e = kt_s["push_e"][0] / max(1, kt_s["push_e"][1]) / 1e3
        steady = {"from_step": st_s["step"], "steps": 1000, "ms_per_step": ms_s / 1000,
                  "value": units_s / (ms_s / 1e3), "unit": UNIT, "electron_step_us": avg_e * 1e6,
                  "electron_step_frac": BYTES_PER_PUSH * st_s["n_e"] / avg_e / 1e9 / peak,
                  "kernel_us_per_step": {k: v[0] / 1000 * 1e3 for k, v in kt_s.items()}}

    # end to end through the public API with host buffers: upload the state, step, read moments
    e2e = None
    if not args.no_e2e:
        host = col.get_state()
        if p.precision == w.MIXED:
            # the precision form's storage: FP32 offsets and velocities (pic_set_state_f32)
            for k in ("off", "vx", "vy", "vz"):
                for sp in ("e", "i"):
                    host[f"{k}_{sp}"] = host[f"{k}_{sp}"].astype(np.float32)
        pinned = {}
        for k, v in host.items():
            if isinstance(v, np.ndarray):
                t = torch.empty(v.shape, dtype=getattr(torch, str(v.dtype)) if v.dtype != np.uint64 else torch.int64,
                                pin_memory=True)
                a = t.numpy().view(v.dtype)
                a[...] = v
                pinned[k] = (t, a)
        hstate = {k: (pinned[k][1] if k in pinned else v) for k, v in host.items()}
        col.close()
        col2 = pb.Column(p)
        local_units = pushed_steps(host["step"], args.steps, host["n_e"], host["n_i"], p.ion_subcycle)
        h2d = sum(a.nbytes for k, (t, a) in pinned.items() if k not in ("Q_e",))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        col2.set_state(hstate)
        col2.step(args.steps)
        mom = col2.moments()
        stx = col2.stats()
        t1 = time.perf_counter()
        d2h = sum(v.nbytes for v in mom.values() if isinstance(v, np.ndarray)) + 8 * 40
        secs = t1 - t0
        secs, local_units = aggregate(dist, torch, secs, local_units)
        e2e = {"value": local_units / secs, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "seconds": secs, "api": ("pic_set_state_f32" if p.precision == w.MIXED else "pic_set_state")
                      + " (host arrays) + pic_step(K) + pic_moments + pic_get_stats"}
        assert stx["step"] == host["step"] + args.steps
        col2.close()

    batch = None
    if rank == 0 and world == 1 and not args.no_batch:
        batch = batched_vs_serial(pb, w, torch, steps=200, warmup=min(args.warmup, 10))

    screen = train = None
    if rank == 0 and world == 1 and not args.no_screen:
        screen = fluid_screen_leg(pb, torch)
    eepf = None
    if rank == 0 and world == 1 and not args.no_eepf:
        eepf = eepf_leg(pb, w, torch, n=args.n)
    bnd = None
    if rank == 0 and world == 1 and not args.no_bounded:
        bnd = bounded_leg(pb, w, torch)
    if rank == 0 and world == 1 and not args.no_train:
        train = closure_training_leg(pb, torch)
    fp64 = small = None
    if rank == 0 and world == 1 and not args.no_fp64:
        fp64 = fp64_form_leg(pb, w, torch, n=args.n)
    if rank == 0 and world == 1 and not args.no_small:
        small = small_column_leg(pb, w, torch)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "particles_per_species": args.n, "n_cells": p.n_cells,
                           "eq2": {k: float(v) for k, v in pb.drive_ri(p).items()},
                           "l2": "inputs larger than L2 (state 1.1 GB)", "parallelism": f"replicas x{world}",
                           "pushed_particle_steps": units},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "batched_vs_serial": batch,
                "ms_per_step_amortized": amort, "steady_state": steady, "fp64_form": fp64, "argon_small_column": small,
                "fluid_screen": screen, "closure_training": train, "eepf": eepf, "bounded_column": bnd,
                "gpu_launches": launches, "ms_per_step_instrumented": ms_inst / args.steps,
                "kernel_ms": {k: v[0] for k, v in kt.items()}, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
