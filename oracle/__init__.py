"""ctypes wrapper of the CPU oracle (pic_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg.  The product path never imports this package.

Two builds of the same C file: FP64 particle storage, and FP32 particle
storage (ORACLE_F32) for the mixed-precision form.  Both are plain,
single-threaded, FP64 in the field.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "pic_oracle.c"
LIBS = {False: HERE / "liboracle_f64.so", True: HERE / "liboracle_f32.so"}
MLP_SRC = HERE / "mlp_oracle.c"
MLP_LIB = HERE / "libmlp_oracle.so"
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall"]


def build(force: bool = False) -> None:
    """Compile both oracle builds with gcc (no CUDA)."""
    if force or not MLP_LIB.exists() or MLP_LIB.stat().st_mtime < MLP_SRC.stat().st_mtime:
        subprocess.run(["gcc", *CFLAGS, "-o", str(MLP_LIB) + ".tmp", str(MLP_SRC), "-lm"], check=True)
        os.replace(str(MLP_LIB) + ".tmp", MLP_LIB)
    for f32, out in LIBS.items():
        if not force and out.exists() and out.stat().st_mtime > max(SRC.stat().st_mtime,
                                                                   (HERE / "pic_oracle.h").stat().st_mtime):
            continue
        cmd = ["gcc", *CFLAGS, *(["-DORACLE_F32"] if f32 else []), "-o", str(out) + ".tmp", str(SRC), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(str(out) + ".tmp", out)


class OraXsec(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32), ("threshold_eV", C.c_double),
                ("energy_eV", C.POINTER(C.c_double)), ("sigma_m2", C.POINTER(C.c_double))]


class OraParams(C.Structure):
    _fields_ = [("gas_mass_amu", C.c_double), ("pressure_torr", C.c_double), ("T_gas_K", C.c_double),
                ("L_m", C.c_double), ("R_m", C.c_double),
                ("drive", C.c_int32), ("field_mode", C.c_int32),
                ("E0_Vpm", C.c_double), ("V_applied", C.c_double), ("I_A", C.c_double),
                ("U_src", C.c_double), ("R_ext_ohm_m2", C.c_double),
                ("n_xsec", C.c_int32), ("pad0", C.c_int32), ("xsec", C.POINTER(OraXsec)),
                ("n_cells", C.c_int32), ("ion_subcycle", C.c_int32), ("dt_s", C.c_double),
                ("n_e0", C.c_int64), ("n_i0", C.c_int64), ("capacity", C.c_int64),
                ("n0_m3", C.c_double), ("Te0_eV", C.c_double), ("Ti0_eV", C.c_double),
                ("loss_mode", C.c_int32), ("precision", C.c_int32), ("nu_w", C.c_double),
                ("seed", C.c_uint64),
                ("diag_every", C.c_int32), ("sort_every", C.c_int32), ("n_table", C.c_int32),
                ("flags", C.c_int32),
                ("eps_max_e_eV", C.c_double), ("eps_max_i_eV", C.c_double),
                ("column", C.c_int32), ("pad1", C.c_int32),
                ("J_emit_Am2", C.c_double), ("T_emit_eV", C.c_double)]


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_U64 = C.POINTER(C.c_uint64)


class OraState(C.Structure):
    _fields_ = [("n_e", C.c_int64), ("n_i", C.c_int64), ("step", C.c_int64), ("next_id", C.c_int64),
                ("E0", C.c_double),
                ("cell_e", _I32), ("off_e", _D), ("vx_e", _D), ("vy_e", _D), ("vz_e", _D), ("id_e", _U64),
                ("cell_i", _I32), ("off_i", _D), ("vx_i", _D), ("vy_i", _D), ("vz_i", _D), ("id_i", _U64),
                ("E", _D), ("Q_e", _I64), ("Q_i", _I64)]


class OraStats(C.Structure):
    _fields_ = [("step", C.c_int64), ("n_e", C.c_int64), ("n_i", C.c_int64), ("next_id", C.c_int64),
                ("n_coll_e", C.c_int64 * 16), ("n_coll_i", C.c_int64 * 16),
                ("births", C.c_int64), ("losses_e", C.c_int64), ("losses_i", C.c_int64),
                ("overflow_e", C.c_int64), ("overflow_i", C.c_int64),
                ("E0", C.c_double), ("n_diag", C.c_int64),
                ("absorbed_e", C.c_int64 * 2), ("absorbed_i", C.c_int64 * 2), ("emitted", C.c_int64)]


class OraMoments(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("n_steps", C.c_int64)] + \
               [(k, _D) for k in ("n_e", "n_i", "gamma_e", "mean_eps_e", "heat_e", "iz_rate",
                                  "gamma_i", "E", "phi")] + [("reset", C.c_int32), ("pad", C.c_int32)]


_libs: dict = {}


def lib(f32: bool = False) -> C.CDLL:
    if f32 not in _libs:
        if not LIBS[f32].exists():
            build()
        L = C.CDLL(str(LIBS[f32]))
        L.ora_create.argtypes = [C.POINTER(OraParams), C.POINTER(C.c_void_p)]
        L.ora_destroy.argtypes = [C.c_void_p]
        L.ora_step.argtypes = [C.c_void_p, C.c_int64]
        L.ora_get_state.argtypes = [C.c_void_p, C.POINTER(OraState)]
        L.ora_set_state.argtypes = [C.c_void_p, C.POINTER(OraState)]
        L.ora_stats_get.argtypes = [C.c_void_p, C.POINTER(OraStats)]
        L.ora_moments_get.argtypes = [C.c_void_p, C.POINTER(OraMoments)]
        L.ora_eepf_config.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double]
        L.ora_eepf_get.argtypes = [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_int64), C.c_int]
        L.ora_last_codes.argtypes = [C.c_void_p, C.c_int, _I32, C.c_int64]
        L.ora_derived.argtypes = [C.c_void_p, _D]
        L.ora_nu_table.argtypes = [C.c_void_p, C.c_int, C.c_int, _D, C.c_int]
        L.ora_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.ora_gauss_table.argtypes = [C.POINTER(C.c_float)]
        L.ora_gauss_sample.argtypes = [C.POINTER(C.c_float), C.c_double]
        L.ora_gauss_sample.restype = C.c_double
        L.ora_i128_to_double.argtypes = [C.c_int64, C.c_uint64]
        L.ora_i128_to_double.restype = C.c_double
        L.ora_field_exact.argtypes = [C.c_int, _I64, _I64, C.c_double, _D]
        L.ora_field_exact_bounded.argtypes = [C.c_int, _I64, _I64, C.c_double, _D]
        L.ora_poisson_thomas.argtypes = [C.c_int, C.c_double, _D, _D]
        _libs[f32] = L
    return _libs[f32]


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().ora_philox4x32_10(c, k, o)
    return list(o)


def gauss_table(f32: bool = False) -> np.ndarray:
    t = np.zeros(4097, dtype=np.float32)
    lib(f32).ora_gauss_table(t.ctypes.data_as(C.POINTER(C.c_float)))
    return t


def gauss_sample(table: np.ndarray, u: float, f32: bool = False) -> float:
    return lib(f32).ora_gauss_sample(table.ctypes.data_as(C.POINTER(C.c_float)), float(u))


def i128_to_double(v: int) -> float:
    lo = v & ((1 << 64) - 1)
    hi = (v >> 64)
    return lib().ora_i128_to_double(hi, lo)


def field_exact(Q_i: np.ndarray, Q_e: np.ndarray, Cfield: float) -> np.ndarray:
    Q_i = np.ascontiguousarray(Q_i, dtype=np.int64)
    Q_e = np.ascontiguousarray(Q_e, dtype=np.int64)
    out = np.zeros(len(Q_i))
    lib().ora_field_exact(len(Q_i), _ptr(Q_i, _I64), _ptr(Q_e, _I64), Cfield, _ptr(out, _D))
    return out


def field_exact_bounded(Q_i: np.ndarray, Q_e: np.ndarray, Cfield: float) -> np.ndarray:
    """Space-charge field at the n_cells faces between two electrodes (n_cells + 1 node charges)."""
    Q_i = np.ascontiguousarray(Q_i, dtype=np.int64)
    Q_e = np.ascontiguousarray(Q_e, dtype=np.int64)
    n = len(Q_i) - 1
    out = np.zeros(n)
    lib().ora_field_exact_bounded(n, _ptr(Q_i, _I64), _ptr(Q_e, _I64), Cfield, _ptr(out, _D))
    return out


def poisson_thomas(rho: np.ndarray, dx: float) -> np.ndarray:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.zeros(len(rho))
    rc = lib().ora_poisson_thomas(len(rho), dx, _ptr(rho, _D), _ptr(phi, _D))
    if rc:
        raise ValueError(rc)
    return phi


def make_params(p, cls=OraParams, xcls=OraXsec):
    """Marshal a workloads.Params into the oracle's struct; returns (struct, keepalive)."""
    keep = []
    xs = (xcls * max(1, len(p.xsec)))()
    for k, x in enumerate(p.xsec):
        e = np.ascontiguousarray(x.energy_eV, dtype=np.float64)
        s = np.ascontiguousarray(x.sigma_m2, dtype=np.float64)
        keep += [e, s]
        xs[k].kind = x.kind
        xs[k].n = len(e)
        xs[k].threshold_eV = x.threshold_eV
        xs[k].energy_eV = _ptr(e, _D)
        xs[k].sigma_m2 = _ptr(s, _D)
    keep.append(xs)
    st = cls()
    for name, _ in cls._fields_:
        if name in ("xsec", "n_xsec") or name.startswith("pad"):
            continue
        setattr(st, name, getattr(p, name))
    st.n_xsec = len(p.xsec)
    st.xsec = C.cast(xs, C.POINTER(xcls))
    return st, keep


class Oracle:
    """One periodic column advanced by the CPU oracle."""

    def __init__(self, params, f32: bool | None = None):
        from_params_f32 = params.precision == 1
        self.f32 = from_params_f32 if f32 is None else f32
        self.L = lib(self.f32)
        if params.drive == 3:
            # (R, I) drive: the homogeneous field and density of eq. 2 from this package's own
            # two-term solve, then the column runs at that field
            from . import two_term
            xs = [(x.kind, x.threshold_eV, x.energy_eV, x.sigma_m2) for x in params.xsec]
            E0, n0, _ = two_term.ri_drive(xs, params.gas_mass_amu, params.pressure_torr, params.T_gas_K,
                                          params.R_m, params.I_A, params.eps_max_e_eV)
            params = params.with_(drive=0, E0_Vpm=float(E0), n0_m3=float(n0))
        self.params = params
        st, self._keep = make_params(params)
        h = C.c_void_p()
        rc = self.L.ora_create(C.byref(st), C.byref(h))
        if rc:
            raise RuntimeError(f"ora_create failed: {rc}")
        self.h = h
        self.N = params.n_cells
        self.nodes = params.n_nodes
        self.cap = params.capacity or (max(params.n_e0, params.n_i0) * 5 // 4 + 1024)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.ora_destroy(h)
            self.h = None

    def step(self, n: int = 1) -> None:
        rc = self.L.ora_step(self.h, n)
        if rc:
            raise RuntimeError(f"ora_step failed: {rc}")

    def stats(self) -> dict:
        s = OraStats()
        self.L.ora_stats_get(self.h, C.byref(s))
        d = {k: getattr(s, k) for k, _ in OraStats._fields_}
        d["n_coll_e"] = list(s.n_coll_e)
        d["n_coll_i"] = list(s.n_coll_i)
        d["absorbed_e"] = list(s.absorbed_e)
        d["absorbed_i"] = list(s.absorbed_i)
        return d

    def derived(self) -> dict:
        o = np.zeros(7)
        self.L.ora_derived(self.h, _ptr(o, _D))
        return dict(zip(["n_g", "nu_star_e", "P_null_e", "nu_star_i", "P_null_i", "w", "dx"], o))

    def nu_table(self, species: int, j: int) -> np.ndarray:
        out = np.zeros(self.params.n_table)
        rc = self.L.ora_nu_table(self.h, species, j, _ptr(out, _D), len(out))
        if rc:
            raise ValueError(rc)
        return out

    def get_state(self) -> dict:
        st = self.stats()
        ne, ni = st["n_e"], st["n_i"]
        d = {
            "cell_e": np.zeros(ne, np.int32), "off_e": np.zeros(ne), "vx_e": np.zeros(ne),
            "vy_e": np.zeros(ne), "vz_e": np.zeros(ne), "id_e": np.zeros(ne, np.uint64),
            "cell_i": np.zeros(ni, np.int32), "off_i": np.zeros(ni), "vx_i": np.zeros(ni),
            "vy_i": np.zeros(ni), "vz_i": np.zeros(ni), "id_i": np.zeros(ni, np.uint64),
            "E": np.zeros(self.nodes), "Q_e": np.zeros(self.nodes, np.int64), "Q_i": np.zeros(self.nodes, np.int64),
        }
        s = OraState()
        for k, t in (("cell", _I32), ("off", _D), ("vx", _D), ("vy", _D), ("vz", _D), ("id", _U64)):
            for sp in ("e", "i"):
                setattr(s, f"{k}_{sp}", _ptr(d[f"{k}_{sp}"], t))
        s.E = _ptr(d["E"], _D)
        s.Q_e = _ptr(d["Q_e"], _I64)
        s.Q_i = _ptr(d["Q_i"], _I64)
        self.L.ora_get_state(self.h, C.byref(s))
        d.update(n_e=s.n_e, n_i=s.n_i, step=s.step, next_id=s.next_id, E0=s.E0)
        return d

    def set_state(self, d: dict, with_E: bool = True, with_Qi: bool = True) -> None:
        s = OraState()
        s.n_e, s.n_i = len(d["cell_e"]), len(d["cell_i"])
        s.step, s.next_id, s.E0 = int(d["step"]), int(d["next_id"]), float(d["E0"])
        keep = []
        for k, dt, t in (("cell", np.int32, _I32), ("off", np.float64, _D), ("vx", np.float64, _D),
                         ("vy", np.float64, _D), ("vz", np.float64, _D), ("id", np.uint64, _U64)):
            for sp in ("e", "i"):
                a = np.ascontiguousarray(d[f"{k}_{sp}"], dtype=dt)
                keep.append(a)
                setattr(s, f"{k}_{sp}", _ptr(a, t))
        if with_E and d.get("E") is not None:
            a = np.ascontiguousarray(d["E"], dtype=np.float64); keep.append(a); s.E = _ptr(a, _D)
        if with_Qi and d.get("Q_i") is not None:
            a = np.ascontiguousarray(d["Q_i"], dtype=np.int64); keep.append(a); s.Q_i = _ptr(a, _I64)
        rc = self.L.ora_set_state(self.h, C.byref(s))
        if rc:
            raise RuntimeError(f"ora_set_state failed: {rc}")

    def codes(self, species: int, n: int) -> np.ndarray:
        out = np.zeros(n, np.int32)
        rc = self.L.ora_last_codes(self.h, species, _ptr(out, _I32), n)
        if rc:
            raise ValueError(rc)
        return out

    def moments(self, reset: bool = False) -> dict:
        names = ("n_e", "n_i", "gamma_e", "mean_eps_e", "heat_e", "iz_rate", "gamma_i", "E", "phi")
        d = {k: np.zeros(self.nodes) for k in names}
        m = OraMoments()
        for k in names:
            setattr(m, k, _ptr(d[k], _D))
        m.reset = int(reset)
        self.L.ora_moments_get(self.h, C.byref(m))
        d["n_samples"], d["n_steps"] = m.n_samples, m.n_steps
        return d

    def eepf_config(self, n_x: int, n_eps: int, eps_max_eV: float) -> None:
        if self.L.ora_eepf_config(self.h, n_x, n_eps, eps_max_eV):
            raise ValueError("bad EEPF histogram shape")
        self._eepf_shape = (n_x, n_eps + 1)

    def eepf(self, reset: bool = False):
        c = np.zeros(self._eepf_shape, np.uint64)
        ns = C.c_int64()
        if self.L.ora_eepf_get(self.h, c.ctypes.data_as(C.POINTER(C.c_uint64)), C.byref(ns), int(reset)):
            raise ValueError("no EEPF histogram")
        return c, ns.value


_mlp = None


def mlp_lib():
    global _mlp
    if _mlp is None:
        if not MLP_LIB.exists():
            build()
        L = C.CDLL(str(MLP_LIB))
        L.mlp_nparam.restype = C.c_int
        L.mlp_forward_backward.argtypes = [_D, _D, _D, C.c_int, C.c_int, _D, _D]
        L.mlp_forward_backward.restype = C.c_double
        L.mlp_adam.argtypes = [_D, _D, _D, _D, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
        _mlp = L
    return _mlp


MLP_NPARAM = 128 * 15 + 128 + 128 * 128 + 128 + 3 * 128 + 3


def mlp_forward_backward(P, X, T, bf16=False, want_grad=True):
    """loss, outputs (n x 3), gradient (flat) of the oracle network."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    n = X.shape[0]
    y = np.zeros((n, 3))
    g = np.zeros(MLP_NPARAM) if want_grad else None
    loss = mlp_lib().mlp_forward_backward(_ptr(P, _D), _ptr(X, _D), _ptr(T, _D), n, int(bf16), _ptr(y, _D),
                                          _ptr(g, _D) if g is not None else None)
    return loss, y, g


def mlp_adam(P, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays."""
    mlp_lib().mlp_adam(_ptr(P, _D), _ptr(np.ascontiguousarray(g, dtype=np.float64), _D), _ptr(m, _D),
                       _ptr(v, _D), t, lr, b1, b2, eps)

