"""Python binding of the GB300 PIC-MCC library (include/pic.h).

Argument marshalling only: every step of the method runs in the CUDA
kernels of libpic.so.  There is no CPU fallback; importing the binding
without the compiled library, or creating a column without a GPU, raises.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path
from typing import Optional

import numpy as np

HERE = Path(__file__).resolve().parent
LIBPATH = HERE / "libpic.so"

PIC_ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ECAPACITY", -5: "ENONFINITE",
              -6: "ETIMEOUT", -7: "EPARAM"}
FLAG_RECORD_CODES = 1
FLAG_NO_GRAPH = 2
FLAG_ALLOW_LARGE_NULL = 4


class PicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{PIC_ERRORS.get(code, code)}: {msg}")
        self.code = code


class Xsec(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32), ("threshold_eV", C.c_double),
                ("energy_eV", C.POINTER(C.c_double)), ("sigma_m2", C.POINTER(C.c_double))]


class Params(C.Structure):
    _fields_ = [("gas_mass_amu", C.c_double), ("pressure_torr", C.c_double), ("T_gas_K", C.c_double),
                ("L_m", C.c_double), ("R_m", C.c_double),
                ("drive", C.c_int32), ("field_mode", C.c_int32),
                ("E0_Vpm", C.c_double), ("V_applied", C.c_double), ("I_A", C.c_double),
                ("U_src", C.c_double), ("R_ext_ohm_m2", C.c_double),
                ("n_xsec", C.c_int32), ("pad0", C.c_int32), ("xsec", C.POINTER(Xsec)),
                ("n_cells", C.c_int32), ("ion_subcycle", C.c_int32), ("dt_s", C.c_double),
                ("n_e0", C.c_int64), ("n_i0", C.c_int64), ("capacity", C.c_int64),
                ("n0_m3", C.c_double), ("Te0_eV", C.c_double), ("Ti0_eV", C.c_double),
                ("loss_mode", C.c_int32), ("precision", C.c_int32), ("nu_w", C.c_double),
                ("seed", C.c_uint64),
                ("diag_every", C.c_int32), ("sort_every", C.c_int32), ("n_table", C.c_int32),
                ("flags", C.c_uint32),
                ("eps_max_e_eV", C.c_double), ("eps_max_i_eV", C.c_double),
                ("column", C.c_int32), ("pad1", C.c_int32),
                ("J_emit_Am2", C.c_double), ("T_emit_eV", C.c_double)]


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_U64 = C.POINTER(C.c_uint64)


class State(C.Structure):
    _fields_ = [("n_e", C.c_int64), ("n_i", C.c_int64), ("step", C.c_int64), ("next_id", C.c_int64),
                ("E0", C.c_double),
                ("cell_e", _I32), ("off_e", _D), ("vx_e", _D), ("vy_e", _D), ("vz_e", _D), ("id_e", _U64),
                ("cell_i", _I32), ("off_i", _D), ("vx_i", _D), ("vy_i", _D), ("vz_i", _D), ("id_i", _U64),
                ("E", _D), ("Q_e", _I64), ("Q_i", _I64)]


_F = C.POINTER(C.c_float)


class StateF32(C.Structure):
    """pic_state_f32: the state with FP32 offsets and velocities (the precision form's storage)."""
    _fields_ = [("n_e", C.c_int64), ("n_i", C.c_int64), ("step", C.c_int64), ("next_id", C.c_int64),
                ("E0", C.c_double),
                ("cell_e", _I32), ("off_e", _F), ("vx_e", _F), ("vy_e", _F), ("vz_e", _F), ("id_e", _U64),
                ("cell_i", _I32), ("off_i", _F), ("vx_i", _F), ("vy_i", _F), ("vz_i", _F), ("id_i", _U64),
                ("E", _D), ("Q_i", _I64)]


class Stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("n_e", C.c_int64), ("n_i", C.c_int64), ("next_id", C.c_int64),
                ("n_coll_e", C.c_int64 * 16), ("n_coll_i", C.c_int64 * 16),
                ("births", C.c_int64), ("losses_e", C.c_int64), ("losses_i", C.c_int64),
                ("overflow_e", C.c_int64), ("overflow_i", C.c_int64),
                ("E0", C.c_double), ("n_diag", C.c_int64),
                ("absorbed_e", C.c_int64 * 2), ("absorbed_i", C.c_int64 * 2), ("emitted", C.c_int64)]


MOMENT_NAMES = ("n_e", "n_i", "gamma_e", "mean_eps_e", "heat_e", "iz_rate", "gamma_i", "E", "phi")


class MomentsOut(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("n_steps", C.c_int64)] + \
               [(k, _D) for k in MOMENT_NAMES] + [("reset", C.c_int32), ("pad", C.c_int32)]


_lib: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    """Load libpic.so (built by build.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        if not LIBPATH.exists():
            raise ImportError(f"{LIBPATH} is missing: run paper_2202_03215_gb300.build.build() (nvcc, sm_103a)")
        L = C.CDLL(str(LIBPATH))
        L.pic_init.argtypes = [C.POINTER(Params), C.POINTER(C.c_void_p)]
        L.pic_check_stability.argtypes = [C.POINTER(Params), _D]
        L.pic_step.argtypes = [C.c_void_p, C.c_int64]
        L.pic_moments.argtypes = [C.c_void_p, C.POINTER(MomentsOut)]
        L.pic_eepf_config.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_double]
        L.pic_eepf_get.argtypes = [C.c_void_p, _U64, C.POINTER(C.c_int64), C.c_int32]
        L.pic_get_state.argtypes = [C.c_void_p, C.POINTER(State)]
        L.pic_set_state.argtypes = [C.c_void_p, C.POINTER(State)]
        L.pic_set_state_f32.argtypes = [C.c_void_p, C.POINTER(StateF32)]
        L.pic_get_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
        L.pic_last_codes.argtypes = [C.c_void_p, C.c_int, _I32, C.c_int64]
        L.pic_derived.argtypes = [C.c_void_p, _D]
        L.pic_stream.argtypes = [C.c_void_p]
        L.pic_stream.restype = C.c_void_p
        L.pic_free.argtypes = [C.c_void_p]
        L.pic_free.restype = None
        L.pic_last_error.argtypes = [C.c_void_p]
        L.pic_last_error.restype = C.c_char_p
        L.pic_test_i128_to_double.argtypes = [_I64, _U64, _D, C.c_int]
        L.pic_abi_version.restype = C.c_int
        L.pic_field_periodic.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double,
                                         C.c_void_p, C.c_void_p, C.c_void_p]
        L.pic_field_periodic_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double,
                                                 C.c_void_p, C.c_void_p, C.c_void_p]
        L.pic_init_batch.argtypes = [C.POINTER(Params), C.c_int, C.POINTER(C.c_void_p)]
        L.pic_step_batch.argtypes = [C.c_void_p, C.c_int64]
        L.pic_batch_column.argtypes = [C.c_void_p, C.c_int]
        L.pic_batch_column.restype = C.c_void_p
        L.pic_batch_size.argtypes = [C.c_void_p]
        L.pic_batch_schedule.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.pic_mlp_nparam.restype = C.c_int
        L.pic_mlp_create.argtypes = [C.c_uint64, C.POINTER(C.c_void_p)]
        L.pic_mlp_free.argtypes = [C.c_void_p]
        L.pic_mlp_free.restype = None
        L.pic_mlp_set_params.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.c_int]
        L.pic_mlp_get_params.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.c_int]
        L.pic_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
        L.pic_mlp_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_float), _D,
                                   C.c_void_p]
        L.pic_mlp_train.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_float,
                                    _D, C.c_void_p]
        L.pic_two_term.argtypes = [C.POINTER(Xsec), C.c_int, C.c_double, _D, C.c_int, C.c_double, C.c_int,
                                   C.POINTER(Transport)]
        L.pic_fluid_init.argtypes = [C.POINTER(FluidColumn), C.c_int, C.POINTER(Transport), C.c_int, C.c_int,
                                     C.c_double, C.c_int, C.c_int, C.POINTER(C.c_void_p)]
        L.pic_fluid_set_state.argtypes = [C.c_void_p, C.c_int, _D, _D]
        L.pic_fluid_get_state.argtypes = [C.c_void_p, C.c_int, _D, _D]
        L.pic_fluid_step.argtypes = [C.c_void_p, C.c_int64]
        L.pic_fluid_modes.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)]
        L.pic_fluid_set_closure.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_float),
                                            C.POINTER(C.c_float), C.c_float, C.c_int]
        L.pic_fluid_set_corrections.argtypes = [C.c_void_p, C.c_void_p]
        L.pic_fluid_features.argtypes = [C.c_void_p, C.c_void_p]
        L.pic_fluid_elapsed.argtypes = [C.c_void_p, _D, _I64]
        L.pic_fluid_stream.argtypes = [C.c_void_p]
        L.pic_fluid_stream.restype = C.c_void_p
        L.pic_fluid_free.argtypes = [C.c_void_p]
        L.pic_fluid_free.restype = None
        L.pic_drive_ri.argtypes = [C.POINTER(Params), _D]
        L.pic_set_timing.argtypes = [C.c_void_p, C.c_int]
        L.pic_kernel_times.argtypes = [C.c_void_p, _D, _I64]
        _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _check(rc: int, h=None) -> None:
    if rc:
        msg = lib().pic_last_error(h)
        raise PicError(rc, msg.decode() if msg else "")


class Transport(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("EN_Td", "mean_eps_eV", "muN", "DN", "mueN", "DeN", "nu_izN", "lossN",
                                           "powerN", "alphaN")]


FLUID_LOSS_FIXED, FLUID_LOSS_PAIR = 0, 1


class FluidColumn(C.Structure):
    _fields_ = [("L_m", C.c_double), ("N_gas_m3", C.c_double), ("mu_iN", C.c_double), ("Gamma_T", C.c_double),
                ("nu_w", C.c_double), ("n_cells", C.c_int32), ("loss", C.c_int32)]


def _xsec_array(xsec):
    keep = []
    xs = (Xsec * max(1, len(xsec)))()
    for k, x in enumerate(xsec):
        e = np.ascontiguousarray(x.energy_eV, dtype=np.float64)
        s = np.ascontiguousarray(x.sigma_m2, dtype=np.float64)
        keep += [e, s]
        xs[k].kind, xs[k].n, xs[k].threshold_eV = x.kind, len(e), x.threshold_eV
        xs[k].energy_eV, xs[k].sigma_m2 = _ptr(e, _D), _ptr(s, _D)
    keep.append(xs)
    return xs, keep


def two_term(xsec, gas_mass_amu: float, EN_Td, eps_max_eV: float = 100.0, n_grid: int = 1000) -> list:
    """pic_two_term: two-term Boltzmann transport at each reduced field (list of dicts)."""
    xs, keep = _xsec_array(xsec)
    en = np.ascontiguousarray(np.atleast_1d(EN_Td), dtype=np.float64)
    out = (Transport * len(en))()
    _check(lib().pic_two_term(xs, len(xsec), gas_mass_amu, _ptr(en, _D), len(en), eps_max_eV, n_grid, out))
    return [{n: getattr(o, n) for n, _ in Transport._fields_} for o in out]


def make_params(p):
    """Marshal a workloads.Params into pic_params; returns (struct, keepalive)."""
    xs, keep = _xsec_array(p.xsec)
    st = Params()
    for name, _ in Params._fields_:
        if name in ("xsec", "n_xsec") or name.startswith("pad"):
            continue
        setattr(st, name, getattr(p, name))
    st.n_xsec = len(p.xsec)
    st.xsec = C.cast(xs, C.POINTER(Xsec))
    return st, keep


def drive_ri(p) -> dict:
    """pic_drive_ri: E0, n0, Te0 and the ion mobility x N of the (R, I) drive of params p."""
    st, keep = make_params(p)
    out = np.zeros(4)
    _check(lib().pic_drive_ri(C.byref(st), _ptr(out, _D)))
    return dict(E0_Vpm=out[0], n0_m3=out[1], Te0_eV=out[2], mu_iN=out[3])


WARN_PLASMA_FREQ, WARN_DEBYE = 1, 2
MLP_HOOK_NO_WEIGHT_COPY, MLP_HOOK_NO_FORWARD_MMA = 1, 2


def check_stability(p) -> dict:
    """pic_check_stability (host only): the resolution limits of Sec. II at the initial state,
    w_pe dt < 0.2 and dx < lambda_De.  Returns the ratios and the PIC_WARN_* bits that fail."""
    st, keep = make_params(p)
    out = np.zeros(2)
    rc = lib().pic_check_stability(C.byref(st), _ptr(out, _D))
    if rc < 0:
        _check(rc)
    return {"wpe_dt": float(out[0]), "dx_over_lambda_De": float(out[1]), "warnings": int(rc)}


def i128_to_double(values) -> np.ndarray:
    """Run the device int128 -> double conversion of the field solve on a list of Python ints."""
    vals = [int(v) for v in values]
    hi = np.array([v >> 64 for v in vals], dtype=np.int64)
    lo = np.array([v & ((1 << 64) - 1) for v in vals], dtype=np.uint64)
    out = np.zeros(len(vals))
    _check(lib().pic_test_i128_to_double(_ptr(hi, _I64), _ptr(lo, _U64), _ptr(out, _D), len(vals)))
    return out


def field_periodic(Q_i, Q_e, C_unit: float, E0: float, stream: int = 0):
    """Periodic Poisson solve on device tensors (int64 node charges, 2^32 per particle).
    Returns (E, E_half) as float64 device tensors of the same length."""
    import torch
    n = _check_field_tensors(Q_i, Q_e)
    E = torch.empty(n, dtype=torch.float64, device=Q_i.device)
    Eh = torch.empty_like(E)
    _check(lib().pic_field_periodic(Q_i.data_ptr(), Q_e.data_ptr(), n, C_unit, E0, E.data_ptr(), Eh.data_ptr(),
                                    stream or None))
    return E, Eh


def _check_field_tensors(Q_i, Q_e, E=None, E_half=None) -> int:
    """Argument checks of the field solves: int64 node charges and float64 outputs, all
    contiguous CUDA tensors on one device, each holding at least n = Q_i.numel() entries.
    Raises ValueError before any device call; returns n."""
    import torch
    n = Q_i.numel()
    dev = Q_i.device
    for name, t, dt in (("Q_i", Q_i, torch.int64), ("Q_e", Q_e, torch.int64), ("E", E, torch.float64),
                        ("E_half", E_half, torch.float64)):
        if t is None:
            continue
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_cuda or t.device != dev:
            raise ValueError(f"{name} must be a CUDA tensor on {dev}, got {t.device}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() < n:
            raise ValueError(f"{name} holds {t.numel()} entries, fewer than the {n} nodes")
    return n


def field_periodic_noalloc(Q_i, Q_e, C_unit: float, E0: float, E, E_half, stream: int = 0) -> None:
    """pic_field_periodic_noalloc: the same solve with caller-provided outputs E, E_half
    (float64 device tensors) and no device allocation inside the call."""
    _check_field_tensors(Q_i, Q_e, E, E_half)
    rc = lib().pic_field_periodic_noalloc(Q_i.data_ptr(), Q_e.data_ptr(), Q_i.numel(), C_unit, E0,
                                          E.data_ptr(), E_half.data_ptr(), stream or None)
    if rc:
        raise PicError(rc, "pic_field_periodic_noalloc failed")


class Column:
    """One periodic positive column on the GPU (pic_init / pic_step / pic_moments / pic_free)."""

    def __init__(self, params, flags: int = 0, _handle=None):
        self.L = lib()
        self.params = params
        self.N = params.n_cells
        self.nodes = params.n_nodes          # node arrays: n_cells, or n_cells + 1 between electrodes
        self.cap = params.capacity or (max(params.n_e0, params.n_i0) * 5 // 4 + 1024)
        self._owned = _handle is None
        if _handle is not None:
            self.h = C.c_void_p(_handle)
            return
        st, keep = make_params(params)
        st.flags = params.flags | flags
        h = C.c_void_p()
        rc = self.L.pic_init(C.byref(st), C.byref(h))
        _check(rc)
        self.h = h
        self.stability = check_stability(params)
        if self.stability["warnings"]:
            import warnings
            warnings.warn(f"resolution limits of the explicit scheme not met: w_pe dt = "
                          f"{self.stability['wpe_dt']:.3g} (< 0.2), dx / lambda_De = "
                          f"{self.stability['dx_over_lambda_De']:.3g} (< 1)", stacklevel=2)

    def close(self) -> None:
        if getattr(self, "h", None):
            if self._owned:
                self.L.pic_free(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def step(self, n: int = 1) -> None:
        _check(self.L.pic_step(self.h, n), self.h)

    def stats(self) -> dict:
        s = Stats()
        _check(self.L.pic_get_stats(self.h, C.byref(s)), self.h)
        d = {k: getattr(s, k) for k, _ in Stats._fields_}
        d["n_coll_e"], d["n_coll_i"] = list(s.n_coll_e), list(s.n_coll_i)
        d["absorbed_e"], d["absorbed_i"] = list(s.absorbed_e), list(s.absorbed_i)
        return d

    def derived(self) -> dict:
        o = np.zeros(7)
        _check(self.L.pic_derived(self.h, _ptr(o, _D)), self.h)
        return dict(zip(["n_g", "nu_star_e", "P_null_e", "nu_star_i", "P_null_i", "w", "dx"], o))

    def stream(self) -> int:
        return self.L.pic_stream(self.h) or 0

    def get_state(self) -> dict:
        st = self.stats()
        ne, ni = st["n_e"], st["n_i"]
        d = {"cell_e": np.zeros(ne, np.int32), "off_e": np.zeros(ne), "vx_e": np.zeros(ne),
             "vy_e": np.zeros(ne), "vz_e": np.zeros(ne), "id_e": np.zeros(ne, np.uint64),
             "cell_i": np.zeros(ni, np.int32), "off_i": np.zeros(ni), "vx_i": np.zeros(ni),
             "vy_i": np.zeros(ni), "vz_i": np.zeros(ni), "id_i": np.zeros(ni, np.uint64),
             "E": np.zeros(self.nodes), "Q_e": np.zeros(self.nodes, np.int64), "Q_i": np.zeros(self.nodes, np.int64)}
        s = State()
        for k, t in (("cell", _I32), ("off", _D), ("vx", _D), ("vy", _D), ("vz", _D), ("id", _U64)):
            for sp in ("e", "i"):
                setattr(s, f"{k}_{sp}", _ptr(d[f"{k}_{sp}"], t))
        s.E, s.Q_e, s.Q_i = _ptr(d["E"], _D), _ptr(d["Q_e"], _I64), _ptr(d["Q_i"], _I64)
        _check(self.L.pic_get_state(self.h, C.byref(s)), self.h)
        d.update(n_e=s.n_e, n_i=s.n_i, step=s.step, next_id=s.next_id, E0=s.E0)
        return d

    def set_state(self, d: dict, with_E: bool = True, with_Qi: bool = True) -> None:
        """pic_set_state; pic_set_state_f32 when the offsets and velocities come as float32
        arrays (the precision form's storage: 28 bytes per particle uploaded instead of 44)."""
        f32 = all(np.asarray(d[f"{k}_{sp}"]).dtype == np.float32 for k in ("off", "vx", "vy", "vz")
                  for sp in ("e", "i"))
        s = StateF32() if f32 else State()
        vt, vp = (np.float32, _F) if f32 else (np.float64, _D)
        s.n_e, s.n_i = len(d["cell_e"]), len(d["cell_i"])
        s.step, s.next_id, s.E0 = int(d["step"]), int(d["next_id"]), float(d["E0"])
        keep = []
        for k, dt, t in (("cell", np.int32, _I32), ("off", vt, vp), ("vx", vt, vp),
                         ("vy", vt, vp), ("vz", vt, vp), ("id", np.uint64, _U64)):
            for sp in ("e", "i"):
                a = np.ascontiguousarray(d[f"{k}_{sp}"], dtype=dt)
                keep.append(a)
                setattr(s, f"{k}_{sp}", _ptr(a, t))
        if with_E and d.get("E") is not None:
            a = np.ascontiguousarray(d["E"], dtype=np.float64); keep.append(a); s.E = _ptr(a, _D)
        if with_Qi and d.get("Q_i") is not None:
            a = np.ascontiguousarray(d["Q_i"], dtype=np.int64); keep.append(a); s.Q_i = _ptr(a, _I64)
        _check((self.L.pic_set_state_f32 if f32 else self.L.pic_set_state)(self.h, C.byref(s)), self.h)

    def set_timing(self, enable: bool) -> None:
        _check(self.L.pic_set_timing(self.h, int(enable)), self.h)

    def kernel_times(self) -> dict:
        """Summed event milliseconds and launch counts per kernel class since the last call."""
        ms = np.zeros(8)
        n = np.zeros(8, np.int64)
        _check(self.L.pic_kernel_times(self.h, _ptr(ms, _D), _ptr(n, _I64)), self.h)
        names = ("push_e", "push_i", "births", "field", "sort", "other")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(names)}

    def codes(self, species: int, n: int) -> np.ndarray:
        out = np.zeros(n, np.int32)
        _check(self.L.pic_last_codes(self.h, species, _ptr(out, _I32), n), self.h)
        return out

    def moments(self, reset: bool = False) -> dict:
        d = {k: np.zeros(self.nodes) for k in MOMENT_NAMES}
        m = MomentsOut()
        for k in MOMENT_NAMES:
            setattr(m, k, _ptr(d[k], _D))
        m.reset = int(reset)
        _check(self.L.pic_moments(self.h, C.byref(m)), self.h)
        d["n_samples"], d["n_steps"] = m.n_samples, m.n_steps
        return d

    def eepf_config(self, n_x: int, n_eps: int, eps_max_eV: float) -> None:
        """Sample the electron energy histogram on every diagnostic step (pic_eepf_config)."""
        _check(self.L.pic_eepf_config(self.h, n_x, n_eps, eps_max_eV), self.h)
        self._eepf_shape = (n_x, n_eps + 1)

    def eepf(self, reset: bool = False):
        """(counts[n_x, n_eps + 1], diagnostic samples) of the energy histogram."""
        c = np.zeros(self._eepf_shape, np.uint64)
        ns = C.c_int64()
        _check(self.L.pic_eepf_get(self.h, _ptr(c, _U64), C.byref(ns), int(reset)), self.h)
        return c, ns.value


def eepf_normalized(counts, eps_max_eV: float):
    """F(x, eps) from an energy histogram (Sec. III.C): per spatial bin, counts / (deps eps^(1/2))
    scaled so that sum eps^(1/2) F deps = 1 over the bins below eps_max (bin centres eps).
    Returns (eps centres, F[n_x, n_eps])."""
    c = np.asarray(counts, float)[:, :-1]
    n_eps = c.shape[1]
    de = eps_max_eV / n_eps
    eps = (np.arange(n_eps) + 0.5) * de
    F = c / (de * np.sqrt(eps))[None, :]
    norm = (F * np.sqrt(eps)[None, :] * de).sum(axis=1, keepdims=True)
    return eps, F / np.where(norm > 0, norm, 1.0)


class Batch:
    """Many independent columns advanced together (pic_init_batch / pic_step_batch)."""

    def __init__(self, params_list, flags: int = 0):
        self.L = lib()
        self.params = list(params_list)
        n = len(self.params)
        arr = (Params * n)()
        self._keep = []
        for i, p in enumerate(self.params):
            st, keep = make_params(p)
            st.flags = p.flags | flags
            arr[i] = st
            self._keep.append(keep)
        h = C.c_void_p()
        _check(self.L.pic_init_batch(arr, n, C.byref(h)))
        self.h = h
        self.columns = [Column(p.with_(column=i), _handle=self.L.pic_batch_column(h, i))
                        for i, p in enumerate(self.params)]

    def step(self, n: int = 1) -> None:
        _check(self.L.pic_step_batch(self.h, n), self.h)

    def schedule(self) -> tuple:
        """(tuned, CTA multiplier of the electrons, of the ions): tuned is False while the next
        steps still time candidate schedules."""
        me, mi = C.c_int(), C.c_int()
        rc = self.L.pic_batch_schedule(self.h, C.byref(me), C.byref(mi))
        _check(min(rc, 0), self.h)
        return rc == 1, me.value, mi.value

    def tune(self, max_steps: int = 1000) -> int:
        """Step until the schedule is tuned (at most max_steps); returns the steps taken."""
        k = 0
        while not self.schedule()[0] and k < max_steps:
            self.step(1)
            k += 1
        return k

    def stream(self) -> int:
        return self.L.pic_stream(self.h) or 0

    def set_timing(self, enable: bool) -> None:
        _check(self.L.pic_set_timing(self.h, int(enable)), self.h)

    def kernel_times(self) -> dict:
        ms = np.zeros(8)
        n = np.zeros(8, np.int64)
        _check(self.L.pic_kernel_times(self.h, _ptr(ms, _D), _ptr(n, _I64)), self.h)
        names = ("push_e", "push_i", "births", "field", "sort", "other")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(names)}

    def close(self) -> None:
        if getattr(self, "h", None):
            for c in self.columns:
                c.h = None
            self.L.pic_free(self.h)
            self.h = None

    def __del__(self):
        self.close()


class Mlp:
    """The closure network on the GPU (pic_mlp_*); data as float32 device tensors."""

    def __init__(self, seed: int = 7):
        self.L = lib()
        h = C.c_void_p()
        _check(self.L.pic_mlp_create(seed, C.byref(h)))
        self.h = h
        self.nparam = self.L.pic_mlp_nparam()

    def close(self) -> None:
        if getattr(self, "h", None):
            self.L.pic_mlp_free(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def params(self) -> np.ndarray:
        out = np.zeros(self.nparam, np.float32)
        _check(self.L.pic_mlp_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_float)), self.nparam))
        return out

    def set_params(self, P) -> None:
        P = np.ascontiguousarray(P, dtype=np.float32)
        _check(self.L.pic_mlp_set_params(self.h, P.ctypes.data_as(C.POINTER(C.c_float)), len(P)))

    def test_hook(self, hook: int, spin: int = 0) -> None:
        """pic_mlp_test_hook: make the selected bounded waits give up after `spin` polls."""
        _check(self.L.pic_mlp_test_hook(self.h, C.c_uint(hook), spin))

    def forward(self, X):
        import torch
        Y = torch.empty((X.shape[0], 3), dtype=torch.float32, device=X.device)
        _check(self.L.pic_mlp_forward(self.h, X.data_ptr(), X.shape[0], Y.data_ptr(), None))
        return Y

    def grad(self, X, T):
        g = np.zeros(self.nparam, np.float32)
        loss = C.c_double()
        _check(self.L.pic_mlp_grad(self.h, X.data_ptr(), T.data_ptr(), X.shape[0],
                                   g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss), None))
        return loss.value, g

    def train(self, X, T, batch: int = 8192, steps: int = 1, lr: float = 1e-3) -> float:
        loss = C.c_double()
        _check(self.L.pic_mlp_train(self.h, X.data_ptr(), T.data_ptr(), X.shape[0], batch, steps, lr,
                                    C.byref(loss), None))
        return loss.value



class Fluid:
    """Many periodic columns of the quasi-neutral fluid model (pic_fluid_*).

    columns: dicts with L_m, N_gas_m3, mu_iN, Gamma_T, nu_w, n_cells and optionally
    loss (FLUID_LOSS_FIXED or FLUID_LOSS_PAIR);
    transport: records of two_term() in increasing Te."""

    def __init__(self, columns, transport, n_T: int = 128, dt_s: float = 2e-8, diag_every: int = 0,
                 n_modes: int = 0):
        self.L = lib()
        self.columns = [dict(c) for c in columns]
        cols = (FluidColumn * len(columns))()
        for k, c in enumerate(columns):
            for name in ("L_m", "N_gas_m3", "mu_iN", "Gamma_T", "nu_w", "n_cells"):
                setattr(cols[k], name, c[name])
            cols[k].loss = c.get("loss", FLUID_LOSS_FIXED)
        tr = (Transport * len(transport))()
        for k, r in enumerate(transport):
            for name, _ in Transport._fields_:
                setattr(tr[k], name, r[name])
        h = C.c_void_p()
        _check(self.L.pic_fluid_init(cols, len(columns), tr, len(transport), n_T, dt_s, diag_every, n_modes,
                                     C.byref(h)))
        self.h = h
        self.n_modes = n_modes
        self.offsets = np.cumsum([0] + [c["n_cells"] for c in columns])
        self._net = None
        self._corr = None

    def set_state(self, col: int, n, T) -> None:
        n = np.ascontiguousarray(n, dtype=np.float64)
        T = np.ascontiguousarray(T, dtype=np.float64)
        _check(self.L.pic_fluid_set_state(self.h, col, _ptr(n, _D), _ptr(T, _D)))

    def get_state(self, col: int):
        N = self.columns[col]["n_cells"]
        n, T = np.zeros(N), np.zeros(N)
        _check(self.L.pic_fluid_get_state(self.h, col, _ptr(n, _D), _ptr(T, _D)))
        return n, T

    def step(self, n: int = 1) -> None:
        _check(self.L.pic_fluid_step(self.h, n))

    def modes(self, max_snaps: int = 100000) -> np.ndarray:
        """Spectral record since the last call: complex array [snap, column, n_modes + 1]
        (entry 0 = mean density)."""
        out = np.zeros((max_snaps, len(self.columns), self.n_modes + 1, 2), dtype=np.float32)
        k = C.c_int()
        _check(self.L.pic_fluid_modes(self.h, out.ctypes.data_as(C.POINTER(C.c_float)), max_snaps, C.byref(k)))
        o = out[:k.value].astype(np.float64)
        return o[..., 0] + 1j * o[..., 1]

    def set_closure(self, net, period: int, feat_scale, targ_scale, nu_bound: float = 0.0, stencil: int = 1) -> None:
        fs = np.ascontiguousarray(feat_scale, dtype=np.float32)
        ts = np.ascontiguousarray(targ_scale, dtype=np.float32)
        _check(self.L.pic_fluid_set_closure(self.h, net.h if net is not None else None, period,
                                            fs.ctypes.data_as(C.POINTER(C.c_float)),
                                            ts.ctypes.data_as(C.POINTER(C.c_float)), nu_bound, stencil))
        self._net = net

    def set_corrections(self, corr) -> None:
        """corr: device float32 tensor (total cells x 3) in SI units, or None."""
        self._corr = corr
        _check(self.L.pic_fluid_set_corrections(self.h, None if corr is None else corr.data_ptr()))

    def features(self):
        import torch
        X = torch.empty((int(self.offsets[-1]), 15), dtype=torch.float32, device="cuda")
        _check(self.L.pic_fluid_features(self.h, X.data_ptr()))
        return X

    def elapsed(self):
        ms = np.zeros(1)
        k = np.zeros(1, dtype=np.int64)
        _check(self.L.pic_fluid_elapsed(self.h, _ptr(ms, _D), _ptr(k, _I64)))
        return float(ms[0]), int(k[0])

    def close(self) -> None:
        if getattr(self, "h", None):
            self.L.pic_fluid_free(self.h)
            self.h = None

    def __del__(self):
        self.close()
