"""ctypes wrapper around oracle/picsar_oracle.c (test infrastructure only).

The C file is a plain FP64 restatement of the PICsar step; this module builds
it with gcc (``build_oracle``) and exposes a small ``Oracle`` class.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "picsar_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libpicsar_oracle.so")
_lock = threading.Lock()
_lib = None

VAC = {"none": 0, "monopole": 1, "monopole_rotator": 2, "uniform_bz": 3, "dipole_corot": 4, "dipole_rotator": 5}
INJECT = {"off": 0, "fixed": 1, "variable": 2}
PUSHER = {"vay": 0, "boris": 1}
ABSORB = {"none": 0, "linear": 1, "quadratic": 2}


class Params(C.Structure):
    _fields_ = [
        ("nr", C.c_int32), ("nth", C.c_int32),
        ("r_min", C.c_double), ("r_max", C.c_double),
        ("r_map", C.c_int32), ("th_map", C.c_int32),
        ("dt", C.c_double),
        ("n_filt", C.c_int32),
        ("absorb_cells", C.c_int32), ("absorb_profile", C.c_int32),
        ("absorb_sigma_max", C.c_double),
        ("vacuum", C.c_int32),
        ("b0", C.c_double), ("omega", C.c_double), ("t_spin", C.c_double),
        ("inject", C.c_int32), ("pairs_per_cell", C.c_int32), ("f_inj", C.c_double),
        ("pusher", C.c_int32),
        ("q_over_m", C.c_double),
        ("inject_smooth", C.c_int32), ("inject_q", C.c_double), ("inject_seed", C.c_uint64),
    ]


def params(**kw) -> Params:
    """Build oracle parameters from keyword values (strings allowed for enums)."""
    p = Params()
    p.q_over_m = 1.0
    p.pairs_per_cell = 2
    for k, v in kw.items():
        if k == "vacuum" and isinstance(v, str):
            v = VAC[v]
        elif k == "inject" and isinstance(v, str):
            v = INJECT[v]
        elif k == "pusher" and isinstance(v, str):
            v = PUSHER[v]
        elif k == "absorb_profile" and isinstance(v, str):
            v = ABSORB[v]
        elif k == "r_map" and isinstance(v, str):
            v = {"linear": 0, "log": 1}[v]
        elif k == "th_map" and isinstance(v, str):
            v = {"linear": 0, "equal_area": 1}[v]
        setattr(p, k, v)
    return p


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    with _lock:
        if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
            return _OUT
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
        return _OUT


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build_oracle())
    P, D, I64, I32 = C.c_void_p, C.POINTER(C.c_double), C.c_int64, C.c_int32
    sig = {
        "orc_create": (P, [C.POINTER(Params)]),
        "orc_destroy": (None, [P]),
        "orc_last_error": (C.c_int, [P]),
        "orc_f_r": (C.c_double, [P, C.c_double]),
        "orc_f_r_inv": (C.c_double, [P, C.c_double]),
        "orc_f_th": (C.c_double, [P, C.c_double]),
        "orc_f_th_inv": (C.c_double, [P, C.c_double]),
        "orc_courant_dt": (C.c_double, [C.POINTER(Params), C.c_double]),
        "orc_load_particles": (None, [P, I64, D, D, D, D, D, D, C.POINTER(C.c_int64)]),
        "orc_num_particles": (I64, [P]),
        "orc_get_particles": (None, [P, D, D, D, D, D, D, C.POINTER(C.c_int64)]),
        "orc_set_clock": (None, [P, I64, I64]),
        "orc_get_step": (I64, [P]),
        "orc_get_fields": (None, [P, D]),
        "orc_get_fields_total": (None, [P, D]),
        "orc_set_fields": (None, [P, D]),
        "orc_ghost": (I32, [P]),
        "orc_get_flux": (None, [P, D]),
        "orc_step": (None, [P, I32]),
        "orc_particles_only": (None, [P]),
        "orc_field_step": (None, [P, I32]),
        "orc_vacuum_fields": (None, [P, C.c_double, C.c_double, C.c_double, D, D]),
        "orc_gather": (None, [P, C.c_double, C.c_double, C.c_double, D, D]),
        "orc_push": (None, [I32, C.c_double, D, D, D]),
        "orc_deposit_path": (C.c_int, [P, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, D, D]),
        "orc_filter_pass": (None, [P, D, I32, I32]),
        "orc_node_charge": (None, [P, I32, D]),
        "orc_gauss_snapshot": (None, [P]),
        "orc_gauss_residual": (C.c_double, [P]),
        "orc_field_energy": (C.c_double, [P]),
        "orc_kinetic_energy": (C.c_double, [P]),
        "orc_divb": (None, [P, D]),
        "orc_luminosity": (None, [P, C.c_double, D]),
        "orc_counters": (None, [P, C.POINTER(C.c_int64)]),
        "orc_splitmix64": (C.c_uint64, [C.c_uint64, C.c_uint64]),
        "orc_axis_ties": (I64, [P]),
        "orc_inject_ties": (I64, [P]),
        "orc_set_axis_hints": (None, [P, I64, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def courant_dt(p: Params, courant: float) -> float:
    return _load().orc_courant_dt(C.byref(p), courant)


def splitmix64(seed: int, n: int) -> int:
    """Output number n + 1 of the SplitMix64 stream seeded with `seed`."""
    return int(_load().orc_splitmix64(seed, n))


def push(pusher, qmdt, E, B, u):
    """One push of momentum u (Cartesian, modified copy returned)."""
    lib = _load()
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    pz = PUSHER[pusher] if isinstance(pusher, str) else pusher
    lib.orc_push(pz, qmdt, _dp(E), _dp(B), _dp(u))
    return u


class Oracle:
    """One oracle simulation (plain FP64, single thread)."""

    def __init__(self, p: Params):
        self.lib = _load()
        self.p = p
        self.h = self.lib.orc_create(C.byref(p))
        if not self.h:
            raise MemoryError("orc_create failed")
        self.nr, self.nth = p.nr, p.nth
        self.g = self.lib.orc_ghost(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc_destroy(h)
            self.h = None

    # -- geometry ---------------------------------------------------------
    def f_r(self, x1):
        return np.vectorize(lambda v: self.lib.orc_f_r(self.h, float(v)))(x1)

    def f_th(self, x2):
        return np.vectorize(lambda v: self.lib.orc_f_th(self.h, float(v)))(x2)

    def f_r_inv(self, r):
        return np.vectorize(lambda v: self.lib.orc_f_r_inv(self.h, float(v)))(r)

    def f_th_inv(self, th):
        return np.vectorize(lambda v: self.lib.orc_f_th_inv(self.h, float(v)))(th)

    @property
    def field_shape(self):
        return (6, self.nr + 1, self.nth + 1)

    @property
    def flux_shape(self):
        return (3, self.nr + 2 * self.g + 1, self.nth + 1)

    # -- state ------------------------------------------------------------
    def load(self, x1, x2, ur, uth, uph, qw, ids=None):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x1, x2, ur, uth, uph, qw)]
        n = len(arrs[0])
        idp = None
        if ids is not None:
            ids = np.ascontiguousarray(ids, dtype=np.int64)
            idp = _ip(ids)
        self.lib.orc_load_particles(self.h, n, *[_dp(a) for a in arrs], idp)

    def particles(self):
        n = self.lib.orc_num_particles(self.h)
        out = {k: np.empty(n) for k in ("x1", "x2", "ur", "uth", "uph", "qw")}
        ids = np.empty(n, dtype=np.int64)
        self.lib.orc_get_particles(self.h, *[_dp(out[k]) for k in ("x1", "x2", "ur", "uth", "uph", "qw")], _ip(ids))
        out["id"] = ids
        return out

    def num_particles(self):
        return self.lib.orc_num_particles(self.h)

    def set_clock(self, step, next_id):
        self.lib.orc_set_clock(self.h, step, next_id)

    def fields(self, total=False):
        """Plasma fields, or with total=True plasma plus analytic field."""
        a = np.zeros(self.field_shape)
        (self.lib.orc_get_fields_total if total else self.lib.orc_get_fields)(self.h, _dp(a))
        return a

    def set_fields(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(self.field_shape)
        self.lib.orc_set_fields(self.h, _dp(a))

    def flux(self):
        a = np.zeros(self.flux_shape)
        self.lib.orc_get_flux(self.h, _dp(a))
        return a

    def step(self, n=1):
        self.lib.orc_step(self.h, n)
        return self.error()

    def particles_only(self):
        """The particle part of one step, fields untouched (sampled replays)."""
        self.lib.orc_particles_only(self.h)
        return self.error()

    def field_step(self, n=1):
        self.lib.orc_field_step(self.h, n)

    def error(self):
        return self.lib.orc_last_error(self.h)

    # -- building blocks --------------------------------------------------
    def vacuum(self, x1, x2, t):
        E, B = np.zeros(3), np.zeros(3)
        self.lib.orc_vacuum_fields(self.h, x1, x2, t, _dp(E), _dp(B))
        return E, B

    def gather(self, x1, x2, t):
        E, B = np.zeros(3), np.zeros(3)
        self.lib.orc_gather(self.h, x1, x2, t, _dp(E), _dp(B))
        return E, B

    def deposit_path(self, qw, a1, a2, b1, b2, fr=None, fth=None):
        if fr is None:
            fr = np.zeros(self.flux_shape[1:])
            fth = np.zeros(self.flux_shape[1:])
        rc = self.lib.orc_deposit_path(self.h, qw, a1, a2, b1, b2, _dp(fr), _dp(fth))
        return rc, fr, fth

    def filter_pass(self, f, half_j, sign):
        f = np.ascontiguousarray(f, dtype=np.float64).copy()
        self.lib.orc_filter_pass(self.h, _dp(f), half_j, sign)
        return f

    # -- diagnostics ------------------------------------------------------
    def node_charge(self, absolute=False):
        q = np.zeros(self.flux_shape[1:])
        self.lib.orc_node_charge(self.h, 1 if absolute else 0, _dp(q))
        return q

    def gauss_snapshot(self):
        self.lib.orc_gauss_snapshot(self.h)

    def gauss_residual(self):
        return self.lib.orc_gauss_residual(self.h)

    def field_energy(self):
        return self.lib.orc_field_energy(self.h)

    def kinetic_energy(self):
        return self.lib.orc_kinetic_energy(self.h)

    def divb(self):
        a = np.zeros((self.nr, self.nth))
        self.lib.orc_divb(self.h, _dp(a))
        return a

    def luminosity(self, t):
        """Radial Poynting flux through the sphere of each node radius."""
        a = np.zeros(self.nr + 1)
        self.lib.orc_luminosity(self.h, t, _dp(a))
        return a

    def axis_ties(self):
        """Ties of the azimuth branch at the polar axis met so far (R15)."""
        return int(self.lib.orc_axis_ties(self.h))

    def inject_ties(self):
        """Variable-count injection draws within 1e-4 n_j of their rounding
        threshold so far (where a surface field held to a lower precision may
        round the cell the other way)."""
        return int(self.lib.orc_inject_ties(self.h))

    def set_axis_hints(self, ties):
        """Follow another run's branches at its logged ties: dict of step, id, sign."""
        st = np.ascontiguousarray(ties["step"], dtype=np.int64)
        ids = np.ascontiguousarray(ties["id"], dtype=np.int64)
        sg = np.ascontiguousarray(ties["sign"], dtype=np.int32)
        self.lib.orc_set_axis_hints(self.h, len(st), _ip(st), _ip(ids), sg.ctypes.data_as(C.POINTER(C.c_int32)))

    def counters(self):
        a = np.zeros(5, dtype=np.int64)
        self.lib.orc_counters(self.h, _ip(a))
        return {"live": int(a[0]), "deleted": int(a[1]), "injected": int(a[2]), "next_id": int(a[3]),
                "capped": int(a[4])}
