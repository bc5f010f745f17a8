"""Thin ctypes binding of the C-ABI in include/picsar.h (argument marshalling only).

Every step of the method runs in the CUDA library ``_build/libpicsar_gb300.so``;
this module only converts Python/NumPy/torch arguments to pointers.  There is
no CPU fallback: if the library is missing the import of ``lib()`` fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpicsar_gb300.so")

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_ECAPACITY, PIC_ENAN, PIC_ECOURANT, PIC_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
PIC_R_LINEAR, PIC_R_LOG = 0, 1
PIC_TH_LINEAR, PIC_TH_EQUAL_AREA = 0, 1
PIC_ABSORB_NONE, PIC_ABSORB_LINEAR, PIC_ABSORB_QUADRATIC = 0, 1, 2
PIC_VAC_NONE, PIC_VAC_MONOPOLE, PIC_VAC_MONOPOLE_ROTATOR, PIC_VAC_UNIFORM_BZ, PIC_VAC_DIPOLE_COROT = 0, 1, 2, 3, 4
PIC_VAC_DIPOLE_ROTATOR = 5
PIC_INJECT_OFF, PIC_INJECT_FIXED, PIC_INJECT_VARIABLE = 0, 1, 2
PIC_FIELDS_PLASMA, PIC_FIELDS_TOTAL = 0, 1
PIC_FP64, PIC_FP32 = 0, 1
PIC_VAY, PIC_BORIS = 0, 1
PIC_MEM_HOST, PIC_MEM_DEVICE = 0, 1

EXPORTS = ["pic_init_grid", "pic_load_particles", "pic_step", "pic_get_fields", "pic_set_fields", "pic_get_flux",
           "pic_get_particles", "pic_get_particles_noalloc", "pic_get_live", "pic_get_moments", "pic_get_luminosity",
           "pic_gauss_snapshot", "pic_set_clock", "pic_profile", "pic_get_profile", "pic_get_launches",
           "pic_ensemble_step", "pic_autotune", "pic_autotune_ensemble", "pic_destroy", "pic_last_error",
           "pic_struct_sizes", "pic_get_charge", "pic_grid_coords", "pic_get_axis_ties", "pic_set_axis_hints",
           "pic_wait_selftest",
           "pic_slabs_init", "pic_slabs_load_particles", "pic_slabs_step", "pic_slabs_get_fields",
           "pic_slabs_get_flux", "pic_slabs_get_particles", "pic_slabs_get_moments", "pic_slabs_destroy"]


class pic_desc(C.Structure):
    _fields_ = [
        ("nr", C.c_int32), ("nth", C.c_int32),
        ("r_min", C.c_double), ("r_max", C.c_double),
        ("r_map", C.c_int32), ("th_map", C.c_int32),
        ("courant", C.c_double), ("dt", C.c_double),
        ("n_filt", C.c_int32),
        ("absorb_cells", C.c_int32), ("absorb_profile", C.c_int32), ("absorb_sigma_max", C.c_double),
        ("vacuum", C.c_int32), ("b0", C.c_double), ("omega", C.c_double), ("t_spin", C.c_double),
        ("inject", C.c_int32), ("pairs_per_cell", C.c_int32), ("f_inj", C.c_double),
        ("precision", C.c_int32), ("pusher", C.c_int32),
        ("q_over_m", C.c_double),
        ("sort_interval", C.c_int32), ("capacity", C.c_int64),
        ("flux_quantum", C.c_double),
        ("tile_shape", C.c_int32),
        ("inject_smooth", C.c_int32), ("inject_q", C.c_double), ("inject_seed", C.c_uint64),
    ]


class pic_moments(C.Structure):
    _fields_ = [
        ("live", C.c_int64), ("deleted", C.c_int64), ("injected", C.c_int64), ("step", C.c_int64),
        ("time", C.c_double), ("dt", C.c_double),
        ("kinetic_energy", C.c_double), ("field_energy", C.c_double),
        ("gauss_residual", C.c_double), ("total_charge", C.c_double),
        ("inject_capped", C.c_int64), ("axis_ties", C.c_int64),
    ]


_lib = None


def lib():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built: run paper_1407_1810_gb300.build.build() (needs nvcc)")
    L = C.CDLL(LIB_PATH)
    P, D, I64, I32 = C.c_void_p, C.POINTER(C.c_double), C.c_int64, C.c_int32
    sig = {
        "pic_init_grid": [C.POINTER(C.c_void_p), C.POINTER(pic_desc), P],
        "pic_load_particles": [P, I64, P, P, P, P, P, P, I32],
        "pic_step": [P, I32],
        "pic_get_fields": [P, I32, P, C.POINTER(C.c_int64), I32],
        "pic_set_fields": [P, P, I32],
        "pic_get_flux": [P, P, C.POINTER(C.c_int64), I32],
        "pic_get_charge": [P, I32, P, C.POINTER(C.c_int64), I32],
        "pic_grid_coords": [P, I64, P, P, P, P, I32],
        "pic_get_particles": [P, C.POINTER(C.c_int64), P, P, P, P, P, P, P, I32],
        "pic_get_moments": [P, C.POINTER(pic_moments)],
        "pic_get_live": [P, C.POINTER(C.c_int64), C.POINTER(C.c_double)],
        "pic_get_luminosity": [P, P, C.POINTER(C.c_int64), I32],
        "pic_get_particles_noalloc": [P, C.POINTER(C.c_int64), P, P, P, P, P, P, P],
        "pic_gauss_snapshot": [P],
        "pic_set_clock": [P, I64, I64],
        "pic_profile": [P, I32],
        "pic_get_profile": [P, D, C.POINTER(C.c_int64)],
        "pic_get_launches": [P, C.POINTER(C.c_int64)],
        "pic_ensemble_step": [C.POINTER(C.c_void_p), I32, I32, C.POINTER(C.c_int64)],
        "pic_autotune": [P, I32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
        "pic_autotune_ensemble": [C.POINTER(C.c_void_p), I32, I32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
        "pic_destroy": [P],
        "pic_get_axis_ties": [P, C.POINTER(C.c_int64), P, P, P],
        "pic_wait_selftest": [I64, I32, P],
        "pic_set_axis_hints": [P, I64, P, P, P],
        "pic_slabs_init": [C.POINTER(C.c_void_p), C.POINTER(pic_desc), I32, C.POINTER(C.c_int32), P],
        "pic_slabs_load_particles": [P, I64, P, P, P, P, P, P, I32],
        "pic_slabs_step": [P, I32],
        "pic_slabs_get_fields": [P, I32, P, C.POINTER(C.c_int64), I32],
        "pic_slabs_get_flux": [P, P, C.POINTER(C.c_int64), I32],
        "pic_slabs_get_particles": [P, C.POINTER(C.c_int64), P, P, P, P, P, P, P, I32],
        "pic_slabs_get_moments": [P, C.POINTER(pic_moments)],
        "pic_slabs_destroy": [P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.pic_last_error.restype = C.c_char_p
    L.pic_last_error.argtypes = []
    _lib = L
    return L


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"picsar error {code}: {msg}")
        self.code = code


def check(rc):
    if rc != PIC_OK:
        raise PicError(rc, lib().pic_last_error().decode())
    return rc


def make_desc(**kw) -> pic_desc:
    d = pic_desc()
    enums = {
        "r_map": {"linear": 0, "log": 1}, "th_map": {"linear": 0, "equal_area": 1},
        "absorb_profile": {"none": 0, "linear": 1, "quadratic": 2},
        "vacuum": {"none": 0, "monopole": 1, "monopole_rotator": 2, "uniform_bz": 3, "dipole_corot": 4,
                   "dipole_rotator": 5},
        "inject": {"off": 0, "fixed": 1, "variable": 2},
        "precision": {"fp64": 0, "fp32": 1}, "pusher": {"vay": 0, "boris": 1},
    }
    for k, v in kw.items():
        if k in enums and isinstance(v, str):
            v = enums[k][v]
        setattr(d, k, v)
    return d


def _ptr(a):
    """(pointer, mem) of a contiguous float64/int64 numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return C.c_void_p(a.ctypes.data), PIC_MEM_HOST
    # torch tensor
    assert a.is_contiguous()
    return C.c_void_p(a.data_ptr()), (PIC_MEM_DEVICE if a.is_cuda else PIC_MEM_HOST)


class Simulation:
    """One context of the library: pic_init_grid .. pic_destroy."""

    def __init__(self, desc: pic_desc, stream: int = 0):
        self.L = lib()
        self.desc = desc
        h = C.c_void_p()
        check(self.L.pic_init_grid(C.byref(h), C.byref(desc), C.c_void_p(stream)))
        self.h = h
        self.nr, self.nth = desc.nr, desc.nth
        self.g = desc.n_filt + 2

    def close(self):
        if getattr(self, "h", None):
            self.L.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, x1, x2, ur, uth, uph, qw):
        ptrs = [_ptr(a) for a in (x1, x2, ur, uth, uph, qw)]
        mems = {m for _, m in ptrs}
        assert len(mems) == 1, "all arrays on the host or all on the device"
        n = len(x1)
        check(self.L.pic_load_particles(self.h, n, *[p for p, _ in ptrs], mems.pop()))

    def step(self, n=1):
        return check(self.L.pic_step(self.h, n))

    def step_rc(self, n=1):
        return self.L.pic_step(self.h, n)

    def fields(self, total=False):
        """Plasma fields (6, nr+1, nth+1), or plasma plus analytic field."""
        which = 1 if total else 0
        n = C.c_int64()
        check(self.L.pic_get_fields(self.h, which, None, C.byref(n), PIC_MEM_HOST))
        out = np.empty(n.value)
        check(self.L.pic_get_fields(self.h, which, C.c_void_p(out.ctypes.data), C.byref(n), PIC_MEM_HOST))
        return out.reshape(6, self.nr + 1, self.nth + 1)

    def charge(self, filtered=False):
        """Node charge (nr+2g+1, nth+1), row i+g: pic_get_charge."""
        n = C.c_int64()
        check(self.L.pic_get_charge(self.h, int(filtered), None, C.byref(n), PIC_MEM_HOST))
        out = np.empty(n.value)
        check(self.L.pic_get_charge(self.h, int(filtered), C.c_void_p(out.ctypes.data), C.byref(n), PIC_MEM_HOST))
        return out.reshape(self.nr + 2 * self.g + 1, self.nth + 1)

    def grid_coords(self, r, th):
        """(x1, x2) of physical positions: pic_grid_coords."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        th = np.ascontiguousarray(th, dtype=np.float64)
        x1, x2 = np.empty_like(r), np.empty_like(r)
        check(self.L.pic_grid_coords(self.h, len(r), C.c_void_p(r.ctypes.data), C.c_void_p(th.ctypes.data),
                                     C.c_void_p(x1.ctypes.data), C.c_void_p(x2.ctypes.data), PIC_MEM_HOST))
        return x1, x2

    def set_fields(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        check(self.L.pic_set_fields(self.h, C.c_void_p(f.ctypes.data), PIC_MEM_HOST))

    def flux(self):
        n = C.c_int64()
        check(self.L.pic_get_flux(self.h, None, C.byref(n), PIC_MEM_HOST))
        out = np.empty(n.value)
        check(self.L.pic_get_flux(self.h, C.c_void_p(out.ctypes.data), C.byref(n), PIC_MEM_HOST))
        return out.reshape(3, self.nr + 2 * self.g + 1, self.nth + 1)

    def particles(self, device=None):
        """Live particles as FP64 arrays (id as int64): numpy on the host, or
        torch tensors on ``device`` when one is given."""
        keys = ("x1", "x2", "ur", "uth", "uph", "qw")
        n = C.c_int64(0)
        check(self.L.pic_get_particles(self.h, C.byref(n), None, None, None, None, None, None, None, PIC_MEM_HOST))
        m = n.value
        if device is not None:
            import torch

            out = {k: torch.empty(m, dtype=torch.float64, device=device) for k in keys}
            out["id"] = torch.empty(m, dtype=torch.int64, device=device)
            ptrs = [C.c_void_p(out[k].data_ptr()) for k in (*keys, "id")]
            check(self.L.pic_get_particles(self.h, C.byref(n), *ptrs, PIC_MEM_DEVICE))
            return out
        out = {k: np.empty(m) for k in keys}
        ids = np.empty(m, dtype=np.int64)
        ptrs = [C.c_void_p(out[k].ctypes.data) for k in keys]
        check(self.L.pic_get_particles(self.h, C.byref(n), *ptrs, C.c_void_p(ids.ctypes.data), PIC_MEM_HOST))
        out["id"] = ids
        return out

    def particles_noalloc(self, out: dict):
        """Live particles into caller-owned device tensors (keys x1, x2, ur,
        uth, uph, qw as float64, id as int64 or None); returns the live count.
        Every tensor must be a contiguous CUDA tensor: the C entry point
        writes up to the smallest buffer's length into each of them."""
        import torch

        keys = ("x1", "x2", "ur", "uth", "uph", "qw")
        bufs = [(k, out[k], torch.float64) for k in keys]
        if out.get("id") is not None:
            bufs.append(("id", out["id"], torch.int64))
        for k, t, dt in bufs:
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and t.dtype == dt):
                raise ValueError(f"particles_noalloc: {k} must be a contiguous CUDA tensor of {dt}")
        cap = min(t.numel() for _, t, _ in bufs)
        n = C.c_int64(cap)
        ptrs = [C.c_void_p(out[k].data_ptr()) for k in keys]
        idp = C.c_void_p(out["id"].data_ptr()) if out.get("id") is not None else None
        check(self.L.pic_get_particles_noalloc(self.h, C.byref(n), *ptrs, idp))
        return n.value

    def live(self):
        n, k = C.c_int64(), C.c_double()
        check(self.L.pic_get_live(self.h, C.byref(n), C.byref(k)))
        return n.value

    def moments(self):
        m = pic_moments()
        check(self.L.pic_get_moments(self.h, C.byref(m)))
        return {k: getattr(m, k) for k, _ in pic_moments._fields_}

    def luminosity(self):
        """Spin-down luminosity through the sphere of each node radius (nr + 1
        values, 0 at the conductors): pic_get_luminosity."""
        n = C.c_int64()
        check(self.L.pic_get_luminosity(self.h, None, C.byref(n), PIC_MEM_HOST))
        out = np.empty(n.value)
        check(self.L.pic_get_luminosity(self.h, C.c_void_p(out.ctypes.data), C.byref(n), PIC_MEM_HOST))
        return out

    def gauss_snapshot(self):
        check(self.L.pic_gauss_snapshot(self.h))

    def set_clock(self, step, next_id):
        check(self.L.pic_set_clock(self.h, step, next_id))

    def profile(self, enable=True):
        check(self.L.pic_profile(self.h, 1 if enable else 0))

    def autotune(self, trial_steps=40):
        """Pick tile shape and sort interval by measurement (pic_autotune)."""
        S, sh = C.c_int32(), C.c_int32()
        check(self.L.pic_autotune(self.h, trial_steps, C.byref(S), C.byref(sh)))
        return {"sort_interval": S.value, "tile_shape": sh.value}

    def axis_ties(self):
        """The logged ties of the azimuth branch at the polar axis: dict of
        step, id (int64) and sign (+1 / -1, the branch taken)."""
        n = C.c_int64(0)
        check(self.L.pic_get_axis_ties(self.h, C.byref(n), None, None, None))
        out = {"step": np.empty(n.value, dtype=np.int64), "id": np.empty(n.value, dtype=np.int64),
               "sign": np.empty(n.value, dtype=np.int32)}
        if n.value:
            check(self.L.pic_get_axis_ties(self.h, C.byref(n), *[C.c_void_p(out[k].ctypes.data)
                                                                  for k in ("step", "id", "sign")]))
        return out

    def set_axis_hints(self, ties):
        """Follow another run's branches at the ties it logged (pic_set_axis_hints)."""
        arr = [np.ascontiguousarray(ties[k], dtype=dt) for k, dt in (("step", np.int64), ("id", np.int64),
                                                                      ("sign", np.int32))]
        check(self.L.pic_set_axis_hints(self.h, len(arr[0]), *[C.c_void_p(a.ctypes.data) for a in arr]))

    def launches(self):
        n = C.c_int64()
        check(self.L.pic_get_launches(self.h, C.byref(n)))
        return n.value

    def get_profile(self):
        ms = (C.c_double * 6)()
        steps = C.c_int64()
        check(self.L.pic_get_profile(self.h, ms, C.byref(steps)))
        names = ["particles", "reduce", "filter", "fields", "inject", "sort"]
        return dict(zip(names, list(ms))), steps.value


class Slabs:
    """One simulation split into radial slabs: pic_slabs_init .. pic_slabs_destroy.
    The methods mirror Simulation's for the whole grid."""

    def __init__(self, desc: pic_desc, nslabs: int, rows=None, stream: int = 0):
        self.L = lib()
        self.desc = desc
        h = C.c_void_p()
        rp = None
        if rows is not None:
            rows = (C.c_int32 * len(rows))(*rows)
            rp = C.cast(rows, C.POINTER(C.c_int32))
        check(self.L.pic_slabs_init(C.byref(h), C.byref(desc), nslabs, rp, C.c_void_p(stream)))
        self.h = h
        self.nr, self.nth = desc.nr, desc.nth
        self.g = desc.n_filt + 2

    def close(self):
        if getattr(self, "h", None):
            self.L.pic_slabs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, x1, x2, ur, uth, uph, qw):
        ptrs = [_ptr(a) for a in (x1, x2, ur, uth, uph, qw)]
        mems = {m for _, m in ptrs}
        assert len(mems) == 1, "all arrays on the host or all on the device"
        check(self.L.pic_slabs_load_particles(self.h, len(x1), *[p for p, _ in ptrs], mems.pop()))

    def step(self, n=1):
        return check(self.L.pic_slabs_step(self.h, n))

    def fields(self, total=False):
        n = C.c_int64()
        check(self.L.pic_slabs_get_fields(self.h, 1 if total else 0, None, C.byref(n), PIC_MEM_HOST))
        out = np.empty(n.value)
        check(self.L.pic_slabs_get_fields(self.h, 1 if total else 0, C.c_void_p(out.ctypes.data), C.byref(n),
                                          PIC_MEM_HOST))
        return out.reshape(6, self.nr + 1, self.nth + 1)

    def flux(self):
        n = C.c_int64()
        check(self.L.pic_slabs_get_flux(self.h, None, C.byref(n), PIC_MEM_HOST))
        out = np.empty(n.value)
        check(self.L.pic_slabs_get_flux(self.h, C.c_void_p(out.ctypes.data), C.byref(n), PIC_MEM_HOST))
        return out.reshape(3, self.nr + 2 * self.g + 1, self.nth + 1)

    def particles(self):
        keys = ("x1", "x2", "ur", "uth", "uph", "qw")
        n = C.c_int64(0)
        check(self.L.pic_slabs_get_particles(self.h, C.byref(n), None, None, None, None, None, None, None,
                                             PIC_MEM_HOST))
        out = {k: np.empty(n.value) for k in keys}
        ids = np.empty(n.value, dtype=np.int64)
        ptrs = [C.c_void_p(out[k].ctypes.data) for k in keys]
        check(self.L.pic_slabs_get_particles(self.h, C.byref(n), *ptrs, C.c_void_p(ids.ctypes.data), PIC_MEM_HOST))
        out = {k: v[: n.value] for k, v in out.items()}
        out["id"] = ids[: n.value]
        return out

    def moments(self):
        m = pic_moments()
        check(self.L.pic_slabs_get_moments(self.h, C.byref(m)))
        return {k: getattr(m, k) for k, _ in pic_moments._fields_}


def wait_selftest(polls, arrive_first, stream=0):
    """Return code of pic_wait_selftest (PIC_ETIMEOUT or PIC_OK expected)."""
    return lib().pic_wait_selftest(polls, 1 if arrive_first else 0, C.c_void_p(stream))


def autotune_ensemble(sims, trial_steps=40):
    """One tile shape and sort interval for all members, by timing the
    batched step on clones (pic_autotune_ensemble)."""
    arr = (C.c_void_p * len(sims))(*[s.h for s in sims])
    S, sh = C.c_int32(0), C.c_int32(0)
    check(lib().pic_autotune_ensemble(arr, len(sims), trial_steps, C.byref(S), C.byref(sh)))
    return {"sort_interval": S.value, "tile_shape": sh.value}


def ensemble_step(sims, nsteps):
    """Advance the simulations together (pic_ensemble_step); returns the
    number of kernel launches the call enqueued."""
    arr = (C.c_void_p * len(sims))(*[s.h for s in sims])
    k = C.c_int64(0)
    check(lib().pic_ensemble_step(arr, len(sims), nsteps, C.byref(k)))
    return k.value
