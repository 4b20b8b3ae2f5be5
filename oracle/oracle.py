"""ctypes wrapper around the plain-C oracle (``rod_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Arrays follow the component-major layout of ``rodgen``.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["rod_oracle.c"]
_LIB_NAME = "liboracle.so"
_lock = threading.RLock()


def oracle_library_path() -> str:
    return os.path.join(_HERE, _LIB_NAME)


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FP contraction).  Returns the .so path."""
    out = oracle_library_path()
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "rod_oracle.h")]
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas",
           "-o", tmp] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, out)
    return out


def build_oracle_omp(force: bool = False) -> str:
    """The same source compiled with -fopenmp: the per-rod loop of the right-hand side and the
    per-item loops of the update run on all host cores (contact stays serial); every item is
    computed by one thread with the same operations, so the results are those of the plain build
    bit for bit.  Returns the .so path (use it through ``using_library``)."""
    out = os.path.join(_HERE, "liboracle_omp.so")
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "rod_oracle.h")]
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas",
           "-o", tmp] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, out)
    return out


def omp_threads(path: str) -> int:
    """Threads the OpenMP build at `path` runs its parallel loops with."""
    lib = C.CDLL(path)
    return int(lib.omp_get_max_threads())


def build_oracle_ad(force: bool = False) -> str:
    """Compile oracle_ad.cpp (the oracle's source over dual and counting number types) with g++,
    same flags as the oracle.  Returns the .so path."""
    out = os.path.join(_HERE, "liboracle_ad.so")
    srcs = [os.path.join(_HERE, s) for s in ("oracle_ad.cpp", "rod_oracle.c", "rod_oracle.h")]
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas",
           "-I", _HERE, "-o", tmp, os.path.join(_HERE, "oracle_ad.cpp"), "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, out)
    return out


_ad_lib = None


def _load_ad():
    global _ad_lib
    with _lock:
        if _ad_lib is None:
            lib = C.CDLL(build_oracle_ad())
            P = C.POINTER(_Params)
            d = C.c_void_p
            lib.orcd_step_jvp.argtypes = [P, C.c_double, C.c_double, C.c_int64] + [d] * 10
            lib.orcd_last_error.restype = C.c_char_p
            lib.orcc_step_count.argtypes = [P, C.c_double, C.c_double, C.c_int64] + [d] * 5
            lib.orcc_last_error.restype = C.c_char_p
            _ad_lib = lib
    return _ad_lib


# operation classes counted by Oracle.step_count, in the library's order
COUNT_NAMES = ("add", "mul", "div", "sqrt", "sincos", "atan2", "floor", "fabs")


class _Params(C.Structure):
    _fields_ = [
        ("n_rods", C.c_int32),
        ("n_elem", C.c_void_p),
        ("rest_len", C.c_void_p),
        ("radius", C.c_void_p),
        ("youngs", C.c_void_p),
        ("shear_mod", C.c_void_p),
        ("density", C.c_void_p),
        ("alpha_c", C.c_double),
        ("clamp_base", C.c_void_p),
        ("rest_kappa", C.c_void_p),
        ("rest_sigma", C.c_void_p),
        ("gravity", C.c_double * 3),
        ("nu_damp", C.c_double),
        ("stokes_gamma", C.c_double),
        ("tip_force", C.c_void_p),
        ("act_amp", C.c_void_p),
        ("act_period", C.c_void_p),
        ("act_phase", C.c_void_p),
        ("elem_couple", C.c_void_p),
        ("contact", C.c_int32),
        ("contact_k", C.c_double),
        ("contact_c", C.c_double),
        ("cell_size", C.c_double),
        ("broad_phase", C.c_int32),
        ("magnetization", C.c_void_p),
        ("field_b0", C.c_double * 3),
        ("field_bc", C.c_double * 3),
        ("field_bs", C.c_double * 3),
        ("field_omega", C.c_double),
        ("muscle_amp", C.c_void_p),
        ("muscle_period", C.c_void_p),
        ("muscle_wavelength", C.c_void_p),
        ("muscle_phase", C.c_void_p),
        ("contact_mu", C.c_double),
        ("contact_vslip", C.c_double),
        ("n_walls", C.c_int32),
        ("wall_point", C.c_void_p),
        ("wall_normal", C.c_void_p),
        ("wall_velocity", C.c_void_p),
        ("wall_k", C.c_double),
        ("wall_c", C.c_double),
        ("wall_mu", C.c_double),
        ("wall_vslip", C.c_double),
    ]


_libs = {}
_active = None  # path of a library that replaces the default one (pin-strength tests only)


def _load():
    with _lock:
        path = _active or build_oracle()
        lib = _libs.get(path)
        if lib is None:
            lib = C.CDLL(path)
            P = C.POINTER(_Params)
            d = C.c_void_p
            lib.orc_rhs.argtypes = [P, C.c_double, d, d, d, d, d, d]
            lib.orc_step.argtypes = [P, C.c_double, C.c_double, C.c_int64, d, d, d, d]
            lib.orc_energy.argtypes = [P, d, d, d, d]
            lib.orc_energy.restype = C.c_double
            lib.orc_strains.argtypes = [P, d, d, d, d, d, d]
            lib.orc_contact_forces.argtypes = [P, d, d, d]
            lib.orc_contact_pairs.argtypes = [P, d, d, C.c_int64]
            lib.orc_contact_pairs.restype = C.c_int64
            lib.orc_segment_closest.argtypes = [d, d, d, d, d, d]
            lib.orc_rot_exp.argtypes = [d, d]
            lib.orc_rot_log.argtypes = [d, d]
            lib.orc_orthonormality_error.argtypes = [P, d]
            lib.orc_orthonormality_error.restype = C.c_double
            lib.orc_last_error.restype = C.c_char_p
            _libs[path] = lib
    return lib


@contextlib.contextmanager
def using_library(path):
    """Within the block, oracles created and module functions called use the oracle library at
    `path` (a build of a patched source, see mutants.py) instead of the default one."""
    global _active
    with _lock:
        prev, _active = _active, path
    try:
        yield
    finally:
        with _lock:
            _active = prev


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _opt(a):
    return None if a is None else _f64(a)


class Oracle:
    """Oracle bound to one ``rodgen.RodProblem`` description (parameters, not state)."""

    def __init__(self, problem, broad_phase: int = 1):
        self.lib = _load()
        p = problem
        self.problem = p
        # keep every array alive for the lifetime of the params struct
        self._keep = {
            "n_elem": np.ascontiguousarray(p.n_elem, dtype=np.int32),
            "rest_len": _f64(p.rest_len),
            "radius": _f64(p.radius),
            "youngs": _f64(p.youngs),
            "shear_mod": _f64(p.shear_mod),
            "density": _f64(p.density),
            "clamp_base": None if p.clamp_base is None else np.ascontiguousarray(p.clamp_base, dtype=np.int8),
            "rest_kappa": None if p.rest_kappa is None else _f64(p.rest_kappa),
            "rest_sigma": None if p.rest_sigma is None else _f64(p.rest_sigma),
            "tip_force": None if p.tip_force is None else _f64(p.tip_force),
            "act_amp": None if p.act_amp is None else _f64(p.act_amp),
            "act_period": None if p.act_period is None else _f64(p.act_period),
            "act_phase": None if p.act_phase is None else _f64(p.act_phase),
            "elem_couple": None if p.elem_couple is None else _f64(p.elem_couple),
            "magnetization": _opt(getattr(p, "magnetization", None)),
            "muscle_amp": _opt(getattr(p, "muscle_amp", None)),
            "muscle_period": _opt(getattr(p, "muscle_period", None)),
            "muscle_wavelength": _opt(getattr(p, "muscle_wavelength", None)),
            "muscle_phase": _opt(getattr(p, "muscle_phase", None)),
            "wall_point": _opt(getattr(p, "wall_point", None)),
            "wall_normal": _opt(getattr(p, "wall_normal", None)),
            "wall_velocity": _opt(getattr(p, "wall_velocity", None)),
        }
        k = self._keep
        prm = _Params()
        prm.n_rods = p.n_rods
        for name in ("n_elem", "rest_len", "radius", "youngs", "shear_mod", "density", "clamp_base",
                     "rest_kappa", "rest_sigma", "tip_force", "act_amp", "act_period", "act_phase",
                     "elem_couple", "magnetization", "muscle_amp", "muscle_period", "muscle_wavelength",
                     "muscle_phase", "wall_point", "wall_normal", "wall_velocity"):
            setattr(prm, name, _ptr(k[name]))
        for name in ("field_b0", "field_bc", "field_bs"):
            setattr(prm, name, (C.c_double * 3)(*[float(g) for g in getattr(p, name, (0.0, 0.0, 0.0))]))
        prm.field_omega = float(getattr(p, "field_omega", 0.0))
        prm.contact_mu = float(getattr(p, "contact_mu", 0.0))
        prm.contact_vslip = float(getattr(p, "contact_vslip", 0.0))
        wp = k["wall_point"]
        prm.n_walls = 0 if wp is None else int(wp.size // 3)
        for name in ("wall_k", "wall_c", "wall_mu", "wall_vslip"):
            setattr(prm, name, float(getattr(p, name, 0.0)))
        prm.alpha_c = p.alpha_c
        prm.gravity = (C.c_double * 3)(*[float(g) for g in p.gravity])
        prm.nu_damp = p.nu_damp
        prm.stokes_gamma = p.stokes_gamma
        prm.contact = 1 if p.contact else 0
        prm.contact_k = p.contact_k
        prm.contact_c = p.contact_c
        prm.cell_size = p.cell_size
        prm.broad_phase = broad_phase
        self.params = prm
        self.N, self.E, self.V = p.n_nodes, p.n_elems, p.n_voronoi

    def _check(self, rc):
        if rc != 0:
            raise RuntimeError("oracle: " + self.lib.orc_last_error().decode())

    def set_broad_phase(self, mode: int):
        self.params.broad_phase = mode

    def rhs(self, x, v, Q, w, t=0.0):
        x, v, Q, w = map(_f64, (x, v, Q, w))
        av = np.empty((3, self.N))
        aw = np.empty((3, self.E))
        self._check(self.lib.orc_rhs(C.byref(self.params), t, _ptr(x), _ptr(v), _ptr(Q), _ptr(w), _ptr(av), _ptr(aw)))
        return av, aw

    def step(self, x, v, Q, w, dt, n_steps, t=0.0):
        """Returns new copies of the state after ``n_steps`` steps."""
        x, v, Q, w = (np.array(a, dtype=np.float64, order="C", copy=True) for a in (x, v, Q, w))
        self._check(self.lib.orc_step(C.byref(self.params), t, dt, int(n_steps), _ptr(x), _ptr(v), _ptr(Q), _ptr(w)))
        return x, v, Q, w

    def step_jvp(self, state, tangents, dt, n_steps, t=0.0, d_rest_kappa=None, d_elem_couple=None):
        """Forward-mode derivative of ``n_steps`` oracle steps (the oracle's source over dual
        numbers): returns (new state, its tangent) for the state tangent ``tangents`` and the
        rest-curvature and element-couple tangents (None: zero).  The state part equals
        ``step`` bit for bit."""
        lib = _load_ad()
        st = [np.array(a, dtype=np.float64, order="C", copy=True) for a in state]
        tg = [np.array(a, dtype=np.float64, order="C", copy=True) for a in tangents]
        dk = None if d_rest_kappa is None else _f64(d_rest_kappa)
        dc = None if d_elem_couple is None else _f64(d_elem_couple)
        rc = lib.orcd_step_jvp(C.byref(self.params), t, dt, int(n_steps), *[_ptr(a) for a in st],
                               *[_ptr(a) for a in tg], _ptr(dk), _ptr(dc))
        if rc != 0:
            raise RuntimeError("oracle (dual): " + lib.orcd_last_error().decode())
        return st, tg

    def step_count(self, state, dt, n_steps, t=0.0):
        """``n_steps`` oracle steps counting the FP64 work: (new state, {class: count}) with the
        classes of COUNT_NAMES."""
        lib = _load_ad()
        st = [np.array(a, dtype=np.float64, order="C", copy=True) for a in state]
        counts = np.zeros(len(COUNT_NAMES), dtype=np.int64)
        rc = lib.orcc_step_count(C.byref(self.params), t, dt, int(n_steps), *[_ptr(a) for a in st], _ptr(counts))
        if rc != 0:
            raise RuntimeError("oracle (counting): " + lib.orcc_last_error().decode())
        return st, dict(zip(COUNT_NAMES, (int(c) for c in counts)))

    def energy(self, x, v, Q, w):
        x, v, Q, w = map(_f64, (x, v, Q, w))
        return self.lib.orc_energy(C.byref(self.params), _ptr(x), _ptr(v), _ptr(Q), _ptr(w))

    def strains(self, x, Q):
        x, Q = map(_f64, (x, Q))
        sig = np.empty((3, self.E))
        kap = np.empty((3, max(self.V, 1)))
        dil = np.empty(self.E)
        vdil = np.empty(max(self.V, 1))
        self._check(self.lib.orc_strains(C.byref(self.params), _ptr(x), _ptr(Q), _ptr(sig), _ptr(kap), _ptr(dil), _ptr(vdil)))
        return sig, kap[:, : self.V], dil, vdil[: self.V]

    def contact_forces(self, x, v=None):
        x = _f64(x)
        v = None if v is None else _f64(v)
        f = np.empty((3, self.N))
        self._check(self.lib.orc_contact_forces(C.byref(self.params), _ptr(x), _ptr(f), _ptr(v)))
        return f

    def contact_pairs(self, x, cap=1 << 20):
        x = _f64(x)
        pairs = np.empty((cap, 2), dtype=np.int64)
        n = self.lib.orc_contact_pairs(C.byref(self.params), _ptr(x), _ptr(pairs), cap)
        if n < 0:
            self._check(-1)
        if n > cap:
            return self.contact_pairs(x, cap=int(n))
        return pairs[:n].copy()

    def orthonormality_error(self, Q):
        Q = _f64(Q)
        return self.lib.orc_orthonormality_error(C.byref(self.params), _ptr(Q))


def rot_exp(phi):
    lib = _load()
    phi = _f64(phi)
    R = np.empty(9)
    lib.orc_rot_exp(_ptr(phi), _ptr(R))
    return R.reshape(3, 3)


def rot_log(R):
    lib = _load()
    R = _f64(np.asarray(R).reshape(9))
    phi = np.empty(3)
    lib.orc_rot_log(_ptr(R), _ptr(phi))
    return phi


def segment_closest(p0, p1, q0, q1):
    lib = _load()
    a = [_f64(z) for z in (p0, p1, q0, q1)]
    s = np.zeros(1)
    u = np.zeros(1)
    lib.orc_segment_closest(*[_ptr(z) for z in a], _ptr(s), _ptr(u))
    return float(s[0]), float(u[0])


