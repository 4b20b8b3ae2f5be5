"""ctypes binding of librod (include/rod.h): argument marshalling only.

Every step of the rod method runs in the CUDA library; this module converts arrays to
pointers, keeps them alive for the duration of a call and turns status codes into
exceptions.  PyTorch provides device memory (for device-side state transfers and for the
outputs of the debug entry points) and the CUDA stream.  There is no CPU fallback: if the
library cannot be loaded, importing or using this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBRARY_PATH = os.path.join(_HERE, "librod.so")

ROD_OK = 0
STATUS_NAMES = {0: "ROD_OK", -1: "ROD_ERR_ARG", -2: "ROD_ERR_CUDA", -3: "ROD_ERR_NONFINITE",
                -4: "ROD_ERR_TIMEOUT", -5: "ROD_ERR_OVERFLOW", -6: "ROD_ERR_STATE"}


class RodError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class SurrogateStats(C.Structure):
    """rod_surrogate_stats."""
    _fields_ = [("surrogate_calls", C.c_int64), ("fallback_calls", C.c_int64), ("checks", C.c_int64),
                ("max_err", C.c_double), ("last_err", C.c_double), ("rejected_err", C.c_double),
                ("sum_err", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RodSystemDesc(C.Structure):
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
        ("cuda_stream", C.c_void_p),
        ("magnetization", C.c_void_p),
        ("field_b0", C.c_double * 3),
        ("field_bc", C.c_double * 3),
        ("field_bs", C.c_double * 3),
        ("field_omega", C.c_double),
        ("muscle_amp", C.c_void_p),
        ("muscle_period", C.c_void_p),
        ("muscle_wavelength", C.c_void_p),
        ("muscle_phase", C.c_void_p),
        ("n_walls", C.c_int32),
        ("wall_point", C.c_void_p),
        ("wall_normal", C.c_void_p),
        ("wall_velocity", C.c_void_p),
        ("wall_k", C.c_double),
        ("wall_c", C.c_double),
        ("wall_mu", C.c_double),
        ("wall_vslip", C.c_double),
    ]


# exported symbols and their signatures (argument types, return type)
_P = C.c_void_p
_SIGNATURES = {
    "rod_system_create": ([C.POINTER(RodSystemDesc), C.POINTER(C.c_void_p)], C.c_int),
    "rod_system_destroy": ([_P], C.c_int),
    "rod_system_sizes": ([_P, _P, _P, _P], C.c_int),
    "rod_system_set_state": ([_P, _P, _P, _P, _P, C.c_int], C.c_int),
    "rod_system_get_state": ([_P, _P, _P, _P, _P, C.c_int], C.c_int),
    "rod_system_set_time": ([_P, C.c_double], C.c_int),
    "rod_system_get_time": ([_P, _P], C.c_int),
    "rod_system_step": ([_P, C.c_int64, C.c_double], C.c_int),
    "rod_system_step_async": ([_P, C.c_int64, C.c_double], C.c_int),
    "rod_system_sync": ([_P], C.c_int),
    "rod_system_contact_config": ([_P, C.c_int, C.c_double, C.c_double, C.c_double], C.c_int),
    "rod_system_friction": ([_P, C.c_double, C.c_double], C.c_int),
    "rod_system_contact_skin": ([_P, C.c_double], C.c_int),
    "rod_system_contact_list_builds": ([_P, _P], C.c_int),
    "rod_system_rhs": ([_P, C.c_double, _P, _P], C.c_int),
    "rod_system_contact_forces": ([_P, _P], C.c_int),
    "rod_system_contact_pairs": ([_P, _P, C.c_int64, _P, _P], C.c_int),
    "rod_system_set_launch": ([_P, C.c_int32, C.c_int32], C.c_int),
    "rod_system_get_launch": ([_P, _P, _P], C.c_int),
    "rod_system_pack_info": ([_P, _P, _P, _P], C.c_int),
    "rod_plan_packs": ([_P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P, _P, _P], C.c_int),
    "rod_system_diagnostics": ([_P, _P, _P], C.c_int),
    "rod_system_set_graphs": ([_P, C.c_int], C.c_int),
    "rod_system_set_params": ([_P, _P, _P, C.c_int], C.c_int),
    "rod_system_autotune": ([_P, C.c_double, C.c_int32, _P, _P, _P], C.c_int),
    "rod_system_forward_checkpointed": ([_P, C.c_int64, C.c_double, C.c_int32], C.c_int),
    "rod_system_backward": ([_P, _P, _P, _P, _P, _P, _P], C.c_int),
    "rod_system_adjoint_of_state": ([_P, _P, _P, _P, _P], C.c_int),
    "rod_system_profile": ([_P, C.c_int], C.c_int),
    "rod_profile_classes": ([], C.c_int32),
    "rod_system_profile_read": ([_P, C.c_int32, _P, _P, _P], C.c_int),
    "rod_system_launch_count": ([_P, _P], C.c_int),
    "rod_contact_forces_noalloc": ([C.c_int32, _P, _P, _P, _P, C.c_double, C.c_double, C.c_double, _P, _P],
                                   C.c_int),
    "rod_surrogate_create": ([C.c_int32, C.c_double, C.POINTER(C.c_void_p)], C.c_int),
    "rod_surrogate_destroy": ([_P], C.c_int),
    "rod_surrogate_num_params": ([], C.c_int64),
    "rod_surrogate_set_params": ([_P, _P, C.c_int], C.c_int),
    "rod_surrogate_get_params": ([_P, _P, C.c_int], C.c_int),
    "rod_surrogate_set_scales": ([_P, _P, _P, _P], C.c_int),
    "rod_surrogate_train_step": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_int32, C.c_float, _P, _P], C.c_int),
    "rod_surrogate_get_grad": ([_P, _P, C.c_int], C.c_int),
    "rod_surrogate_forward": ([_P, _P, _P, _P, _P, _P, C.c_int32, _P, _P], C.c_int),
    "rod_surrogate_debug_buffer": ([_P, C.c_int32, _P, C.c_int64, _P], C.c_int),
    "rod_surrogate_set_wait_polls": ([_P, C.c_uint32], C.c_int),
    "rod_surrogate_apply_debug": ([_P, _P, _P, _P, C.c_int64], C.c_int),
    "rod_surrogate_set_prior": ([_P, C.c_int32], C.c_int),
    "rod_surrogate_raw_features": ([_P, _P, _P, _P, _P, _P, C.c_int32, _P, _P, _P], C.c_int),
    "rod_surrogate_raw_targets": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_int32, _P, _P], C.c_int),
    "rod_surrogate_perturb": ([_P, _P, _P, _P, _P, C.c_int32, _P, _P, _P, _P, _P, C.c_double, _P, _P, _P, _P, _P, _P],
                              C.c_int),
    "rod_surrogate_apply": ([_P, _P, C.c_int64], C.c_int),
    "rod_surrogate_rollout": ([_P, _P, _P, _P, C.c_int32, C.c_int64, C.c_int32, C.c_double, _P], C.c_int),
    "rod_surrogate_rollout_local": ([_P, _P, _P, C.c_int32, _P, C.c_int32, C.c_int64, C.c_int32, C.c_double, _P],
                                    C.c_int),
    "rod_max_elements_per_rod": ([], C.c_int32),
    "rod_last_error": ([], C.c_char_p),
    "rod_version": ([], C.c_char_p),
}

_lib = None
_lock = threading.Lock()


def load_library(path: Optional[str] = None):
    """Load librod.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIBRARY_PATH
            if not os.path.exists(p):
                raise ImportError(f"librod.so not found at {p}; build it with paper_2605_13766_gb300.build.build()")
            lib = C.CDLL(p)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _check(status: int):
    if status != ROD_OK:
        raise RodError(status, _lib.rod_last_error().decode(errors="replace"))


def _host(a, dtype=np.float64):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


class RodSystem:
    """One ensemble of rods on the GPU (a handle on ``rod_system``).

    ``problem`` is any object with the attributes of ``rodgen.RodProblem`` (sizes, materials,
    loads, optional contact settings).  The state is set separately with ``set_state``.
    """

    def __init__(self, problem, stream=None, use_torch_stream: bool = True):
        lib = load_library()
        self.lib = lib
        p = problem
        keep = {
            "n_elem": _host(p.n_elem, np.int32),
            "rest_len": _host(p.rest_len),
            "radius": _host(p.radius),
            "youngs": _host(p.youngs),
            "shear_mod": _host(p.shear_mod),
            "density": _host(p.density),
            "clamp_base": _host(getattr(p, "clamp_base", None), np.int8),
            "rest_kappa": _host(getattr(p, "rest_kappa", None)),
            "rest_sigma": _host(getattr(p, "rest_sigma", None)),
            "tip_force": _host(getattr(p, "tip_force", None)),
            "act_amp": _host(getattr(p, "act_amp", None)),
            "act_period": _host(getattr(p, "act_period", None)),
            "act_phase": _host(getattr(p, "act_phase", None)),
            "elem_couple": _host(getattr(p, "elem_couple", None)),
            "magnetization": _host(getattr(p, "magnetization", None)),
            "muscle_amp": _host(getattr(p, "muscle_amp", None)),
            "muscle_period": _host(getattr(p, "muscle_period", None)),
            "muscle_wavelength": _host(getattr(p, "muscle_wavelength", None)),
            "muscle_phase": _host(getattr(p, "muscle_phase", None)),
            "wall_point": _host(getattr(p, "wall_point", None)),
            "wall_normal": _host(getattr(p, "wall_normal", None)),
            "wall_velocity": _host(getattr(p, "wall_velocity", None)),
        }
        d = RodSystemDesc()
        d.n_rods = int(keep["n_elem"].shape[0])
        for k, v in keep.items():
            setattr(d, k, _ptr(v))
        d.alpha_c = float(getattr(p, "alpha_c", 4.0 / 3.0))
        d.gravity = (C.c_double * 3)(*[float(g) for g in getattr(p, "gravity", (0.0, 0.0, 0.0))])
        d.nu_damp = float(getattr(p, "nu_damp", 0.0))
        d.stokes_gamma = float(getattr(p, "stokes_gamma", 0.0))
        for name in ("field_b0", "field_bc", "field_bs"):
            setattr(d, name, (C.c_double * 3)(*[float(g) for g in getattr(p, name, (0.0, 0.0, 0.0))]))
        d.field_omega = float(getattr(p, "field_omega", 0.0))
        d.n_walls = 0 if keep["wall_point"] is None else int(keep["wall_point"].size // 3)
        for name in ("wall_k", "wall_c", "wall_mu", "wall_vslip"):
            setattr(d, name, float(getattr(p, name, 0.0)))
        self.torch_stream = None
        if stream is None and use_torch_stream:
            import torch
            cur = torch.cuda.current_stream()
            # the legacy default stream has handle 0, which the library reads as "make your
            # own stream"; give the system a torch stream of its own instead and keep it, so
            # that callers can order torch work and record events on the stream it runs on
            self.torch_stream = cur if cur.cuda_stream else torch.cuda.Stream()
            stream = self.torch_stream.cuda_stream
        d.cuda_stream = stream
        handle = C.c_void_p()
        _check(lib.rod_system_create(C.byref(d), C.byref(handle)))
        self.handle = handle
        n, e, v = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib.rod_system_sizes(handle, C.byref(n), C.byref(e), C.byref(v)))
        self.n_nodes, self.n_elems, self.n_voronoi = n.value, e.value, v.value
        self.n_rods = d.n_rods
        if getattr(p, "contact", False):
            self.contact_config(True, p.contact_k, p.contact_c, p.cell_size)
        if float(getattr(p, "contact_mu", 0.0)) > 0:
            self.friction(p.contact_mu, p.contact_vslip)

    # -- lifetime
    def close(self):
        if getattr(self, "handle", None):
            self.lib.rod_system_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state
    def set_state(self, x, v, Q, w):
        """Host numpy arrays (copied synchronously) or CUDA torch tensors (copied on the stream)."""
        on_dev = not isinstance(x, np.ndarray)
        if on_dev:
            import torch
            arrs = [a.contiguous() for a in (x, v, Q, w)]
            for a in arrs:
                if a.dtype != torch.float64 or not a.is_cuda:
                    raise TypeError("device state must be float64 CUDA tensors")
            if self.torch_stream is not None:
                self.torch_stream.wait_stream(torch.cuda.current_stream())
        else:
            arrs = [_host(a) for a in (x, v, Q, w)]
        self._check_shapes(arrs)
        _check(self.lib.rod_system_set_state(self.handle, *[_ptr(a) for a in arrs], 1 if on_dev else 0))
        self._keep_state_inputs = arrs  # alive until the stream has copied them

    def get_state(self, device: bool = False, out=None):
        """The state (x, v, Q, w).  out: four caller arrays to fill (host numpy, pinned or not,
        or CUDA float64 tensors when device=True) instead of new ones."""
        if out is not None:
            out = list(out)
            if device:
                import torch
                for a in out:
                    if a.dtype != torch.float64 or not a.is_cuda or not a.is_contiguous():
                        raise TypeError("device outputs must be contiguous float64 CUDA tensors")
            else:
                for a in out:
                    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
                        raise TypeError("host outputs must be C-contiguous float64 numpy arrays")
            self._check_shapes(out)
        elif device:
            import torch
            out = [torch.empty((3, self.n_nodes), dtype=torch.float64, device="cuda"),
                   torch.empty((3, self.n_nodes), dtype=torch.float64, device="cuda"),
                   torch.empty((9, self.n_elems), dtype=torch.float64, device="cuda"),
                   torch.empty((3, self.n_elems), dtype=torch.float64, device="cuda")]
        else:
            out = [np.empty((3, self.n_nodes)), np.empty((3, self.n_nodes)),
                   np.empty((9, self.n_elems)), np.empty((3, self.n_elems))]
        _check(self.lib.rod_system_get_state(self.handle, *[_ptr(a) for a in out], 1 if device else 0))
        if device and self.torch_stream is not None:
            import torch
            torch.cuda.current_stream().wait_stream(self.torch_stream)
        return tuple(out)

    def _check_shapes(self, arrs):
        want = [(3, self.n_nodes), (3, self.n_nodes), (9, self.n_elems), (3, self.n_elems)]
        for a, s in zip(arrs, want):
            if tuple(a.shape) != s and (int(np.prod(a.shape)) != s[0] * s[1]):
                raise ValueError(f"state array of shape {tuple(a.shape)}, expected {s}")

    @property
    def time(self) -> float:
        t = C.c_double()
        _check(self.lib.rod_system_get_time(self.handle, C.byref(t)))
        return t.value

    @time.setter
    def time(self, t: float):
        _check(self.lib.rod_system_set_time(self.handle, float(t)))

    # -- stepping
    def step(self, n_steps: int, dt: float):
        _check(self.lib.rod_system_step(self.handle, int(n_steps), float(dt)))

    def step_async(self, n_steps: int, dt: float):
        _check(self.lib.rod_system_step_async(self.handle, int(n_steps), float(dt)))

    def sync(self):
        _check(self.lib.rod_system_sync(self.handle))

    def contact_config(self, enable: bool, k: float = 0.0, c: float = 0.0, cell_size: float = 0.0):
        _check(self.lib.rod_system_contact_config(self.handle, 1 if enable else 0, float(k), float(c),
                                                  float(cell_size)))

    def contact_skin(self, skin: float):
        """Skin list for the contact search: candidates within r_a + r_b + skin, rebuilt on the
        device once a node has moved by skin / 2 (0: search the cell grid at every step)."""
        _check(self.lib.rod_system_contact_skin(self.handle, float(skin)))

    def contact_list_builds(self) -> int:
        """Skin-list builds since the contact grid was last set up (0 without a skin list)."""
        n = C.c_int64(0)
        _check(self.lib.rod_system_contact_list_builds(self.handle, C.byref(n)))
        return int(n.value)

    def friction(self, mu: float, v_slip: float):
        """Rod-rod friction: -mu f_n v_t / max(|v_t|, v_slip) at every contact."""
        _check(self.lib.rod_system_friction(self.handle, float(mu), float(v_slip)))

    # -- debug / parity entry points (device outputs)

    def rhs(self, t: float = 0.0):
        import torch
        av = torch.empty((3, self.n_nodes), dtype=torch.float64, device="cuda")
        aw = torch.empty((3, self.n_elems), dtype=torch.float64, device="cuda")
        _check(self.lib.rod_system_rhs(self.handle, float(t), av.data_ptr(), aw.data_ptr()))
        return av, aw

    def contact_forces(self):
        import torch
        f = torch.empty((3, self.n_nodes), dtype=torch.float64, device="cuda")
        _check(self.lib.rod_system_contact_forces(self.handle, f.data_ptr()))
        return f

    def contact_pair_count(self):
        """(segment pairs in contact, candidate pairs that reached the FP64 test) at the current
        state, by the cell-grid search."""
        n, nc = C.c_int64(0), C.c_int64(0)
        _check(self.lib.rod_system_contact_pairs(self.handle, None, 0, C.byref(n), C.byref(nc)))
        return int(n.value), int(nc.value)

    def contact_pairs(self, cap: Optional[int] = None):
        """Pairs (a, b), a < b, of segments of different rods in contact at the current state,
        found by the cell-grid search: (int64 array [n, 2] sorted by rows, candidates that
        reached the FP64 test).  cap=None counts first and then fetches them all."""
        n, nc = C.c_int64(0), C.c_int64(0)
        if cap is None:
            _check(self.lib.rod_system_contact_pairs(self.handle, None, 0, C.byref(n), C.byref(nc)))
            cap = int(n.value)
        buf = np.zeros((max(int(cap), 1), 2), dtype=np.int64)
        _check(self.lib.rod_system_contact_pairs(self.handle, buf.ctypes.data if cap > 0 else None, int(cap),
                                                 C.byref(n), C.byref(nc)))
        got = buf[:min(int(n.value), int(cap))]
        got = got[np.lexsort((got[:, 1], got[:, 0]))] if len(got) else got.reshape(0, 2)
        return got, int(nc.value)

    # -- differentiation
    def set_params(self, rest_kappa=None, elem_couple=None):
        """Replace the rest curvature (3, V) and/or element couples (3, E): numpy or CUDA tensors."""
        arrs = [rest_kappa, elem_couple]
        on_dev = any(a is not None and not isinstance(a, np.ndarray) for a in arrs)
        if on_dev:
            import torch
            arrs = [None if a is None else a.detach().to(torch.float64).contiguous() for a in arrs]
            if self.torch_stream is not None:
                self.torch_stream.wait_stream(torch.cuda.current_stream())
        else:
            arrs = [_host(a) for a in arrs]
        _check(self.lib.rod_system_set_params(self.handle, _ptr(arrs[0]), _ptr(arrs[1]), 1 if on_dev else 0))
        self._keep_params = arrs

    def forward_checkpointed(self, n_steps: int, dt: float, every: int = 100):
        _check(self.lib.rod_system_forward_checkpointed(self.handle, int(n_steps), float(dt), int(every)))

    def backward(self, gx, gv, gQ, gw):
        """Adjoint of the final state (CUDA tensors) -> (grad rest curvature (3, V), grad couples (3, E))."""
        import torch
        gs = [g.detach().to(torch.float64).contiguous() for g in (gx, gv, gQ, gw)]
        if self.torch_stream is not None:
            self.torch_stream.wait_stream(torch.cuda.current_stream())
        gk = torch.empty((3, max(self.n_voronoi, 1)), dtype=torch.float64, device="cuda")
        gc = torch.empty((3, self.n_elems), dtype=torch.float64, device="cuda")
        _check(self.lib.rod_system_backward(self.handle, *[g.data_ptr() for g in gs], gk.data_ptr(), gc.data_ptr()))
        return gk[:, : self.n_voronoi], gc

    def adjoint_of_state(self):
        import torch
        out = [torch.empty((3, self.n_nodes), dtype=torch.float64, device="cuda"),
               torch.empty((3, self.n_nodes), dtype=torch.float64, device="cuda"),
               torch.empty((9, self.n_elems), dtype=torch.float64, device="cuda"),
               torch.empty((3, self.n_elems), dtype=torch.float64, device="cuda")]
        _check(self.lib.rod_system_adjoint_of_state(self.handle, *[o.data_ptr() for o in out]))
        return tuple(out)

    def use_graphs(self, enable: bool = True):
        _check(self.lib.rod_system_set_graphs(self.handle, 1 if enable else 0))

    # -- tracing
    def profile(self, enable: bool = True):
        _check(self.lib.rod_system_profile(self.handle, 1 if enable else 0))

    def profile_read(self):
        """{kernel class: (total device ms, launches)} from the event pairs recorded so far."""
        out = {}
        for k in range(self.lib.rod_profile_classes()):
            name, ms, n = C.c_char_p(), C.c_double(), C.c_int64()
            _check(self.lib.rod_system_profile_read(self.handle, k, C.byref(name), C.byref(ms), C.byref(n)))
            out[name.value.decode()] = (ms.value, n.value)
        return out

    @property
    def launch_count(self) -> int:
        n = C.c_int64()
        _check(self.lib.rod_system_launch_count(self.handle, C.byref(n)))
        return n.value

    # -- launch shape
    def set_launch(self, elems_per_block: int = 0, threads_per_block: int = 0):
        _check(self.lib.rod_system_set_launch(self.handle, int(elems_per_block), int(threads_per_block)))

    def autotune(self, dt: float, trial_steps: int = 20):
        """Pick the fastest launch shape by timing; returns (elements per block, threads, ms per step)."""
        e, t, ms = C.c_int32(), C.c_int32(), C.c_double()
        _check(self.lib.rod_system_autotune(self.handle, float(dt), int(trial_steps), C.byref(e), C.byref(t),
                                            C.byref(ms)))
        return e.value, t.value, ms.value

    def get_launch(self):
        e, t = C.c_int32(), C.c_int32()
        _check(self.lib.rod_system_get_launch(self.handle, C.byref(e), C.byref(t)))
        return e.value, t.value

    def diagnostics(self, per_rod: bool = True):
        """Energy parts and director orthonormality of the current state.

        Returns (rows, totals): rows a [9, R] device tensor (translational kinetic, rotational
        kinetic, shear/stretch, bend/twist, work potential, max |Q Q^T - I|, tip x, y, z per rod)
        or None, and totals a numpy array of 6 (rows 0-4 summed, row 5 maximised)."""
        import torch
        rows = torch.empty((9, self.n_rods), dtype=torch.float64, device="cuda") if per_rod else None
        tot = np.zeros(6)
        # with totals the call synchronises the system's stream, so the rows are complete on return
        _check(self.lib.rod_system_diagnostics(self.handle, rows.data_ptr() if rows is not None else None,
                                               tot.ctypes.data_as(C.c_void_p)))
        return rows, tot

    def energy(self) -> float:
        """Total energy: kinetic + strain energy + work potential of gravity and tip forces."""
        return float(self.diagnostics(per_rod=False)[1][:5].sum())

    def pack_info(self):
        """(block packs, of which list their rods, rods on the cooperative path)."""
        n, l, g = C.c_int32(), C.c_int32(), C.c_int32()
        _check(self.lib.rod_system_pack_info(self.handle, C.byref(n), C.byref(l), C.byref(g)))
        return n.value, l.value, g.value


class Surrogate:
    """Handle on ``rod_surrogate``: the learned window-of-steps surrogate (BF16 tensor cores).

    Features, outputs and the kinematic prior are described with the C ABI (include/rod.h)."""

    N_FEATURES = 24
    N_OUTPUTS = 15
    POSITIONS = 51

    def __init__(self, window_steps: int = 50, dt: float = 1e-5):
        self.lib = load_library()
        h = C.c_void_p()
        _check(self.lib.rod_surrogate_create(int(window_steps), float(dt), C.byref(h)))
        self.handle = h
        self.window = int(window_steps)
        self.dt = float(dt)
        self.n_params = int(self.lib.rod_surrogate_num_params())
        self.scales = None

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rod_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        if isinstance(params, np.ndarray):
            p = np.ascontiguousarray(params, dtype=np.float32)
            if p.size != self.n_params:
                raise ValueError(f"need {self.n_params} parameters, got {p.size}")
            _check(self.lib.rod_surrogate_set_params(self.handle, p.ctypes.data, 0))
        else:
            p = params.detach().float().contiguous()
            if p.numel() != self.n_params:
                raise ValueError(f"need {self.n_params} parameters, got {p.numel()}")
            _check(self.lib.rod_surrogate_set_params(self.handle, p.data_ptr(), 1))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.n_params, dtype=np.float32)
        _check(self.lib.rod_surrogate_get_params(self.handle, p.ctypes.data, 0))
        return p

    # shapes of rod_surrogate_debug_buffer's arrays per window: (rows, channels)
    _DEBUG_SHAPES = {0: (64, 32), 1: (64, 64), 2: (64, 64), 3: (64, 64), 4: (64, 64), 5: (64, 64), 6: (64, 64),
                     7: (51, 16), 8: (51, 16), 9: (64, 16), 10: (64, 64), 11: (64, 64), 12: (64, 64)}

    def debug_buffer(self, which: int) -> np.ndarray:
        """Intermediate array `which` of the last training step (see include/rod.h), as
        float32 [windows, rows, channels]."""
        n = C.c_int64(0)
        _check(self.lib.rod_surrogate_debug_buffer(self.handle, int(which), None, 0, C.byref(n)))
        out = np.empty(int(n.value), dtype=np.float32)
        _check(self.lib.rod_surrogate_debug_buffer(self.handle, int(which), out.ctypes.data, out.size, C.byref(n)))
        rows, ch = self._DEBUG_SHAPES[int(which)]
        return out.reshape(-1, rows, ch)

    def set_wait_polls(self, polls: int):
        """Polls of the fused kernel's tensor-core waits before ROD_ERR_TIMEOUT (0: default)."""
        _check(self.lib.rod_surrogate_set_wait_polls(self.handle, int(polls)))

    def apply_debug(self, system):
        """One window call with every layer's arrays captured: (pre, act), each float32
        [4 layers, rods, 51 positions, 64 channels] (see include/rod.h)."""
        n = 4 * system.n_rods * 51 * 64
        pre = np.zeros(n, dtype=np.float32)
        act = np.zeros(n, dtype=np.float32)
        _check(self.lib.rod_surrogate_apply_debug(self.handle, system.handle, pre.ctypes.data, act.ctypes.data, n))
        shape = (4, system.n_rods, 51, 64)
        return pre.reshape(shape), act.reshape(shape)

    def get_grad(self) -> np.ndarray:
        g = np.empty(self.n_params, dtype=np.float32)
        _check(self.lib.rod_surrogate_get_grad(self.handle, g.ctypes.data, 0))
        return g

    def set_scales(self, in_shift, in_scale, out_scale):
        sh = np.ascontiguousarray(in_shift, dtype=np.float64)
        sc = np.ascontiguousarray(in_scale, dtype=np.float64)
        o = np.ascontiguousarray(out_scale, dtype=np.float64)
        if sh.size != self.N_FEATURES or sc.size != self.N_FEATURES or o.size != self.N_OUTPUTS:
            raise ValueError("need 24 input shifts, 24 input scales and 15 output scales")
        _check(self.lib.rod_surrogate_set_scales(self.handle, sh.ctypes.data, sc.ctypes.data, o.ctypes.data))
        self.scales = (sh, sc, o)

    def set_prior(self, positions: bool = True, directors: bool = True, velocity_residual: bool = True,
                  omega_residual: bool = True):
        """Form of the update: kinematic priors x + T v for positions and exp([-T w]x) Q for
        directors; velocities / angular velocities as residuals (v + output) or output alone."""
        flags = (int(bool(positions)) | (int(bool(directors)) << 1) | (int(not velocity_residual) << 2)
                 | (int(not omega_residual) << 3))
        _check(self.lib.rod_surrogate_set_prior(self.handle, flags))
        self.prior = flags

    def train_step(self, start, end, act, lr: float, stream=None):
        """start/end: (x, v, Q, w) CUDA float64 tensors of nwin rods of 50 elements; act (3, nwin).
        Returns the mean-square loss of the batch (before the update)."""
        import torch
        nwin = int(act.shape[1])
        arrs = [a.contiguous() for a in list(start) + list(end) + [act]]
        loss = C.c_float()
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(self.lib.rod_surrogate_train_step(self.handle, *[a.data_ptr() for a in arrs], nwin, float(lr),
                                                 C.byref(loss), s))
        return loss.value

    def raw_features(self, state, act, stream=None):
        """Unscaled FP64 features (nwin, 24, 51) and their mask (int8, 1 where defined)."""
        import torch
        nwin = int(act.shape[1])
        arrs = [a.contiguous() for a in list(state) + [act]]
        out = torch.empty((nwin, self.N_FEATURES, self.POSITIONS), dtype=torch.float64, device="cuda")
        mask = torch.empty((nwin, self.N_FEATURES, self.POSITIONS), dtype=torch.int8, device="cuda")
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(self.lib.rod_surrogate_raw_features(self.handle, *[a.data_ptr() for a in arrs], nwin, out.data_ptr(),
                                                   mask.data_ptr(), s))
        return out, mask

    def raw_targets(self, start, end, stream=None):
        """Unscaled FP64 targets (nwin, 15, 51): change over the window minus the kinematic prior."""
        import torch
        nwin = int(start[0].shape[1]) // self.POSITIONS
        arrs = [a.contiguous() for a in list(start) + list(end)]
        out = torch.empty((nwin, self.N_OUTPUTS, self.POSITIONS), dtype=torch.float64, device="cuda")
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(self.lib.rod_surrogate_raw_targets(self.handle, *[a.data_ptr() for a in arrs], nwin, out.data_ptr(), s))
        return out

    def perturb(self, state, draws, spread, noise: float, held=None, stream=None):
        """Window starts (x, v, Q, w) (CUDA float64) plus noise (rod_surrogate_perturb): draws =
        standard normal tensors shaped like (x, v, w, w), or None with noise = 0; spread: the 15
        output scales; held: CUDA int8 (nwin,) or None.  Returns new tensors."""
        import torch
        nwin = int(state[0].shape[1]) // self.POSITIONS
        src = [a.contiguous() for a in state]
        out = [torch.empty_like(a) for a in src]
        dr = [None] * 4 if draws is None else [a.contiguous() for a in draws]
        sp = np.ascontiguousarray(spread, dtype=np.float64)
        if sp.size != self.N_OUTPUTS:
            raise ValueError("spread holds the 15 output scales")
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        ptr = lambda a: None if a is None else a.data_ptr()
        _check(self.lib.rod_surrogate_perturb(self.handle, *[a.data_ptr() for a in src], nwin, *[ptr(a) for a in dr],
                                              sp.ctypes.data, float(noise), ptr(held), *[a.data_ptr() for a in out], s))
        return out

    def forward(self, state, act, stream=None):
        """Raw network outputs (nwin, 51, 16) float32 for the states (x, v, Q, w) of nwin rods."""
        import torch
        nwin = int(act.shape[1])
        arrs = [a.contiguous() for a in list(state) + [act]]
        out = torch.empty((nwin, self.POSITIONS, 16), dtype=torch.float32, device="cuda")
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(self.lib.rod_surrogate_forward(self.handle, *[a.data_ptr() for a in arrs], nwin, out.data_ptr(), s))
        torch.cuda.current_stream().synchronize()
        return out

    def apply(self, system, n_calls: int):
        """Advance every rod of ``system`` (50 elements each, no contact) by n_calls windows."""
        _check(self.lib.rod_surrogate_apply(self.handle, system.handle, int(n_calls)))

    def rollout(self, system, shadow, sample_rods, n_calls: int, check_every: int, bound: float) -> dict:
        """n_calls windows with a check of the sampled rods against ``shadow`` every check_every
        calls and a plain-step redo of any segment whose sampled tip error exceeds ``bound``."""
        idx = np.ascontiguousarray(sample_rods, dtype=np.int32)
        st = SurrogateStats()
        _check(self.lib.rod_surrogate_rollout(self.handle, system.handle, shadow.handle, idx.ctypes.data, int(idx.size),
                                              int(n_calls), int(check_every), float(bound), C.byref(st)))
        return st.as_dict()

    def rollout_local(self, system, shadows, sample_rods, n_calls: int, check_every: int, bound: float) -> dict:
        """n_calls windows with pipelined local checks: the check of each segment restarts the
        plain step from the surrogate's state of the sampled rods on one of ``shadows`` (each
        holding those rods); a segment above ``bound`` is undone and redone with the plain step."""
        idx = np.ascontiguousarray(sample_rods, dtype=np.int32)
        arr = (C.c_void_p * len(shadows))(*[sh.handle.value for sh in shadows])
        st = SurrogateStats()
        _check(self.lib.rod_surrogate_rollout_local(self.handle, system.handle, arr, len(shadows), idx.ctypes.data,
                                                    int(idx.size), int(n_calls), int(check_every), float(bound),
                                                    C.byref(st)))
        return st.as_dict()


def contact_forces_noalloc(node_off, radius, x, v, k: float, c: float, cell_size: float, f, stream=None):
    """rod_contact_forces_noalloc on CUDA torch tensors (int32 node offsets [R+1], float64 radius
    [R], x, v, f [3, N]); f is overwritten.  Uses torch's current stream unless one is given."""
    lib = load_library()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib.rod_contact_forces_noalloc(int(radius.shape[0]), node_off.data_ptr(), radius.data_ptr(),
                                          x.data_ptr(), v.data_ptr(), float(k), float(c), float(cell_size),
                                          f.data_ptr(), stream))


def plan_packs(n_elem, cap_elems: int, cap_rods: int) -> dict:
    """The thread-block packing of rods with these element counts for a launch shape of
    cap_elems elements and at most cap_rods rods per block (rod_plan_packs; host only, no GPU).
    Returns {"packs": int32 [n_packs, 10] (first rod, rods, first element, elements, first node,
    nodes, first Voronoi point, Voronoi points, listed, list offset) in launch order,
    "list": int32 [n_list, 2] (global rod, first pack-local element), "n_long": rods on the
    cooperative path}."""
    lib = load_library()
    n = np.ascontiguousarray(n_elem, dtype=np.int32)
    npk, nl, ng = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib.rod_plan_packs(n.ctypes.data, int(n.size), int(cap_elems), int(cap_rods), C.byref(npk), C.byref(nl),
                              C.byref(ng), None, None))
    packs = np.zeros((npk.value, 10), dtype=np.int32)
    lst = np.zeros((nl.value, 2), dtype=np.int32)
    _check(lib.rod_plan_packs(n.ctypes.data, int(n.size), int(cap_elems), int(cap_rods), None, None, None,
                              packs.ctypes.data if packs.size else None, lst.ctypes.data if lst.size else None))
    return {"packs": packs, "list": lst, "n_long": ng.value}


def exported_symbols():
    return list(_SIGNATURES)
