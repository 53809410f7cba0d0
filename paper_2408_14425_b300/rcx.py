"""Thin ctypes binding of librcx.so (argument marshalling only).

Every step of the formal solution runs in the library's CUDA kernels; this
module checks tensor dtypes/devices/shapes, passes raw pointers and the
current CUDA stream, and turns status codes into exceptions.  There is no
fallback: if librcx.so is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librcx.so")

RC_OK = 0
STATUS = {0: "RC_OK", -1: "RC_ERR_ARG", -2: "RC_ERR_OOM", -3: "RC_ERR_CUDA",
          -4: "RC_ERR_TIMEOUT", -5: "RC_ERR_NOT_CONVERGED", -6: "RC_ERR_UNSUPPORTED"}
PRECISION = {"f32": 0, "fp32": 0, "f16": 1, "fp16": 1, "bf16": 2}

# every symbol include/rcx.h declares
EXPORTS = [
    "rc_options_default", "rc_plan", "rc_plan_destroy", "rc_plan_reserve",
    "rc_plan_scratch_bytes", "rc_formal_solve", "rc_formal_solve_host", "rc_plan_cascade",
    "rc_plan_last_launch_count", "rc_last_error", "rc_status_string", "rc_plan_set_timing",
    "rc_plan_launch_times", "rc_plan_launch_name", "rc_formal_solve_noalloc",
    "rc_formal_solve_mali", "rc_atom_create", "rc_atom_destroy", "rc_atom_n_lambda", "rc_lte",
    "rc_emis_opac", "rc_stat_eq", "rc_nlte_solve", "rc_plan_set_lane_layout",
    "rc_plan_set_march", "rc_plan_get_march", "rc_line_integrals", "rc_stat_eq_integrals",
    "rc_formal_solve_host_async", "rc_plan_wait", "rc_plan_get_march_cascades",
    "rc_plan_set_top_list", "rc_plan_get_top_list",
    "rc_plan_get_lane_layout", "rc_plan_autotune", "rc_batch_create", "rc_batch_run",
    "rc_batch_info", "rc_batch_destroy", "rc_formal_solve_batched", "rc_mlp_create",
    "rc_mlp_destroy", "rc_mlp_n_params", "rc_mlp_set_params", "rc_mlp_get_params",
    "rc_mlp_fit_normalization", "rc_mlp_forward", "rc_mlp_loss_grad", "rc_mlp_train",
    "rc_surrogate_features", "rc_surrogate_targets", "rc_surrogate_seed", "rc_plan_set_active",
    "rc_plan_active_probes", "rc_emergent", "rc_mlp_use_tensor_cores", "rc_mlp_tensor_core_status",
    "rc_selftest_bounded_wait", "rc_surrogate_init", "rc_surrogate_train_step",
    "rc_surrogate_predict", "rc_batch_solo_domains",
]


class RcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


class rc_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int), ("voxel_size", ctypes.c_double)]


class rc_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("n_incl", ctypes.c_int),
                ("interval_rule", ctypes.c_int), ("lambda_block", ctypes.c_int),
                ("bilinear_fix", ctypes.c_int), ("lambda_per_lane", ctypes.c_int),
                ("strips", ctypes.c_int), ("reserved", ctypes.c_int)]


class rc_atom_desc(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("E_eV", ctypes.POINTER(ctypes.c_double)),
                ("g", ctypes.POINTER(ctypes.c_double)), ("n_lines", ctypes.c_int),
                ("lower", ctypes.POINTER(ctypes.c_int)), ("upper", ctypes.POINTER(ctypes.c_int)),
                ("A_ul", ctypes.POINTER(ctypes.c_double)), ("n_per_line", ctypes.c_int),
                ("x_max", ctypes.c_double), ("T_ref", ctypes.c_double),
                ("mass_amu", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p


def load():
    """Load librcx.so (raises if it is missing: there is no non-CUDA path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"librcx.so not built at {LIB_PATH}; run paper_2408_14425_b300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    L.rc_options_default.argtypes = [ctypes.POINTER(rc_options)]
    L.rc_options_default.restype = None
    L.rc_plan.argtypes = [ctypes.POINTER(rc_grid), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.c_float, ctypes.POINTER(rc_options), ctypes.POINTER(_vp)]
    L.rc_plan.restype = ctypes.c_int
    L.rc_plan_destroy.argtypes = [_vp]
    L.rc_plan_destroy.restype = None
    L.rc_plan_reserve.argtypes = [_vp, ctypes.c_int]
    L.rc_plan_reserve.restype = ctypes.c_int
    L.rc_plan_scratch_bytes.argtypes = [_vp]
    L.rc_plan_scratch_bytes.restype = ctypes.c_size_t
    L.rc_formal_solve.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp]
    L.rc_formal_solve.restype = ctypes.c_int
    L.rc_formal_solve_host.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp]
    L.rc_formal_solve_host.restype = ctypes.c_int
    L.rc_formal_solve_host_async.argtypes = L.rc_formal_solve_host.argtypes
    L.rc_formal_solve_host_async.restype = ctypes.c_int
    L.rc_plan_wait.argtypes = [_vp]
    L.rc_plan_wait.restype = ctypes.c_int
    L.rc_plan_cascade.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.rc_plan_cascade.restype = ctypes.c_int
    L.rc_plan_last_launch_count.argtypes = [_vp]
    L.rc_plan_last_launch_count.restype = ctypes.c_int
    L.rc_last_error.argtypes = []
    L.rc_last_error.restype = ctypes.c_char_p
    L.rc_status_string.argtypes = [ctypes.c_int]
    L.rc_status_string.restype = ctypes.c_char_p
    L.rc_plan_set_timing.argtypes = [_vp, ctypes.c_int]
    L.rc_plan_set_timing.restype = ctypes.c_int
    L.rc_plan_launch_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]
    L.rc_plan_launch_times.restype = ctypes.c_int
    L.rc_plan_launch_name.argtypes = [_vp, ctypes.c_int]
    L.rc_plan_launch_name.restype = ctypes.c_char_p
    L.rc_formal_solve_noalloc.argtypes = [ctypes.POINTER(rc_grid), ctypes.c_int, ctypes.c_int,
                                          ctypes.c_float, _vp, _vp, ctypes.c_int, _vp, _vp, _vp]
    L.rc_formal_solve_noalloc.restype = ctypes.c_int
    L.rc_formal_solve_mali.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
    L.rc_formal_solve_mali.restype = ctypes.c_int
    L.rc_atom_create.argtypes = [ctypes.POINTER(rc_atom_desc), ctypes.POINTER(_vp)]
    L.rc_atom_create.restype = ctypes.c_int
    L.rc_atom_destroy.argtypes = [_vp]
    L.rc_atom_destroy.restype = None
    L.rc_atom_n_lambda.argtypes = [_vp]
    L.rc_atom_n_lambda.restype = ctypes.c_int
    L.rc_lte.argtypes = [_vp, _vp, _vp, ctypes.c_longlong, _vp, _vp, _vp, _vp]
    L.rc_lte.restype = ctypes.c_int
    L.rc_emis_opac.argtypes = [_vp, _vp, _vp, ctypes.c_longlong, _vp, _vp, _vp]
    L.rc_emis_opac.restype = ctypes.c_int
    L.rc_stat_eq.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_longlong, _vp,
                             ctypes.POINTER(ctypes.c_double), _vp]
    L.rc_stat_eq.restype = ctypes.c_int
    L.rc_line_integrals.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_longlong, _vp, _vp]
    L.rc_line_integrals.restype = ctypes.c_int
    L.rc_stat_eq_integrals.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_longlong, _vp,
                                       ctypes.POINTER(ctypes.c_double), _vp]
    L.rc_stat_eq_integrals.restype = ctypes.c_int
    L.rc_nlte_solve.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double), _vp]
    L.rc_nlte_solve.restype = ctypes.c_int
    _ip = ctypes.POINTER(ctypes.c_int)
    L.rc_emergent.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_longlong, ctypes.c_float,
                              _vp, _vp, _vp]
    L.rc_emergent.restype = ctypes.c_int
    L.rc_plan_set_active.argtypes = [_vp, _vp, _vp]
    L.rc_plan_set_active.restype = ctypes.c_int
    L.rc_plan_active_probes.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong)]
    L.rc_plan_active_probes.restype = ctypes.c_int
    L.rc_plan_set_lane_layout.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
    L.rc_plan_set_lane_layout.restype = ctypes.c_int
    L.rc_plan_get_lane_layout.argtypes = [_vp, _ip, _ip]
    L.rc_plan_get_lane_layout.restype = ctypes.c_int
    L.rc_plan_set_march.argtypes = [_vp, ctypes.c_int]
    L.rc_plan_set_march.restype = ctypes.c_int
    L.rc_plan_get_march.argtypes = [_vp, _ip]
    L.rc_plan_get_march.restype = ctypes.c_int
    L.rc_plan_get_march_cascades.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint)]
    L.rc_plan_get_march_cascades.restype = ctypes.c_int
    L.rc_plan_set_top_list.argtypes = [_vp, ctypes.c_int]
    L.rc_plan_set_top_list.restype = ctypes.c_int
    L.rc_plan_get_top_list.argtypes = [_vp, _ip, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_longlong)]
    L.rc_plan_get_top_list.restype = ctypes.c_int
    L.rc_plan_autotune.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _ip, _ip]
    L.rc_plan_autotune.restype = ctypes.c_int
    _pp = ctypes.POINTER(_vp)
    L.rc_batch_create.argtypes = [ctypes.c_int, _pp, _pp, _pp, _ip, _pp, ctypes.c_int,
                                  ctypes.POINTER(_vp)]
    L.rc_batch_create.restype = ctypes.c_int
    L.rc_batch_run.argtypes = [_vp, _vp]
    L.rc_batch_run.restype = ctypes.c_int
    L.rc_batch_info.argtypes = [_vp, _ip, _ip, _ip]
    L.rc_batch_info.restype = ctypes.c_int
    L.rc_batch_solo_domains.argtypes = [_vp]
    L.rc_batch_solo_domains.restype = ctypes.c_int
    L.rc_batch_destroy.argtypes = [_vp]
    L.rc_batch_destroy.restype = None
    L.rc_formal_solve_batched.argtypes = [ctypes.c_int, _pp, _pp, _pp, _ip, _pp, _vp]
    L.rc_formal_solve_batched.restype = ctypes.c_int
    _fp = ctypes.POINTER(ctypes.c_float)
    L.rc_mlp_create.argtypes = [ctypes.c_ulonglong, ctypes.POINTER(_vp)]
    L.rc_mlp_create.restype = ctypes.c_int
    L.rc_mlp_destroy.argtypes = [_vp]
    L.rc_mlp_destroy.restype = None
    L.rc_mlp_n_params.argtypes = [_vp]
    L.rc_mlp_n_params.restype = ctypes.c_int
    L.rc_mlp_set_params.argtypes = [_vp, _fp, _fp, _fp]
    L.rc_mlp_set_params.restype = ctypes.c_int
    L.rc_mlp_get_params.argtypes = [_vp, _fp, _fp, _fp]
    L.rc_mlp_get_params.restype = ctypes.c_int
    L.rc_mlp_fit_normalization.argtypes = [_vp, _vp, ctypes.c_longlong, _vp]
    L.rc_mlp_fit_normalization.restype = ctypes.c_int
    L.rc_mlp_use_tensor_cores.argtypes = [_vp, ctypes.c_int]
    L.rc_mlp_use_tensor_cores.restype = ctypes.c_int
    L.rc_mlp_tensor_core_status.argtypes = [_vp]
    L.rc_selftest_bounded_wait.argtypes = [_vp]
    L.rc_selftest_bounded_wait.restype = ctypes.c_int
    L.rc_surrogate_init.argtypes = [ctypes.c_ulonglong, ctypes.POINTER(_vp)]
    L.rc_surrogate_init.restype = ctypes.c_int
    L.rc_surrogate_train_step.argtypes = [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_int,
                                          ctypes.c_float, ctypes.POINTER(ctypes.c_float), _vp]
    L.rc_surrogate_train_step.restype = ctypes.c_int
    L.rc_surrogate_predict.argtypes = [_vp, _vp, ctypes.c_longlong, _vp, _vp]
    L.rc_surrogate_predict.restype = ctypes.c_int
    L.rc_mlp_tensor_core_status.restype = ctypes.c_int
    L.rc_mlp_forward.argtypes = [_vp, _vp, ctypes.c_longlong, _vp, _vp]
    L.rc_mlp_forward.restype = ctypes.c_int
    L.rc_mlp_loss_grad.argtypes = [_vp, _vp, _vp, ctypes.c_longlong, _vp, _vp, _vp]
    L.rc_mlp_loss_grad.restype = ctypes.c_int
    L.rc_mlp_train.argtypes = [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                               ctypes.c_float, _fp, _vp]
    L.rc_mlp_train.restype = ctypes.c_int
    L.rc_surrogate_features.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_longlong, _vp, _vp]
    L.rc_surrogate_features.restype = ctypes.c_int
    L.rc_surrogate_targets.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_longlong, _vp, _vp]
    L.rc_surrogate_targets.restype = ctypes.c_int
    L.rc_surrogate_seed.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_longlong, _vp,
                                    ctypes.POINTER(ctypes.c_int), _vp]
    L.rc_surrogate_seed.restype = ctypes.c_int
    _lib = L
    return L


def check(status: int):
    if status != RC_OK:
        msg = load().rc_last_error().decode(errors="replace")
        raise RcError(status, msg)


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, name, shape, dtype_name="float32"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != getattr(torch, dtype_name):
        raise TypeError(f"{name} must be {dtype_name}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a, name, shape):
    if hasattr(a, "numpy") and not isinstance(a, np.ndarray):  # torch CPU tensor
        if a.is_cuda:
            raise TypeError(f"{name} must be in host memory")
        if not a.is_contiguous() or str(a.dtype) != "torch.float32":
            raise TypeError(f"{name} must be a contiguous float32 host tensor")
        if tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(a.shape)}, expected {tuple(shape)}")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float32 or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous float32 array")
    if a.shape != tuple(shape):
        raise ValueError(f"{name} has shape {a.shape}, expected {tuple(shape)}")
    return ctypes.c_void_p(a.ctypes.data)


class Plan:
    """rc_plan: cascade geometry of an nx x nz grid (see include/rcx.h)."""

    def __init__(self, nx: int, nz: int, n_cascades: int, dirs0: int = 4, branching: int = 4,
                 interval0: float = 1.0, voxel_size: float = 1.0, precision: str = "f32",
                 interval_rule: int = 0, lambda_block: int = 0, n_incl: int = 1,
                 bilinear_fix: bool = False, lambda_per_lane: int = 0, strips: int = 0):
        L = load()
        self.nx, self.nz, self.n_cascades = nx, nz, n_cascades
        g = rc_grid(nx, nz, voxel_size)
        o = rc_options()
        L.rc_options_default(ctypes.byref(o))
        o.precision = PRECISION[precision]
        o.interval_rule = interval_rule
        o.lambda_block = lambda_block
        o.n_incl = n_incl
        o.bilinear_fix = int(bilinear_fix)
        o.lambda_per_lane = lambda_per_lane
        o.strips = strips
        h = _vp()
        check(L.rc_plan(ctypes.byref(g), n_cascades, dirs0, branching, interval0, ctypes.byref(o),
                        ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().rc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def reserve(self, n_lambda: int):
        check(load().rc_plan_reserve(self._h, n_lambda))

    def scratch_bytes(self) -> int:
        return int(load().rc_plan_scratch_bytes(self._h))

    def last_launch_count(self) -> int:
        return int(load().rc_plan_last_launch_count(self._h))

    def set_timing(self, enable: bool = True):
        check(load().rc_plan_set_timing(self._h, int(enable)))

    def launch_times(self):
        """[(kernel name, ms)] of the last timed solve (waits for it)."""
        buf = (ctypes.c_float * 64)()
        n = ctypes.c_int()
        check(load().rc_plan_launch_times(self._h, buf, 64, ctypes.byref(n)))
        return [(load().rc_plan_launch_name(self._h, j).decode(), float(buf[j]))
                for j in range(n.value)]

    def emergent(self, chi, eta, rays, mu: float = 0.0, want_contrib: bool = False, stream=None):
        """rc_emergent: I [n_lambda][n_rays] (and the contribution map) along device rays [n][4]."""
        import torch
        nl = chi.shape[0]
        shape = (nl, self.nz, self.nx)
        n = rays.shape[0]
        I = torch.empty((nl, n), dtype=torch.float32, device=chi.device)
        C = torch.zeros(shape, dtype=torch.float32, device=chi.device) if want_contrib else None
        check(load().rc_emergent(self._h, _dev_ptr(chi, "chi", shape), _dev_ptr(eta, "eta", shape), nl,
                                 _dev_ptr(rays, "rays", (n, 4)), n, mu, _dev_ptr(I, "I", I.shape),
                                 _dev_ptr(C, "contrib", shape) if C is not None else None,
                                 _stream_ptr(stream)))
        return (I, C) if want_contrib else I

    def set_active(self, active=None, stream=None):
        """rc_plan_set_active: device uint8 [nz][nx] mask of the active cells, or None."""
        ptr = None
        if active is not None:
            ptr = _dev_ptr(active, "active", (self.nz, self.nx), "uint8")
        check(load().rc_plan_set_active(self._h, ptr, _stream_ptr(stream)))

    def active_probes(self):
        out = (ctypes.c_longlong * self.n_cascades)()
        check(load().rc_plan_active_probes(self._h, out))
        return list(out)

    def set_lane_layout(self, lambda_block: int, lambda_per_lane: int):
        check(load().rc_plan_set_lane_layout(self._h, lambda_block, lambda_per_lane))

    def lane_layout(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        check(load().rc_plan_get_lane_layout(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    MARCH_LANE_GROUP, MARCH_SHARED_DDA, MARCH_SHARED_DDA_ALL, MARCH_TUNED = 0, 1, 2, 3

    def march_cascades(self):
        """rc_plan_get_march_cascades: the cascades that take the shared-DDA march."""
        m = ctypes.c_uint()
        check(load().rc_plan_get_march_cascades(self._h, ctypes.byref(m)))
        return [i for i in range(self.n_cascades) if (m.value >> i) & 1]

    def set_march(self, mode: int):
        """rc_plan_set_march: 0 lane-group DDA everywhere, 1 shared DDA on the short cascades
        (default), 2 shared DDA on every cascade >= 1 where it applies."""
        check(load().rc_plan_set_march(self._h, int(mode)))

    def march(self) -> int:
        m = ctypes.c_int()
        check(load().rc_plan_get_march(self._h, ctypes.byref(m)))
        return m.value

    def set_top_list(self, enable: bool):
        """rc_plan_set_top_list: march only the listed CTAs of the highest launched cascade
        (default) or every CTA."""
        check(load().rc_plan_set_top_list(self._h, 1 if enable else 0))

    def top_list(self):
        """rc_plan_get_top_list: (cascade or -1, listed CTAs, CTAs of that cascade)."""
        c, n, t = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
        check(load().rc_plan_get_top_list(self._h, ctypes.byref(c), ctypes.byref(n), ctypes.byref(t)))
        return c.value, n.value, t.value

    def autotune(self, chi, eta, J, stream=None):
        """rc_plan_autotune: keep the fastest lane layout for these inputs; returns it."""
        nl = chi.shape[0]
        shape = (nl, self.nz, self.nx)
        a, b = ctypes.c_int(), ctypes.c_int()
        check(load().rc_plan_autotune(self._h, _dev_ptr(chi, "chi", shape), _dev_ptr(eta, "eta", shape),
                                      nl, _dev_ptr(J, "J", shape), _stream_ptr(stream),
                                      ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def cascade(self, i: int):
        px, pz = ctypes.c_int(), ctypes.c_int()
        w = ctypes.c_longlong()
        a, b = ctypes.c_double(), ctypes.c_double()
        check(load().rc_plan_cascade(self._h, i, ctypes.byref(px), ctypes.byref(pz),
                                     ctypes.byref(w), ctypes.byref(a), ctypes.byref(b)))
        return dict(Px=px.value, Pz=pz.value, W=w.value, a=a.value, b=b.value)

    def formal_solve(self, chi, eta, J=None, alo=None, want_alo: bool = False, stream=None):
        """J (and the diagonal ALO) of device FP32 chi/eta [n_lambda][nz][nx]."""
        import torch
        if chi.dim() == 2:
            chi = chi.unsqueeze(0)
            eta = eta.unsqueeze(0)
        nl = chi.shape[0]
        shape = (nl, self.nz, self.nx)
        pc = _dev_ptr(chi, "chi", shape)
        pe = _dev_ptr(eta, "eta", shape)
        if J is None:
            J = torch.empty(shape, dtype=torch.float32, device=chi.device)
        pj = _dev_ptr(J, "J", shape)
        if want_alo and alo is None:
            alo = torch.empty(shape, dtype=torch.float32, device=chi.device)
        pa = _dev_ptr(alo, "alo", shape) if alo is not None else None
        check(load().rc_formal_solve(self._h, pc, pe, nl, pj, pa, _stream_ptr(stream)))
        return (J, alo) if alo is not None else J

    def formal_solve_mali(self, chi, eta, J=None, J_eff=None, alo_c=None, alo=None, stream=None):
        """J, J_eff = J - Lambda* S_local (no cancellation) and 1 - Lambda* (rc_formal_solve_mali)."""
        import torch
        nl = chi.shape[0]
        shape = (nl, self.nz, self.nx)

        def out(t):
            return torch.empty(shape, dtype=torch.float32, device=chi.device) if t is None else t
        J, J_eff, alo_c = out(J), out(J_eff), out(alo_c)
        check(load().rc_formal_solve_mali(
            self._h, _dev_ptr(chi, "chi", shape), _dev_ptr(eta, "eta", shape), nl,
            _dev_ptr(J, "J", shape), _dev_ptr(alo, "alo", shape) if alo is not None else None,
            _dev_ptr(J_eff, "J_eff", shape), _dev_ptr(alo_c, "alo_c", shape), _stream_ptr(stream)))
        return J, J_eff, alo_c

    def formal_solve_host(self, chi, eta, J=None, alo=None, want_alo: bool = False):
        """Same on host FP32 arrays (numpy or CPU tensors); copies are inside the call."""
        nl = chi.shape[0]
        shape = (nl, self.nz, self.nx)
        if J is None:
            J = np.empty(shape, dtype=np.float32)
        if want_alo and alo is None:
            alo = np.empty(shape, dtype=np.float32)
        check(load().rc_formal_solve_host(
            self._h, _host_ptr(chi, "chi", shape), _host_ptr(eta, "eta", shape), nl,
            _host_ptr(J, "J", shape), _host_ptr(alo, "alo", shape) if alo is not None else None))
        return (J, alo) if alo is not None else J

    def formal_solve_host_async(self, chi, eta, J, alo=None):
        """rc_formal_solve_host_async: enqueues the host-buffer solve and returns; the buffers
        must stay alive and chi / eta unmodified until wait() (consecutive calls pipeline)."""
        nl = chi.shape[0]
        shape = (nl, self.nz, self.nx)
        check(load().rc_formal_solve_host_async(
            self._h, _host_ptr(chi, "chi", shape), _host_ptr(eta, "eta", shape), nl,
            _host_ptr(J, "J", shape), _host_ptr(alo, "alo", shape) if alo is not None else None))

    def wait(self):
        """rc_plan_wait: every enqueued host-buffer solve has completed."""
        check(load().rc_plan_wait(self._h))


def formal_solve_noalloc(chi, eta, n_cascades: int, dirs0: int = 4, interval0: float = 1.0,
                         voxel_size: float = 1.0, J=None, alo=None, stream=None):
    """rc_formal_solve_noalloc: the formal solution with no device allocation by the library.

    For callers that cannot let a library call cudaMalloc (memory owned by another allocator,
    fixed device-memory budgets).  Scratch is a 32 MiB static device array shared by every
    call; calls that overlap on the GPU race on it.  J (and alo) may be passed in so that this
    call allocates nothing either; if J is None a torch tensor is created for it here.
    """
    import torch
    if chi.dim() == 2:
        chi = chi.unsqueeze(0)
        eta = eta.unsqueeze(0)
    nl, nz, nx = chi.shape
    shape = (nl, nz, nx)
    pc = _dev_ptr(chi, "chi", shape)
    pe = _dev_ptr(eta, "eta", shape)
    if J is None:
        J = torch.empty(shape, dtype=torch.float32, device=chi.device)
    pj = _dev_ptr(J, "J", shape)
    pa = _dev_ptr(alo, "alo", shape) if alo is not None else None
    g = rc_grid(nx, nz, voxel_size)
    check(load().rc_formal_solve_noalloc(ctypes.byref(g), n_cascades, dirs0, interval0, pc, pe, nl,
                                         pj, pa, _stream_ptr(stream)))
    return (J, alo) if alo is not None else J


class Atom:
    """rc_atom_create: a model atom with non-overlapping Gaussian lines (include/rcx.h)."""

    def __init__(self, desc: dict):
        L = load()
        E = (ctypes.c_double * len(desc["E_eV"]))(*desc["E_eV"])
        g = (ctypes.c_double * len(desc["g"]))(*desc["g"])
        lines = desc["lines"]
        lo = (ctypes.c_int * len(lines))(*[int(x[0]) for x in lines])
        up = (ctypes.c_int * len(lines))(*[int(x[1]) for x in lines])
        A = (ctypes.c_double * len(lines))(*[float(x[2]) for x in lines])
        d = rc_atom_desc(len(desc["E_eV"]), E, g, len(lines), lo, up, A, int(desc["n_per_line"]),
                         float(desc["x_max"]), float(desc["T_ref"]), float(desc["mass_amu"]))
        h = _vp()
        check(L.rc_atom_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.n_levels = len(desc["E_eV"])
        self.n_lambda = L.rc_atom_n_lambda(h)
        self.n_per_line = int(desc["n_per_line"])

    def close(self):
        if getattr(self, "_h", None):
            load().rc_atom_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lte(self, T, nH, stream=None):
        """(n_e, n_atom, pops[n_levels][ncell]) from device FP64 T, n_H (flattened cells)."""
        import torch
        n = T.numel()
        ne = torch.empty(n, dtype=torch.float64, device=T.device)
        na = torch.empty_like(ne)
        pops = torch.empty((self.n_levels, n), dtype=torch.float64, device=T.device)
        check(load().rc_lte(self._h, _dev_ptr(T.reshape(-1), "T", (n,), "float64"),
                            _dev_ptr(nH.reshape(-1), "nH", (n,), "float64"), n,
                            _dev_ptr(ne, "ne", (n,), "float64"), _dev_ptr(na, "n_atom", (n,), "float64"),
                            _dev_ptr(pops, "pops", (self.n_levels, n), "float64"), _stream_ptr(stream)))
        return ne, na, pops

    def emis_opac(self, T, pops, stream=None):
        import torch
        n = T.numel()
        chi = torch.empty((self.n_lambda, n), dtype=torch.float32, device=T.device)
        eta = torch.empty_like(chi)
        check(load().rc_emis_opac(self._h, _dev_ptr(T.reshape(-1), "T", (n,), "float64"),
                                  _dev_ptr(pops, "pops", (self.n_levels, n), "float64"), n,
                                  _dev_ptr(chi, "chi", chi.shape), _dev_ptr(eta, "eta", eta.shape),
                                  _stream_ptr(stream)))
        return chi, eta

    def stat_eq(self, T, ne, n_atom, J_eff, alo_c, pops, stream=None):
        """Updates pops (device FP64 [n_levels][ncell]) in place; returns the max relative change."""
        n = T.numel()
        ch = ctypes.c_double()
        shp = (self.n_lambda, n)
        check(load().rc_stat_eq(
            self._h, _dev_ptr(T.reshape(-1), "T", (n,), "float64"),
            _dev_ptr(ne.reshape(-1), "ne", (n,), "float64"),
            _dev_ptr(n_atom.reshape(-1), "n_atom", (n,), "float64"),
            _dev_ptr(J_eff.reshape(shp), "J_eff", shp),
            _dev_ptr(alo_c.reshape(shp), "alo_c", shp) if alo_c is not None else None, n,
            _dev_ptr(pops, "pops", (self.n_levels, n), "float64"), ctypes.byref(ch),
            _stream_ptr(stream)))
        return ch.value

    def line_integrals(self, T, J_eff, alo_c, lambda_begin: int, stream=None):
        """rc_line_integrals: (Jeff_bar, (1 - Lambda*)_bar) per line over the grid wavelengths
        [lambda_begin, lambda_begin + J_eff.shape[0]); device FP64 [n_lines][2][ncell]."""
        import torch
        n = T.numel()
        cnt = int(J_eff.shape[0])
        n_lines = self.n_lambda // self.n_per_line
        out = torch.empty((n_lines, 2, n), dtype=torch.float64, device=T.device)
        shp = (cnt, n)
        check(load().rc_line_integrals(
            self._h, _dev_ptr(T.reshape(-1), "T", (n,), "float64"),
            _dev_ptr(J_eff.reshape(shp), "J_eff", shp),
            _dev_ptr(alo_c.reshape(shp), "alo_c", shp) if alo_c is not None else None,
            int(lambda_begin), cnt, n, _dev_ptr(out, "out", out.shape, "float64"),
            _stream_ptr(stream)))
        return out

    def stat_eq_integrals(self, T, ne, n_atom, integrals, pops, stream=None):
        """rc_stat_eq_integrals: updates pops in place from summed line integrals; returns the
        max relative change."""
        n = T.numel()
        ch = ctypes.c_double()
        n_lines = self.n_lambda // self.n_per_line
        check(load().rc_stat_eq_integrals(
            self._h, _dev_ptr(T.reshape(-1), "T", (n,), "float64"),
            _dev_ptr(ne.reshape(-1), "ne", (n,), "float64"),
            _dev_ptr(n_atom.reshape(-1), "n_atom", (n,), "float64"),
            _dev_ptr(integrals, "integrals", (n_lines, 2, n), "float64"), n,
            _dev_ptr(pops, "pops", (self.n_levels, n), "float64"), ctypes.byref(ch),
            _stream_ptr(stream)))
        return ch.value


def nlte_solve(plan: Plan, atom: Atom, T, ne, n_atom, pops, tol: float = 1e-3,
               max_iter: int = 500, stream=None):
    """rc_nlte_solve: iterate pops (device FP64, in place) to max relative change < tol.
    Returns (converged, iterations, history)."""
    n = T.numel()
    it = ctypes.c_int()
    fin = ctypes.c_double()
    hist = (ctypes.c_double * max_iter)()
    st = load().rc_nlte_solve(
        plan.handle, atom._h, _dev_ptr(T.reshape(-1), "T", (n,), "float64"),
        _dev_ptr(ne.reshape(-1), "ne", (n,), "float64"),
        _dev_ptr(n_atom.reshape(-1), "n_atom", (n,), "float64"),
        _dev_ptr(pops, "pops", (atom.n_levels, n), "float64"), tol, max_iter, ctypes.byref(it),
        ctypes.byref(fin), hist, _stream_ptr(stream))
    if st not in (RC_OK, -5):
        check(st)
    return st == RC_OK, it.value, [hist[i] for i in range(it.value)]


class Batch:
    """rc_batch_create: fixed batch of domains, one launch per cascade, CUDA graph."""

    def __init__(self, plans, chis, etas, Js, autotune: bool = False):
        L = load()
        n = len(plans)
        arr = lambda xs: (_vp * n)(*[_vp(x) for x in xs])  # noqa: E731
        self._keep = (plans, chis, etas, Js)
        for p, c, e, j in zip(plans, chis, etas, Js):
            shape = (c.shape[0], p.nz, p.nx)
            _dev_ptr(c, "chi", shape)
            _dev_ptr(e, "eta", shape)
            _dev_ptr(j, "J", shape)
        nl = (ctypes.c_int * n)(*[int(c.shape[0]) for c in chis])
        h = _vp()
        check(L.rc_batch_create(n, arr([p.handle.value for p in plans]),
                                arr([c.data_ptr() for c in chis]), arr([e.data_ptr() for e in etas]),
                                nl, arr([j.data_ptr() for j in Js]), int(autotune), ctypes.byref(h)))
        self._h = h

    def run(self, stream=None):
        check(load().rc_batch_run(self._h, _stream_ptr(stream)))

    def info(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(load().rc_batch_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return dict(launches=a.value, lambda_block=b.value, lambda_per_lane=c.value,
                    solo_domains=load().rc_batch_solo_domains(self._h))

    def close(self):
        if getattr(self, "_h", None):
            load().rc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """rc_mlp_create: the 6-64-64-3 surrogate network trained and run by librcx.so."""

    def __init__(self, seed: int = 0):
        h = _vp()
        check(load().rc_mlp_create(seed, ctypes.byref(h)))
        self._h = h
        self.n_params = load().rc_mlp_n_params(h)

    def close(self):
        if getattr(self, "_h", None):
            load().rc_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta=None, mean=None, std=None):
        def p(a, n):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float32)
            assert a.size == n
            self._hold = getattr(self, "_hold", []) + [a]
            return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        check(load().rc_mlp_set_params(self._h, p(theta, self.n_params), p(mean, 6), p(std, 6)))
        self._hold = []

    def get_params(self):
        th = np.empty(self.n_params, np.float32)
        mu = np.empty(6, np.float32)
        sd = np.empty(6, np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        check(load().rc_mlp_get_params(self._h, th.ctypes.data_as(fp), mu.ctypes.data_as(fp),
                                       sd.ctypes.data_as(fp)))
        return th, mu, sd

    def use_tensor_cores(self, enable: bool = True, training: bool = False):
        """rc_mlp_use_tensor_cores: inference with the 64 x 64 layer on tcgen05 tensor cores
        (bf16 in, FP32 out) when enable; training's 64-wide products on them when training."""
        check(load().rc_mlp_use_tensor_cores(self._h, (1 if enable else 0) | (2 if training else 0)))

    def tensor_core_status(self):
        check(load().rc_mlp_tensor_core_status(self._h))

    def fit_normalization(self, X, stream=None):
        check(load().rc_mlp_fit_normalization(self._h, _dev_ptr(X, "X", (X.shape[0], 6)), X.shape[0],
                                              _stream_ptr(stream)))

    def forward(self, X, stream=None):
        import torch
        Y = torch.empty((X.shape[0], 3), dtype=torch.float32, device=X.device)
        check(load().rc_mlp_forward(self._h, _dev_ptr(X, "X", (X.shape[0], 6)), X.shape[0],
                                    _dev_ptr(Y, "Y", Y.shape), _stream_ptr(stream)))
        return Y

    def loss_grad(self, X, Yt, stream=None):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=X.device)
        l = torch.empty(1, dtype=torch.float32, device=X.device)
        check(load().rc_mlp_loss_grad(self._h, _dev_ptr(X, "X", (X.shape[0], 6)),
                                      _dev_ptr(Yt, "Y", (X.shape[0], 3)), X.shape[0],
                                      _dev_ptr(g, "grad", g.shape), _dev_ptr(l, "loss", (1,)),
                                      _stream_ptr(stream)))
        return float(l.item()), g

    def train(self, X, Yt, batch: int, steps: int, lr: float, record: bool = True, stream=None):
        hist = (ctypes.c_float * max(steps, 1))() if record else None
        check(load().rc_mlp_train(self._h, _dev_ptr(X, "X", (X.shape[0], 6)),
                                  _dev_ptr(Yt, "Y", (X.shape[0], 3)), X.shape[0], batch, steps, lr,
                                  hist, _stream_ptr(stream)))
        return [hist[i] for i in range(steps)] if record else None


def surrogate_features(atom: Atom, T, ne, nH, J, stream=None):
    import torch
    n = T.numel()
    X = torch.empty((n, 6), dtype=torch.float32, device=T.device)
    check(load().rc_surrogate_features(
        atom._h, _dev_ptr(T.reshape(-1), "T", (n,), "float64"), _dev_ptr(ne.reshape(-1), "ne", (n,), "float64"),
        _dev_ptr(nH.reshape(-1), "nH", (n,), "float64"), _dev_ptr(J.reshape(atom.n_lambda, n), "J", (atom.n_lambda, n)),
        n, _dev_ptr(X, "X", X.shape), _stream_ptr(stream)))
    return X


def surrogate_targets(atom: Atom, T, n_atom, pops, stream=None):
    import torch
    n = T.numel()
    Y = torch.empty((n, 3), dtype=torch.float32, device=T.device)
    check(load().rc_surrogate_targets(
        atom._h, _dev_ptr(T.reshape(-1), "T", (n,), "float64"),
        _dev_ptr(n_atom.reshape(-1), "n_atom", (n,), "float64"),
        _dev_ptr(pops, "pops", (atom.n_levels, n), "float64"), n, _dev_ptr(Y, "Y", Y.shape),
        _stream_ptr(stream)))
    return Y


def surrogate_seed(atom: Atom, net: MLP, X, T, n_atom, pops, stream=None):
    """Writes seeded populations into pops (device FP64); returns the LTE-fallback cell count."""
    n = T.numel()
    fb = ctypes.c_int()
    check(load().rc_surrogate_seed(
        atom._h, net._h, _dev_ptr(X, "X", (n, 6)), _dev_ptr(T.reshape(-1), "T", (n,), "float64"),
        _dev_ptr(n_atom.reshape(-1), "n_atom", (n,), "float64"), n,
        _dev_ptr(pops, "pops", (atom.n_levels, n), "float64"), ctypes.byref(fb), _stream_ptr(stream)))
    return fb.value
