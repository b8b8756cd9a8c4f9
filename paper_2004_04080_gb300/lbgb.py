"""Thin ctypes binding of the C ABI in ``include/lbgb.h``.

The module-level functions carry the C names and only marshal arguments;
every step of the method runs in the CUDA kernels of ``liblbgb.so``.  There is
no fallback: if the library is missing or no GPU is present the calls raise.
PyTorch serves only as the device allocator (the workspace tensor) and for the
current CUDA stream.

``LBLattice`` is a convenience owner of one context and its workspace.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

LB_OK, LB_ERR_ARG, LB_ERR_STATE, LB_ERR_CUDA, LB_ERR_NOMEM = 0, -1, -2, -3, -4
LB_ERR_NONFINITE, LB_ERR_OVERLAP, LB_ERR_TIMEOUT = -5, -6, -7
LB_FP64, LB_FP32, LB_FP16 = 0, 1, 2
LB_ONE_COMPONENT = 0x100
PREC = {"fp64": LB_FP64, "fp32": LB_FP32, "fp16": LB_FP16}
TERMS = {"F_liq": 0, "T_liq": 1, "F_d": 2, "T_d": 3, "F_c": 4, "T_c": 5, "F_s": 6,
         "T_s": 7, "F_pair": 8, "F_total": 9, "T_total": 10}

# every symbol declared in include/lbgb.h
EXPORTS = ["lb_workspace_bytes", "lb_create", "lb_set_params", "lb_init_fields", "lb_add_colloids",
           "lb_step", "lb_get_fields", "lb_get_colloids", "lb_get_colloid_terms", "lb_get_totals",
           "lb_get_populations", "lb_get_owner", "lb_profile", "lb_profile_read", "lb_profile_read_kernel",
           "lb_set_rounding",
           "lb_state_bytes",
           "lb_get_state", "lb_set_state", "lb_adjoint_bytes", "lb_adjoint_seed", "lb_adjoint_step",
           "lb_adjoint_initial", "lb_adjoint_step_async", "lb_drag_gradient", "lb_record", "lb_totals_static",
           "lb_launch_count", "lb_pair_list_builds", "lb_fused_kernel", "lb_destroy", "lb_last_error"]


class LbParams(C.Structure):
    """Mirror of ``lb_params`` (field order and types as in lbgb.h)."""

    _fields_ = [
        ("tau", C.c_double * 2), ("G", C.c_double), ("zeta", C.c_double * 2),
        ("rho0", C.c_double * 2), ("bc", C.c_int * 3), ("wall_u_lo", C.c_double * 3),
        ("wall_u_hi", C.c_double * 3), ("body_force", C.c_double * 3), ("hertz_K", C.c_double),
        ("hertz_sigma", C.c_double), ("hertz_rcap", C.c_double), ("lub_on", C.c_int),
        ("lub_hn", C.c_double), ("lub_hmin", C.c_double), ("lub_scale", C.c_double),
        ("side_wall_k", C.c_double), ("side_wall_d", C.c_double), ("rotate", C.c_int),
        ("janus", C.c_int), ("janus_theta0", C.c_double), ("janus_width", C.c_double),
        ("rcut", C.c_double), ("delr", C.c_double),
        ("open", C.c_int * 2), ("open_rho", C.c_double * 4), ("open_extrap", C.c_int),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblbgb.so (building it first if asked); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("liblbgb.so is not built (run __graft_entry__.build())")
        _build.build()
    lib = C.CDLL(path)
    P, D, I = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
    lib.lb_workspace_bytes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]
    lib.lb_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, C.c_size_t, P, C.POINTER(P)]
    lib.lb_set_params.argtypes = [P, C.POINTER(LbParams)]
    lib.lb_init_fields.argtypes = [P, D, D, D]
    lib.lb_add_colloids.argtypes = [P, C.c_int, D, D, D, D, D, D]
    lib.lb_step.argtypes = [P, C.c_int]
    lib.lb_get_fields.argtypes = [P, D, D, D]
    lib.lb_get_colloids.argtypes = [P, D, D, D, D, D, D]
    lib.lb_get_colloid_terms.argtypes = [P, C.c_int, D]
    lib.lb_get_totals.argtypes = [P, D]
    lib.lb_get_populations.argtypes = [P, C.c_int, D]
    lib.lb_get_owner.argtypes = [P, I]
    lib.lb_profile.argtypes = [P, C.c_int]
    lib.lb_profile_read.argtypes = [P, D, C.POINTER(C.c_longlong)]
    lib.lb_profile_read_kernel.argtypes = [P, C.c_int, D, C.POINTER(C.c_longlong)]
    lib.lb_state_bytes.argtypes = [P, C.POINTER(C.c_size_t)]
    lib.lb_get_state.argtypes = [P, P]
    lib.lb_set_state.argtypes = [P, P]
    lib.lb_adjoint_bytes.argtypes = [P, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
    lib.lb_adjoint_seed.argtypes = [P, C.c_double, P, P, D]
    lib.lb_adjoint_step.argtypes = [P, P, P, P, P, D, D]
    lib.lb_adjoint_initial.argtypes = [P, P, P]
    lib.lb_adjoint_step_async.argtypes = [P, P, P, P, P, P, D]
    lib.lb_drag_gradient.argtypes = [P, P, C.c_double, C.c_double, P]
    lib.lb_record.argtypes = [P, P, P, C.c_int]
    lib.lb_set_rounding.argtypes = [P, C.c_int, C.c_ulonglong]
    lib.lb_totals_static.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_longlong, P, D, P, P]
    lib.lb_launch_count.argtypes = [P]
    lib.lb_launch_count.restype = C.c_longlong
    lib.lb_pair_list_builds.argtypes = [P]
    lib.lb_pair_list_builds.restype = C.c_longlong
    lib.lb_fused_kernel.argtypes = [P]
    lib.lb_destroy.argtypes = [P]
    lib.lb_last_error.argtypes = [P]
    lib.lb_last_error.restype = C.c_char_p
    _lib = lib
    return lib


class LBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (status %d)" % (msg, code))
        self.code = code


def _dp(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).ravel()
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def make_params(**kw) -> LbParams:
    from .workloads import default_params

    d = default_params()
    unknown = set(kw) - set(d)
    if unknown:
        raise KeyError("unknown parameters: %s" % sorted(unknown))
    d.update(kw)
    p = LbParams()
    for name, _t in LbParams._fields_:
        v = d[name]
        field = getattr(p, name)
        if hasattr(field, "__len__"):
            for i, x in enumerate(v):
                field[i] = x
        else:
            setattr(p, name, v)
    return p


# ------------------------------------------------- C-named thin wrappers
def lb_workspace_bytes(nx, ny, nz, prec, max_colloids) -> int:
    out = C.c_size_t(0)
    rc = load().lb_workspace_bytes(nx, ny, nz, prec, max_colloids, C.byref(out))
    if rc:
        raise LBError(rc, "lb_workspace_bytes")
    return out.value


def lb_create(nx, ny, nz, prec, max_colloids, workspace_ptr: int, nbytes: int, stream_ptr: int):
    h = C.c_void_p()
    rc = load().lb_create(nx, ny, nz, prec, max_colloids, C.c_void_p(workspace_ptr), nbytes,
                          C.c_void_p(stream_ptr), C.byref(h))
    if rc:
        raise LBError(rc, "lb_create")
    return h


def _check(h, rc, what):
    if rc < 0:
        raise LBError(rc, "%s: %s" % (what, load().lb_last_error(h).decode()))
    return rc


def lb_set_params(h, **params):
    p = make_params(**params)
    return _check(h, load().lb_set_params(h, C.byref(p)), "lb_set_params")


def lb_init_fields(h, rhoA, rhoB, u=None):
    a, b = _f64(rhoA), _f64(rhoB)  # rhoB may be None on a one-component lattice
    uu = _f64(u, 3 * a.size)
    return _check(h, load().lb_init_fields(h, _dp(a), _dp(b), _dp(uu)), "lb_init_fields")


def lb_add_colloids(h, pos, radius, mass, vel=None, omega=None, quat=None):
    pos = _f64(pos)
    n = pos.size // 3
    rad = _f64(np.broadcast_to(np.asarray(radius, dtype=np.float64), (n,)))
    mas = _f64(np.broadcast_to(np.asarray(mass, dtype=np.float64), (n,)))
    rc = load().lb_add_colloids(h, n, _dp(pos), _dp(_f64(vel, 3 * n)), _dp(_f64(omega, 3 * n)),
                                _dp(_f64(quat, 4 * n)), _dp(rad), _dp(mas))
    return _check(h, rc, "lb_add_colloids")


def lb_step(h, nsteps: int):
    return _check(h, load().lb_step(h, nsteps), "lb_step")


def lb_get_fields(h, rhoA: np.ndarray, rhoB: np.ndarray, u: np.ndarray):
    return _check(h, load().lb_get_fields(h, _dp(rhoA), _dp(rhoB), _dp(u)), "lb_get_fields")


def lb_get_colloids(h, pos, vel, omega, quat, force, torque):
    return _check(h, load().lb_get_colloids(h, *[_dp(a) for a in (pos, vel, omega, quat, force, torque)]),
                  "lb_get_colloids")


def lb_get_colloid_terms(h, which: int, out: np.ndarray):
    return _check(h, load().lb_get_colloid_terms(h, which, _dp(out)), "lb_get_colloid_terms")


def lb_get_totals(h, out: np.ndarray):
    return _check(h, load().lb_get_totals(h, _dp(out)), "lb_get_totals")


def lb_get_populations(h, k: int, out: np.ndarray):
    return _check(h, load().lb_get_populations(h, k, _dp(out)), "lb_get_populations")


def lb_get_owner(h, out: np.ndarray):
    return _check(h, load().lb_get_owner(h, out.ctypes.data_as(C.POINTER(C.c_int))), "lb_get_owner")


def lb_profile(h, enable: bool):
    return _check(h, load().lb_profile(h, int(bool(enable))), "lb_profile")


LB_KERNEL_FUSED, LB_KERNEL_DENSITY = 0, 1
LB_ROUND_NEAREST, LB_ROUND_STOCHASTIC = 0, 1


def lb_set_rounding(h, mode: int, seed: int = 0):
    """Rounding of the FP16 deviation stores (LB_ROUND_NEAREST or
    LB_ROUND_STOCHASTIC, bits from ``seed``)."""
    return _check(h, load().lb_set_rounding(h, int(mode), int(seed) & ((1 << 64) - 1)), "lb_set_rounding")


def lb_profile_read(h):
    """(summed fused-kernel time in ms, number of timed launches)"""
    t, n = C.c_double(0.0), C.c_longlong(0)
    _check(h, load().lb_profile_read(h, C.byref(t), C.byref(n)), "lb_profile_read")
    return t.value, n.value


def lb_profile_read_kernel(h, kernel: int):
    """(summed time in ms, number of timed launches) of LB_KERNEL_FUSED or
    LB_KERNEL_DENSITY"""
    t, n = C.c_double(0.0), C.c_longlong(0)
    _check(h, load().lb_profile_read_kernel(h, int(kernel), C.byref(t), C.byref(n)), "lb_profile_read_kernel")
    return t.value, n.value


def lb_state_bytes(h) -> int:
    out = C.c_size_t(0)
    _check(h, load().lb_state_bytes(h, C.byref(out)), "lb_state_bytes")
    return out.value


def lb_get_state(h, d_dst: int):
    return _check(h, load().lb_get_state(h, C.c_void_p(d_dst)), "lb_get_state")


def lb_set_state(h, d_src: int):
    return _check(h, load().lb_set_state(h, C.c_void_p(d_src)), "lb_set_state")


def lb_adjoint_bytes(h):
    fb, sb = C.c_size_t(0), C.c_size_t(0)
    _check(h, load().lb_adjoint_bytes(h, C.byref(fb), C.byref(sb)), "lb_adjoint_bytes")
    return fb.value, sb.value


def lb_adjoint_seed(h, weight: float, d_adj: int, d_scratch: int) -> float:
    v = C.c_double(0.0)
    _check(h, load().lb_adjoint_seed(h, float(weight), C.c_void_p(d_adj), C.c_void_p(d_scratch), C.byref(v)),
           "lb_adjoint_seed")
    return v.value


def lb_adjoint_step(h, d_state: int, d_adj_in: int, d_adj_out: int, d_scratch: int, dJdF, grads: np.ndarray):
    g = None if dJdF is None else _f64(dJdF)
    return _check(h, load().lb_adjoint_step(h, C.c_void_p(d_state), C.c_void_p(d_adj_in), C.c_void_p(d_adj_out),
                                            C.c_void_p(d_scratch), _dp(g), _dp(grads)), "lb_adjoint_step")


def lb_adjoint_step_async(h, d_state: int, d_adj_in: int, d_adj_out: int, d_scratch: int, d_dJdF, grads=None):
    """d_dJdF: device pointer or None; grads: host array of 5 (read and clear
    the accumulated gradients, synchronising) or None (keep accumulating)."""
    return _check(h, load().lb_adjoint_step_async(h, C.c_void_p(d_state), C.c_void_p(d_adj_in),
                                                  C.c_void_p(d_adj_out), C.c_void_p(d_scratch),
                                                  C.c_void_p(d_dJdF or None), _dp(grads)),
                  "lb_adjoint_step_async")


def lb_drag_gradient(h, d_F: int, weight: float, eps: float, d_dJdF: int):
    return _check(h, load().lb_drag_gradient(h, C.c_void_p(d_F), float(weight), float(eps), C.c_void_p(d_dJdF)),
                  "lb_drag_gradient")


def lb_record(h, d_states, d_forces, nsteps: int):
    """d_states / d_forces: device pointers or None."""
    return _check(h, load().lb_record(h, C.c_void_p(d_states or None), C.c_void_p(d_forces or None), int(nsteps)),
                  "lb_record")


def lb_adjoint_initial(h, d_adj: int, d_grad: int):
    return _check(h, load().lb_adjoint_initial(h, C.c_void_p(d_adj), C.c_void_p(d_grad)), "lb_adjoint_initial")


def lb_totals_static(d_pops: int, prec: int, nx: int, ny: int, nz: int, plane_stride: int, d_mask: int,
                     rho0, d_out: int, stream_ptr: int) -> int:
    """Allocation-free global totals of caller-held device populations (see
    lbgb.h); pointers are device addresses as integers (0 for NULL)."""
    r0 = None if rho0 is None else _f64(rho0, 2)
    rc = load().lb_totals_static(C.c_void_p(d_pops), prec, nx, ny, nz, plane_stride,
                                 C.c_void_p(d_mask or None), _dp(r0), C.c_void_p(d_out),
                                 C.c_void_p(stream_ptr or None))
    if rc:
        raise LBError(rc, "lb_totals_static")
    return rc


def lb_launch_count(h) -> int:
    return int(load().lb_launch_count(h))


def lb_pair_list_builds(h) -> int:
    """Particle pair-list builds so far (synchronises the context's stream)."""
    n = int(load().lb_pair_list_builds(h))
    if n < 0:
        raise LBError(LB_ERR_CUDA, "lb_pair_list_builds")
    return n


LB_FUSED_MOMENTUM, LB_FUSED_TWO_PASS, LB_FUSED_PLAIN, LB_FUSED_SINGLE = 1, 2, 3, 4
FUSED_KERNEL_NAMES = {LB_FUSED_MOMENTUM: "k_lean", LB_FUSED_TWO_PASS: "k_fused_async",
                      LB_FUSED_PLAIN: "k_fused", LB_FUSED_SINGLE: "k1_step"}


def lb_fused_kernel(h) -> int:
    """Which fused lattice kernel lb_step launches now (LB_FUSED_*)."""
    return _check(h, load().lb_fused_kernel(h), "lb_fused_kernel")


def lb_destroy(h):
    return load().lb_destroy(h)


def lb_last_error(h) -> str:
    return load().lb_last_error(h).decode()


# ------------------------------------------------------- convenience
class LBLattice:
    """One lattice context with a torch-allocated device workspace
    (components=1: the one-component fluid, LB_ONE_COMPONENT)."""

    def __init__(self, shape, prec="fp32", max_colloids=0, device=None, stream=None, components=2):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("LBLattice needs a CUDA device; there is no CPU fallback")
        self.shape = tuple(int(v) for v in shape)
        self.N = int(np.prod(self.shape))
        self.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        self.components = int(components)
        flag = LB_ONE_COMPONENT if self.components == 1 else 0
        self.device = torch.device(device or "cuda:0")
        nbytes = lb_workspace_bytes(*self.shape, self.prec | flag, max_colloids)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h = lb_create(*self.shape, self.prec | flag, max_colloids, self.workspace.data_ptr(), nbytes,
                           self.stream.cuda_stream)
        self.nc = 0

    def close(self):
        if getattr(self, "h", None):
            lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, **kw):
        lb_set_params(self.h, **kw)

    def init_fields(self, rhoA, rhoB=None, u=None):
        lb_init_fields(self.h, rhoA, rhoB, u)
        self.nc = 0

    def add_colloids(self, pos, radius, mass, vel=None, omega=None, quat=None):
        lb_add_colloids(self.h, pos, radius, mass, vel, omega, quat)
        self.nc += np.asarray(pos).size // 3

    def step(self, n=1):
        return lb_step(self.h, n)

    def get_fields(self):
        a, b, u = np.empty(self.N), np.empty(self.N), np.empty((3, self.N))
        lb_get_fields(self.h, a, b, u)
        return a, b, u

    def totals(self):
        out = np.empty(8)
        lb_get_totals(self.h, out)
        return out

    def get_colloids(self):
        n = self.nc
        arrs = [np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 4)),
                np.empty((n, 3)), np.empty((n, 3))]
        if n:
            lb_get_colloids(self.h, *arrs)
        return dict(zip(("pos", "vel", "omega", "quat", "force", "torque"), arrs))

    def term(self, name):
        out = np.empty((max(self.nc, 1), 3))
        lb_get_colloid_terms(self.h, TERMS[name], out)
        return out[: self.nc]

    def populations(self, k):
        out = np.empty((19, self.N))
        lb_get_populations(self.h, k, out)
        return out

    def owner(self):
        out = np.empty(self.N, dtype=np.int32)
        lb_get_owner(self.h, out)
        return out

    def launch_count(self):
        return lb_launch_count(self.h)

    def pair_list_builds(self):
        return lb_pair_list_builds(self.h)

    def profile(self, enable=True):
        lb_profile(self.h, enable)

    def profile_read(self, kernel: int = LB_KERNEL_FUSED):
        return lb_profile_read_kernel(self.h, kernel)

    def set_rounding(self, mode: int, seed: int = 0):
        lb_set_rounding(self.h, mode, seed)

    def fused_kernel(self) -> str:
        """Name of the fused lattice kernel lb_step launches now."""
        return FUSED_KERNEL_NAMES[lb_fused_kernel(self.h)]
