"""ctypes binding of the plain C FP64 oracle (``lbgb_oracle.c``).

Test infrastructure only.  The oracle shares no code with the CUDA library:
it is compiled from its own C file with gcc (-O2 -ffp-contract=off -fopenmp;
every thread count gives the same bits), it keeps
its own table of parameter defaults (DEFAULTS below), and only the seeded
input generators of ``paper_2004_04080_gb300.workloads`` (initial densities,
particle placements, named parameter sets) feed both.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbgb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbgb_oracle.so")
_lib = None
_lock = threading.Lock()


class OrcParams(C.Structure):
    """Mirror of ``orc_params`` in lbgb_oracle.c (field order matters)."""

    _fields_ = [
        ("tau", C.c_double * 2),
        ("G", C.c_double),
        ("zeta", C.c_double * 2),
        ("rho0", C.c_double * 2),
        ("bc", C.c_int * 3),
        ("wall_u_lo", C.c_double * 3),
        ("wall_u_hi", C.c_double * 3),
        ("body_force", C.c_double * 3),
        ("hertz_K", C.c_double),
        ("hertz_sigma", C.c_double),
        ("hertz_rcap", C.c_double),
        ("lub_on", C.c_int),
        ("lub_hn", C.c_double),
        ("lub_hmin", C.c_double),
        ("lub_scale", C.c_double),
        ("side_wall_k", C.c_double),
        ("side_wall_d", C.c_double),
        ("rotate", C.c_int),
        ("janus", C.c_int),
        ("janus_theta0", C.c_double),
        ("janus_width", C.c_double),
        ("open", C.c_int * 2),
        ("open_rho", C.c_double * 4),
        ("open_extrap", C.c_int),
    ]


def build_oracle(force: bool = False) -> str:
    """Compile the oracle shared library (plain gcc, no GPU needed)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build_oracle())
        P = C.c_void_p
        D = C.POINTER(C.c_double)
        I = C.POINTER(C.c_int)
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
        lib.orc_destroy.argtypes = [P]
        lib.orc_set_params.argtypes = [P, C.POINTER(OrcParams)]
        lib.orc_init_fields.argtypes = [P, D, D, D]
        lib.orc_add_colloids.argtypes = [P, C.c_int, D, D, D, D, D, D]
        lib.orc_step.argtypes = [P, C.c_int]
        lib.orc_get_fields.argtypes = [P, D, D, D]
        lib.orc_totals.argtypes = [P, D]
        lib.orc_get_colloids.argtypes = [P, D, D, D, D, D, D]
        lib.orc_get_colloid_terms.argtypes = [P, C.c_int, D]
        lib.orc_get_populations.argtypes = [P, C.c_int, D]
        lib.orc_set_populations.argtypes = [P, C.c_int, D]
        lib.orc_get_owner.argtypes = [P, I]
        lib.orc_get_psi.argtypes = [P, C.c_int, D]
        lib.orc_set_colloid_state.argtypes = [P, C.c_int, D, D, D, D]
        lib.orc_feq.argtypes = [C.c_double, D, D]
        lib.orc_lattice.argtypes = [I, I, I, D, I]
        lib.orc_pair_force.argtypes = [C.POINTER(OrcParams), D, C.c_double, C.c_double, D, D, D]
        lib.orc_integrate_one.argtypes = [D, D, D, D, C.c_double, C.c_double, D, D, C.c_int, I]
        lib.orc_set_threads.argtypes = [C.c_int]
        lib.orc_set_threads.restype = C.c_int
        _lib = lib
        return lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


# Values of the parameters a caller leaves out: a plain two-component BGK
# fluid at tau = 1 without coupling, wetting, walls, body force or particle
# pair forces; reference density 1/2 per component (the 50/50 mixture of the
# benchmark workloads); lubrication off, with the cut-off gap 0.67 and floor
# 0.5 of App. D and the prefactor 0.1; rotation integrated (Eqs. 33-34);
# Janus wettability off, with the switch at 108 degrees and 10 degrees wide of
# the benchmark input (App. D) for when it is turned on; rcut and delr (App. A)
# only size a neighbour list in the GPU library, so the oracle, which
# evaluates every pair, accepts and ignores them; the z faces are walls unless
# opened (Sec. 2.2: open=(lo, hi) types, open_rho = (lo A, lo B, hi A, hi B)),
# with the face values of pressure and velocity faces taken at the boundary
# node unless open_extrap = 1 (first-order extrapolation, Sec. 2.2).
DEFAULTS = dict(
    tau=(1.0, 1.0), G=0.0, zeta=(0.0, 0.0), rho0=(0.5, 0.5), bc=(1, 1, 1),
    wall_u_lo=(0.0, 0.0, 0.0), wall_u_hi=(0.0, 0.0, 0.0), body_force=(0.0, 0.0, 0.0),
    hertz_K=0.0, hertz_sigma=0.0, hertz_rcap=0.0,
    lub_on=0, lub_hn=0.67, lub_hmin=0.5, lub_scale=0.1,
    side_wall_k=0.0, side_wall_d=0.0, rotate=1,
    janus=0, janus_theta0=108.0, janus_width=10.0,
    rcut=0.0, delr=0.0,
    open=(0, 0), open_rho=(1.0, 1.0, 1.0, 1.0), open_extrap=0,
)


def make_params(**kw) -> OrcParams:
    """Fill an OrcParams from keyword arguments (same names as lb_params),
    the rest from DEFAULTS."""
    unknown = set(kw) - set(DEFAULTS)
    if unknown:
        raise KeyError("unknown parameters: %s" % sorted(unknown))
    d = dict(DEFAULTS)
    d.update(kw)
    p = OrcParams()
    for name, _t in OrcParams._fields_:
        v = d[name]
        field = getattr(p, name)
        if hasattr(field, "__len__"):
            for i, x in enumerate(v):
                field[i] = x
        else:
            setattr(p, name, v)
    return p


TERMS = {"F_liq": 0, "T_liq": 1, "F_d": 2, "T_d": 3, "F_c": 4, "T_c": 5, "F_s": 6,
         "T_s": 7, "F_pair": 8, "F_total": 9, "T_total": 10}


class Oracle:
    """One oracle lattice: ``Oracle(nx, ny, nz, max_colloids)``."""

    def __init__(self, nx: int, ny: int, nz: int, max_colloids: int = 0):
        self.lib = _load()
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        self.h = self.lib.orc_create(nx, ny, nz, max_colloids)
        if not self.h:
            raise MemoryError("orc_create failed")
        self.nc = 0

    def close(self):
        if self.h:
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc, what):
        if rc != 0:
            raise RuntimeError("%s failed with status %d" % (what, rc))
        return rc

    def set_params(self, **kw):
        self.params = make_params(**kw)
        self._chk(self.lib.orc_set_params(self.h, C.byref(self.params)), "orc_set_params")

    def init_fields(self, rhoA, rhoB, u=None):
        a, b = _f64(rhoA).ravel(), _f64(rhoB).ravel()
        uu = None if u is None else _f64(u).reshape(3, self.N)
        self._chk(self.lib.orc_init_fields(self.h, _dp(a), _dp(b), _dp(uu)), "orc_init_fields")

    def add_colloids(self, pos, radius, mass, vel=None, omega=None, quat=None):
        pos = _f64(pos).reshape(-1, 3)
        n = pos.shape[0]
        rad = _f64(np.broadcast_to(radius, (n,)))
        mas = _f64(np.broadcast_to(mass, (n,)))
        v = None if vel is None else _f64(vel).reshape(n, 3)
        w = None if omega is None else _f64(omega).reshape(n, 3)
        q = None if quat is None else _f64(quat).reshape(n, 4)
        rc = self.lib.orc_add_colloids(self.h, n, _dp(pos), _dp(v), _dp(w), _dp(q), _dp(rad), _dp(mas))
        self._chk(rc, "orc_add_colloids")
        self.nc += n

    def step(self, n: int = 1, check: bool = True) -> int:
        rc = self.lib.orc_step(self.h, n)
        if check:
            self._chk(rc, "orc_step")
        return rc

    def get_fields(self):
        a = np.empty(self.N)
        b = np.empty(self.N)
        u = np.empty((3, self.N))
        self._chk(self.lib.orc_get_fields(self.h, _dp(a), _dp(b), _dp(u)), "orc_get_fields")
        return a, b, u

    def totals(self):
        out = np.empty(8)
        self._chk(self.lib.orc_totals(self.h, _dp(out)), "orc_totals")
        return out

    def get_colloids(self):
        n = self.nc
        pos, vel, om = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3))
        q, F, T = np.empty((n, 4)), np.empty((n, 3)), np.empty((n, 3))
        self.lib.orc_get_colloids(self.h, _dp(pos), _dp(vel), _dp(om), _dp(q), _dp(F), _dp(T))
        return dict(pos=pos, vel=vel, omega=om, quat=q, force=F, torque=T)

    def term(self, name: str):
        out = np.empty((max(self.nc, 1), 3))
        self._chk(self.lib.orc_get_colloid_terms(self.h, TERMS[name], _dp(out)), "orc_get_colloid_terms")
        return out[: self.nc]

    def populations(self, k: int):
        out = np.empty((19, self.N))
        self._chk(self.lib.orc_get_populations(self.h, k, _dp(out)), "orc_get_populations")
        return out

    def set_populations(self, k: int, f):
        f = _f64(f).reshape(19, self.N)
        self._chk(self.lib.orc_set_populations(self.h, k, _dp(f)), "orc_set_populations")

    def psi(self, k: int):
        """psi^k of the last force evaluation: virtual densities (Eq. 20)
        on particle frontier nodes, 0 elsewhere."""
        out = np.empty(self.N)
        self._chk(self.lib.orc_get_psi(self.h, k, _dp(out)), "orc_get_psi")
        return out

    def owner(self):
        out = np.empty(self.N, dtype=np.int32)
        self._chk(self.lib.orc_get_owner(self.h, out.ctypes.data_as(C.POINTER(C.c_int))), "orc_get_owner")
        return out

    def set_colloid_state(self, p, pos=None, vel=None, omega=None, quat=None):
        args = [None if a is None else _f64(a) for a in (pos, vel, omega, quat)]
        self._chk(self.lib.orc_set_colloid_state(self.h, p, *[_dp(a) for a in args]), "orc_set_colloid_state")


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's site loops (0: all cores); returns the count."""
    return int(_load().orc_set_threads(int(n)))


def lattice():
    """(c [19,3] int, w [19], opp [19]) as tabulated by the oracle."""
    lib = _load()
    cx, cy, cz, opp = (np.empty(19, dtype=np.int32) for _ in range(4))
    w = np.empty(19)
    ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
    lib.orc_lattice(ip(cx), ip(cy), ip(cz), _dp(w), ip(opp))
    return np.stack([cx, cy, cz], axis=1), w, opp


def feq(rho: float, u) -> np.ndarray:
    lib = _load()
    uu = _f64(u)
    out = np.empty(19)
    lib.orc_feq(float(rho), _dp(uu), _dp(out))
    return out


def pair_force(rij, Ri, Rj, vi=(0, 0, 0), vj=(0, 0, 0), **params):
    lib = _load()
    p = make_params(**params)
    out = np.empty(3)
    r, a, b = _f64(rij), _f64(vi), _f64(vj)
    lib.orc_pair_force(C.byref(p), _dp(r), float(Ri), float(Rj), _dp(a), _dp(b), _dp(out))
    return out


def integrate_one(r, v, w, q, m, R, F, T, rotate=1, L=(0, 0, 0)):
    """One leap-frog + Svanberg step; returns new (r, v, w, q)."""
    lib = _load()
    r, v, w, q = (_f64(a).copy() for a in (r, v, w, q))
    F, T = _f64(F), _f64(T)
    Ls = np.asarray(L, dtype=np.int32)
    lib.orc_integrate_one(_dp(r), _dp(v), _dp(w), _dp(q), float(m), float(R), _dp(F), _dp(T),
                          int(rotate), Ls.ctypes.data_as(C.POINTER(C.c_int)))
    return r, v, w, q
