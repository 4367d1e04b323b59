"""Python handle on the plain FP64 CPU oracle (``iblbm_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously-correct reference
the CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package; the library
in ``paper_2609_02298_b300`` never does, and nothing here imports that library.

The C source is compiled with gcc into ``oracle/liboracle.so`` on first use
(or by :func:`build`).  Everything is FP64 and in lattice units.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iblbm_oracle.c")
_HDR = os.path.join(_HERE, "iblbm_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
# all-cores build of the same source (OpenMP over the node loops), used when the
# environment sets IBLBM_ORACLE_OPENMP=1 (the all-cores CPU baseline)
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")

PERIODIC, VELOCITY, NEUMANN = 0, 1, 2
BGK, TRT, CMMRT, STREAM_ONLY = 0, 1, 2, 3
HAT, PESKIN4 = 0, 1
DF, MDF, DFC = 0, 1, 2
FIXED, PRESCRIBED, FREE, FREE_TRANSLATION = 0, 1, 2, 3

_lib = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add); returns the .so path.
    ``openmp`` builds the all-cores copy (the node loops' OpenMP pragmas enabled)."""
    out = _LIB_OMP if openmp else _LIB
    stale = not os.path.exists(out) or any(
        os.path.getmtime(p) > os.path.getmtime(out) for p in (_SRC, _HDR))
    if force or stale:
        tmp = out + ".tmp%d" % os.getpid()
        flags = ["-fopenmp"] if openmp else ["-Wno-unknown-pragmas"]
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
                               "-Wall"] + flags + ["-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class LatticeParams(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("bc", C.c_int * 4),
                ("ubc", (C.c_double * 2) * 4), ("collision", C.c_int), ("tau", C.c_double),
                ("trt_lambda", C.c_double), ("cm_sq", C.c_double), ("cm_se", C.c_double),
                ("gfx", C.c_double), ("gfy", C.c_double), ("wall_closure", C.c_int)]


class BodyParams(C.Structure):
    _fields_ = [("xc", C.c_double), ("yc", C.c_double), ("radius", C.c_double),
                ("rho_ratio", C.c_double), ("motion", C.c_int), ("gx", C.c_double),
                ("gy", C.c_double), ("internal_mass", C.c_int), ("mdf_nmin", C.c_int),
                ("mdf_nmax", C.c_int), ("mdf_tol", C.c_double), ("mdf_omega", C.c_double),
                ("osc_amp", C.c_double), ("osc_period", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build(openmp=os.environ.get("IBLBM_ORACLE_OPENMP") == "1"))
        P = C.POINTER
        d, i, vp = C.c_double, C.c_int, C.c_void_p
        pd, pi = P(C.c_double), P(C.c_int)
        sig = {
            "orc_create": (vp, [P(LatticeParams)]),
            "orc_destroy": (None, [vp]),
            "orc_add_body": (i, [vp, pd, i, d, i, i, P(BodyParams)]),
            "orc_set_uniform": (None, [vp, d, d, d]),
            "orc_set_populations": (None, [vp, pd]),
            "orc_get_populations": (None, [vp, pd]),
            "orc_step": (i, [vp, i]),
            "orc_get_macro": (None, [vp, pd, pd, pd]),
            "orc_body_forces": (None, [vp, i, pd]),
            "orc_body_state": (None, [vp, i, pd]),
            "orc_force_history": (i, [vp, i, pd, i]),
            "orc_marker_data": (None, [vp, i, pd]),
            "orc_marker_stencils": (None, [vp, i, pi]),
            "orc_mdf_iterations": (i, [vp, i]),
            "orc_mdf_omega": (d, [vp, i]),
            "orc_mdf_residual": (d, [vp, i]),
            "orc_mdf_omega_end": (d, [vp, i]),
            "orc_phi": (d, [i, d]),
            "orc_feq": (None, [d, d, d, pd]),
            "orc_guo": (None, [d, d, d, d, d, pd]),
            "orc_collide_node": (None, [P(LatticeParams), pd, d, d]),
            "orc_interp": (None, [i, i, i, pd, pd, i, pd]),
            "orc_spread": (None, [i, i, i, pd, pd, i, d, pd]),
            "orc_dfc_lambda": (None, [i, i, i, pd, i, d, pd]),
            "orc_mdf_norm_A": (d, [i, i, i, pd, i, d]),
            "orc_verlet_free_fall": (None, [d, d, d, d, i, i, pd, pd]),
            "orc_local_diagnostics_fields": (i, [i, i, i, pd, pd, pd, pd, i, d, pd, d, d, pd, vp]),
            "orc_local_diagnostics": (i, [vp, i, d, d, pd, vp]),
            "orc_set_marker_velocity": (i, [vp, i, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lattice_params(nx, ny, bc=(PERIODIC,) * 4, ubc=((0.0, 0.0),) * 4, collision=BGK, tau=0.8,
                   trt_lambda=0.25, cm_sq=1.2, cm_se=1.4, force=(0.0, 0.0), wall_closure=0) -> LatticeParams:
    p = LatticeParams()
    p.nx, p.ny = nx, ny
    for s in range(4):
        p.bc[s] = bc[s]
        p.ubc[s][0], p.ubc[s][1] = ubc[s]
    p.collision, p.tau, p.trt_lambda, p.cm_sq, p.cm_se = collision, tau, trt_lambda, cm_sq, cm_se
    p.gfx, p.gfy = force
    p.wall_closure = wall_closure
    return p


# ---- primitives ---------------------------------------------------------------
def phi(kernel: int, r: float) -> float:
    return lib().orc_phi(kernel, float(r))


def feq(rho, ux, uy) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, _dp(out))
    return out


def guo(tau, ux, uy, Fx, Fy) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_guo(tau, ux, uy, Fx, Fy, _dp(out))
    return out


def collide_node(params: LatticeParams, f: np.ndarray, Fx=0.0, Fy=0.0) -> np.ndarray:
    v = np.ascontiguousarray(f, dtype=np.float64).copy()
    lib().orc_collide_node(C.byref(params), _dp(v), Fx, Fy)
    return v


def interp(kernel, field: np.ndarray, xy: np.ndarray) -> np.ndarray:
    g = np.ascontiguousarray(field, dtype=np.float64)
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    out = np.zeros(len(xy))
    lib().orc_interp(kernel, g.shape[1], g.shape[0], _dp(g), _dp(xy), len(xy), _dp(out))
    return out


def spread(kernel, Fk: np.ndarray, xy: np.ndarray, ds: float, nx: int, ny: int) -> np.ndarray:
    Fk = np.ascontiguousarray(Fk, dtype=np.float64)
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    out = np.zeros((ny, nx))
    lib().orc_spread(kernel, nx, ny, _dp(Fk), _dp(xy), len(xy), ds, _dp(out))
    return out


def dfc_lambda(kernel, xy: np.ndarray, ds: float, nx: int, ny: int) -> np.ndarray:
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    out = np.zeros(len(xy))
    lib().orc_dfc_lambda(kernel, nx, ny, _dp(xy), len(xy), ds, _dp(out))
    return out


def local_diagnostics_fields(kernel, rho, ux, uy, md, ds, body, u_ref, kappa=2.0, per_marker=False):
    """Sec. 2.8 diagnostics from node fields [ny, nx] and marker data [n, 7]; returns
    out[8] (and the [n, 5] per-marker table when ``per_marker``)."""
    rho, ux, uy = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy))
    md = np.ascontiguousarray(md, dtype=np.float64).reshape(-1, 7)
    body = np.ascontiguousarray(body, dtype=np.float64)
    out = np.zeros(8)
    pm = np.zeros((len(md), 5)) if per_marker else None
    rc = lib().orc_local_diagnostics_fields(kernel, rho.shape[1], rho.shape[0], _dp(rho), _dp(ux), _dp(uy),
                                            _dp(md), len(md), ds, _dp(body), u_ref, kappa, _dp(out),
                                            pm.ctypes.data if pm is not None else None)
    if rc:
        raise ValueError("stencil or probe node outside the lattice")
    return (out, pm) if per_marker else out


def mdf_norm_A(kernel, xy: np.ndarray, ds: float, nx: int, ny: int) -> float:
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    return lib().orc_mdf_norm_A(kernel, nx, ny, _dp(xy), len(xy), ds)


def verlet_free_fall(rho_ratio, radius, gx, gy, internal_mass, nsteps):
    v = np.zeros((nsteps, 2))
    x = np.zeros((nsteps, 2))
    lib().orc_verlet_free_fall(rho_ratio, radius, gx, gy, internal_mass, nsteps, _dp(v), _dp(x))
    return v, x


# ---- whole case -------------------------------------------------------------------
class Case:
    """One oracle simulation (post-collision state between steps)."""

    def __init__(self, params: LatticeParams):
        self.nx, self.ny = params.nx, params.ny
        self._p = params
        self._h = lib().orc_create(C.byref(params))
        if not self._h:
            raise ValueError("invalid lattice parameters")
        self.body_n = []

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def add_body(self, xy, ds, kernel, scheme, body: BodyParams) -> int:
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        rc = lib().orc_add_body(self._h, _dp(xy), len(xy), ds, kernel, scheme, C.byref(body))
        if rc < 0:
            raise ValueError("orc_add_body failed: %d" % rc)
        self.body_n.append(len(xy))
        return rc

    def set_uniform(self, rho, ux, uy):
        lib().orc_set_uniform(self._h, rho, ux, uy)

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        lib().orc_set_populations(self._h, _dp(f))

    def populations(self) -> np.ndarray:
        out = np.zeros((9, self.ny, self.nx))
        lib().orc_get_populations(self._h, _dp(out))
        return out

    def step(self, n: int = 1):
        rc = lib().orc_step(self._h, n)
        if rc:
            raise RuntimeError("orc_step failed: %d" % rc)

    def macro(self):
        r = np.zeros((self.ny, self.nx))
        ux = np.zeros_like(r)
        uy = np.zeros_like(r)
        lib().orc_get_macro(self._h, _dp(r), _dp(ux), _dp(uy))
        return r, ux, uy

    def body_forces(self, b: int) -> np.ndarray:
        out = np.zeros(3)
        lib().orc_body_forces(self._h, b, _dp(out))
        return out

    def body_state(self, b: int) -> np.ndarray:
        out = np.zeros(6)
        lib().orc_body_state(self._h, b, _dp(out))
        return out

    def force_history(self, b: int, cap: int = 1 << 22) -> np.ndarray:
        out = np.zeros((cap, 3))
        n = lib().orc_force_history(self._h, b, _dp(out), cap)
        return out[:n].copy()

    def marker_data(self, b: int) -> np.ndarray:
        out = np.zeros((self.body_n[b], 7))
        lib().orc_marker_data(self._h, b, _dp(out))
        return out

    def marker_stencils(self, b: int) -> np.ndarray:
        out = np.zeros((self.body_n[b], 2), dtype=np.int32)
        lib().orc_marker_stencils(self._h, b, out.ctypes.data_as(C.POINTER(C.c_int)))
        return out

    def mdf_iterations(self, b: int) -> int:
        return lib().orc_mdf_iterations(self._h, b)

    def mdf_omega(self, b: int) -> float:
        return lib().orc_mdf_omega(self._h, b)

    def mdf_residual(self, b: int) -> float:
        return lib().orc_mdf_residual(self._h, b)

    def mdf_omega_end(self, b: int) -> float:
        return lib().orc_mdf_omega_end(self._h, b)

    def set_marker_velocity(self, b: int, ud=None) -> None:
        if ud is None:
            rc = lib().orc_set_marker_velocity(self._h, b, None)
        else:
            ud = np.ascontiguousarray(ud, dtype=np.float64).reshape(-1, 2)
            rc = lib().orc_set_marker_velocity(self._h, b, ud.ctypes.data)
        if rc:
            raise ValueError("orc_set_marker_velocity: bad body or moving body")

    def local_diagnostics(self, b: int, u_ref: float, kappa: float = 2.0, per_marker: bool = False):
        out = np.zeros(8)
        pm = np.zeros((self.body_n[b], 5)) if per_marker else None
        rc = lib().orc_local_diagnostics(self._h, b, u_ref, kappa, _dp(out),
                                         pm.ctypes.data if pm is not None else None)
        if rc:
            raise ValueError("stencil or probe node outside the lattice")
        return (out, pm) if per_marker else out
