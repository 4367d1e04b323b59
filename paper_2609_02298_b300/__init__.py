"""B300 (sm_103a) immersed-boundary lattice Boltzmann library: Python binding.

A thin ctypes layer over ``libiblbm.so`` (C ABI in ``include/iblbm.h``): it
marshals arguments, installs PyTorch's caching allocator as the library's
device allocator and converts status codes to exceptions.  Every step of the
method runs in the library's CUDA kernels; there is no CPU fallback -- loading
fails loudly when the shared library is missing.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref
from typing import Iterable, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libiblbm.so")

BC_PERIODIC, BC_VELOCITY, BC_NEUMANN = 0, 1, 2
BGK, TRT, CMMRT, STREAM_ONLY = 0, 1, 2, 3
HAT, PESKIN4 = 0, 1
DF, MDF, DFC = 0, 1, 2
F64, F32, F16S = 0, 1, 2
FIXED, PRESCRIBED, FREE, FREE_TRANSLATION = 0, 1, 2, 3

OK = 0
WARN_MDF_NOT_CONVERGED = 1


class IblbmError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s failed: %s (%d)" % (what, strerror(code), code))
        self.code = code


class LatticeDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("storage", C.c_int), ("bc", C.c_int * 4),
                ("u_bc", (C.c_double * 2) * 4), ("trt_lambda", C.c_double), ("cm_sq", C.c_double),
                ("cm_se", C.c_double), ("force", C.c_double * 2), ("init_rho", C.c_double),
                ("init_u", C.c_double * 2), ("cuda_stream", C.c_void_p), ("wall_closure", C.c_int)]


class BodyDesc(C.Structure):
    _fields_ = [("xc", C.c_double), ("yc", C.c_double), ("radius", C.c_double),
                ("rho_ratio", C.c_double), ("motion", C.c_int), ("gx", C.c_double),
                ("gy", C.c_double), ("internal_mass", C.c_int), ("mdf_nmin", C.c_int),
                ("mdf_nmax", C.c_int), ("mdf_tol", C.c_double), ("mdf_omega", C.c_double),
                ("osc_amp", C.c_double), ("osc_period", C.c_double), ("history_cap", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

# (name, restype, argtypes) of every exported call
_P = C.POINTER
_d, _i, _vp, _sz, _ll = C.c_double, C.c_int, C.c_void_p, C.c_size_t, C.c_longlong
_pd, _pi = _P(C.c_double), _P(C.c_int)
SIGNATURES = [
    ("iblbm_set_allocator", _i, [ALLOC_FN, FREE_FN, _vp]),
    ("iblbm_create", _i, [_P(LatticeDesc), _i, _d, _P(_vp)]),
    ("iblbm_destroy", None, [_vp]),
    ("iblbm_add_body", _i, [_vp, _pd, _i, _d, _i, _i, _P(BodyDesc), _pi]),
    ("iblbm_step", _i, [_vp, _i]),
    ("iblbm_sync", _i, [_vp]),
    ("iblbm_steps_done", _ll, [_vp]),
    ("iblbm_body_forces", _i, [_vp, _i, _pd]),
    ("iblbm_body_state", _i, [_vp, _i, _pd]),
    ("iblbm_force_history", _i, [_vp, _i, _pd, _i, _pi]),
    ("iblbm_move_body", _i, [_vp, _i, _pd, _pd]),
    ("iblbm_marker_data", _i, [_vp, _i, _pd]),
    ("iblbm_marker_stencils", _i, [_vp, _i, _pi]),
    ("iblbm_mdf_info", _i, [_vp, _i, _pi, _pd, _pd]),
    ("iblbm_mdf_relaxation", _i, [_vp, _i, _pd]),
    ("iblbm_local_diagnostics", _i, [_vp, _i, C.c_double, C.c_double, _pd, _vp]),
    ("iblbm_set_marker_velocity", _i, [_vp, _i, _vp]),
    ("iblbm_get_populations", _i, [_vp, _pd, _i]),
    ("iblbm_set_populations", _i, [_vp, _pd]),
    ("iblbm_get_macro", _i, [_vp, _pd, _pd, _pd]),
    ("iblbm_snapshot", _i, [_vp, _vp, _sz, _P(_sz)]),
    ("iblbm_restore", _i, [_vp, _vp, _sz]),
    ("iblbm_device_bytes", _sz, [_vp]),
    ("iblbm_strerror", C.c_char_p, [_i]),
    ("iblbm_step_batch", _i, [_P(_vp), _i, _i]),
    ("iblbm_set_timing", _i, [_vp, _i]),
    ("iblbm_kernel_timing", _i, [_vp, _pd, _pi]),
    ("iblbm_stage_timing", _i, [_vp, _pd, _pi]),
    ("iblbm_dfc_lambda_noalloc", _i, [_vp, _i, _d, _i, _i, _i, _vp, _vp]),
    ("iblbm_set_kernel_variant", _i, [_i, _i, _i]),
    ("iblbm_kernel_variant", _i, [_i, _i, _pi, _pd]),
    ("iblbm_test_set_consumer_poll_limit", _i, [C.c_long]),
    ("iblbm_test_set_ib_fast", _i, [_i]),
    ("iblbm_server_create", _i, [_sz, _i, _vp, _P(_vp)]),
    ("iblbm_server_destroy", None, [_vp]),
    ("iblbm_server_submit", _i, [_vp, _P(LatticeDesc), _i, _d, _P(BodyDesc), _pd, _i, _d, _i, _i, _i,
                                 _P(_ll)]),
    ("iblbm_server_tick", _i, [_vp, _i, _pi, _pi]),
    ("iblbm_server_poll", _i, [_vp, _ll, _pd, _i, _pi, _pd]),
    ("iblbm_server_stats", _i, [_vp, _P(_sz), _pi, _pi]),
    ("iblbm_server_set_graphs", _i, [_vp, _i]),
]

_lib = None
_alloc_cb = None
_free_cb = None
_live = weakref.WeakSet()


@atexit.register
def _close_all():
    # release device memory while the allocator behind the callbacks still exists
    for lat in list(_live):
        try:
            lat.close()
        except Exception:
            pass


def _host_buffer(obj):
    """(address, bytes) of a contiguous host buffer: numpy array or CPU torch tensor."""
    if hasattr(obj, "data_ptr"):
        if obj.device.type != "cpu" or not obj.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor")
        return obj.data_ptr(), obj.numel() * obj.element_size()
    arr = np.asarray(obj)
    if not arr.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a contiguous array")
    return arr.ctypes.data, arr.nbytes


def load_library(path: str = LIB_PATH):
    """Loads libiblbm.so (building it first if the sources are newer); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        try:
            from . import build as _build
            _build.build()
        except Exception as exc:  # no toolchain: fail loudly, never fall back
            raise ImportError("libiblbm.so is missing and could not be built: %s" % exc) from exc
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load_library().iblbm_strerror(code).decode()


def _check(code: int, what: str) -> int:
    if code < 0:
        raise IblbmError(code, what)
    return code


def use_torch_allocator() -> None:
    """Routes the library's device allocations through PyTorch's caching allocator."""
    global _alloc_cb, _free_cb
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    _alloc_cb, _free_cb = ALLOC_FN(_alloc), FREE_FN(_free)
    _check(load_library().iblbm_set_allocator(_alloc_cb, _free_cb, None), "iblbm_set_allocator")


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Lattice:
    """One lattice with its bodies (an ``iblbm_ctx``)."""

    def __init__(self, nx: int, ny: int, collision: int = BGK, tau: float = 0.8, storage: int = F32,
                 bc: Sequence[int] = (BC_PERIODIC,) * 4,
                 u_bc: Sequence[Sequence[float]] = ((0.0, 0.0),) * 4, trt_lambda: float = 3.0 / 16.0,
                 cm_sq: float = 1.2, cm_se: float = 1.4, force=(0.0, 0.0), init_rho: float = 1.0,
                 init_u=(0.0, 0.0), stream: Optional[int] = None, wall_closure: int = 0):
        lib = load_library()
        d = LatticeDesc()
        d.nx, d.ny, d.storage = nx, ny, storage
        for s in range(4):
            d.bc[s] = bc[s]
            d.u_bc[s][0], d.u_bc[s][1] = u_bc[s]
        d.trt_lambda, d.cm_sq, d.cm_se = trt_lambda, cm_sq, cm_se
        d.force[0], d.force[1] = force
        d.init_rho = init_rho
        d.init_u[0], d.init_u[1] = init_u
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        d.cuda_stream = stream
        d.wall_closure = wall_closure
        h = C.c_void_p()
        _check(lib.iblbm_create(C.byref(d), collision, tau, C.byref(h)), "iblbm_create")
        self._h = h
        self.nx, self.ny, self.storage = nx, ny, storage
        self.body_n = []
        _live.add(self)

    @classmethod
    def from_spec(cls, spec, storage: Optional[int] = None, stream: Optional[int] = None) -> "Lattice":
        """Builds a lattice and its bodies from a case description object with the
        attributes nx, ny, bc, ubc, collision, tau, storage, trt_lambda, cm_sq,
        cm_se, force, init_u and bodies (each with xy, ds, kernel, scheme, xc,
        yc, radius, rho_ratio, motion, gx, gy, internal_mass, mdf_*, osc_*)."""
        lat = cls(spec.nx, spec.ny, spec.collision, spec.tau,
                  spec.storage if storage is None else storage, spec.bc, spec.ubc, spec.trt_lambda,
                  spec.cm_sq, spec.cm_se, spec.force, 1.0, spec.init_u, stream,
                  getattr(spec, "wall_closure", 0))
        for b in spec.bodies:
            lat.add_body(b.xy, b.ds, b.kernel, b.scheme, xc=b.xc, yc=b.yc, radius=b.radius,
                         rho_ratio=b.rho_ratio, motion=b.motion, gx=b.gx, gy=b.gy,
                         internal_mass=b.internal_mass, mdf_nmin=b.mdf_nmin, mdf_nmax=b.mdf_nmax,
                         mdf_tol=b.mdf_tol, mdf_omega=b.mdf_omega, osc_amp=b.osc_amp,
                         osc_period=b.osc_period)
        return lat

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load_library().iblbm_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def add_body(self, xy, ds: float, kernel: int, scheme: int, xc: float, yc: float, radius: float,
                 rho_ratio: float = 1.0, motion: int = FIXED, gx: float = 0.0, gy: float = 0.0,
                 internal_mass: int = 1, mdf_nmin: int = 5, mdf_nmax: int = 20, mdf_tol: float = 1e-4,
                 mdf_omega: float = 0.0, osc_amp: float = 0.0, osc_period: float = 1.0,
                 history_cap: int = 0) -> int:
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        b = BodyDesc()
        b.xc, b.yc, b.radius, b.rho_ratio, b.motion = xc, yc, radius, rho_ratio, motion
        b.gx, b.gy, b.internal_mass = gx, gy, internal_mass
        b.mdf_nmin, b.mdf_nmax, b.mdf_tol, b.mdf_omega = mdf_nmin, mdf_nmax, mdf_tol, mdf_omega
        b.osc_amp, b.osc_period, b.history_cap = osc_amp, osc_period, history_cap
        bid = C.c_int(-1)
        _check(load_library().iblbm_add_body(self._h, _dp(xy), len(xy), ds, kernel, scheme,
                                             C.byref(b), C.byref(bid)), "iblbm_add_body")
        self.body_n.append(len(xy))
        return bid.value

    def step(self, n: int = 1) -> None:
        _check(load_library().iblbm_step(self._h, n), "iblbm_step")

    def sync(self) -> int:
        return _check(load_library().iblbm_sync(self._h), "iblbm_sync")

    @property
    def steps_done(self) -> int:
        return load_library().iblbm_steps_done(self._h)

    @property
    def device_bytes(self) -> int:
        return load_library().iblbm_device_bytes(self._h)

    def body_forces(self, b: int = 0) -> np.ndarray:
        out = np.zeros(3)
        _check(load_library().iblbm_body_forces(self._h, b, _dp(out)), "iblbm_body_forces")
        return out

    def body_state(self, b: int = 0) -> np.ndarray:
        out = np.zeros(6)
        _check(load_library().iblbm_body_state(self._h, b, _dp(out)), "iblbm_body_state")
        return out

    def force_history(self, b: int = 0, cap: int = 65536) -> np.ndarray:
        out = np.zeros((cap, 3))
        n = C.c_int(0)
        _check(load_library().iblbm_force_history(self._h, b, _dp(out), cap, C.byref(n)),
               "iblbm_force_history")
        return out[:n.value].copy()

    def move_body(self, b: int, xy=None, uvw=None) -> None:
        pxy = None
        puvw = None
        if xy is not None:
            xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
            pxy = _dp(xy)
        if uvw is not None:
            uvw = np.ascontiguousarray(uvw, dtype=np.float64)
            puvw = _dp(uvw)
        _check(load_library().iblbm_move_body(self._h, b, pxy, puvw), "iblbm_move_body")

    def marker_data(self, b: int = 0) -> np.ndarray:
        out = np.zeros((self.body_n[b], 7))
        _check(load_library().iblbm_marker_data(self._h, b, _dp(out)), "iblbm_marker_data")
        return out

    def marker_stencils(self, b: int = 0) -> np.ndarray:
        out = np.zeros((self.body_n[b], 2), dtype=np.int32)
        _check(load_library().iblbm_marker_stencils(self._h, b, out.ctypes.data_as(C.POINTER(C.c_int))),
               "iblbm_marker_stencils")
        return out

    def mdf_info(self, b: int = 0):
        it, res, om = C.c_int(0), C.c_double(0), C.c_double(0)
        _check(load_library().iblbm_mdf_info(self._h, b, C.byref(it), C.byref(res), C.byref(om)),
               "iblbm_mdf_info")
        return it.value, res.value, om.value

    def mdf_relaxation(self, b: int = 0) -> float:
        """Relaxation in use when the last MDF iteration ended (coupled path: halved per rejection)."""
        om = C.c_double(0)
        _check(load_library().iblbm_mdf_relaxation(self._h, b, C.byref(om)), "iblbm_mdf_relaxation")
        return om.value

    def set_marker_velocity(self, b: int, ud=None) -> None:
        """Desired velocity per marker of a fixed body (``[n, 2]``), or None for the
        rigid velocity again (iblbm_set_marker_velocity)."""
        if ud is None:
            _check(load_library().iblbm_set_marker_velocity(self._h, b, None), "iblbm_set_marker_velocity")
            return
        ud = np.ascontiguousarray(ud, dtype=np.float64).reshape(-1, 2)
        if len(ud) != self.body_n[b]:
            raise ValueError("expected %d marker velocities" % self.body_n[b])
        _check(load_library().iblbm_set_marker_velocity(self._h, b, ud.ctypes.data), "iblbm_set_marker_velocity")

    def local_diagnostics(self, b: int = 0, u_ref: float = 0.1, kappa: float = 2.0, per_marker: bool = False):
        """Sec. 2.8 diagnostics of body ``b`` (iblbm_local_diagnostics): out[8] =
        slip mean, slip max, bilinear slip max, net and gross leakage, interior
        residual, interior node count, sum |F_k|; with ``per_marker`` also the
        [n, 5] table (kernel slip, bilinear slip, normal velocity, pressure
        residual, |F_k|)."""
        out = np.zeros(8)
        pm = np.zeros((self.body_n[b], 5)) if per_marker else None
        _check(load_library().iblbm_local_diagnostics(self._h, b, u_ref, kappa, _dp(out),
                                                       pm.ctypes.data if pm is not None else None),
               "iblbm_local_diagnostics")
        return (out, pm) if per_marker else out

    def populations(self, shifted: bool = False) -> np.ndarray:
        out = np.zeros((9, self.ny, self.nx))
        _check(load_library().iblbm_get_populations(self._h, _dp(out), 1 if shifted else 0),
               "iblbm_get_populations")
        return out

    def set_populations(self, f: np.ndarray) -> None:
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        _check(load_library().iblbm_set_populations(self._h, _dp(f)), "iblbm_set_populations")

    def macro(self):
        r = np.zeros((self.ny, self.nx))
        ux, uy = np.zeros_like(r), np.zeros_like(r)
        _check(load_library().iblbm_get_macro(self._h, _dp(r), _dp(ux), _dp(uy)), "iblbm_get_macro")
        return r, ux, uy

    def snapshot_bytes(self) -> int:
        """Size of a checkpoint of this lattice."""
        n = C.c_size_t(0)
        _check(load_library().iblbm_snapshot(self._h, None, 0, C.byref(n)), "iblbm_snapshot")
        return n.value

    def snapshot(self, out=None):
        """Checkpoint to host memory: a new ``bytes`` object, or written into ``out``
        (a uint8 numpy array or CPU torch tensor, e.g. pinned, of at least
        ``snapshot_bytes()`` bytes), which is then returned."""
        n = C.c_size_t(0)
        lib = load_library()
        if out is None:
            size = self.snapshot_bytes()
            buf = C.create_string_buffer(size)
            _check(lib.iblbm_snapshot(self._h, buf, size, C.byref(n)), "iblbm_snapshot")
            return buf.raw
        ptr, size = _host_buffer(out)
        _check(lib.iblbm_snapshot(self._h, C.c_void_p(ptr), size, C.byref(n)), "iblbm_snapshot")
        return out

    def restore(self, blob) -> None:
        """Restore a checkpoint from ``bytes`` or from a host buffer as accepted by
        ``snapshot(out=...)`` (read in place: a pinned buffer is copied by DMA)."""
        if isinstance(blob, (bytes, bytearray)):
            buf = C.create_string_buffer(bytes(blob), len(blob))
            _check(load_library().iblbm_restore(self._h, buf, len(blob)), "iblbm_restore")
            return
        ptr, size = _host_buffer(blob)
        _check(load_library().iblbm_restore(self._h, C.c_void_p(ptr), size), "iblbm_restore")

    def set_timing(self, enable: bool) -> None:
        _check(load_library().iblbm_set_timing(self._h, 1 if enable else 0), "iblbm_set_timing")

    def kernel_timing(self):
        ms, n = C.c_double(0), C.c_int(0)
        _check(load_library().iblbm_kernel_timing(self._h, C.byref(ms), C.byref(n)), "iblbm_kernel_timing")
        return ms.value, n.value

    def stage_timing(self):
        """{stage: (ms, launches)} for the IB stage, stream-collide, lattice edges and counters."""
        ms = (C.c_double * 4)()
        n = (C.c_int * 4)()
        _check(load_library().iblbm_stage_timing(self._h, ms, n), "iblbm_stage_timing")
        return {k: (ms[i], n[i]) for i, k in enumerate(("ib", "stream_collide", "edges", "counters"))}


def set_kernel_variant(storage: int, collision: int, variant: int) -> None:
    """Fixes the stream-collide variant (0 vector, 1 / 2 nodes per lane, 3 bulk-staged; -1 retune)."""
    _check(load_library().iblbm_set_kernel_variant(storage, collision, variant), "iblbm_set_kernel_variant")


KERNEL_VARIANTS = 4   # IBLBM_KERNEL_VARIANTS


def test_set_consumer_poll_limit(polls: int) -> None:
    """Test hook: polls after which the bulk sweep's consumers give up (negative: default)."""
    _check(load_library().iblbm_test_set_consumer_poll_limit(int(polls)), "iblbm_test_set_consumer_poll_limit")


def test_set_ib_fast(enable: bool) -> None:
    """Test hook: False sends every IB stage through the general path (default True)."""
    _check(load_library().iblbm_test_set_ib_fast(1 if enable else 0), "iblbm_test_set_ib_fast")


def kernel_variant(storage: int, collision: int):
    """(chosen variant or -1, [tuning time in ms of each variant])."""
    v = C.c_int(-1)
    ms = (C.c_double * KERNEL_VARIANTS)()
    _check(load_library().iblbm_kernel_variant(storage, collision, C.byref(v), ms), "iblbm_kernel_variant")
    return v.value, list(ms)


def step_batch(lattices: Iterable[Lattice], nsteps: int) -> None:
    """Advances every lattice by nsteps in one launch sequence per step."""
    lats = list(lattices)
    arr = (C.c_void_p * len(lats))(*[l.handle.value for l in lats])
    _check(load_library().iblbm_step_batch(arr, len(lats), nsteps), "iblbm_step_batch")


def _lattice_desc(spec, storage=None, stream=0) -> LatticeDesc:
    d = LatticeDesc()
    d.nx, d.ny = spec.nx, spec.ny
    d.storage = spec.storage if storage is None else storage
    for s in range(4):
        d.bc[s] = spec.bc[s]
        d.u_bc[s][0], d.u_bc[s][1] = spec.ubc[s]
    d.trt_lambda, d.cm_sq, d.cm_se = spec.trt_lambda, spec.cm_sq, spec.cm_se
    d.force[0], d.force[1] = spec.force
    d.init_rho = 1.0
    d.init_u[0], d.init_u[1] = spec.init_u
    d.cuda_stream = stream
    return d


class Server:
    """Continuous-batching serving loop (``iblbm_server_*``)."""

    def __init__(self, hbm_budget: int, max_slots: int = 64, stream: Optional[int] = None):
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        self._stream = stream
        h = C.c_void_p()
        _check(load_library().iblbm_server_create(int(hbm_budget), max_slots, stream, C.byref(h)),
               "iblbm_server_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().iblbm_server_destroy(self._h)
        self._h = None

    def set_graphs(self, enable: bool) -> None:
        """Ticks replay captured step graphs (True, the default) or launch step by step."""
        _check(load_library().iblbm_server_set_graphs(self._h, 1 if enable else 0), "iblbm_server_set_graphs")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, spec, nsteps: int, storage=None) -> int:
        """Queues a case described like ``Lattice.from_spec`` (at most one body)."""
        d = _lattice_desc(spec, storage, self._stream)
        rid = C.c_longlong(0)
        if spec.bodies:
            b0 = spec.bodies[0]
            b = BodyDesc()
            b.xc, b.yc, b.radius, b.rho_ratio, b.motion = b0.xc, b0.yc, b0.radius, b0.rho_ratio, b0.motion
            b.gx, b.gy, b.internal_mass = b0.gx, b0.gy, b0.internal_mass
            b.mdf_nmin, b.mdf_nmax, b.mdf_tol, b.mdf_omega = b0.mdf_nmin, b0.mdf_nmax, b0.mdf_tol, b0.mdf_omega
            b.osc_amp, b.osc_period, b.history_cap = b0.osc_amp, b0.osc_period, max(nsteps, 1)
            xy = np.ascontiguousarray(b0.xy, dtype=np.float64).reshape(-1, 2)
            rc = load_library().iblbm_server_submit(self._h, C.byref(d), spec.collision, spec.tau, C.byref(b),
                                                    _dp(xy), len(xy), b0.ds, b0.kernel, b0.scheme, nsteps,
                                                    C.byref(rid))
        else:
            rc = load_library().iblbm_server_submit(self._h, C.byref(d), spec.collision, spec.tau, None, None,
                                                    0, 0.0, 0, 0, nsteps, C.byref(rid))
        _check(rc, "iblbm_server_submit")
        return rid.value

    def tick(self, max_steps: int):
        res, que = C.c_int(0), C.c_int(0)
        done = _check(load_library().iblbm_server_tick(self._h, max_steps, C.byref(res), C.byref(que)),
                      "iblbm_server_tick")
        return done, res.value, que.value

    def poll(self, req_id: int, cap: int = 1 << 20):
        """Returns None while pending, else (force history (n, 3), latency seconds)."""
        out = np.zeros((cap, 3))
        n, lat = C.c_int(0), C.c_double(0)
        rc = load_library().iblbm_server_poll(self._h, req_id, _dp(out), cap, C.byref(n), C.byref(lat))
        if rc == 0:
            return None
        _check(rc, "iblbm_server_poll")
        return out[:n.value].copy(), lat.value

    def stats(self):
        used, res, que = C.c_size_t(0), C.c_int(0), C.c_int(0)
        _check(load_library().iblbm_server_stats(self._h, C.byref(used), C.byref(res), C.byref(que)),
               "iblbm_server_stats")
        return used.value, res.value, que.value
