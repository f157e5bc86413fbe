"""ctypes binding of include/cteno.h: one Python function per C entry point, same names, plus a
small ``Solver`` convenience class. Arguments are marshalled (numpy arrays for host memory,
integer addresses for device memory); every step of the computation runs in libcteno.so."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

CTENO_SCHEME_CTENO, CTENO_SCHEME_CTENOZ, CTENO_SCHEME_CWENO, CTENO_SCHEME_TENO = 0, 1, 2, 3
CTENO_FP64, CTENO_MIXED = 0, 1
CTENO_BOUNDARY_TRANSMISSIVE = 0
CTENO_BOUNDARY_WALL = 1
CTENO_BOUNDARY_STATE_A = 2
CTENO_BOUNDARY_SHOCK_AB = 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libcteno.so")
_lib = None


class CtenoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cteno error {code}: {msg}")
        self.code = code


class cteno_params(C.Structure):
    _fields_ = [("dim", C.c_int), ("degree", C.c_int), ("scheme", C.c_int), ("precision", C.c_int),
                ("lam_gamma", C.c_int), ("positivity_guard", C.c_int), ("ctenoz_form", C.c_int),
                ("characteristic", C.c_int), ("rk", C.c_int), ("C_T", C.c_double),
                ("lambda1p", C.c_double), ("eps", C.c_double), ("cfl", C.c_double),
                ("gamma", C.c_double)]


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libcteno.so (built in-tree). Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                           "`python -m paper_2312_17042_gb300.build` (nvcc, sm_103a)")
    lib = C.CDLL(_LIB_PATH)
    P, I, I64, D, V = C.POINTER, C.c_int, C.c_int64, C.c_double, C.c_void_p
    sig = {
        "cteno_default_params": (None, [P(cteno_params)]),
        "cteno_create": (I, [P(V), P(cteno_params), V]),
        "cteno_mesh_build": (I, [V, I64, V, I64, V, V, I, P(C.c_int32)]),
        "cteno_stencil_build": (I, [V]),
        "cteno_lsq_build": (I, [V]),
        "cteno_set_state": (I, [V, C.c_int32, V, I]),
        "cteno_rk_stage": (I, [V, I, V]),
        "cteno_run": (I, [V, I]),
        "cteno_get_state": (I, [V, C.c_int32, V, I]),
        "cteno_get_state_noalloc": (I, [V, C.c_int32, V]),
        "cteno_set_state_all": (I, [V, V, I]),
        "cteno_get_state_all": (I, [V, V, I]),
        "cteno_get_dt": (I, [V, V]),
        "cteno_record_flags": (I, [V, I]),
        "cteno_get_flags": (I, [V, C.c_int32, V]),
        "cteno_get_face_states": (I, [V, C.c_int32, V]),
        "cteno_get_stencil": (I, [V, C.c_int32, I64, V, V, V]),
        "cteno_info": (I, [V, C.c_int32, V]),
        "cteno_boundary_region": (I, [V, C.c_int32, V, V, I]),
        "cteno_boundary_states": (I, [V, V, V, D, D, D]),
        "cteno_set_time": (I, [V, D]),
        "cteno_get_time": (I, [V, V]),
        "cteno_sync": (I, [V, P(I64)]),
        "cteno_set_launch": (I, [V, I, I]),
        "cteno_autotune": (I, [V, V]),
        "cteno_kernel_stats": (I, [V, V]),
        "cteno_profile_step": (I, [V, I, V]),
        "cteno_set_timing": (I, [V, I]),
        "cteno_last_kernel_ms": (I, [V, V]),
        "cteno_measure_alu_peak": (I, [P(D), P(D)]),
        "cteno_test_wait_timeout": (I, [V, I64]),
        "cteno_last_error": (C.c_char_p, [V]),
        "cteno_destroy": (None, [V]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def _check(ctx, rc):
    if rc != 0:
        msg = load_library().cteno_last_error(ctx)
        raise CtenoError(rc, msg.decode() if msg else "")


# ---- thin wrappers with the C names ------------------------------------------------------------
def cteno_default_params() -> cteno_params:
    p = cteno_params()
    load_library().cteno_default_params(C.byref(p))
    return p


def cteno_create(params: cteno_params, stream: int = 0):
    h = C.c_void_p()
    rc = load_library().cteno_create(C.byref(h), C.byref(params), C.c_void_p(stream or None))
    _check(None, rc)
    return h


def cteno_mesh_build(ctx, xyz: np.ndarray, cells: np.ndarray, period=None, boundary: int = 0) -> int:
    xyz = np.ascontiguousarray(xyz, np.float64)
    cells = np.ascontiguousarray(cells, np.int32)
    per = None if period is None else np.ascontiguousarray(period, np.float64)
    mid = C.c_int32(-1)
    rc = load_library().cteno_mesh_build(ctx, xyz.shape[0], _ptr(xyz), cells.shape[0], _ptr(cells),
                                         None if per is None else _ptr(per),
                                         int(boundary), C.byref(mid))
    _check(ctx, rc)
    return mid.value


def cteno_stencil_build(ctx):
    _check(ctx, load_library().cteno_stencil_build(ctx))


def cteno_lsq_build(ctx):
    _check(ctx, load_library().cteno_lsq_build(ctx))


def cteno_set_state(ctx, mesh_id: int, U, is_device: bool = False):
    """U: numpy [nv, ncells] float64 (host) or, with is_device, a device address (int)."""
    if is_device:
        _check(ctx, load_library().cteno_set_state(ctx, mesh_id, C.c_void_p(U), 1))
    else:
        U = np.ascontiguousarray(U, np.float64)
        _check(ctx, load_library().cteno_set_state(ctx, mesh_id, _ptr(U), 0))


def cteno_rk_stage(ctx, stage: int, dt=None):
    """dt: the time step of each mesh, or None for the CFL step of the current state (stage 0)."""
    if dt is None:
        _check(ctx, load_library().cteno_rk_stage(ctx, stage, None))
        return
    dt = np.ascontiguousarray(np.atleast_1d(dt), np.float64)
    _check(ctx, load_library().cteno_rk_stage(ctx, stage, _ptr(dt)))


def cteno_run(ctx, nsteps: int):
    _check(ctx, load_library().cteno_run(ctx, nsteps))


def cteno_get_state(ctx, mesh_id: int, out=None, is_device: bool = False):
    if is_device:
        _check(ctx, load_library().cteno_get_state(ctx, mesh_id, C.c_void_p(out), 1))
        return out
    info = cteno_info(ctx, mesh_id)
    if out is None:
        out = np.empty((info[4], info[7]))
    _check(ctx, load_library().cteno_get_state(ctx, mesh_id, _ptr(out), 0))
    return out


def cteno_set_state_all(ctx, U, is_device: bool = False):
    """All meshes at once. U: a flat float64 array holding mesh after mesh, each block
    [nv, ncells] (or a list of those blocks), or with is_device a device address (int)."""
    if is_device:
        _check(ctx, load_library().cteno_set_state_all(ctx, C.c_void_p(U), 1))
        return
    if isinstance(U, (list, tuple)):
        U = np.concatenate([np.ascontiguousarray(u, np.float64).ravel() for u in U])
    U = np.ascontiguousarray(U, np.float64)
    _check(ctx, load_library().cteno_set_state_all(ctx, _ptr(U), 0))


def cteno_get_state_all(ctx, out=None, is_device: bool = False):
    """All meshes at once into a flat float64 array (mesh after mesh, [nv, ncells] blocks)."""
    if is_device:
        _check(ctx, load_library().cteno_get_state_all(ctx, C.c_void_p(out), 1))
        return out
    if out is None:
        info = cteno_info(ctx, -1)
        out = np.empty(int(info[4]) * int(info[1]))
    _check(ctx, load_library().cteno_get_state_all(ctx, _ptr(out), 0))
    return out


def cteno_get_state_noalloc(ctx, mesh_id: int, out=None):
    """Host read-back through the library's fixed staging array (no device allocation)."""
    info = cteno_info(ctx, mesh_id)
    if out is None:
        out = np.empty((info[4], info[7]))
    _check(ctx, load_library().cteno_get_state_noalloc(ctx, mesh_id, _ptr(out)))
    return out


def cteno_get_dt(ctx) -> np.ndarray:
    out = np.empty(cteno_info(ctx, -1)[0])
    _check(ctx, load_library().cteno_get_dt(ctx, _ptr(out)))
    return out


def cteno_record_flags(ctx, enable: bool = True):
    _check(ctx, load_library().cteno_record_flags(ctx, int(enable)))


def cteno_get_flags(ctx, mesh_id: int) -> np.ndarray:
    """[ncells, nv] flags, or [ncells, (d+1) nv] (face-major) with the characteristic
    reconstruction."""
    info = cteno_info(ctx, mesh_id)
    out = np.empty((info[7], info[9]), np.uint8)
    _check(ctx, load_library().cteno_get_flags(ctx, mesh_id, _ptr(out)))
    return out


def cteno_get_face_states(ctx, mesh_id: int) -> np.ndarray:
    info = cteno_info(ctx, mesh_id)
    out = np.empty((info[7], info[5], info[6], info[4]))
    _check(ctx, load_library().cteno_get_face_states(ctx, mesh_id, _ptr(out)))
    return out


def cteno_get_stencil(ctx, mesh_id: int, cell: int, with_admissibility: bool = True):
    info = cteno_info(ctx, mesh_id)
    M, nf = int(info[2]), int(info[5])
    d = nf - 1
    central = np.empty(M, np.int32)
    dirm = np.empty((nf, int(info[8])), np.int32)
    dok = np.empty(nf, np.int32) if with_admissibility else None
    _check(ctx, load_library().cteno_get_stencil(ctx, mesh_id, int(cell), _ptr(central), _ptr(dirm),
                                                 _ptr(dok) if dok is not None else None))
    return central, dirm, dok


def cteno_boundary_region(ctx, mesh_id: int, lo, hi, kind: int):
    lo = np.ascontiguousarray(lo, np.float64)
    hi = np.ascontiguousarray(hi, np.float64)
    _check(ctx, load_library().cteno_boundary_region(ctx, mesh_id, _ptr(lo), _ptr(hi), int(kind)))


def cteno_boundary_states(ctx, A, B, xs0: float = 0.0, sy: float = 0.0, vs: float = 0.0):
    A = np.ascontiguousarray(A, np.float64)
    B = np.ascontiguousarray(B, np.float64)
    _check(ctx, load_library().cteno_boundary_states(ctx, _ptr(A), _ptr(B), float(xs0), float(sy), float(vs)))


def cteno_set_time(ctx, t: float):
    _check(ctx, load_library().cteno_set_time(ctx, float(t)))


def cteno_get_time(ctx) -> np.ndarray:
    out = np.empty(cteno_info(ctx, -1)[0])
    _check(ctx, load_library().cteno_get_time(ctx, _ptr(out)))
    return out


def cteno_info(ctx, mesh_id: int = -1) -> np.ndarray:
    out = np.zeros(10, np.int64)
    _check(ctx, load_library().cteno_info(ctx, mesh_id, _ptr(out)))
    return out


def cteno_sync(ctx) -> int:
    g = C.c_int64(0)
    _check(ctx, load_library().cteno_sync(ctx, C.byref(g)))
    return g.value


def cteno_set_launch(ctx, recon_block: int = 0, flux_block: int = 0):
    _check(ctx, load_library().cteno_set_launch(ctx, recon_block, flux_block))


def cteno_autotune(ctx):
    best = np.zeros(2, np.int32)
    _check(ctx, load_library().cteno_autotune(ctx, _ptr(best)))
    return tuple(int(x) for x in best)


def cteno_kernel_stats(ctx) -> np.ndarray:
    out = np.zeros(4)
    _check(ctx, load_library().cteno_kernel_stats(ctx, _ptr(out)))
    return out


def cteno_profile_step(ctx, nsteps: int) -> np.ndarray:
    out = np.zeros(2)
    _check(ctx, load_library().cteno_profile_step(ctx, nsteps, _ptr(out)))
    return out


def cteno_set_timing(ctx, enable: bool = True):
    _check(ctx, load_library().cteno_set_timing(ctx, int(enable)))


def cteno_last_kernel_ms(ctx) -> np.ndarray:
    out = np.zeros(2)
    _check(ctx, load_library().cteno_last_kernel_ms(ctx, _ptr(out)))
    return out


def cteno_measure_alu_peak():
    """(fp64_tflops, fp32_tflops) of the current device."""
    a, b = C.c_double(0), C.c_double(0)
    _check(None, load_library().cteno_measure_alu_peak(C.byref(a), C.byref(b)))
    return a.value, b.value


def cteno_test_wait_timeout(ctx, limit_ns: int):
    _check(ctx, load_library().cteno_test_wait_timeout(ctx, int(limit_ns)))


def cteno_last_error(ctx) -> str:
    m = load_library().cteno_last_error(ctx)
    return m.decode() if m else ""


def cteno_destroy(ctx):
    load_library().cteno_destroy(ctx)


# ---- convenience ---------------------------------------------------------------------------------
class Solver:
    """One context holding one or more meshes of the same dimension.

    ``meshes`` are objects with ``xyz``, ``cells`` and ``period`` attributes (see workloads.Mesh).
    ``stream`` is a CUDA stream handle (e.g. torch.cuda.current_stream().cuda_stream); 0 uses the
    legacy default stream.
    """

    def __init__(self, meshes, dim: int, degree: int = 2, scheme: int = 0, precision: int = 0,
                 stream: int = 0, build: bool = True, boundary: int = 0, regions=None, states=None, **kw):
        p = cteno_default_params()
        p.dim, p.degree, p.scheme, p.precision = dim, degree, scheme, precision
        for k, v in kw.items():
            setattr(p, k, v)
        self.params = p
        self.ctx = cteno_create(p, stream)
        self.mesh_ids = [cteno_mesh_build(self.ctx, m.xyz, m.cells, m.period, boundary) for m in meshes]
        # boundary regions and states (e.g. workloads.dmr_boundary()): applied to every mesh
        for lo, hi, kind in (regions or ()):
            for mid in self.mesh_ids:
                cteno_boundary_region(self.ctx, mid, lo, hi, kind)
        if states is not None:
            cteno_boundary_states(self.ctx, *states)
        if build:
            cteno_stencil_build(self.ctx)
            cteno_lsq_build(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            cteno_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, U, mesh_id: int = 0):
        cteno_set_state(self.ctx, mesh_id, U)

    def get_state(self, mesh_id: int = 0):
        return cteno_get_state(self.ctx, mesh_id)

    def stage(self, s: int, dt=None):
        cteno_rk_stage(self.ctx, s, dt)

    def step(self, dt=None):
        for s in range(self.params.rk):
            cteno_rk_stage(self.ctx, s, dt)

    def run(self, nsteps: int):
        cteno_run(self.ctx, nsteps)

    def dt(self):
        return cteno_get_dt(self.ctx)

    def sync(self) -> int:
        return cteno_sync(self.ctx)
