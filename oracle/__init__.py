"""Python handle on the plain FP64 CPU oracle (oracle/cteno_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by the
CPU-baseline leg of bench.py. The CUDA library never imports or calls anything here.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build_oracle import LIB, build

_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # CTENO_ORACLE_LIB names another build of the oracle to load instead (the mutation tests point
    # it at deliberately altered copies to show that the pins catch them)
    alt = os.environ.get("CTENO_ORACLE_LIB")
    if alt:
        lib = C.CDLL(alt)
    else:
        build()
        lib = C.CDLL(LIB)
    V = C.c_void_p
    lib.orc_create.restype = V
    lib.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                               C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, _dp, C.c_int,
                               _ip, _dp, C.POINTER(C.c_int)]
    lib.orc_destroy.argtypes = [V]
    lib.orc_setup_all.argtypes = [V]
    lib.orc_setup_cells.argtypes = [V, C.c_int, _ip]
    lib.orc_set_state.argtypes = [V, _dp]
    lib.orc_get_state.argtypes = [V, _dp]
    lib.orc_dt.restype = C.c_double
    lib.orc_dt.argtypes = [V]
    lib.orc_stage.argtypes = [V, C.c_int, C.c_double]
    lib.orc_step.restype = C.c_double
    lib.orc_step.argtypes = [V, C.c_double]
    lib.orc_residual.argtypes = [V, _dp]
    lib.orc_residual_cells.argtypes = [V, C.c_int, _ip, _dp]
    lib.orc_reconstruct_cells.argtypes = [V, C.c_int, _ip]
    lib.orc_residual_subset.argtypes = [V, C.c_int, _ip, _dp]
    lib.orc_get_chi.argtypes = [V, _dp]
    lib.orc_select.restype = C.c_uint
    lib.orc_select.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                               _dp, _dp]
    lib.orc_info.argtypes = [V, _ip]
    lib.orc_get_geometry.argtypes = [V, V, V, V, V, V, V, V]
    lib.orc_get_face_points.argtypes = [V, V, V]
    lib.orc_get_stencil.argtypes = [V, C.c_int, _ip, _ip, _ip]
    lib.orc_get_lsq.argtypes = [V, C.c_int, _dp, _dp]
    lib.orc_lsq_apply.argtypes = [V, C.c_int, _dp, C.c_double, _dp]
    lib.orc_get_face_states.argtypes = [V, _dp]
    lib.orc_get_flags.argtypes = [V, _u8]
    lib.orc_get_si.argtypes = [V, _dp]
    lib.orc_get_stmask.argtypes = [V, _ip]
    lib.orc_get_guarded.argtypes = [V, _u8]
    lib.orc_get_coeffs.argtypes = [V, _dp]
    lib.orc_get_refmap.argtypes = [V, C.c_int, _dp, _dp]
    lib.orc_get_exponents.argtypes = [V, _ip]
    lib.orc_psibar.restype = C.c_double
    lib.orc_psibar.argtypes = [V, C.c_int]
    lib.orc_hllc.argtypes = [V, _dp, _dp, _dp, _dp]
    lib.orc_euler_flux.argtypes = [V, _dp, _dp, _dp]
    lib.orc_smoothness.restype = C.c_double
    lib.orc_smoothness.argtypes = [V, _dp, C.c_int, C.c_int]
    lib.orc_simplex_monomial.restype = C.c_double
    lib.orc_simplex_monomial.argtypes = [V, _dp, C.c_int]
    lib.orc_num_threads.restype = C.c_int
    lib.orc_eigen.argtypes = [V, _dp, _dp, _dp, _dp]
    lib.orc_boundary_region.argtypes = [V, _dp, _dp, C.c_int]
    lib.orc_boundary_states.argtypes = [V, _dp, _dp, C.c_double, C.c_double, C.c_double]
    lib.orc_set_time.argtypes = [V, C.c_double]
    lib.orc_get_time.restype = C.c_double
    lib.orc_get_time.argtypes = [V]
    _lib = lib
    return lib


def num_threads() -> int:
    return int(_load().orc_num_threads())


DEFAULTS = dict(degree=2, scheme=0, lam_gamma=1, ctenoz_form=0, characteristic=0, boundary=0, rk=3, C_T=1e-6,
                lambda1p=1e15, eps=1e-24, gamma=1.4, cfl=0.5, guard=1)


def select(SI, scheme=0, ctenoz_form=0, lam_gamma=1, C_T=1e-6, lambda1p=1e15, eps=1e-24):
    """The oracle's selection (eqs. 19-23, Alg. 1 / 2) of one cell and variable from its smoothness
    indicators SI[0] (central) .. SI[s_t - 1] (admissible directional stencils): (delta bits, chi)."""
    SI = np.ascontiguousarray(SI, np.float64)
    chi = np.empty(SI.size)
    bits = _load().orc_select(scheme, ctenoz_form, lam_gamma, C_T, lambda1p, eps, SI.size, SI, chi)
    return int(bits), chi


class Oracle:
    """One mesh, one scheme configuration, FP64 state on the host."""

    def __init__(self, mesh, setup: bool = True, **params):
        p = dict(DEFAULTS)
        p.update(params)
        self.p = p
        self.lib = _load()
        self.dim = mesh.dim
        self.mesh = mesh
        xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
        cells = np.ascontiguousarray(mesh.cells, dtype=np.int32)
        period = np.ascontiguousarray(mesh.period, dtype=np.float64)
        err = C.c_int(0)
        self.h = self.lib.orc_create(self.dim, p["degree"], p["scheme"], p["lam_gamma"], p["ctenoz_form"],
                                     p["characteristic"], p["boundary"], p["rk"], p["C_T"], p["lambda1p"], p["eps"],
                                     p["gamma"], p["cfl"],
                                     p["guard"],
                                     mesh.nverts, xyz, mesh.ncells, cells, period, C.byref(err))
        if err.value:
            raise RuntimeError(f"oracle mesh set-up failed ({err.value})")
        info = np.zeros(8, np.int32)
        self.lib.orc_info(self.h, info)
        self.nv, self.nf, self.nq, self.nk, self.M = (int(x) for x in info[:5])
        self.dmax = int(info[7])   # members kept per directional stencil
        self.ncells = mesh.ncells
        # selections per cell: one per variable, or per face and characteristic field
        self.sel_shape = (self.nf, self.nv) if p["characteristic"] else (self.nv,)
        if setup:
            rc = self.lib.orc_setup_all(self.h)
            if rc:
                raise RuntimeError(f"oracle stencil/least-squares set-up failed ({rc})")

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    # state -------------------------------------------------------------------------------
    def set_state(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == (self.nv, self.ncells)
        self.lib.orc_set_state(self.h, U)

    def get_state(self):
        out = np.empty((self.nv, self.ncells))
        self.lib.orc_get_state(self.h, out)
        return out

    def dt(self) -> float:
        return float(self.lib.orc_dt(self.h))

    def stage(self, s: int, dt: float):
        self.lib.orc_stage(self.h, s, dt)

    def step(self, dt: float = 0.0) -> float:
        return float(self.lib.orc_step(self.h, dt))

    def run(self, nsteps: int, dt: float = 0.0):
        dts = [self.step(dt) for _ in range(nsteps)]
        return np.array(dts)

    def residual(self):
        out = np.empty((self.nv, self.ncells))
        self.lib.orc_residual(self.h, out)
        return out

    def residual_cells(self, ids):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        out = np.empty((ids.size, self.nv))
        rc = self.lib.orc_residual_cells(self.h, ids.size, ids, out)
        if rc:
            raise RuntimeError(f"oracle set-up failed ({rc})")
        return out

    def residual_subset(self, ids):
        """Residual of the (set-up) cells `ids`, reconstructing them and their face neighbours
        once each: [len(ids), nv]."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        out = np.empty((ids.size, self.nv))
        rc = self.lib.orc_residual_subset(self.h, ids.size, ids, out)
        if rc:
            raise RuntimeError(f"oracle subset residual failed ({rc}): cells not set up")
        return out

    def reconstruct_cells(self, ids):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        rc = self.lib.orc_reconstruct_cells(self.h, ids.size, ids)
        if rc:
            raise RuntimeError(f"oracle set-up failed ({rc})")

    def setup_cells(self, ids):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        rc = self.lib.orc_setup_cells(self.h, ids.size, ids)
        if rc:
            raise RuntimeError(f"oracle set-up failed ({rc})")

    # debug accessors -----------------------------------------------------------------------
    def geometry(self):
        n, d, nf = self.ncells, self.dim, self.nf
        g = dict(vol=np.empty(n), cen=np.empty((n, d)), cells=np.empty((n, d + 1), np.int32),
                 area=np.empty((n, nf)), normal=np.empty((n, nf, d)),
                 nbr=np.empty((n, nf), np.int32), nbr_face=np.empty((n, nf), np.int32))
        ptr = lambda a: a.ctypes.data_as(C.c_void_p)
        self.lib.orc_get_geometry(self.h, ptr(g["vol"]), ptr(g["cen"]), ptr(g["cells"]),
                                  ptr(g["area"]), ptr(g["normal"]), ptr(g["nbr"]),
                                  ptr(g["nbr_face"]))
        return g

    def face_points(self):
        fq = np.empty((self.ncells, self.nf, self.nq, self.dim))
        fw = np.empty(self.nq)
        self.lib.orc_get_face_points(self.h, fq.ctypes.data_as(C.c_void_p),
                                     fw.ctypes.data_as(C.c_void_p))
        return fq, fw

    def stencil(self, i: int):
        d = self.dim
        central = np.empty(self.M, np.int32)
        dirm = np.empty((self.nf, self.dmax), np.int32)
        dok = np.empty(self.nf, np.int32)
        self.lib.orc_get_stencil(self.h, int(i), central, dirm, dok)
        return central, dirm, dok

    def lsq(self, i: int):
        A = np.empty((self.M, self.nk))
        Vp = np.empty(self.M)
        self.lib.orc_get_lsq(self.h, int(i), A, Vp)
        return A, Vp

    def lsq_apply(self, i: int, Um, U0: float):
        a = np.empty(self.nk)
        self.lib.orc_lsq_apply(self.h, int(i), np.ascontiguousarray(Um, np.float64), float(U0), a)
        return a

    def face_states(self):
        out = np.empty((self.ncells, self.nf, self.nq, self.nv))
        self.lib.orc_get_face_states(self.h, out)
        return out

    def flags(self):
        """Selection flags of the last reconstruction: [ncells, nv], or [ncells, nf, nv] (face,
        characteristic field) for the characteristic reconstruction."""
        out = np.empty((self.ncells,) + self.sel_shape, np.uint8)
        self.lib.orc_get_flags(self.h, out)
        return out

    def smoothness_indicators(self):
        out = np.empty((self.ncells,) + self.sel_shape + (1 + self.nf,))
        self.lib.orc_get_si(self.h, out)
        return out

    def chi(self):
        """chi_s of eq. 22 of the last reconstruction: [ncells, nv, 1 + nf] (central, then the
        directional stencil of each local face; 0 where not admissible); [ncells, nf, nv, 1 + nf]
        for the characteristic reconstruction."""
        out = np.empty((self.ncells,) + self.sel_shape + (1 + self.nf,))
        self.lib.orc_get_chi(self.h, out)
        return out

    def coefficients(self):
        out = np.empty((self.ncells,) + self.sel_shape + (self.nk,))
        self.lib.orc_get_coeffs(self.h, out)
        return out

    # boundary kinds (oracle readings): 0 transmissive, 1 wall, 2 fixed state A, 3 moving shock
    # (state A where xs0 + sy y + vs t exceeds the face midpoint's x, else B)
    def boundary_region(self, lo, hi, kind: int):
        """Every boundary face whose midpoint lies in the box [lo, hi] gets `kind`."""
        self.lib.orc_boundary_region(self.h, np.ascontiguousarray(lo, np.float64),
                                     np.ascontiguousarray(hi, np.float64), int(kind))

    def boundary_states(self, A, B, xs0=0.0, sy=0.0, vs=0.0):
        self.lib.orc_boundary_states(self.h, np.ascontiguousarray(A, np.float64),
                                     np.ascontiguousarray(B, np.float64), xs0, sy, vs)

    def set_time(self, t: float):
        self.lib.orc_set_time(self.h, float(t))

    def time(self) -> float:
        return float(self.lib.orc_get_time(self.h))

    def eigen(self, u, n):
        """(R, L): right and left eigenvectors of the Euler flux Jacobian in unit direction n at
        the conserved state u, as the characteristic reconstruction uses them."""
        u = np.ascontiguousarray(u, np.float64)
        n = np.ascontiguousarray(n, np.float64)
        R = np.empty((self.nv, self.nv))
        L = np.empty((self.nv, self.nv))
        self.lib.orc_eigen(self.h, u, n, R, L)
        return R, L

    def refmap(self, i: int):
        X = np.empty((self.dim + 1, self.dim))
        Ji = np.empty((self.dim, self.dim))
        self.lib.orc_get_refmap(self.h, int(i), X, Ji)
        return X, Ji

    def stencil_mask(self):
        out = np.empty(self.ncells, np.int32)
        self.lib.orc_get_stmask(self.h, out)
        return out

    def exponents(self):
        ex = np.empty((self.nk, 3), np.int32)
        self.lib.orc_get_exponents(self.h, ex)
        return ex[:, : self.dim]

    def psibar(self):
        return np.array([self.lib.orc_psibar(self.h, k) for k in range(self.nk)])

    def guarded(self):
        """Cells whose last reconstruction fell back to the cell mean (positivity guard)."""
        out = np.empty(self.ncells, np.uint8)
        self.lib.orc_get_guarded(self.h, out)
        return out.astype(bool)

    def nguard(self) -> int:
        info = np.zeros(8, np.int32)
        self.lib.orc_info(self.h, info)
        return int(info[6])

    def hllc(self, uL, uR, n):
        F = np.empty(self.nv)
        self.lib.orc_hllc(self.h, np.ascontiguousarray(uL, np.float64),
                          np.ascontiguousarray(uR, np.float64), np.ascontiguousarray(n, np.float64), F)
        return F

    def euler_flux(self, u, n):
        F = np.empty(self.nv)
        self.lib.orc_euler_flux(self.h, np.ascontiguousarray(u, np.float64),
                                np.ascontiguousarray(n, np.float64), F)
        return F

    def smoothness(self, a, deg: int):
        a = np.ascontiguousarray(a, np.float64)
        return float(self.lib.orc_smoothness(self.h, a, a.size, deg))

    def simplex_monomial(self, xi, k: int):
        return float(self.lib.orc_simplex_monomial(self.h, np.ascontiguousarray(xi, np.float64), k))
