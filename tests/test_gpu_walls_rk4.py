"""Reflective walls, the classical RK4 step and the triple-point workload on the GPU, through the
C ABI, against the oracle (same readings: a wall's outside state is the mirror image of the
reconstructed inside state; RK4 accumulates U^n + dt/6 (k1 + 2 k2 + 2 k3 + k4) stage by stage).

Tolerances: FP64 1e-12 of each component's scale (at degree 4, max(1e-12, 50 cond(A) u) as for
the other high-degree tests); mixed path 1e-5; mass and energy in a closed box constant to 1e-13
(FP64) and 1e-8 (mixed: FP32 wall fluxes).
"""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

WALL = 1
U_EPS = np.finfo(float).eps / 2


def _native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_17042_gb300 import build, native
    build.build()
    return native


def _solver(native, meshes, dim, **kw):
    import torch
    return native.Solver(meshes, dim, stream=torch.cuda.current_stream().cuda_stream, **kw)


def _relerr(a, b):
    scale = np.maximum(np.abs(b).max(axis=-1, keepdims=True), 1e-300)
    return float((np.abs(a - b) / scale).max())


def _uniform(mesh, rho, vel, p):
    prim = np.zeros((mesh.ncells, mesh.dim + 2))
    prim[:, 0] = rho
    prim[:, 1:1 + mesh.dim] = vel
    prim[:, -1] = p
    return W.primitive_to_conserved(prim).T.copy()


@pytest.mark.parametrize("degree", [2, 3])
def test_flow_into_a_wall_fp64_matches_oracle(degree):
    native = _native()
    from oracle import Oracle
    mesh = W.tri_mesh(100, 5, lx=2.0, ly=0.1, periodic=False)
    U = _uniform(mesh, 1.0, [0.5, 0.0], 1.0)
    o = Oracle(mesh, degree=degree, boundary=WALL, cfl=0.4)
    o.set_state(U)
    dts = o.run(10)
    s = _solver(native, [mesh], 2, degree=degree, boundary=WALL, cfl=0.4)
    s.set_state(U)
    s.run(10)
    err = _relerr(s.get_state(), o.get_state())
    print(f"wall channel, degree {degree}: max rel {err:.2e}")
    assert err < 1e-12
    assert abs(s.dt()[0] - dts[-1]) < 1e-13 * dts[-1]
    s.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("rk", [3, 4])
def test_closed_box_3d_conserves_mass_and_energy(rk, precision):
    native = _native()
    from oracle import Oracle
    mesh = W.tet_mesh(6, periodic=False)
    U = _uniform(mesh, 1.0 + 0.5 * W.cell_centroids(mesh)[:, 0], [0.6, -0.3, 0.2], 1.0)
    vol = W.cell_volumes(mesh)
    s = _solver(native, [mesh], 3, degree=2, boundary=WALL, rk=rk, cfl=0.4, precision=precision)
    s.set_state(U)
    s.run(6)
    Un = s.get_state()
    # FP64: the mass and energy fluxes through a wall vanish to rounding; the mixed path computes
    # HLLC in FP32, where the contact speed of a state against its mirror image is zero only to
    # FP32 rounding (measured: 2.5e-10 of the mass after 6 steps)
    tol = 1e-13 if precision == 0 else 1e-8
    for v in (0, 4):
        rel = abs((vol * Un[v]).sum() - (vol * U[v]).sum()) / (vol * U[v]).sum()
        assert rel < tol, (v, rel)
    if precision == 0:
        o = Oracle(mesh, degree=2, boundary=WALL, rk=rk, cfl=0.4)
        o.set_state(U)
        o.run(6)
        assert _relerr(Un, o.get_state()) < 1e-12
    s.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_rk4_matches_oracle_and_stage_calls(precision):
    """Density wave, CTENO degree 3, 10 RK4 steps: FP64 within 1e-12 of the oracle (the mixed path
    within 1e-5); four cteno_rk_stage calls (CFL step at stage 0) equal one cteno_run step bit for
    bit."""
    native = _native()
    from oracle import Oracle
    wl = W.density_wave_2d(24)
    o = Oracle(wl.mesh, degree=3, rk=4, cfl=0.5)
    o.set_state(wl.U0)
    dts = o.run(10)
    s = _solver(native, [wl.mesh], 2, degree=3, rk=4, cfl=0.5, precision=precision)
    s.set_state(wl.U0)
    s.run(10)
    U10 = s.get_state()
    err = _relerr(U10, o.get_state())
    print(f"RK4 wave, precision {precision}: max rel {err:.2e}")
    assert err < (1e-12 if precision == 0 else 1e-5)
    if precision == 0:
        assert abs(s.dt()[0] - dts[-1]) < 1e-13 * dts[-1]
    s.run(1)
    U11 = s.get_state()
    s.set_state(U10)
    for st in range(4):
        s.stage(st)            # dt = NULL: the CFL step of the state at stage 0
    assert np.array_equal(s.get_state(), U11)
    with pytest.raises(native.CtenoError):
        s.stage(4)
    s.close()


@pytest.mark.parametrize("degree,scheme", [(2, 0), (4, 1), (4, 2)], ids=["CTENO3", "CTENOZ5", "CWENO5"])
def test_triple_point_reduced_matches_oracle(degree, scheme):
    """The triple-point workload's construction at 70 x 30 squares (4200 triangles), walls all round,
    lambda_1' = 1e4 as in Sec. 3.4, 5 FP64 steps."""
    native = _native()
    from oracle import Oracle
    wl = W.triple_point_2d(70, 30)
    o = Oracle(wl.mesh, degree=degree, scheme=scheme, lambda1p=1e4, boundary=WALL, cfl=0.4)
    tol = 1e-12
    if degree >= 4:
        tol = max(tol, 50 * max(np.linalg.cond(o.lsq(i)[0]) for i in range(wl.mesh.ncells)) * U_EPS)
    o.set_state(wl.U0)
    o.run(5)
    s = _solver(native, [wl.mesh], 2, degree=degree, scheme=scheme, lambda1p=1e4, boundary=WALL, cfl=0.4)
    s.set_state(wl.U0)
    s.run(5)
    err = _relerr(s.get_state(), o.get_state())
    print(f"triple point 70x30, degree {degree}, scheme {scheme}: max rel {err:.2e} (tol {tol:.1e})")
    assert err < 10 * tol
    s.close()


@pytest.mark.parametrize("degree,lam", [(2, 1e15), (4, 1e15)], ids=["CTENO3", "CTENO5"])
def test_double_mach_reflection_reduced_matches_oracle(degree, lam):
    """The double Mach reflection's construction (Sec. 3.3) at 48 x 12 squares (1152 triangles):
    inflow, wall, moving-shock and transmissive boundary faces, 10 FP64 steps against the oracle;
    the library's physical time equals the sum of the steps."""
    native = _native()
    from oracle import Oracle
    wl = W.dmr_2d(12)
    regions, states = W.dmr_boundary()
    o = Oracle(wl.mesh, degree=degree, scheme=0, lambda1p=lam, cfl=0.4)
    for lo, hi, kind in regions:
        o.boundary_region(lo, hi, kind)
    o.boundary_states(*states)
    tol = 1e-12
    if degree >= 4:
        tol = max(tol, 50 * max(np.linalg.cond(o.lsq(i)[0]) for i in range(wl.mesh.ncells)) * U_EPS)
    o.set_state(wl.U0)
    dts = o.run(10)
    s = _solver(native, [wl.mesh], 2, degree=degree, scheme=0, lambda1p=lam, cfl=0.4, regions=regions,
                states=states)
    s.set_state(wl.U0)
    s.run(10)
    err = _relerr(s.get_state(), o.get_state())
    t = native.cteno_get_time(s.ctx)[0]
    print(f"DMR 48x12, degree {degree}: max rel {err:.2e} (tol {tol:.1e}), t = {t:.6f}")
    assert err < 10 * tol
    assert abs(t - dts.sum()) < 1e-14 and abs(o.time() - dts.sum()) < 1e-14
    s.close()
