"""Pins of the oracle's reflective walls (Sec. 3.3 / 3.4 use walls; reading in residual_cell) and
of its classical fourth-order Runge-Kutta step (Sec. 2: "3rd- or 4th-order" explicit RK).

  * Walls close the box: with every boundary face a wall, mass and energy stay constant to
    rounding while the flow runs into them (transmissive boundaries let mass out).
  * A uniform flow into a wall: the reflected shock leaves the fluid at rest behind it with the
    density and pressure of the exact Riemann solution of the state against its mirror image.
  * RK4 is fourth order in time: successive differences fall by 2^4 (RK3's by 2^3); a uniform
    flow (zero residual) passes through its stages unchanged.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from tests import exact as X


def _uniform(mesh, rho, vel, p):
    prim = np.zeros((mesh.ncells, mesh.dim + 2))
    prim[:, 0] = rho
    prim[:, 1:1 + mesh.dim] = vel
    prim[:, -1] = p
    return W.primitive_to_conserved(prim).T.copy()


def _primitive(U, g=1.4):
    """(rho, velocity, p) per cell from conserved U [nv, ncells]."""
    rho = U[0]
    vel = U[1:-1] / rho
    p = (g - 1.0) * (U[-1] - 0.5 * rho * (vel ** 2).sum(axis=0))
    return np.vstack([rho, vel, p]).T


@pytest.mark.parametrize("rk", [3, 4])
@pytest.mark.parametrize("dim", [2, 3])
def test_walls_conserve_mass_and_energy(dim, rk):
    mesh = W.tri_mesh(16, 16, periodic=False) if dim == 2 else W.tet_mesh(4, periodic=False)
    vel = [0.6, -0.3] if dim == 2 else [0.6, -0.3, 0.2]
    U = _uniform(mesh, 1.0 + 0.5 * W.cell_centroids(mesh)[:, 0], vel, 1.0)   # denser towards x = 1
    vol = W.cell_volumes(mesh)
    for boundary in (1, 0):
        o = Oracle(mesh, degree=2, boundary=boundary, rk=rk, cfl=0.4)
        o.set_state(U)
        o.run(5)
        Un = o.get_state()
        dm = abs((vol * Un[0]).sum() - (vol * U[0]).sum()) / (vol * U[0]).sum()
        de = abs((vol * Un[-1]).sum() - (vol * U[-1]).sum()) / (vol * U[-1]).sum()
        if boundary == 1:
            assert dm < 1e-14 and de < 1e-14, (dm, de)
        else:
            assert dm > 1e-3


def test_flow_into_a_wall_against_the_exact_reflection():
    """rho = 1, u = 0.5, p = 1 towards the wall at x = 2 of the channel [0,2] x [0,0.1] (walls all
    round): the star state of the Riemann problem (rho, u, p) | (rho, -u, p) is at rest; behind the
    reflected shock the scheme reaches its density and pressure, ahead of it (and behind the
    rarefaction leaving the wall at x = 0) the flow is untouched."""
    mesh = W.tri_mesh(100, 5, lx=2.0, ly=0.1, periodic=False)
    U = _uniform(mesh, 1.0, [0.5, 0.0], 1.0)
    o = Oracle(mesh, degree=2, boundary=1, cfl=0.4)
    o.set_state(U)
    t, T = 0.0, 0.2
    while t < T - 1e-14:
        dt = min(o.dt(), T - t)
        o.step(dt)
        t += dt
    Uf = o.get_state()
    star = X.riemann_exact((1.0, 0.5, 1.0), (1.0, -0.5, 1.0), np.array([0.0]))[0]   # (rho, u, p)
    rho_s, p_s = star[0], star[2]
    assert abs(star[1]) < 1e-12
    # shock speed from the mass balance: S = -rho u / (rho_s - rho)
    S = -0.5 / (rho_s - 1.0)
    cen = W.cell_centroids(mesh)
    x_shock = 2.0 + S * T
    behind = cen[:, 0] > x_shock + 0.06
    ahead = (cen[:, 0] < x_shock - 0.08) & (cen[:, 0] > 1.68 * T + 0.1)   # right of the rarefaction
    assert behind.sum() >= 20 and ahead.sum() >= 200
    prim = _primitive(Uf)
    assert np.abs(prim[behind, 0] - rho_s).max() < 0.02 * rho_s
    assert np.abs(prim[behind, 3] - p_s).max() < 0.02 * p_s
    assert np.abs(prim[behind, 1]).max() < 0.02
    assert np.abs(prim[ahead, 0] - 1.0).max() < 5e-3   # the smeared feet of the two waves


@pytest.mark.parametrize("rk,order", [(3, 3), (4, 4)])
def test_runge_kutta_order_in_time(rk, order):
    """Fixed mesh (8^2 x 2, central reconstruction), 4, 8, 16 steps: successive differences fall
    by 2^order."""
    wl = W.density_wave_2d(8)
    T = 0.02
    sols = []
    for nst in (4, 8, 16):
        o = Oracle(wl.mesh, degree=2, C_T=0.0, rk=rk)
        o.set_state(wl.U0)
        o.run(nst, T / nst)
        sols.append(o.get_state())
    e1 = np.abs(sols[0] - sols[1]).max()
    e2 = np.abs(sols[1] - sols[2]).max()
    assert order - 0.3 < math.log2(e1 / e2) < order + 0.3, math.log2(e1 / e2)


def test_rk4_step_of_a_uniform_flow_is_exact():
    """The residual of a uniform periodic flow is zero, so every RK4 stage must give back U^n (a
    stage that drops U^n or the accumulated sum shows); the weights are pinned by the order."""
    wl = W.density_wave_2d(8)
    U = _uniform(wl.mesh, 1.3, [0.4, -0.2], 0.9)
    o = Oracle(wl.mesh, degree=2, rk=4)
    o.set_state(U)
    o.run(3, 0.01)
    assert np.abs(o.get_state() - U).max() < 1e-14


def test_fixed_state_boundary_keeps_a_matching_uniform_flow():
    """Every boundary face of the fixed-state kind: with A equal to the interior uniform state the
    residual vanishes to rounding; with another A exactly the cells that own a boundary face move."""
    mesh = W.tri_mesh(12, 6, ly=0.5, periodic=False)
    U = _uniform(mesh, 1.3, [0.7, -0.4], 2.0)
    o = Oracle(mesh, degree=2)
    o.boundary_region((-1, -1), (2, 2), 2)
    o.boundary_states(U[:, 0], U[:, 0])
    o.set_state(U)
    assert np.abs(o.residual()).max() < 1e-12
    o.boundary_states(_uniform(mesh, 1.0, [0.0, 0.0], 1.0)[:, 0], U[:, 0])
    R = o.residual()
    touched = (o.geometry()["nbr"] < 0).any(axis=1)
    assert np.array_equal(np.abs(R).max(axis=0) > 1e-12, touched)


def test_moving_shock_boundary_switches_at_the_line():
    """Kind 3 on every boundary face, line x = 0.2 + 0.5 t (xs0 = 0.2, sy = 0, vs = 0.5), A equal to
    the interior state, B another: only cells with a boundary face whose midpoint lies right of the
    line at the stage's time see B, so their residual is the only nonzero one; one step later the
    line has moved by 0.5 dt and fewer faces see B."""
    mesh = W.tri_mesh(16, 4, ly=0.25, periodic=False, jitter=0.0)
    U = _uniform(mesh, 1.0, [0.0, 0.0], 1.0)
    B = _uniform(mesh, 0.5, [0.0, 0.0], 0.4)[:, 0]
    o = Oracle(mesh, degree=2)
    o.boundary_region((-1, -1), (2, 2), 3)
    o.boundary_states(U[:, 0], B, 0.2, 0.0, 0.5)
    g = o.geometry()
    cells = g["cells"]
    xyz = mesh.xyz
    nb = g["nbr"]

    def expected(t):
        hit = np.zeros(mesh.ncells, bool)
        for i in range(mesh.ncells):
            for f in range(3):
                if nb[i, f] < 0:
                    mid = np.delete(xyz[cells[i]], f, axis=0).mean(0)
                    hit[i] |= not (0.2 + 0.5 * t > mid[0])
        return hit
    for t in (0.0, 0.3):
        o.set_time(t)
        o.set_state(U)
        R = o.residual()
        got = np.abs(R).max(axis=0) > 1e-12
        assert np.array_equal(got, expected(t)), t
    assert expected(0.0).sum() > expected(0.3).sum() > 0
    o.set_time(0.0)
    o.step(0.01)
    assert abs(o.time() - 0.01) < 1e-16
