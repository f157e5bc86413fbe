"""Pins of the oracle's characteristic-variable reconstruction (Sec. 2.2 and 3.2: the
reconstruction applied to characteristic variables; the readings are in the oracle's
euler_eigen and recon_cell comments).

  * The eigenvectors: L R = I, and A_n R = R diag(u_n - c, u_n, .., u_n, u_n + c) with A_n the
    Jacobian of the Euler flux in direction n, taken by central differences of an independent
    flux (tests/exact.py), in 2D and 3D.
  * Linearity: where every field keeps the central polynomial (a smooth field), the
    characteristic reconstruction gives the conserved one's face states (R L = I).
  * A contact (density jump at constant velocity and pressure) is a jump in the entropy field
    alone: the other fields see no variation and keep the central stencil everywhere, while the
    conserved reconstruction drops it for every variable that jumps.
  * Sod: the exact Riemann solution within the bounds of the conserved case; conservation on a
    periodic mesh.
"""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from tests import exact as X


def _jacobian(u, n, g=1.4, h=1e-6):
    nv = u.size
    A = np.empty((nv, nv))
    for k in range(nv):
        e = np.zeros(nv)
        e[k] = h * max(1.0, abs(u[k]))
        A[:, k] = (X.euler_flux(u + e, n, g) - X.euler_flux(u - e, n, g)) / (2 * e[k])
    return A


@pytest.mark.parametrize("dim", [2, 3])
def test_eigenvectors_diagonalise_the_flux_jacobian(dim):
    mesh = W.tri_mesh(4, 4) if dim == 2 else W.tet_mesh(4)
    o = Oracle(mesh, setup=False)
    rng = np.random.default_rng(dim)
    for _ in range(20):
        rho, p = rng.uniform(0.2, 3.0, 2)
        vel = rng.uniform(-2, 2, dim)
        u = np.concatenate([[rho], rho * vel, [p / 0.4 + 0.5 * rho * vel @ vel]])
        n = rng.normal(size=dim)
        n /= np.linalg.norm(n)
        R, L = o.eigen(u, n)
        assert np.allclose(L @ R, np.eye(dim + 2), atol=1e-13)
        c = np.sqrt(1.4 * p / rho)
        un = vel @ n
        lam = np.array([un - c] + [un] * dim + [un + c])
        A = _jacobian(u, n)
        assert np.allclose(A @ R, R * lam, rtol=1e-6, atol=1e-6 * np.abs(A).max())
        # the shear fields are orthogonal to n
        for m in range(dim - 1):
            assert abs(R[1:dim + 1, 2 + m] @ n) < 1e-14


@pytest.mark.parametrize("dim,degree", [(2, 2), (2, 3), (3, 2), (2, 5)])
def test_smooth_field_characteristic_equals_conserved(dim, degree):
    """In every cell where both reconstructions keep the central polynomial for every variable,
    field and face (nearly all cells of the smooth wave, CTENOZ), their face states agree."""
    wl = W.density_wave_2d(12 if degree < 5 else 14) if dim == 2 else W.density_wave_3d(5)
    oc = Oracle(wl.mesh, degree=degree, scheme=1)
    oc.set_state(wl.U0)
    oc.residual()
    och = Oracle(wl.mesh, degree=degree, scheme=1, characteristic=1)
    och.set_state(wl.U0)
    och.residual()
    fl = och.flags()
    assert fl.shape == (wl.mesh.ncells, dim + 1, dim + 2)
    central = np.all(oc.flags() == 1, axis=1) & np.all(fl == 1, axis=(1, 2))
    assert central.mean() > 0.9, central.mean()
    fs_c, fs_w = oc.face_states()[central], och.face_states()[central]
    assert np.abs(fs_w - fs_c).max() < 1e-12 * np.abs(fs_c).max()


@pytest.mark.parametrize("scheme", [0, 1])
def test_contact_is_an_entropy_field_jump(scheme):
    mesh = W.tri_mesh(16, 8, periodic=False, jitter=0.1, seed=3)
    cen = W.cell_centroids(mesh)
    prim = np.zeros((mesh.ncells, 4))
    prim[:, 0] = np.where(cen[:, 0] < 0.5, 1.0, 0.125)
    prim[:, 1] = 0.3
    prim[:, 2] = -0.2
    prim[:, 3] = 1.0
    U = W.primitive_to_conserved(prim).T.copy()
    oc = Oracle(mesh, degree=2, scheme=scheme, eps=1e-24, ctenoz_form=1)
    oc.set_state(U)
    oc.residual()
    och = Oracle(mesh, degree=2, scheme=scheme, eps=1e-24, ctenoz_form=1, characteristic=1)
    och.set_state(U)
    och.residual()
    flc, flw = oc.flags(), och.flags()                  # [cells, 4], [cells, 3 faces, 4 fields]
    dropped_c = (flc & 1) == 0
    dropped_w = (flw & 1) == 0
    # conserved: rho, both momenta and E all jump, and all drop the central stencil somewhere
    assert all(dropped_c[:, v].sum() >= 10 for v in range(4))
    # characteristic: only the entropy field (index 1) sees the jump
    assert not dropped_w[:, :, [0, 2, 3]].any()
    assert dropped_w[:, :, 1].sum() >= 10
    # and where it does, the cell's conserved density also dropped it
    assert np.all(dropped_c[dropped_w[:, :, 1].any(axis=1), 0])


def test_sod_characteristic_against_exact_riemann_solution():
    wl = W.shock_tube_2d(nx=80, ny=8)
    o = Oracle(wl.mesh, degree=2, scheme=0, cfl=0.4, characteristic=1)
    o.set_state(wl.U0)
    t, T = 0.0, 0.15
    while t < T - 1e-14:
        dt = min(o.dt(), T - t)
        o.step(dt)
        t += dt
    U = o.get_state()
    xs = W.cell_centroids(wl.mesh)[:, 0]
    ref = X.riemann_exact((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (xs - 0.5) / T)[:, 0]
    vol = W.cell_volumes(wl.mesh)
    l1 = np.sum(vol * np.abs(U[0] - ref)) / vol.sum()
    assert l1 < 0.012, l1
    assert U[0].max() < 1.0 + 0.03 and U[0].min() > 0.125 - 0.03
    assert np.abs(U[2]).max() < 0.05


def test_characteristic_conservation_periodic():
    wl = W.density_wave_2d(10)
    U = wl.U0.copy()
    U[0, ::7] += 0.3        # rough data, so that every selection path is taken
    U[3, ::5] += 0.5
    o = Oracle(wl.mesh, degree=3, scheme=0, characteristic=1)
    vol = W.cell_volumes(wl.mesh)
    o.set_state(U)
    o.residual()
    assert (o.flags() & 1 == 0).any()
    before = (vol * U).sum(axis=1)
    for _ in range(3):
        o.step(0.2 * o.dt())
    after = (vol * o.get_state()).sum(axis=1)
    assert np.allclose(after, before, rtol=1e-13, atol=1e-14)
