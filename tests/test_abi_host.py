"""C-ABI checks that need no GPU: the library loads, exports every entry point of
include/cteno.h, validates its arguments, and its host-side stencil search (integer results)
agrees exactly with the oracle's."""
from __future__ import annotations

import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cteno.h")


def _lib():
    from paper_2312_17042_gb300 import build, native
    build.build()
    return native


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cteno_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    native = _lib()
    lib = native.load_library()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_parameter_validation_without_gpu():
    native = _lib()
    p = native.cteno_default_params()
    assert (p.dim, p.degree, p.C_T, p.lambda1p, p.eps, p.ctenoz_form) == (2, 2, 1e-6, 1e15, 1e-24, 0)
    for dim, degree in ((2, 7), (2, 1), (3, 4)):   # 2D: degrees 2 to 6; 3D: 2 and 3
        p.dim, p.degree = dim, degree
        with pytest.raises(native.CtenoError):
            native.cteno_create(p)
    p = native.cteno_default_params()
    ctx = native.cteno_create(p)
    # rk_stage before lsq_build is an ordering error, not a crash
    with pytest.raises(native.CtenoError) as e:
        native.cteno_rk_stage(ctx, 0, [1e-3])
    assert e.value.code == -2
    # degenerate cell
    xyz = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]])
    with pytest.raises(native.CtenoError) as e:
        native.cteno_mesh_build(ctx, xyz, np.array([[0, 1, 2]]))
    assert e.value.code == -3
    # mesh too small for M = 12
    m = W.tri_mesh(2, 2, periodic=False)
    native.cteno_mesh_build(ctx, m.xyz, m.cells, m.period)
    with pytest.raises(native.CtenoError) as e:
        native.cteno_stencil_build(ctx)
    assert e.value.code == -4
    native.cteno_destroy(ctx)


@pytest.mark.parametrize("mesh,degree", [
    (W.tri_mesh(12, 12, periodic=True, seed=1), 2),
    (W.tri_mesh(14, 9, periodic=False, seed=2), 3),
    (W.tet_mesh(6, periodic=True, seed=3), 2),
    (W.tet_mesh(5, periodic=False, seed=4), 3),
    (W.tri_mesh(16, 16, periodic=True, seed=5), 4),
    (W.tri_mesh(18, 14, periodic=False, seed=6), 5),
    (W.tri_mesh(20, 20, periodic=True, seed=7), 6),
], ids=["tri-per-r2", "tri-r3", "tet-per-r2", "tet-r3", "tri-per-r4", "tri-r5", "tri-per-r6"])
def test_host_stencils_match_oracle_exactly(mesh, degree):
    """Central stencils (ids, nearest-first order) and directional member positions are integer
    results of the same readings, computed independently: they must agree exactly."""
    native = _lib()
    from oracle import Oracle
    o = Oracle(mesh, degree=degree)
    p = native.cteno_default_params()
    p.dim, p.degree = mesh.dim, degree
    ctx = native.cteno_create(p)
    mid = native.cteno_mesh_build(ctx, mesh.xyz, mesh.cells, mesh.period)
    native.cteno_stencil_build(ctx)
    for i in range(mesh.ncells):
        c_lib, d_lib, _ = native.cteno_get_stencil(ctx, mid, i, with_admissibility=False)
        c_orc, d_orc, _ = o.stencil(i)
        assert np.array_equal(c_lib, c_orc), i
        assert np.array_equal(d_lib, d_orc), i
    native.cteno_destroy(ctx)


def test_launch_values_of_the_lane_only_paths_without_gpu():
    """Degrees 4-6 and the characteristic reconstruction run the variable-per-lane schedule only:
    every other reconstruction launch value is refused before anything runs."""
    native = _lib()
    for kw in (dict(degree=5), dict(characteristic=1), dict(dim=3, degree=3, characteristic=1)):
        p = native.cteno_default_params()
        for k, v in kw.items():
            setattr(p, k, v)
        p.precision = 1
        ctx = native.cteno_create(p)
        for bad in (128, -64, 2048 + 64, 3072 + 128, 4096, 5120 + 8, 6144 + 4):
            with pytest.raises(native.CtenoError) as e:
                native.cteno_set_launch(ctx, bad, 0)
            assert e.value.code == -1
        if kw.get("characteristic"):   # the 64-register build of degrees 4-6: no projection
            with pytest.raises(native.CtenoError):
                native.cteno_set_launch(ctx, 1536 + 64, 0)
        else:
            native.cteno_set_launch(ctx, 1536 + 64, 0)
        native.cteno_set_launch(ctx, 1024 + 256, 8192 + 128)   # lanes + face-based flux
        native.cteno_destroy(ctx)


def test_boundary_region_validation_without_gpu():
    native = _lib()
    p = native.cteno_default_params()
    p.dim = 3
    ctx = native.cteno_create(p)
    m = W.tet_mesh(3, periodic=False)
    mid = native.cteno_mesh_build(ctx, m.xyz, m.cells, m.period)
    native.cteno_boundary_region(ctx, mid, (-1, -1, -1), (2, 2, 0.0), native.CTENO_BOUNDARY_WALL)
    for kind in (native.CTENO_BOUNDARY_SHOCK_AB, 7, -1):   # the moving shock is 2D only
        with pytest.raises(native.CtenoError):
            native.cteno_boundary_region(ctx, mid, (-1, -1, -1), (2, 2, 2), kind)
    with pytest.raises(native.CtenoError):
        native.cteno_boundary_region(ctx, 5, (-1, -1, -1), (2, 2, 2), 0)
    native.cteno_destroy(ctx)


def test_corrupt_meshes_are_refused_without_gpu():
    """Host-side fault injection: corrupt connectivity, a degenerate (non-finite) vertex, a face
    shared by three cells, an empty mesh and a periodic box too small for the stencils each return
    an error code from the call that sees them, before any device work."""
    native = _lib()
    m = W.tri_mesh(8, 8, periodic=False)
    out_of_range = m.cells.copy()
    out_of_range[3, 1] = m.nverts + 5
    negative = m.cells.copy()
    negative[3, 1] = -1
    nan_xyz = m.xyz.copy()
    nan_xyz[2] = np.nan
    cases = [(m.xyz, out_of_range, -3), (m.xyz, negative, -3),
             (m.xyz, np.vstack([m.cells, m.cells[:1]]), -3),   # a repeated cell: faces shared three times
             (nan_xyz, m.cells, -3), (m.xyz, m.cells[:0], -1)]
    for xyz, cells, code in cases:
        ctx = native.cteno_create(native.cteno_default_params())
        with pytest.raises(native.CtenoError) as e:
            native.cteno_mesh_build(ctx, xyz, cells, m.period)
        assert e.value.code == code, (e.value.code, str(e.value))
        native.cteno_destroy(ctx)
    small = W.tri_mesh(3, 3, periodic=True)
    ctx = native.cteno_create(native.cteno_default_params())
    native.cteno_mesh_build(ctx, small.xyz, small.cells, small.period)
    with pytest.raises(native.CtenoError) as e:   # a stencil would span more than 0.4 of the box
        native.cteno_stencil_build(ctx)
    assert e.value.code == -4
    native.cteno_destroy(ctx)


@pytest.mark.parametrize("mesh", [W.tri_mesh(10, 9, periodic=False, seed=8), W.tet_mesh(4, periodic=False, seed=9)],
                         ids=["tri", "tet"])
def test_cell_orientation_does_not_change_the_stencils(mesh):
    """Reference map (reading R5): every cell is brought to the positive vertex order, so a mesh
    given with every cell negatively oriented (two vertices swapped) gets the same central and
    directional stencils, face for face, as the same mesh given positively."""
    native = _lib()
    d = mesh.dim
    p = native.cteno_default_params()
    p.dim = d
    flipped = mesh.cells.copy()
    flipped[:, [1, 2]] = flipped[:, [2, 1]]
    got = []
    for cells in (mesh.cells, flipped):
        ctx = native.cteno_create(p)
        native.cteno_mesh_build(ctx, mesh.xyz, cells, mesh.period)
        native.cteno_stencil_build(ctx)
        got.append([native.cteno_get_stencil(ctx, 0, i, with_admissibility=False)[:2]
                    for i in range(0, mesh.ncells, 7)])
        native.cteno_destroy(ctx)
    for (c0, s0), (c1, s1) in zip(*got):
        assert np.array_equal(c0, c1)
        # directional stencils per face: the same member sets, whichever local numbering
        assert sorted(tuple(sorted(c0[j] for j in row if j >= 0)) for row in s0) == \
               sorted(tuple(sorted(c1[j] for j in row if j >= 0)) for row in s1)
