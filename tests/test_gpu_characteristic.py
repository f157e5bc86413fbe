"""Characteristic-variable reconstruction (Sec. 2.2, 3.2) on the GPU against the oracle's, through
the C ABI. Per face, the library projects each lane's conserved coefficients onto the
characteristic fields of the face's normal direction at the cell's mean state (shuffles within the
cell's lane group), selects per field and transforms the face's Gauss-point values back.

Tolerances (relative to each component's scale, at least 1e-3 of the largest component's): FP64
face states and updates 1e-12 at degrees 2 and 3 (max(1e-12, 50 cond(A) u) at
degree 5, as for the conserved reconstruction) and flags equal per face and field; the mixed path
keeps its contract (flags equal outside the 1e-4 band of the cut-off, face states within 1e-5 of
their scale).
"""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from tests.test_gpu_parity import flag_band

pytestmark = pytest.mark.gpu

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
    """Max |a - b| relative to each component's scale, floored at 1e-3 of the largest component:
    a component that vanishes identically in the oracle (the momenta of a fluid at rest) is
    compared at the state's scale, since projecting through the eigenvectors and back leaves
    rounding-level momenta."""
    scale = np.abs(b).max(axis=-1, keepdims=True)
    scale = np.maximum(scale, 1e-3 * scale.max())
    return float((np.abs(a - b) / scale).max())


def _sod_state(wl, steps=8):
    from oracle import Oracle
    o = Oracle(wl.mesh, degree=2, scheme=0, cfl=0.4)
    o.set_state(wl.U0)
    o.run(steps)
    return o.get_state()


CASES = [
    ("tri-sod-r2", lambda: W.shock_tube_2d(40, 10), 2, True),
    ("tri-sod-r3", lambda: W.shock_tube_2d(40, 10), 3, True),
    ("tri-wave-r5", lambda: W.density_wave_2d(14), 5, False),
    ("tet-blast-r2", lambda: W.blast_3d(6), 2, False),
    ("tet-blast-r3", lambda: W.blast_3d(6), 3, False),
]


@pytest.mark.parametrize("scheme,form", [(0, 0), (1, 1), (2, 0), (3, 0)], ids=["CTENO", "CTENOZ-wenoz", "CWENO", "TENO"])
@pytest.mark.parametrize("name,make,degree,smear", CASES, ids=[c[0] for c in CASES])
def test_one_stage_characteristic_fp64(name, make, degree, smear, scheme, form):
    native = _native()
    from oracle import Oracle
    wl = make()
    d = wl.mesh.dim
    U = _sod_state(wl) if smear else wl.U0
    o = Oracle(wl.mesh, degree=degree, scheme=scheme, ctenoz_form=form, characteristic=1)
    o.set_state(U)
    dt = 0.5 * o.dt()
    tol = 1e-12
    if degree >= 4:
        tol = max(tol, 50 * max(np.linalg.cond(o.lsq(i)[0]) for i in range(wl.mesh.ncells)) * U_EPS)
    s = _solver(native, [wl.mesh], d, degree=degree, scheme=scheme, ctenoz_form=form, characteristic=1)
    native.cteno_record_flags(s.ctx, True)
    s.set_state(U)
    s.stage(0, dt)
    fs = native.cteno_get_face_states(s.ctx, 0)
    fl = native.cteno_get_flags(s.ctx, 0).reshape(wl.mesh.ncells, d + 1, d + 2)
    U1 = s.get_state()
    o.stage(0, dt)
    e_fs = _relerr(fs.reshape(-1, d + 2).T, o.face_states().reshape(-1, d + 2).T)
    e_u = _relerr(U1, o.get_state())
    ref = o.flags()
    dropped = int(((ref & 1) == 0).sum())
    print(f"{name} scheme {scheme}/{form}: face {e_fs:.2e} update {e_u:.2e} tol {tol:.1e}, "
          f"{dropped} (face, field) selections without the central stencil")
    assert e_fs < tol and e_u < tol
    if degree >= 4:
        band = flag_band(o, rel=1000 * tol / 50)
        assert not ((fl != ref) & ~band).any()
    else:
        assert np.array_equal(fl, ref)
    s.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_characteristic_10_steps_sod(precision):
    """Sod on the 64x16 copy of the shock-tube mesh, CTENO degree 3, characteristic variables,
    10 steps: FP64 within 1e-12 of the oracle, the mixed path within 1e-5."""
    native = _native()
    from oracle import Oracle
    wl = W.shock_tube_2d(64, 16)
    o = Oracle(wl.mesh, degree=3, scheme=0, cfl=0.4, characteristic=1)
    o.set_state(wl.U0)
    o.run(10)
    ref = o.get_state()
    s = _solver(native, [wl.mesh], 2, degree=3, scheme=0, cfl=0.4, characteristic=1, precision=precision)
    s.set_state(wl.U0)
    s.run(10)
    err = _relerr(s.get_state(), ref)
    print(f"characteristic Sod, precision {precision}: max rel {err:.2e}")
    assert err < (1e-12 if precision == 0 else 1e-5)
    s.close()


@pytest.mark.parametrize("name,make,degree", [("tri-sod-r2", lambda: W.shock_tube_2d(40, 10), 2),
                                               ("tet-blast-r3", lambda: W.blast_3d(6), 3)])
def test_mixed_characteristic_flags_and_face_states(name, make, degree):
    native = _native()
    from oracle import Oracle
    wl = make()
    d = wl.mesh.dim
    U = _sod_state(wl) if d == 2 else wl.U0
    o = Oracle(wl.mesh, degree=degree, scheme=1, ctenoz_form=1, characteristic=1)
    o.set_state(U)
    dt = 0.5 * o.dt()
    s = _solver(native, [wl.mesh], d, degree=degree, scheme=1, ctenoz_form=1, characteristic=1, precision=1)
    native.cteno_record_flags(s.ctx, True)
    s.set_state(U)
    s.stage(0, dt)
    fs = native.cteno_get_face_states(s.ctx, 0)
    fl = native.cteno_get_flags(s.ctx, 0).reshape(wl.mesh.ncells, d + 1, d + 2)
    o.stage(0, dt)
    e_fs = _relerr(fs.reshape(-1, d + 2).T, o.face_states().reshape(-1, d + 2).T)
    band = flag_band(o)
    bad = (fl != o.flags()) & ~band
    print(f"mixed characteristic {name}: face {e_fs:.2e}, band {int(band.sum())}")
    assert e_fs < 1e-5
    assert not bad.any(), np.argwhere(bad)[:10]
    s.close()
