"""Central degrees 4 to 6 in 2D (CTENO5-7: Sec. 2.3 and Fig. 1, directional stencils of degree 2;
Tables 1-3 for the orders) on the GPU, through the C ABI, against the FP64 oracle.

Tolerances. Both sides solve eq. 12 by Householder QR (the oracle R a = Q^T b for every solve, the
library once through the pseudo-inverse R^-1 Q^T diag|V'_m|). Each is backward stable, so their
coefficients may differ by a few cond(A) u |a|, and at these degrees cond(A) is large: up to ~2e5
on periodic meshes and ~1e7 on the one-sided stencils of boundary cells at degree 6. Face states
and updates must agree within max(1e-12, 50 kappa u), kappa the largest cond(A) of the mesh's
central stencils (from the oracle's own A). Smoothness indicators inherit the same relative
difference (times about 12 through the sixth power of gamma), so the FP64 flags must equal the
oracle's outside the band where some chi_s of the oracle lies within 1000 kappa u (relative) of
C_T; the mixed path keeps the 1e-4 band of the lower degrees.
"""
from __future__ import annotations

import math

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
    scale = np.maximum(np.abs(b).max(axis=-1, keepdims=True), 1e-300)
    return float((np.abs(a - b) / scale).max())


def _kappa(o, ncells):
    """Largest condition number of the central least-squares matrices A (eq. 10) of the mesh."""
    return max(np.linalg.cond(o.lsq(i)[0]) for i in range(ncells))


MESHES = [
    ("wave-per", lambda: W.density_wave_2d(16)),
    ("sod", lambda: W.shock_tube_2d(40, 10)),
]
SCHEMES = [(0, 0), (1, 0), (1, 1), (2, 0), (3, 0)]


@pytest.mark.parametrize("scheme,form", SCHEMES, ids=["CTENO", "CTENOZ", "CTENOZ-wenoz", "CWENO", "TENO"])
@pytest.mark.parametrize("degree", [4, 5, 6])
@pytest.mark.parametrize("name,make", MESHES, ids=[m[0] for m in MESHES])
def test_one_stage_high_degree_fp64(name, make, degree, scheme, form):
    native = _native()
    from oracle import Oracle
    wl = make()
    if name == "sod":  # a smeared state with shocks, contact and rarefaction
        o0 = Oracle(wl.mesh, degree=2, scheme=0, cfl=0.4)
        o0.set_state(wl.U0)
        o0.run(8)
        U = o0.get_state()
    else:
        U = wl.U0
    o = Oracle(wl.mesh, degree=degree, scheme=scheme, ctenoz_form=form)
    o.set_state(U)
    dt = 0.5 * o.dt()
    kappa = _kappa(o, wl.mesh.ncells)
    tol = max(1e-12, 50 * kappa * U_EPS)
    s = _solver(native, [wl.mesh], 2, degree=degree, scheme=scheme, ctenoz_form=form)
    native.cteno_record_flags(s.ctx, True)
    s.set_state(U)
    s.stage(0, dt)
    fs_gpu = native.cteno_get_face_states(s.ctx, 0)
    fl_gpu = native.cteno_get_flags(s.ctx, 0)
    U_gpu = s.get_state()
    o.stage(0, dt)
    fs_orc = o.face_states()
    assert fs_gpu.shape == fs_orc.shape == (wl.mesh.ncells, 3, (degree + 2) // 2, 4)
    e_fs = _relerr(fs_gpu.reshape(-1, 4).T, fs_orc.reshape(-1, 4).T)
    e_u = _relerr(U_gpu, o.get_state())
    band = flag_band(o, rel=1000 * kappa * U_EPS)
    bad = (fl_gpu != o.flags()) & ~band
    print(f"{name} r={degree} scheme {scheme}/{form}: kappa {kappa:.2e} tol {tol:.1e} face {e_fs:.2e} "
          f"update {e_u:.2e} flags in band {int(band.sum())}")
    assert e_fs < tol and e_u < tol
    assert not bad.any(), np.argwhere(bad)[:10]
    for i in range(0, wl.mesh.ncells, 13):
        _, dirm, dok = native.cteno_get_stencil(s.ctx, 0, i)
        _, dirm_o, dok_o = o.stencil(i)
        assert np.array_equal(dirm, dirm_o) and np.array_equal(dok, dok_o)
    s.close()


@pytest.mark.parametrize("scheme", [0, 1], ids=["CTENO", "CTENOZ"])
@pytest.mark.parametrize("degree", [4, 5, 6])
def test_shock_tube_high_degree_10_steps_fp64(degree, scheme):
    """Sod on the 64x16 copy of the shock-tube mesh, CFL 0.4, 10 FP64 steps (the positivity guard
    active on both sides)."""
    native = _native()
    from oracle import Oracle
    wl = W.shock_tube_2d(64, 16)
    o = Oracle(wl.mesh, degree=degree, scheme=scheme, cfl=0.4)
    kappa = _kappa(o, wl.mesh.ncells)
    o.set_state(wl.U0)
    dts = o.run(10)
    s = _solver(native, [wl.mesh], 2, degree=degree, scheme=scheme, cfl=0.4)
    s.set_state(wl.U0)
    s.run(10)
    err = _relerr(s.get_state(), o.get_state())
    print(f"Sod 64x16 r={degree} scheme {scheme}: kappa {kappa:.2e} max rel after 10 steps {err:.2e}, "
          f"dt {abs(s.dt()[0] - dts[-1]) / dts[-1]:.1e}")
    assert err < max(1e-12, 50 * kappa * U_EPS) * 10
    s.close()


@pytest.mark.parametrize("degree", [4, 5, 6])
def test_mixed_high_degree_against_oracle(degree):
    """Mixed path (FP32 operators and arithmetic on FP64-accurate differences): one stage on the
    periodic wave and on the smeared Sod state; flags equal the oracle's outside the 1e-4 band."""
    native = _native()
    from oracle import Oracle
    for make in (lambda: W.density_wave_2d(16), lambda: W.shock_tube_2d(40, 10)):
        wl = make()
        o = Oracle(wl.mesh, degree=degree, scheme=1)
        o.set_state(wl.U0)
        dt = 0.5 * o.dt()
        s = _solver(native, [wl.mesh], 2, degree=degree, scheme=1, precision=1)
        native.cteno_record_flags(s.ctx, True)
        s.set_state(wl.U0)
        s.stage(0, dt)
        fs = native.cteno_get_face_states(s.ctx, 0)
        fl = native.cteno_get_flags(s.ctx, 0)
        o.stage(0, dt)
        e_fs = _relerr(fs.reshape(-1, 4).T, o.face_states().reshape(-1, 4).T)
        band = flag_band(o)
        bad = (fl != o.flags()) & ~band
        print(f"mixed r={degree} {wl.mesh.ncells} cells: face states max rel {e_fs:.2e}, band {int(band.sum())}")
        assert not bad.any(), np.argwhere(bad)[:10]
        assert e_fs < 1e-4
        s.close()


def _l1_wave(native, n, degree, scheme, lambda1p, precision=0, T=0.1):
    """L1 density error of the smooth wave on n^2 x 2 periodic triangles at time T. The Courant
    number shrinks as (16/n)^((r+1)/3 - 1) from 0.1 at n = 16, so that the third-order time error
    falls like h^(r+1) with the spatial one and the observed order is the reconstruction's."""
    wl = W.density_wave_2d(n)
    cfl = 0.1 * (16.0 / n) ** max(0.0, (degree + 1) / 3.0 - 1.0)
    s = _solver(native, [wl.mesh], 2, degree=degree, scheme=scheme, lambda1p=lambda1p, cfl=cfl,
                precision=precision)
    s.set_state(wl.U0)
    s.stage(0)                 # the CFL step of the initial state (dt = NULL)
    dt0 = s.dt()[0]
    s.set_state(wl.U0)
    nst = int(math.ceil(T / dt0))
    for _ in range(nst):
        for st in range(3):
            s.stage(st, T / nst)
    U = s.get_state()
    s.close()
    vol = W.cell_volumes(wl.mesh)
    return float(np.sum(vol * np.abs(U[0] - wl.exact(T)[0])) / vol.sum())


STUDY_N = (16, 24, 32, 48, 64)


def test_orders_and_lambda1p_study():
    """Sec. 3.1.1, Tables 1-3: L1 density errors of the smooth wave at t = 0.1 on 16^2 .. 64^2 x 2
    periodic triangles at lambda_1' = 1e15 and 1e4, CTENO and CTENOZ, degrees 2 to 6, FP64
    (printed with the observed orders between successive meshes). Asserted: at 1e15 CTENOZ
    converges at high order at every degree on the finest pair, and each degree is more accurate
    than the one below."""
    native = _native()
    rows = []
    for degree in (2, 3, 4, 5, 6):
        for scheme in (0, 1):
            for lam in (1e15, 1e4):
                e = [_l1_wave(native, n, degree, scheme, lam) for n in STUDY_N]
                orders = [math.log(e[k] / e[k + 1]) / math.log(STUDY_N[k + 1] / STUDY_N[k])
                          for k in range(len(e) - 1)]
                rows.append((degree, scheme, lam, e, orders))
    print("degree scheme lambda1p  L1 at n = " + " ".join(str(n) for n in STUDY_N) + "  |  orders")
    for degree, scheme, lam, e, orders in rows:
        print(f"{degree} {'CTENOZ' if scheme else 'CTENO '} {lam:.0e}  " + " ".join(f"{x:.3e}" for x in e) +
              "  |  " + " ".join(f"{o:.2f}" for o in orders))
    z = {d: (e, orders) for d, sc, lam, e, orders in rows if sc == 1 and lam == 1e15}
    for degree, (e, orders) in z.items():
        assert orders[-1] > degree + 1 - 0.8, (degree, orders, e)
    f = [z[d][0][-1] for d in (2, 3, 4, 5, 6)]
    assert all(a > b for a, b in zip(f, f[1:])), f


@pytest.mark.parametrize("scheme", [0, 1], ids=["CTENO", "CTENOZ"])
@pytest.mark.parametrize("degree", [4, 5, 6])
def test_64_register_build_matches_default(degree, scheme):
    """The mixed reconstruction of degrees 4-6 compiled for at most 64 registers per thread (launch
    values 1536 + b) is the same arithmetic as the default build (1024 + b): face states and the
    update agree on the smeared Sod state and the flags equal the oracle's outside the 1e-4 band;
    the FP64 path, the characteristic reconstruction and degree 3 refuse the launch value."""
    native = _native()
    from oracle import Oracle
    wl = W.shock_tube_2d(40, 10)
    o = Oracle(wl.mesh, degree=2, scheme=0, cfl=0.4)
    o.set_state(wl.U0)
    o.run(8)
    U = o.get_state()
    o = Oracle(wl.mesh, degree=degree, scheme=scheme)
    o.set_state(U)
    dt = 0.5 * o.dt()
    o.stage(0, dt)
    out = []
    for launch in (1024 + 128, 1536 + 64, 1536 + 256):
        s = _solver(native, [wl.mesh], 2, degree=degree, scheme=scheme, precision=1)
        native.cteno_set_launch(s.ctx, launch, 0)
        native.cteno_record_flags(s.ctx, True)
        s.set_state(U)
        s.stage(0, dt)
        out.append((native.cteno_get_face_states(s.ctx, 0), s.get_state(), native.cteno_get_flags(s.ctx, 0)))
        s.close()
    band = flag_band(o)
    for fs, Un, fl in out[1:]:
        assert np.abs(fs - out[0][0]).max() <= 1e-6 * np.abs(out[0][0]).max()
        assert _relerr(Un, out[0][1]) < 1e-6
        assert not ((fl != o.flags()) & ~band).any()
    for kw in (dict(degree=3, precision=1), dict(degree=degree, precision=0),
               dict(degree=degree, precision=1, characteristic=1)):
        s = _solver(native, [wl.mesh], 2, **kw)
        with pytest.raises(native.CtenoError):
            native.cteno_set_launch(s.ctx, 1536 + 64, 0)
        s.close()
