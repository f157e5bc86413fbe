"""Accuracy on the smooth 3D density wave (periodic unit cube, n^3 cubes x 6 tetrahedra,
rho = 1 + 0.2 sin 2 pi (x+y+z), u = v = w = p = 1, degree 2), advanced with equal CFL-0.5 steps to
a final time reached exactly.

- The configured case (CTENO, T = 0.2): the L1 density error of the mixed path stays within 1.05x
  of the FP64 path at 32^3, 48^3 and 64^3 (both advanced with the same time steps).
- Order: CTENOZ shows the scheme's third order (> 2.9 between 32^3, 48^3 and 64^3). CTENO with
  lambda_1' = 1e15 rejects the central stencil in a few smooth cells at some stages on these
  jittered tetrahedra and is measured at about 2.2 at T = 0.2 (third order when the central stencil
  is always kept, i.e. C_T = 0); it is asserted to stay above second order."""
from __future__ import annotations

import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_17042_gb300 import build, native
    build.build()
    return native


def _wave(n):
    mesh = W.tet_mesh(n, 1.0, periodic=True, jitter=0.08, seed=0)
    prim = W._wave_prim(3, 0.0)
    return mesh, W.cell_average(mesh, prim, n_rule=4)


def _l1_errors(native, T, scheme, precisions, sizes=(32, 48, 64)):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    errs = {}
    for n in sizes:
        mesh, U0 = _wave(n)
        exact = W.cell_average(mesh, W._wave_prim(3, T), n_rule=4)[0]
        vol = W.cell_volumes(mesh)
        # time step: the FP64 CFL step of the initial state, then equal steps reaching T exactly
        probe = native.Solver([mesh], 3, degree=2, precision=0, cfl=0.5, stream=stream)
        probe.set_state(U0)
        probe.run(1)
        nst = int(math.ceil(T / probe.dt()[0]))
        probe.close()
        dt = T / nst
        for precision in precisions:
            s = native.Solver([mesh], 3, degree=2, scheme=scheme, precision=precision, stream=stream)
            s.set_state(U0)
            for _ in range(nst):
                s.step(dt)
            rho = s.get_state()[0]
            errs[(n, precision)] = float(np.sum(vol * np.abs(rho - exact)) / vol.sum())
            s.close()
    return errs


def _orders(errs, precision, sizes=(32, 48, 64)):
    return [math.log(errs[(a, precision)] / errs[(b, precision)]) / math.log(b / a)
            for a, b in zip(sizes, sizes[1:])]


def test_mixed_vs_fp64_l1_error_3d_wave_cteno_t02():
    native = _native()
    errs = _l1_errors(native, 0.2, 0, (0, 1))
    print("CTENO T=0.2 L1 errors", errs, "FP64 orders", _orders(errs, 0))
    for n in (32, 48, 64):
        assert errs[(n, 1)] <= 1.05 * errs[(n, 0)], (n, errs)
    assert min(_orders(errs, 0)) > 2.0, errs


def test_third_order_3d_wave_ctenoz():
    native = _native()
    errs = _l1_errors(native, 0.05, 1, (0, 1))
    o = _orders(errs, 0)
    print("CTENOZ T=0.05 L1 errors", errs, "FP64 orders", o, "mixed orders", _orders(errs, 1))
    assert min(o) > 2.9, (o, errs)
    for n in (32, 48, 64):
        assert errs[(n, 1)] <= 1.05 * errs[(n, 0)], (n, errs)
