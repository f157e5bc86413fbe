"""Failure detection on the GPU without faulting it, and checkpoint / resume.

  * A non-finite state (a NaN written into one cell's mean on the host) reaches the update
    kernels, which record it in the context's error word; the next synchronising call returns
    CTENO_ERR_DEVICE, and a new context works.
  * The bounded waits of the staged schedules: a test hook makes each block first wait, for 1 ms,
    on a shared-memory barrier that nothing completes; the wait runs out, the kernel records the
    timeout, lets its own bulk copies land and returns; the host sees CTENO_ERR_DEVICE and the
    device stays usable.
  * Resume: reading every mesh's state back (cteno_get_state_all) and setting it again
    (cteno_set_state_all) between steps reproduces an uninterrupted run bit for bit.
"""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

CTENO_ERR_DEVICE = -7


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


def _fresh_context_works(native):
    wl = W.shock_tube_2d(16, 8)
    s = _solver(native, [wl.mesh], 2, degree=2, precision=1, cfl=0.4)
    s.set_state(wl.U0)
    s.run(2)
    assert s.sync() >= 0
    U = s.get_state()
    assert np.isfinite(U).all()
    s.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_non_finite_state_is_reported(precision):
    native = _native()
    wl = W.shock_tube_2d(32, 8)
    s = _solver(native, [wl.mesh], 2, degree=2, precision=precision, cfl=0.4)
    U = wl.U0.copy()
    U[3, 100] = np.nan                  # energy of one cell
    s.set_state(U)
    s.run(1)
    with pytest.raises(native.CtenoError) as e:
        s.sync()
    assert e.value.code == CTENO_ERR_DEVICE
    assert "non-finite" in str(e.value)
    s.close()
    _fresh_context_works(native)


@pytest.mark.parametrize("launch", [2048 + 64, 3072 + 128, 4096, 4097, 5120 + 8, 6144 + 4, 7168 + 4])
def test_bounded_wait_timeout_is_reported(launch):
    native = _native()
    wl = W.shock_tube_2d(64, 16)
    s = _solver(native, [wl.mesh], 2, degree=2, precision=1, cfl=0.4)
    native.cteno_set_launch(s.ctx, launch, 0)
    s.set_state(wl.U0)
    s.run(1)
    assert s.sync() >= 0                # the schedule runs cleanly without the hook
    native.cteno_test_wait_timeout(s.ctx, 1_000_000)   # 1 ms on a barrier nothing completes
    s.run(1)
    with pytest.raises(native.CtenoError) as e:
        s.sync()
    assert e.value.code == CTENO_ERR_DEVICE
    assert "timed out" in str(e.value)
    s.close()
    _fresh_context_works(native)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_resume_from_read_back_state_is_bit_identical(precision):
    native = _native()
    wls = W.quadrants_batch(4, seed=9, nmin=12, nmax=30)
    meshes = [w.mesh for w in wls]
    flat = np.concatenate([w.U0.ravel() for w in wls])
    a = _solver(native, meshes, 2, degree=2, scheme=1, precision=precision, cfl=0.4)
    native.cteno_set_state_all(a.ctx, flat)
    a.run(6)
    ref, ref_dt = native.cteno_get_state_all(a.ctx), a.dt()
    a.close()
    b = _solver(native, meshes, 2, degree=2, scheme=1, precision=precision, cfl=0.4)
    native.cteno_set_state_all(b.ctx, flat)
    b.run(3)
    checkpoint = native.cteno_get_state_all(b.ctx)
    b.close()
    c = _solver(native, meshes, 2, degree=2, scheme=1, precision=precision, cfl=0.4)   # a new process would do the same
    native.cteno_set_state_all(c.ctx, checkpoint)
    c.run(3)
    assert np.array_equal(native.cteno_get_state_all(c.ctx), ref)
    assert np.array_equal(c.dt(), ref_dt)
    c.close()
