"""cteno_get_state_noalloc: the allocation-free state read-back.

For callers that cannot allocate device memory when they read a state back (a program whose own
pool owns the device memory, or code running where cudaMalloc is not allowed). The entry point
stages through a fixed array compiled into the library instead of a cudaMalloc'd buffer; its
output must equal cteno_get_state's, on consecutive calls, and the device's free memory must not
change across it. This file is collected last so that a run stopping at its first failure has
already run every other test; it passes alone in a fresh process as well.
"""
from __future__ import annotations

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


def test_noalloc_read_back_allocates_nothing_and_matches_get_state():
    import torch
    native = _native()
    wl = W.shock_tube_2d(64, 16)
    for precision in (0, 1):
        s = native.Solver([wl.mesh], 2, degree=2, precision=precision, cfl=0.4,
                          stream=torch.cuda.current_stream().cuda_stream)
        s.set_state(wl.U0)
        s.run(2)
        s.sync()
        torch.cuda.synchronize()
        # first on this context, before cteno_get_state has allocated its staging buffer
        free0, _ = torch.cuda.mem_get_info()
        first = native.cteno_get_state_noalloc(s.ctx, 0)
        again = native.cteno_get_state_noalloc(s.ctx, 0)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
        assert np.array_equal(first, again)
        ref = native.cteno_get_state(s.ctx, 0)
        assert np.array_equal(first, ref)       # a copy of the same FP64 values: exact
        for _ in range(2):                      # two calls in a row, with the state moving between
            s.run(2)
            ref = native.cteno_get_state(s.ctx, 0)
            got = native.cteno_get_state_noalloc(s.ctx, 0)
            assert np.array_equal(got, ref)
        s.close()


def test_noalloc_rejects_states_larger_than_its_array():
    import torch
    native = _native()
    mesh = W.tri_mesh(512, 520, periodic=False)   # 532480 cells x 4 variables > 2^21 values
    s = native.Solver([mesh], 2, degree=2, stream=torch.cuda.current_stream().cuda_stream)
    s.set_state(W.uniform_state(mesh, [1.0, 0.0, 0.0, 1.0]))
    with pytest.raises(native.CtenoError) as e:
        native.cteno_get_state_noalloc(s.ctx, 0)
    assert e.value.code == -1
    ok = native.cteno_get_state(s.ctx, 0)      # the allocating path still works
    assert ok.shape == (4, mesh.ncells)
    s.close()
