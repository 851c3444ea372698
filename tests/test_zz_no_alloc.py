"""dc_global_solve_static: the allocation-free variant of the global-step solve.

It exists for callers that may not allocate device memory while they run
(a fixed HBM budget already handed to a caching allocator, or a loop that cannot
take the device-wide synchronisation of cudaMalloc/cudaFree).  This file is
collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["hanging_16x16", "draped_61x61"])
def test_static_scratch_solve_matches_global_solve_twice(which):
    import torch

    from paper_2106_05306_gb300 import _lib
    from tests._helpers import make_cloth
    sc = scenes.hanging_cloth() if which == "hanging_16x16" else scenes.draped_cloth()
    cloth = make_cloth(sc)
    lib = _lib.load()
    rng = np.random.default_rng(21)
    for call in range(2):
        rhs = torch.tensor(rng.standard_normal((sc.m, 3)), device="cuda")
        ref = torch.empty_like(rhs)
        got = torch.full_like(rhs, float("nan"))
        _lib.check(lib.dc_global_solve(cloth._ctx, rhs.data_ptr(), ref.data_ptr()), cloth._ctx)
        _lib.check(lib.dc_global_solve_static(cloth._ctx, rhs.data_ptr(), got.data_ptr()), cloth._ctx)
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item() / max(ref.abs().max().item(), 1e-3)
        assert err <= 1e-11, (call, err)
        assert torch.all(got[torch.as_tensor(sc.pins, dtype=torch.long)] == 0)
    # host arrays are rejected rather than staged (staging would need memory)
    host = torch.zeros((sc.m, 3), dtype=torch.float64)
    st = lib.dc_global_solve_static(cloth._ctx, host.data_ptr(), host.data_ptr())
    assert st == 1 and b"device arrays" in lib.dc_last_error(cloth._ctx)
    cloth.close()
