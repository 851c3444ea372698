"""dc_global_solve_static: the allocation-free variant of the global-step solve.

It exists for callers that may not allocate device memory while they run
(a fixed HBM budget already handed to a caching allocator, or a loop that cannot
take the device-wide synchronisation of cudaMalloc/cudaFree).  This file is
collected last so that a failure here leaves every other test already run.
"""
import os

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which,solver,sweeps", [("hanging_16x16", 0, "tree"), ("draped_61x61", 0, "tree"),
                                                 ("hanging_16x16", 1, "tree"), ("draped_61x61", 1, "tree"),
                                                 ("draped_61x61", 1, "level")])
def test_static_scratch_solve_matches_global_solve_twice(which, solver, sweeps):
    """Two calls in a row with different right-hand sides agree with dc_global_solve
    (1e-11); with global_solver 1 the supernodal sweeps (one launch per sweep, or
    one per tree level) also use the context's sweep vectors and flags, and no
    bounded wait gives up (the sticky fault word stays clear)."""
    import torch

    from paper_2106_05306_gb300 import _lib
    from tests._helpers import make_cloth
    sc = scenes.hanging_cloth() if which == "hanging_16x16" else scenes.draped_cloth()
    if sweeps == "level":
        os.environ["DC_LEVEL_SOLVES"] = "1"
    try:
        cloth = make_cloth(sc, global_solver=solver)
    finally:
        os.environ.pop("DC_LEVEL_SOLVES", None)
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
    cloth.sync()          # raises DC_ERR_TIMEOUT if a sweep's bounded wait gave up
    # the component-major layout goes through the same fixed array
    cloth.set_layout("component_major")
    rhs_t = rhs.t().contiguous()
    got_t = torch.full_like(rhs_t, float("nan"))
    _lib.check(lib.dc_global_solve_static(cloth._ctx, rhs_t.data_ptr(), got_t.data_ptr()), cloth._ctx)
    torch.cuda.synchronize()
    assert torch.equal(got_t.t(), got)
    # host arrays are rejected rather than staged (staging would need memory)
    host = torch.zeros((sc.m, 3), dtype=torch.float64)
    st = lib.dc_global_solve_static(cloth._ctx, host.data_ptr(), host.data_ptr())
    assert st == 1 and b"device arrays" in lib.dc_last_error(cloth._ctx)
    cloth.close()
