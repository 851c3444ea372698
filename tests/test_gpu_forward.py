"""GPU forward parity: libdc (through the C ABI) against the CPU oracle on the same
seeded inputs.  Every step starts from the oracle's own state, so each step is
compared on identical inputs (max-norm relative error <= 1e-9)."""
import numpy as np
import pytest

import scenes
from oracle import cloth as oc
from tests._helpers import STATE_TOL, cuda, make_cloth, oracle_model, rel_inf

pytestmark = pytest.mark.gpu


def _per_step_parity(sc, n_steps, stride=1, **over):
    cloth = make_cloth(sc, **over)
    M = oracle_model(sc, **over)
    xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, n_steps, n_iters=over.get("n_pd_iters"))
    worst = 0.0
    n_cases = np.zeros(3, int)
    for n in range(0, n_steps, stride):
        x1, v1 = cloth.step(cuda(xs[n]), cuda(vs[n]))
        ex = rel_inf(x1.cpu().numpy(), xs[n + 1])
        ev = rel_inf(v1.cpu().numpy(), vs[n + 1])
        worst = max(worst, ex, ev)
        assert ex <= STATE_TOL and ev <= STATE_TOL, (n, ex, ev)
        if len(recs[n].cases):
            n_cases += np.bincount(recs[n].cases, minlength=3)
    cloth.close()
    return worst, n_cases, xs, vs


def test_global_solve_matches_banded_cholesky():
    for sc in (scenes.small_scene(5, seed=1), scenes.hanging_cloth(), scenes.draped_cloth()):
        cloth = make_cloth(sc)
        M = oracle_model(sc)
        rng = np.random.default_rng(3)
        rhs = rng.standard_normal((sc.m, 3))
        got = cloth.global_solve(cuda(rhs)).cpu().numpy()
        want = np.zeros_like(rhs)
        want[M.free] = M.solve_P(rhs[M.free])
        assert rel_inf(got, want) < 1e-11
        assert np.all(got[M.pins] == 0.0)
        st = cloth.stats()
        assert st["n_free"] == len(M.free) and st["factor_nnz"] > 0
        cloth.close()


@pytest.mark.parametrize("contact,drop,pinned", [("sphere", False, True), ("sphere", True, False),
                                                 ("plane", True, True), ("capsule", False, False),
                                                 ("both", True, True), ("none", False, True)])
def test_step_parity_small_scenes(contact, drop, pinned):
    sc = scenes.small_scene(5, seed=3, contact=contact, drop=drop, pinned=pinned)
    _per_step_parity(sc, 3)


def test_step_parity_hanging_cloth_16x16():
    """The 16x16 two-corner-pinned cloth over a sphere and the ground, 50 steps."""
    sc = scenes.hanging_cloth()
    worst, n_cases, xs, vs = _per_step_parity(sc, sc.n_steps)
    assert n_cases.sum() > 0
    # whole rollout on the GPU alone (errors may grow through contact switches)
    cloth = make_cloth(sc)
    xN, vN, tr = cloth.rollout(cuda(sc.x0), cuda(sc.v0), sc.n_steps, traj=True)
    tr = tr.cpu().numpy()
    assert rel_inf(tr[10], xs[10]) < 1e-8
    assert rel_inf(xN.cpu().numpy(), xs[-1]) < 1e-6
    st = cloth.stats()
    assert st["steps"] == sc.n_steps
    cloth.close()


def test_step_parity_draped_61x61_sampled():
    """The 61x61 draped cloth at full size; every 6th step of the first 48."""
    sc = scenes.draped_cloth()
    worst, n_cases, _, _ = _per_step_parity(sc, 48, stride=6)
    assert n_cases.sum() > 0


def test_step_parity_collapsed_triangle():
    """A triangle collapsed onto a line at x_n: the first local step takes reading
    R1's degenerate rule on both sides (the kernel's closed form would divide by
    det F^T F = 0)."""
    sc = scenes.collapsed_triangle_scene()
    M = oracle_model(sc)
    assert oc.polar_degenerate(M.deformation_gradients(sc.x0))[0]
    _per_step_parity(sc, 3)


@pytest.mark.parametrize("n", [2, 3, 7])
def test_ragged_and_tiny_grids(n):
    sc = scenes.small_scene(n, seed=n, contact="both", drop=True, pinned=(n > 2))
    _per_step_parity(sc, 2)


def test_zero_iterations_and_no_obstacles():
    sc = scenes.small_scene(4, seed=2, contact="sphere", drop=True)
    _per_step_parity(sc, 2, n_pd_iters=0)
    sc2 = scenes.small_scene(4, seed=2, contact="none")
    _per_step_parity(sc2, 2, n_pd_iters=1)


def test_irregular_pins():
    sc = scenes.small_scene(6, seed=4, contact="both", drop=True)
    sc.pins = np.array([0, 7, 13, 35], dtype=np.int32)
    sc.v0[sc.pins] = 0.0
    _per_step_parity(sc, 2)


def test_bitwise_repeatable_and_host_device_pointers_agree():
    import torch
    sc = scenes.hanging_cloth()
    cloth = make_cloth(sc)
    x, v = cuda(sc.x0), cuda(sc.v0)
    for _ in range(12):
        x, v = cloth.step(x, v)
    a = cloth.step(x, v)
    b = cloth.step(x, v)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    c = cloth.step(x.cpu().pin_memory(), v.cpu().pin_memory())
    d = cloth.step(x.cpu(), v.cpu())
    assert torch.equal(a[0].cpu(), c[0]) and torch.equal(a[1].cpu(), d[1])
    cloth.close()


def test_invalid_inputs_are_rejected():
    import paper_2106_05306_gb300 as dc
    sc = scenes.small_scene(3, seed=0)
    with pytest.raises(dc.DCError):
        dc.Cloth(sc.rest_pos, np.array([[0, 1, 99]]), [])
    cloth = dc.Cloth(sc.rest_pos, sc.tris, sc.pins)
    with pytest.raises(dc.DCError):
        cloth.step(cuda(sc.x0), cuda(sc.v0))          # no parameters yet
    with pytest.raises(dc.DCError):
        cloth.set_params(h=float("nan"))
    with pytest.raises(dc.DCError):
        cloth.set_params(h=1e-2, obstacles=[{"kind": "sphere", "center": (0, 0, 0), "radius": -1.0}])
    cloth.close()
