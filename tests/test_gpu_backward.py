"""GPU adjoint parity: dc_backward (checkpointed recomputation + preconditioned
GMRES per step) against the oracle's direct KKT adjoint, to 1e-7 relative."""
import numpy as np
import pytest

import scenes
from oracle import cloth as oc
from tests._helpers import GRAD_TOL, cuda, make_cloth, oracle_model, rel_l2

pytestmark = pytest.mark.gpu


def _grad_parity(sc, n_steps, ck=1, dtraj=False, **over):
    cloth = make_cloth(sc, checkpoint_every=ck, **over)
    M = oracle_model(sc, **over)
    xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, n_steps)
    rng = np.random.default_rng(11)
    gT = rng.standard_normal((n_steps + 1, sc.m, 3)) * 0.1 if dtraj else None
    gv = rng.standard_normal((sc.m, 3)) * 0.3
    want = oc.rollout_gradient(M, recs, sc.loss_w, gv, gT)
    cloth.rollout(cuda(sc.x0), cuda(sc.v0), n_steps)
    dx0, dv0, dth = cloth.backward(cuda(sc.loss_w), cuda(gv), cuda(gT) if dtraj else None)
    got = (dx0.cpu().numpy(), dv0.cpu().numpy(), dth.cpu().numpy())
    st = cloth.stats()
    cloth.close()
    assert rel_l2(got[0], want[0]) <= GRAD_TOL, rel_l2(got[0], want[0])
    assert rel_l2(got[1], want[1]) <= GRAD_TOL, rel_l2(got[1], want[1])
    scale = np.max(np.abs(want[2]))
    for q in range(3):
        assert abs(got[2][q] - want[2][q]) <= GRAD_TOL * max(abs(want[2][q]), 1e-6 * scale), (q, got[2], want[2])
    assert st["adj_nonconverged"] == 0
    return got, want, st, recs


@pytest.mark.parametrize("contact,drop,pinned", [("sphere", True, True), ("plane", True, False),
                                                 ("capsule", False, True), ("both", True, True),
                                                 ("none", False, True)])
def test_backward_parity_small(contact, drop, pinned):
    sc = scenes.small_scene(5, seed=3, contact=contact, drop=drop, pinned=pinned)
    _grad_parity(sc, 3)


@pytest.mark.parametrize("precond", [0, 1])
def test_backward_parity_hanging_cloth_16x16(precond):
    """precond 0: per-step multifrontal LDL^T; 1: node-block inverse + projected P^-1."""
    sc = scenes.hanging_cloth()
    got, want, st, recs = _grad_parity(sc, sc.n_steps, ck=10, adj_precond=precond)
    assert sum(len(r.contacts) for r in recs) > 0
    assert st["adj_steps"] == sc.n_steps
    if precond == 0:
        assert st["adj_max_iters_seen"] <= 40


def test_backward_parity_through_a_collapsed_triangle():
    """With no PD iteration the step ends where it started, so the adjoint is
    linearised at a state with a triangle collapsed onto a line: both sides take
    its projection as locally constant (reading R1, dR = 0)."""
    sc = scenes.collapsed_triangle_scene(n_steps=1)
    M = oracle_model(sc)
    assert oc.polar_degenerate(M.deformation_gradients(sc.x0))[0]
    got, want, st, recs = _grad_parity(sc, 1, n_pd_iters=0)
    assert np.all(np.isfinite(got[0])) and np.all(np.isfinite(got[2]))


def test_backward_with_per_step_loss_and_checkpoint_invariance():
    import torch
    sc = scenes.small_scene(5, seed=1, contact="both", drop=True, n_steps=6)
    got, _, _, _ = _grad_parity(sc, 6, ck=4, dtraj=True)
    outs = []
    for ck in (1, 3, 6):
        cloth = make_cloth(sc, checkpoint_every=ck)
        cloth.rollout(cuda(sc.x0), cuda(sc.v0), 6)
        outs.append(cloth.backward(cuda(sc.loss_w)))
        cloth.close()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)


def test_backward_parity_draped_61x61_short():
    sc = scenes.draped_cloth()
    # start just before the cloth reaches the sphere so that contacts appear
    M = oracle_model(sc)
    xs, vs, _ = oc.rollout(M, sc.x0, sc.v0, 20)
    sc.x0, sc.v0 = xs[-1], vs[-1]
    got, want, st, recs = _grad_parity(sc, 4, ck=2)
    assert sum(len(r.contacts) for r in recs) > 0


def test_autograd_function_matches_backward():
    import torch
    import paper_2106_05306_gb300 as dc
    sc = scenes.small_scene(5, seed=3, contact="both", drop=True, n_steps=3)
    cloth = make_cloth(sc)
    p = sc.params
    x0 = cuda(sc.x0).requires_grad_(True)
    v0 = cuda(sc.v0).requires_grad_(True)
    th = torch.tensor([p.k_stretch, p.k_bend, p.mu], dtype=torch.float64, requires_grad=True)
    xN, vN = dc.rollout_fn(cloth, x0, v0, th, 3)
    L = (xN * cuda(sc.loss_w)).sum()
    gx0, gv0, gth = torch.autograd.grad(L, (x0, v0, th))
    M = oracle_model(sc)
    xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, 3)
    want = oc.rollout_gradient(M, recs, sc.loss_w)
    assert rel_l2(gx0.cpu().numpy(), want[0]) <= GRAD_TOL
    assert rel_l2(gv0.cpu().numpy(), want[1]) <= GRAD_TOL
    assert rel_l2(gth.numpy(), want[2]) <= GRAD_TOL
    cloth.close()
