"""Oracle parity of the configurations the benchmark times, at their own sizes.

- The batched workload's path: a ClothBatch with global_solver 1 (tree-scheduled
  supernodal sweeps with the contact solve fused in, fronts of more than 64 nodes
  on the CTA path), CUDA graphs and autotuned block sizes, over cloths of 62x62,
  57x57 and 41x41 nodes (the stiffest of the workload's seeds among them), 26
  steps from rest so that the last ~9 have contacts, forward and adjoint.
- The single draped 61x61 cloth as configured: 125 steps, checkpoints every 25,
  gradient through the autograd Function.

The oracle recomputes every step from the GPU's own state (one step at a time,
in a pool of processes) and solves the direct adjoint along those steps, so each
comparison is on identical inputs: states to 1e-9 per step; gradients to 1e-7,
or to the oracle's own rounding spread scaled to the GPU adjoint's backward error
(a relative residual of 1e-12; the benchmark runs at 1e-10), whichever is larger.
"""
import numpy as np
import pytest

import scenes
from tests._helpers import GRAD_TOL, STATE_TOL, cuda, make_batch, make_cloth, oracle_along, rel_inf, \
    spawn_pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    p = spawn_pool()
    yield p
    p.close()
    p.join()


ADJ_TOL = 1e-12          # the GPU adjoint's relative residual in these tests
EPS = 2.0 ** -52


def _check_grad(got, pair, label=""):
    """GPU gradient against the oracle's: within GRAD_TOL relative, or within the
    oracle's own spread between two sparse-LU orderings scaled from the direct
    solve's backward error (eps) to the GPU's (ADJ_TOL).  The spread is what the
    ill-conditioned adjoint systems make of a backward error of eps; to first
    order the forward error grows linearly with the backward error, and the GPU's
    Krylov solve stops at a relative residual of ADJ_TOL, not at eps (reading
    R10).  dL/dtheta sums per-step terms that cancel by two to three orders of
    magnitude, so it shows this first."""
    want, want2 = pair
    for k, name in enumerate(("dL/dx0", "dL/dv0", "dL/dtheta")):
        err = np.linalg.norm(np.ravel(got[k]) - np.ravel(want[k]))
        spread = np.linalg.norm(np.ravel(want2[k]) - np.ravel(want[k]))
        ref = np.linalg.norm(np.ravel(want[k]))
        print(f"{label} {name}: |GPU - oracle| / |oracle| = {err / ref:.2e}, oracle ordering spread "
              f"{spread / ref:.2e}, scaled to the GPU's residual {spread * ADJ_TOL / EPS / ref:.2e}")
        assert err <= max(GRAD_TOL * ref, spread * ADJ_TOL / EPS), (name, err / ref, spread / ref)


def test_batched_workload_solver1_parity(pool):
    seeds = (15, 21, 45)
    n_steps = 26
    scs = [scenes.batch_instance(s, n_steps=n_steps) for s in seeds]
    assert max(s.n for s in scs) > 60
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):       # the context's stream: capturable, unlike the legacy default one
        b = make_batch(scs, checkpoint_every=1, global_solver=1, adj_tol=ADJ_TOL)
        b.autotune()
        b.set_graphs(True)
    cat = lambda k: np.concatenate([getattr(s, k) for s in scs])
    with torch.cuda.stream(stream):
        xN, vN, tr = b.rollout(cuda(cat("x0")), cuda(cat("v0")), n_steps, traj=True)
        # the rollout replayed as a graph gives the same bits as the traced one
        xN2, vN2 = b.rollout(cuda(cat("x0")), cuda(cat("v0")), n_steps)
        dx0, dv0, dth = b.backward(cuda(cat("loss_w")), allow_nonconverged=True)
    torch.cuda.synchronize()
    assert torch.equal(xN, xN2) and torch.equal(vN, vN2)
    st = b.stats()
    assert st["graph_replays"] > 0 and st["global_solver"] == 1
    tr = tr.cpu().numpy()
    o = b.node_offsets
    specs = [("batch", s, ()) for s in seeds]
    trajs = [tr[:, o[i]:o[i + 1]] for i in range(len(seeds))]
    recs, grads = oracle_along(specs, trajs, [s.v0 for s in scs], scs[0].params.h, [s.loss_w for s in scs], pool,
                               second_ordering=True)
    n_contact = 0
    for i, sc in enumerate(scs):
        v = sc.v0
        for n in range(n_steps):
            rec = recs[i][n]
            assert rel_inf(trajs[i][n + 1], rec.x_np1) <= STATE_TOL, (seeds[i], n)
            v_gpu = (trajs[i][n + 1] - trajs[i][n]) / sc.params.h
            assert rel_inf(v_gpu, rec.v_np1) <= 1e-7, (seeds[i], n)   # v from differenced positions
            n_contact += len(rec.contacts)
        got = (dx0.cpu().numpy()[o[i]:o[i + 1]], dv0.cpu().numpy()[o[i]:o[i + 1]], dth.cpu().numpy()[i])
        _check_grad(got, grads[i], f"cloth {seeds[i]} (n = {sc.n})")
    assert n_contact > 1000
    print(f"contact node-steps {n_contact}; adjoint fallbacks {st['adj_fallbacks']}, "
          f"non-converged {st['adj_nonconverged']}")
    b.close()


def test_draped_61x61_checkpointed_gradient_parity(pool):
    """The draped cloth as configured: rollout_fn over 125 steps with checkpoints
    every 25; the gradient w.r.t. x0, v0 and (k_stretch, k_bend, mu) against the
    oracle's direct adjoint along the same 125 steps."""
    import torch

    import paper_2106_05306_gb300 as dc
    sc = scenes.draped_cloth()
    p = sc.params
    cloth = make_cloth(sc, checkpoint_every=25, adj_tol=ADJ_TOL)
    cloth.allow_nonconverged = True   # steps ended at their rounding floor are still compared below
    x0 = cuda(sc.x0).requires_grad_(True)
    v0 = cuda(sc.v0).requires_grad_(True)
    th = torch.tensor([p.k_stretch, p.k_bend, p.mu], dtype=torch.float64, requires_grad=True)
    xN, _ = dc.rollout_fn(cloth, x0, v0, th, sc.n_steps)
    L = (xN * cuda(sc.loss_w)).sum()
    gx0, gv0, gth = torch.autograd.grad(L, (x0, v0, th))
    st = cloth.stats()
    _, _, tr = cloth.rollout(cuda(sc.x0), cuda(sc.v0), sc.n_steps, traj=True)
    tr = tr.cpu().numpy()
    assert np.array_equal(tr[-1], xN.detach().cpu().numpy())
    cloth.close()
    recs, grads = oracle_along([("draped", 0, ())], [tr], [sc.v0], p.h, [sc.loss_w], pool, second_ordering=True)
    for n, rec in enumerate(recs[0]):
        assert rel_inf(tr[n + 1], rec.x_np1) <= STATE_TOL, n
    assert sum(len(r.contacts) for r in recs[0]) > 10000
    got = (gx0.cpu().numpy(), gv0.cpu().numpy(), gth.numpy())
    print(f"adjoint fallbacks {st['adj_fallbacks']}, non-converged {st['adj_nonconverged']}, |dL/dx0| "
          f"{np.linalg.norm(grads[0][0][0]):.3e}")
    _check_grad(got, grads[0], "draped 61x61")


def test_large_capsule_field_200x200(pool):
    """The large configuration: a 200x200 cloth (40,000 nodes, 120k DOF) dropped on
    8 capsules and the ground, mu 0.4, h = 1/240, checkpoints every 10 steps.  Its
    top fronts exceed one CTA's shared memory, so their factorisation level runs
    with the panel scratch in global memory.  Forward states for every step of a
    46-step prefix; the gradient over a 5-step window once the cloth touches the
    highest capsule (steps 46-50), against the oracle's direct adjoint."""
    import torch
    sc = scenes.capsule_field()
    h = sc.params.h
    cloth = make_cloth(sc, checkpoint_every=10, global_solver=1, adj_tol=ADJ_TOL)
    n0, n1 = 46, 5                 # the highest capsule is reached at about step 43
    _, _, tr = cloth.rollout(cuda(sc.x0), cuda(sc.v0), n0, traj=True)
    tr = tr.cpu().numpy()
    spec = ("capsules", 0, ())
    recs, _ = oracle_along([spec], [tr], [sc.v0], h, [None], pool, gradient=False)
    for n, rec in enumerate(recs[0]):
        assert rel_inf(tr[n + 1], rec.x_np1) <= STATE_TOL, n
    x0 = tr[n0]
    v0 = (tr[n0] - tr[n0 - 1]) / h
    _, _, tr2 = cloth.rollout(cuda(x0), cuda(v0), n1, traj=True)
    dx0, dv0, dth = cloth.backward(cuda(sc.loss_w), allow_nonconverged=True)
    st = cloth.stats()
    tr2 = tr2.cpu().numpy()
    recs2, grads = oracle_along([spec], [tr2], [v0], h, [sc.loss_w], pool, second_ordering=True)
    assert sum(len(r.contacts) for r in recs2[0]) > 0
    _check_grad((dx0.cpu().numpy(), dv0.cpu().numpy(), dth.cpu().numpy()), grads[0], "capsules 200x200")
    print(f"contact node-steps in the window {sum(len(r.contacts) for r in recs2[0])}; "
          f"fallbacks {st['adj_fallbacks']}, non-converged {st['adj_nonconverged']}")
    cloth.close()
