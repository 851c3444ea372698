"""GPU parity of the supernodal substitution of P (global_solver = 1): the
global solve against the oracle's banded Cholesky, forward steps and adjoint
gradients against the oracle, a batch against the same cloths alone (bitwise),
the tree-scheduled sweeps against one launch per level (bitwise), and the
allocation-free entry point against dc_global_solve."""
import numpy as np
import pytest

import scenes
from oracle import cloth as oc
from tests._helpers import (GRAD_TOL, STATE_TOL, cuda, make_batch, make_cloth, oracle_model, rel_inf,
                            rel_l2)

pytestmark = pytest.mark.gpu


def test_supernodal_global_solve_matches_banded_cholesky():
    import torch
    for sc in (scenes.small_scene(5, seed=1), scenes.hanging_cloth(), scenes.draped_cloth(),
               scenes.batch_instance(15)):
        cloth = make_cloth(sc, global_solver=1)
        assert cloth.stats()["global_solver"] == 1 and cloth.stats()["psolve_flops"] > 0
        M = oracle_model(sc)
        rng = np.random.default_rng(3)
        rhs = rng.standard_normal((sc.m, 3))
        got = cloth.global_solve(cuda(rhs)).cpu().numpy()
        want = np.zeros_like(rhs)
        want[M.free] = M.solve_P(rhs[M.free])
        assert rel_inf(got, want) < 1e-11
        assert np.all(got[M.pins] == 0.0)
        dst = torch.empty((sc.m, 3), dtype=torch.float64, device="cuda")
        assert cloth._lib.dc_global_solve_static(cloth._ctx, cuda(rhs).data_ptr(), dst.data_ptr()) == 0
        torch.cuda.synchronize()
        assert torch.equal(dst, torch.tensor(got, device="cuda"))
        cloth.close()


@pytest.mark.parametrize("contact,drop,pinned", [("sphere", True, True), ("both", True, False),
                                                 ("capsule", False, True)])
def test_supernodal_rollout_and_adjoint_parity(contact, drop, pinned):
    sc = scenes.small_scene(6, seed=5, contact=contact, drop=drop, pinned=pinned, n_steps=4)
    M = oracle_model(sc)
    xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps)
    gv = 0.3 * np.random.default_rng(2).standard_normal((sc.m, 3))
    want = oc.rollout_gradient(M, recs, sc.loss_w, gv)
    for ck in (1, 3):
        cloth = make_cloth(sc, global_solver=1, checkpoint_every=ck)
        xN, vN = cloth.rollout(cuda(sc.x0), cuda(sc.v0), sc.n_steps)
        assert rel_inf(xN.cpu().numpy(), xs[-1]) <= STATE_TOL
        assert rel_inf(vN.cpu().numpy(), vs[-1]) <= STATE_TOL
        dx0, dv0, dth = cloth.backward(cuda(sc.loss_w), cuda(gv))
        cloth.close()
        assert rel_l2(dx0.cpu().numpy(), want[0]) <= GRAD_TOL
        assert rel_l2(dv0.cpu().numpy(), want[1]) <= GRAD_TOL
        scale = np.max(np.abs(want[2]))
        for q in range(3):
            assert abs(dth[q].item() - want[2][q]) <= GRAD_TOL * max(abs(want[2][q]), 1e-6 * scale)


def test_supernodal_batch_is_bitwise_the_cloths_alone():
    import torch
    scs = [scenes.small_scene(4, seed=1, contact="sphere", drop=True),
           scenes.small_scene(7, seed=2, contact="plane", drop=True, pinned=False),
           scenes.small_scene(5, seed=3, contact="both", drop=True)]
    cat = lambda k: cuda(np.concatenate([getattr(s, k) for s in scs]))
    b = make_batch(scs, global_solver=1, checkpoint_every=1)
    xN, vN = b.rollout(cat("x0"), cat("v0"), 3)
    dx0, dv0, dth = b.backward(cat("loss_w"))
    parts = [b.split(t) for t in (xN, vN, dx0, dv0)]
    b.close()
    for i, sc in enumerate(scs):
        cl = make_cloth(sc, global_solver=1, checkpoint_every=1)
        ax, av = cl.rollout(cuda(sc.x0), cuda(sc.v0), 3)
        adx, adv, ath = cl.backward(cuda(sc.loss_w))
        cl.close()
        for a, p in zip((ax, av, adx, adv), (q[i] for q in parts)):
            assert torch.equal(a, p), i
        assert torch.equal(ath, dth[i])


def test_supernodal_tree_schedule_is_bitwise_the_level_launches(monkeypatch):
    """One launch per sweep, fronts taken in dependency order by whichever CTA is
    free, gives the bits of one launch per tree level: a front's arithmetic does
    not depend on when or where it runs.  This holds for the supernodal sweeps of
    the forward step and for the multifrontal solves of the adjoint's
    preconditioner (the gradients).  Cloths of 35-49 nodes a side have fronts on
    both the CTA path and the warp path."""
    import torch
    scs = [scenes.batch_instance(s, n_steps=3) for s in (0, 1, 2, 5)]
    assert max(sc.n for sc in scs) >= 40
    cat = lambda k: cuda(np.concatenate([getattr(s, k) for s in scs]))
    runs = []
    for levels in (True, False):
        if levels:
            monkeypatch.setenv("DC_LEVEL_SOLVES", "1")
        else:
            monkeypatch.delenv("DC_LEVEL_SOLVES", raising=False)
        b = make_batch(scs, global_solver=1, checkpoint_every=1)
        xN, vN = b.rollout(cat("x0"), cat("v0"), 3)
        dx0, dv0, dth = b.backward(cat("loss_w"), allow_nonconverged=True)
        rhs = cuda(np.random.default_rng(9).standard_normal((sum(sc.m for sc in scs), 3)))
        sol = b.global_solve(rhs)
        b.stats()   # raises if a dependency wait of a sweep gave up
        b.close()
        runs.append((xN, vN, dx0, dv0, dth, sol))
    for a, c in zip(*runs):
        assert torch.equal(a, c)


def test_supernodal_rejects_block_preconditioner():
    import paper_2106_05306_gb300 as dc
    sc = scenes.small_scene(4, seed=1)
    with pytest.raises(dc.DCError, match="DC_ERR_INVALID"):
        make_cloth(sc, global_solver=1, adj_precond=1)


def test_supernodal_sweep_wait_gives_up_and_reports():
    """A sweep started past its first work item leaves a parent waiting for a child
    that never runs (a flag that nothing sets): the bounded wait gives up after
    about a second, the context reports DC_ERR_TIMEOUT from then on, and the GPU
    stays usable for a new context."""
    import time

    import paper_2106_05306_gb300 as dc
    from paper_2106_05306_gb300._lib import check
    sc = scenes.batch_instance(0, n_steps=2)     # 43 x 43 nodes: a 9-level tree
    cloth = make_cloth(sc, global_solver=1)
    with pytest.raises(dc.DCError, match="DC_ERR_INVALID"):
        check(cloth._lib.dc_debug_sweep_wait_timeout(cloth._ctx, 0), cloth._ctx)
    t0 = time.perf_counter()
    st = cloth._lib.dc_debug_sweep_wait_timeout(cloth._ctx, 1)
    elapsed = time.perf_counter() - t0
    with pytest.raises(dc.DCError, match="DC_ERR_TIMEOUT.*gave up"):
        check(st, cloth._ctx)
    assert elapsed < 60.0
    with pytest.raises(dc.DCError, match="DC_ERR_TIMEOUT"):
        cloth.stats()
    with pytest.raises(dc.DCError, match="DC_ERR_TIMEOUT"):
        cloth.sync()
    cloth.close()
    fresh = make_cloth(sc, global_solver=1)
    M = oracle_model(sc)
    rhs = np.random.default_rng(4).standard_normal((sc.m, 3))
    got = fresh.global_solve(cuda(rhs)).cpu().numpy()
    want = np.zeros_like(rhs)
    want[M.free] = M.solve_P(rhs[M.free])
    assert rel_inf(got, want) < 1e-11
    fresh.stats()
    fresh.close()


def test_fused_sweeps_are_bitwise_the_two_launches():
    """Both substitution sweeps of a global step in one tree-scheduled launch (the
    default) give the same bits as the forward and backward sweeps launched one
    after the other (DC_SEPARATE_SWEEPS=1), for a rollout and its gradient."""
    import os

    import torch
    scs = [scenes.batch_instance(s, n_steps=3) for s in (3, 15)]
    for sc in scs:
        sc.x0 = sc.x0 - np.array([0.0, 0.3, 0.0])   # start near the sphere: contacts in three steps
    out = []
    for separate in (False, True):
        if separate:
            os.environ["DC_SEPARATE_SWEEPS"] = "1"
        try:
            b = make_batch(scs, global_solver=1, checkpoint_every=1)
        finally:
            os.environ.pop("DC_SEPARATE_SWEEPS", None)
        cat = lambda k: np.concatenate([getattr(s, k) for s in scs])
        xN, vN = b.rollout(cuda(cat("x0")), cuda(cat("v0")), 3)
        g = b.backward(cuda(cat("loss_w")), allow_nonconverged=True)
        st = b.stats()
        out.append((xN, vN) + tuple(g))
        b.close()
    assert st["contacts_stick"] + st["contacts_slip"] > 0
    for a, c in zip(out[0], out[1]):
        assert torch.equal(a, c)
