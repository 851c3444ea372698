"""GPU batched path: cloths of different sizes, pins, materials and obstacles
packed into one context (dc_create_batch / dc_set_params_batch).  Every
instance must match the oracle (states 1e-9, gradients 1e-7) and be bitwise
identical to the same cloth run alone; CUDA graphs and the block-size
autotuner must not change a bit either."""
import numpy as np
import pytest

import scenes
from oracle import cloth as oc
from tests._helpers import (GRAD_TOL, STATE_TOL, cuda, make_batch, make_cloth, oracle_model, rel_inf,
                            rel_l2)

pytestmark = pytest.mark.gpu


def _mixed_scenes():
    a = scenes.small_scene(4, seed=1, contact="sphere", drop=True, pinned=True)
    b = scenes.small_scene(6, seed=2, contact="plane", drop=True, pinned=False)
    b.params.k_stretch = 300.0
    b.params.mu = 0.9
    c = scenes.small_scene(5, seed=3, contact="both", drop=True, pinned=True)
    c.params.k_bend = 3e-3
    c.params.density = 0.2
    d = scenes.small_scene(3, seed=4, contact="none", pinned=True)
    e = scenes.small_scene(5, seed=5, contact="capsule", drop=False, pinned=True)
    return [a, b, c, d, e]


def _cat(arrs):
    return cuda(np.concatenate([np.asarray(a) for a in arrs], axis=0))


def _run_batch(batch, scs, n_steps, gv_list):
    batch.rollout(_cat([s.x0 for s in scs]), _cat([s.v0 for s in scs]), n_steps)
    xN, vN = batch.rollout(_cat([s.x0 for s in scs]), _cat([s.v0 for s in scs]), n_steps)
    dx0, dv0, dth = batch.backward(_cat([s.loss_w for s in scs]), _cat(gv_list))
    return xN, vN, dx0, dv0, dth


def test_batch_forward_and_adjoint_match_oracle_and_alone():
    import torch
    scs = _mixed_scenes()
    n_steps = 3
    rng = np.random.default_rng(7)
    gvs = [0.3 * rng.standard_normal((s.m, 3)) for s in scs]
    batch = make_batch(scs, checkpoint_every=2)
    xN, vN, dx0, dv0, dth = _run_batch(batch, scs, n_steps, gvs)
    assert dth.shape == (len(scs), 3)
    parts = [batch.split(t) for t in (xN, vN, dx0, dv0)]
    st = batch.stats()
    assert st["n_instances"] == len(scs) and st["adj_nonconverged"] == 0
    batch.close()
    n_contacts = 0
    for i, sc in enumerate(scs):
        M = oracle_model(sc)
        xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, n_steps)
        n_contacts += sum(len(r.contacts) for r in recs)
        assert rel_inf(parts[0][i].cpu().numpy(), xs[-1]) <= STATE_TOL, i
        assert rel_inf(parts[1][i].cpu().numpy(), vs[-1]) <= STATE_TOL, i
        want = oc.rollout_gradient(M, recs, sc.loss_w, gvs[i])
        assert rel_l2(parts[2][i].cpu().numpy(), want[0]) <= GRAD_TOL, i
        assert rel_l2(parts[3][i].cpu().numpy(), want[1]) <= GRAD_TOL, i
        got = dth[i].cpu().numpy()
        scale = np.max(np.abs(want[2]))
        for q in range(3):
            assert abs(got[q] - want[2][q]) <= GRAD_TOL * max(abs(want[2][q]), 1e-6 * scale), (i, q, got, want[2])
        # the same cloth alone: bitwise the same numbers
        cl = make_cloth(sc, checkpoint_every=2)
        ax, av = cl.rollout(cuda(sc.x0), cuda(sc.v0), n_steps)
        adx, adv, ath = cl.backward(cuda(sc.loss_w), cuda(gvs[i]))
        cl.close()
        assert torch.equal(ax, parts[0][i]) and torch.equal(av, parts[1][i]), i
        assert torch.equal(adx, parts[2][i]) and torch.equal(adv, parts[3][i]), i
        assert torch.equal(ath, dth[i]), i
    assert n_contacts > 0


@pytest.mark.parametrize("solver", [0, 1])
def test_batch_graphs_and_autotune_change_no_bit(solver):
    import torch
    scs = _mixed_scenes()[:3]
    rng = np.random.default_rng(8)
    gvs = [0.3 * rng.standard_normal((s.m, 3)) for s in scs]
    ref = make_batch(scs, checkpoint_every=2, global_solver=solver)
    want = _run_batch(ref, scs, 5, gvs)
    ref.close()
    # graphs need a capturable (non-default) stream
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = make_batch(scs, checkpoint_every=2, global_solver=solver)
        b.set_graphs(True)
        b.autotune()
        got = _run_batch(b, scs, 5, gvs)
        got2 = _run_batch(b, scs, 5, gvs)      # replays the captured graphs
        st = b.stats()
        b.close()
    s.synchronize()
    assert st["graphs"] == 1 and st["graph_replays"] >= 4
    for k in ("block_local", "block_gather", "block_node", "block_elem"):
        assert st[k] in (64, 128, 256, 512)
    for a, b2, c in zip(want, got, got2):
        assert torch.equal(a, b2) and torch.equal(a, c)


def test_batch_of_workload_instances_forward():
    """Three members of the batched workload (grid 16..20), forward parity."""
    scs = [scenes.batch_instance(seed, n_lo=16, n_hi=20, n_steps=2) for seed in range(3)]
    batch = make_batch(scs)
    xN, vN = batch.rollout(_cat([s.x0 for s in scs]), _cat([s.v0 for s in scs]), 2)
    parts = batch.split(xN), batch.split(vN)
    batch.close()
    for i, sc in enumerate(scs):
        xs, vs, _ = oc.rollout(oracle_model(sc), sc.x0, sc.v0, 2)
        assert rel_inf(parts[0][i].cpu().numpy(), xs[-1]) <= STATE_TOL
        assert rel_inf(parts[1][i].cpu().numpy(), vs[-1]) <= STATE_TOL


def test_batch_parameter_checks():
    import paper_2106_05306_gb300 as dc
    from tests._helpers import params_kw
    scs = _mixed_scenes()[:2]
    batch = make_batch(scs)
    kws = [params_kw(s) for s in scs]
    kws[1]["h"] = 0.5 * kws[0]["h"]     # h is shared by a batch
    with pytest.raises(dc.DCError, match="DC_ERR_INVALID"):
        batch.set_params(kws)
    with pytest.raises(dc.DCError, match="DC_ERR_INVALID"):
        batch.set_params([params_kw(scs[0])] * 3)
    batch.close()


def test_batch_autograd_function_matches_backward():
    """rollout_fn over a ClothBatch: per-instance theta (B, 3) gets each instance's
    dL/d(k_stretch, k_bend, mu), equal to dc_backward's."""
    import torch
    import paper_2106_05306_gb300 as dc
    scs = _mixed_scenes()[:3]
    b = make_batch(scs, checkpoint_every=1)
    x0 = _cat([s.x0 for s in scs]).requires_grad_(True)
    v0 = _cat([s.v0 for s in scs]).requires_grad_(True)
    th = torch.tensor([[s.params.k_stretch, s.params.k_bend, s.params.mu] for s in scs], dtype=torch.float64,
                      requires_grad=True)
    xi = _cat([s.loss_w for s in scs])
    xN, vN = dc.rollout_fn(b, x0, v0, th, 3)
    gx0, gv0, gth = torch.autograd.grad((xN * xi).sum(), (x0, v0, th))
    b.rollout(x0.detach(), v0.detach(), 3)
    dx0, dv0, dth = b.backward(xi)
    b.close()
    assert torch.equal(gx0, dx0) and torch.equal(gv0, dv0) and torch.equal(gth, dth.cpu())
