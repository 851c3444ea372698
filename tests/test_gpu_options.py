"""GPU tests of the boundary's options and error paths: the contact-compliance
choices (parity with the oracle, the printed mass splitting's divergence), the
component-major node layout, host-injected non-finite input, the adjoint
fallback and DC_ERR_NONCONVERGED, DC_ERR_NOT_SPD, and dc_batch_hbm_bytes against
the device memory a context actually held.  Every failure here is made on the
host (a parameter, an input array); none faults the GPU."""
import dataclasses

import numpy as np
import pytest

import scenes
from oracle import cloth as oc
from tests._helpers import GRAD_TOL, STATE_TOL, cuda, make_batch, make_cloth, oracle_model, rel_inf, rel_l2

pytestmark = pytest.mark.gpu


def _soft(sc, ks=0.15):
    return dataclasses.replace(sc, params=dataclasses.replace(sc.params, k_stretch=ks, k_bend=1e-7))


@pytest.mark.parametrize("mode,soft", [("diag_pinv", False), ("diag_p", False), ("diag_pinv", True),
                                       ("diag_p", True), ("mass", True), ("rowsum", True)])
def test_compliance_choices_match_the_oracle(mode, soft):
    """Each step from the oracle's state, K = 20 iterations, both sides with the
    same compliance choice (reading R5 and its ablations)."""
    sc = scenes.small_scene(5, seed=3, contact="both", drop=True, n_steps=3)
    if soft:
        sc = _soft(sc)
    for solver in (0, 1):
        cloth = make_cloth(sc, contact_compliance=mode, global_solver=solver)
        M = oracle_model(sc, contact_compliance=mode)
        xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps)
        assert sum(len(r.contacts) for r in recs) > 0
        for n in range(sc.n_steps):
            x1, v1 = cloth.step(cuda(xs[n]), cuda(vs[n]))
            assert rel_inf(x1.cpu().numpy(), xs[n + 1]) <= STATE_TOL
            assert rel_inf(v1.cpu().numpy(), vs[n + 1]) <= STATE_TOL, (mode, solver, n)
        assert cloth.stats()["contact_compliance"] == oc_mode_code(mode)
        cloth.close()


def oc_mode_code(mode):
    return {"rowsum": 0, "diag_pinv": 1, "diag_p": 2, "mass": 3}[mode]


def test_mass_splitting_diverges_at_cloth_stiffness():
    """The printed splitting at the hanging cloth's stiffness: the states blow up
    and the forward step reports DC_ERR_NONFINITE once they overflow."""
    import paper_2106_05306_gb300 as dc
    sc = scenes.hanging_cloth()
    cloth = make_cloth(sc, contact_compliance="mass")
    x, v = sc.x0.copy(), sc.v0.copy()
    x1, v1 = cloth.step(x, v)                     # host arrays: synchronous, flags checked
    assert np.max(np.abs(v1.numpy())) > 1e20
    with pytest.raises(dc.DCError, match="DC_ERR_NONFINITE"):
        for _ in range(20):
            x, v = cloth.step(x, v)
            x, v = x.numpy(), v.numpy()
    cloth.close()


def test_component_major_layout_gives_the_same_numbers():
    """A batch with [3][m] node arrays: rollout (with trajectory), backward (with a
    per-step loss) and the global solve are the transposes of the [m][3] results,
    bit for bit (the layout only changes the boundary permutation)."""
    import torch
    scs = [scenes.small_scene(5, seed=3, contact="both", drop=True, n_steps=4),
           scenes.small_scene(4, seed=1, contact="sphere", drop=True, n_steps=4)]
    n = 4
    res = {}
    for layout in ("node_major", "component_major"):
        b = make_batch(scs, checkpoint_every=2)
        b.set_layout(layout)
        cat = lambda k: np.concatenate([getattr(s, k) for s in scs])
        x0, v0, xi = cat("x0"), cat("v0"), cat("loss_w")
        rng = np.random.default_rng(3)
        gT = 0.1 * rng.standard_normal((n + 1, b.m, 3))
        if layout == "component_major":
            x0, v0, xi = x0.T.copy(), v0.T.copy(), xi.T.copy()
            gT = gT.transpose(0, 2, 1).copy()
        xN, vN, tr = b.rollout(cuda(x0), cuda(v0), n, traj=True)
        dx0, dv0, dth = b.backward(cuda(xi), None, cuda(gT))
        sol = b.global_solve(cuda(x0))
        out = [xN, vN, dx0, dv0, sol]
        if layout == "component_major":
            out = [a.t() for a in out]
            tr = tr.transpose(1, 2)
        res[layout] = [a.cpu() for a in out] + [tr.cpu(), dth.cpu()]
        b.close()
    for a, c in zip(res["node_major"], res["component_major"]):
        assert torch.equal(a.contiguous(), c.contiguous())


def test_nan_input_is_reported_once():
    import paper_2106_05306_gb300 as dc
    sc = scenes.small_scene(4, seed=2, contact="plane", drop=True)
    cloth = make_cloth(sc)
    x = sc.x0.copy()
    x[5, 1] = np.nan
    with pytest.raises(dc.DCError, match="DC_ERR_NONFINITE"):
        cloth.step(x, sc.v0)                      # host arrays: the call synchronises and reports
    x1, v1 = cloth.step(sc.x0, sc.v0)             # reported once; a finite step is fine again
    assert np.all(np.isfinite(x1.numpy()))
    xd = cuda(x)
    cloth.rollout(xd, cuda(sc.v0), 2)             # device arrays: asynchronous, reported at the next sync
    with pytest.raises(dc.DCError, match="DC_ERR_NONFINITE"):
        cloth.sync()
    cloth.close()


def test_adjoint_fallback_and_nonconverged():
    """adj_max_iters = 1 stops every adjoint step far above adj_tol.  With the
    fallback off, dc_backward reports DC_ERR_NONCONVERGED (after writing its
    outputs); with it on, the fallback pass finishes each step and the gradient
    matches the oracle's direct adjoint."""
    import paper_2106_05306_gb300 as dc
    sc = scenes.small_scene(5, seed=3, contact="both", drop=True, n_steps=3)
    M = oracle_model(sc)
    xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps)
    want = oc.rollout_gradient(M, recs, sc.loss_w)
    off = make_cloth(sc, adj_max_iters=1, adj_fallback=0)
    off.rollout(cuda(sc.x0), cuda(sc.v0), sc.n_steps)
    with pytest.raises(dc.DCError, match="DC_ERR_NONCONVERGED"):
        off.backward(cuda(sc.loss_w))
    st = off.stats()
    assert st["adj_nonconverged"] == sc.n_steps and st["adj_fallbacks"] == 0
    off.close()
    for solver in (0, 1):
        on = make_cloth(sc, adj_max_iters=1, adj_fallback=1, global_solver=solver)
        on.rollout(cuda(sc.x0), cuda(sc.v0), sc.n_steps)
        dx0, dv0, dth = on.backward(cuda(sc.loss_w))
        st = on.stats()
        assert st["adj_fallbacks"] == sc.n_steps and st["adj_nonconverged"] == 0
        assert rel_l2(dx0.cpu().numpy(), want[0]) <= GRAD_TOL
        assert rel_l2(dv0.cpu().numpy(), want[1]) <= GRAD_TOL
        assert rel_l2(dth.cpu().numpy(), want[2]) <= GRAD_TOL
        on.close()


def test_nonconverged_counts_per_instance():
    """dc_get_instance_nonconverged: with adj_max_iters = 1 and the fallback off,
    every adjoint step an instance takes stops above adj_tol, and the steps past
    an instance's own count (its adjoint passes through) are not counted."""
    import paper_2106_05306_gb300 as dc
    scs = [scenes.small_scene(5, seed=3, contact="both", drop=True), scenes.small_scene(4, seed=1, contact="sphere",
                                                                                        drop=True),
           scenes.small_scene(5, seed=2, contact="plane", drop=True)]
    steps = [3, 1, 2]
    b = make_batch(scs, adj_max_iters=1, adj_fallback=0)
    b.set_instance_steps(steps)
    cat = lambda k: np.concatenate([getattr(s, k) for s in scs])
    b.rollout(cuda(cat("x0")), cuda(cat("v0")), max(steps))
    with pytest.raises(dc.DCError, match="DC_ERR_NONCONVERGED"):
        b.backward(cuda(cat("loss_w")))
    assert list(b.instance_nonconverged()) == steps
    assert b.stats()["adj_nonconverged"] == sum(steps)
    b.close()


def test_underflowing_mass_is_not_spd():
    """A density so small that the lumped masses underflow to 0, with no stiffness:
    P = M has a zero pivot, which the factorisation reports."""
    import paper_2106_05306_gb300 as dc
    sc = scenes.small_scene(4, seed=1)
    cloth = dc.Cloth(sc.rest_pos, sc.tris, sc.pins)
    with pytest.raises(dc.DCError, match="DC_ERR_NOT_SPD"):
        cloth.set_params(density=5e-324, k_stretch=0.0, k_bend=0.0)
    cloth.set_params()                            # the context is still usable
    cloth.close()


def test_batch_hbm_bytes_bounds_the_memory_held():
    """dc_batch_hbm_bytes is an upper bound of what the context holds through the
    rollout and backward it was asked about, and not far above it."""
    import paper_2106_05306_gb300 as dc
    scs = [scenes.batch_instance(s, n_steps=6) for s in (3, 4, 5)]
    kw = [dict(k_stretch=s.params.k_stretch, k_bend=s.params.k_bend, mu=s.params.mu, obstacles=s.obstacles,
               checkpoint_every=2, global_solver=1) for s in scs]
    est = dc.batch_hbm_bytes([(s.rest_pos, s.tris, s.pins) for s in scs], kw, 6)
    b = dc.ClothBatch([(s.rest_pos, s.tris, s.pins) for s in scs])
    b.set_params(kw)
    cat = lambda k: np.concatenate([getattr(s, k) for s in scs])
    b.rollout(cuda(cat("x0")), cuda(cat("v0")), 6)
    b.backward(cuda(cat("loss_w")), allow_nonconverged=True)
    peak = b.stats()["device_bytes_peak"]
    b.close()
    assert peak <= est <= 1.5 * peak, (peak, est)


@pytest.mark.parametrize("which", ["hanging_16x16", "draped_61x61", "batch_3", "capsules_200x200"])
def test_gpu_factorisation_of_P_matches_the_host_factor(which):
    """factor_on_gpu: P's numeric Cholesky on the GPU (multifrontal, FP64, into the
    supernodal panels) solves the global step like the host factor and like the
    oracle's banded Cholesky to 2e-11 (two factorisations in different orders
    differ by about cond(P) eps, and cond(P) reaches 1e5 here); a short rollout and
    its gradient agree with the host-factor context to 1e-9 / 1e-7 (gradients
    below 1e-9 in absolute value, such as that of the bending stiffness of a
    cloth still in free fall, are rounding and compared absolutely)."""
    import time

    import torch
    if which == "batch_3":
        scs = [scenes.batch_instance(s, n_steps=4) for s in (3, 15, 21)]
    else:
        scs = [{"hanging_16x16": scenes.hanging_cloth, "draped_61x61": scenes.draped_cloth,
                "capsules_200x200": scenes.capsule_field}[which]()]
    ctx, secs = [], []
    for gpu in (0, 1):
        t0 = time.perf_counter()
        b = make_batch(scs, global_solver=1, factor_on_gpu=gpu, checkpoint_every=2)
        torch.cuda.synchronize()
        secs.append(time.perf_counter() - t0)
        ctx.append(b)
    print(f"{which}: context + parameters with the host factor {secs[0]:.2f} s, GPU factor {secs[1]:.2f} s")
    rhs = cuda(np.random.default_rng(5).standard_normal((ctx[0].m, 3)))
    a, g = ctx[0].global_solve(rhs), ctx[1].global_solve(rhs)
    assert rel_inf(g.cpu().numpy(), a.cpu().numpy()) <= 2e-11
    if which == "draped_61x61":
        M = oracle_model(scs[0])
        want = np.zeros((scs[0].m, 3))
        want[M.free] = M.solve_P(rhs.cpu().numpy()[M.free])
        assert rel_inf(g.cpu().numpy(), want) <= 2e-11
    if which != "capsules_200x200":
        cat = lambda k: np.concatenate([getattr(s, k) for s in scs])
        outs = []
        for b in ctx:
            xN, vN = b.rollout(cuda(cat("x0")), cuda(cat("v0")), 4)
            outs.append((xN.cpu().numpy(), vN.cpu().numpy()) + tuple(
                t.cpu().numpy() for t in b.backward(cuda(cat("loss_w")), allow_nonconverged=True)))
        for k in range(2):
            assert rel_inf(outs[1][k], outs[0][k]) <= STATE_TOL
        for k in range(2, 5):
            d = np.linalg.norm(np.ravel(outs[1][k] - outs[0][k]))
            assert d <= GRAD_TOL * np.linalg.norm(np.ravel(outs[0][k])) + 1e-9, (k, d)
    for b in ctx:
        b.close()


def test_gpu_factorisation_reports_a_non_positive_pivot():
    import paper_2106_05306_gb300 as dc
    sc = scenes.small_scene(4, seed=1)
    cloth = dc.Cloth(sc.rest_pos, sc.tris, sc.pins)
    with pytest.raises(dc.DCError, match="DC_ERR_NOT_SPD"):
        cloth.set_params(density=5e-324, k_stretch=0.0, k_bend=0.0, global_solver=1, factor_on_gpu=1)
    cloth.set_params(global_solver=1, factor_on_gpu=1)
    cloth.close()


@pytest.mark.parametrize("ck", [1, 2])
def test_instances_of_different_lengths_in_one_batch(ck):
    """dc_set_instance_steps: each instance of a batch takes its own number of steps
    (then keeps its state, and its adjoint passes through the remaining steps):
    every output is bitwise that of the instance rolled out alone for its steps."""
    import torch
    scs = [scenes.small_scene(5, seed=3, contact="both", drop=True), scenes.small_scene(4, seed=1, contact="sphere",
                                                                                      drop=True),
           scenes.small_scene(5, seed=2, contact="plane", drop=True)]
    steps = [3, 6, 4]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = make_batch(scs, checkpoint_every=ck)
        b.set_graphs(True)
        b.set_instance_steps(steps)
        cat = lambda k: np.concatenate([getattr(s, k) for s in scs])
        xN, vN = b.rollout(cuda(cat("x0")), cuda(cat("v0")), max(steps))
        dx0, dv0, dth = b.backward(cuda(cat("loss_w")))
    torch.cuda.synchronize()
    o = b.node_offsets
    for i, (sc, n) in enumerate(zip(scs, steps)):
        c = make_cloth(sc, checkpoint_every=ck)
        x1, v1 = c.rollout(cuda(sc.x0), cuda(sc.v0), n)
        g = c.backward(cuda(sc.loss_w))
        sl = slice(int(o[i]), int(o[i + 1]))
        assert torch.equal(xN[sl], x1) and torch.equal(vN[sl], v1)
        assert torch.equal(dx0[sl], g[0]) and torch.equal(dv0[sl], g[1]) and torch.equal(dth[i], g[2])
        c.close()
    b.close()
