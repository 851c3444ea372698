"""GPU request server (dc_server_*): requests of different sizes, step counts and
parameters are all submitted at once, so that most of them arrive while others
run.  Each result must be bitwise the result of the same request run alone, the
first ones must match the oracle, and the slot and HBM-budget bounds must hold."""
import numpy as np
import pytest

import scenes
from oracle import cloth as oc
from tests._helpers import GRAD_TOL, STATE_TOL, cuda, make_cloth, oracle_model, params_kw, rel_inf, rel_l2

pytestmark = pytest.mark.gpu


def _requests():
    out = []
    specs = [(4, 1, "sphere", True, True, 3), (6, 2, "plane", True, False, 4), (5, 3, "both", True, True, 2),
             (3, 4, "none", False, True, 5), (5, 5, "capsule", False, True, 3), (7, 6, "both", True, False, 2),
             (4, 7, "sphere", True, True, 4), (6, 8, "plane", True, True, 3)]
    for n, seed, contact, drop, pinned, steps in specs:
        sc = scenes.small_scene(n, seed=seed, contact=contact, drop=drop, pinned=pinned, n_steps=steps)
        sc.params.k_stretch *= 1.0 + 0.1 * seed
        gv = 0.3 * np.random.default_rng(seed).standard_normal((sc.m, 3))
        out.append((sc, gv, params_kw(sc, checkpoint_every=2)))
    return out


def _submit_all(srv, reqs):
    return [srv.submit(sc.rest_pos, sc.tris, sc.pins, sc.x0, sc.v0, sc.loss_w, sc.n_steps, kw, dL_dv=gv)
            for sc, gv, kw in reqs]


@pytest.mark.parametrize("max_batch", [1, 4])
def test_server_results_match_alone_and_oracle(max_batch):
    """max_batch 4: the requests submitted together are packed into batch contexts
    of up to four cloths with their own step counts; each result is still bitwise
    the request run alone."""
    import paper_2106_05306_gb300 as dc
    reqs = _requests()
    srv = dc.Server(n_slots=3, n_prep_threads=2, max_batch=max_batch)
    res = [srv.wait(t) for t in _submit_all(srv, reqs)]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert 1 <= st["peak_in_flight"] <= 3 * max_batch
    assert st["cloth_steps"] == sum(sc.n_steps for sc, _, _ in reqs)
    for i, ((sc, gv, kw), r) in enumerate(zip(reqs, res)):
        assert r["status"] == "DC_OK", r["message"]
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        assert r["device_bytes"] >= r["device_bytes_peak"] > 0, (r["device_bytes"], r["device_bytes_peak"])
        cl = make_cloth(sc, checkpoint_every=2)
        xN, vN = cl.rollout(cuda(sc.x0), cuda(sc.v0), sc.n_steps)
        dx0, dv0, dth = cl.backward(cuda(sc.loss_w), cuda(gv))
        cl.close()
        assert np.array_equal(r["x_final"], xN.cpu().numpy()), i
        assert np.array_equal(r["v_final"], vN.cpu().numpy()), i
        assert np.array_equal(r["dL_dx0"], dx0.cpu().numpy()), i
        assert np.array_equal(r["dL_dv0"], dv0.cpu().numpy()), i
        assert np.array_equal(r["dL_dparams"], dth.cpu().numpy()), i
        if i < 3:
            M = oracle_model(sc)
            xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps)
            assert rel_inf(r["x_final"], xs[-1]) <= STATE_TOL
            want = oc.rollout_gradient(M, recs, sc.loss_w, gv)
            assert rel_l2(r["dL_dx0"], want[0]) <= GRAD_TOL
            assert rel_l2(r["dL_dv0"], want[1]) <= GRAD_TOL


def test_server_hbm_budget_bounds_admission():
    import paper_2106_05306_gb300 as dc
    reqs = _requests()[:5]
    srv = dc.Server(n_slots=4, n_prep_threads=2)
    first = [srv.wait(t) for t in _submit_all(srv, reqs)]
    srv.close()
    sizes = [r["device_bytes"] for r in first]
    # room for the largest request plus a little: never two large ones at once
    budget = int(max(sizes) * 1.05)
    srv = dc.Server(n_slots=4, n_prep_threads=2, hbm_budget_bytes=budget)
    res = [srv.wait(t) for t in _submit_all(srv, reqs)]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs)
    assert st["peak_bytes_reserved"] <= budget
    for a, b in zip(first, res):
        assert np.array_equal(a["dL_dx0"], b["dL_dx0"]) and np.array_equal(a["x_final"], b["x_final"])
    # a request larger than the whole budget is refused
    srv = dc.Server(n_slots=1, n_prep_threads=1, hbm_budget_bytes=min(sizes) // 2)
    sc, gv, kw = reqs[0]
    r = srv.wait(srv.submit(sc.rest_pos, sc.tris, sc.pins, sc.x0, sc.v0, sc.loss_w, sc.n_steps, kw))
    srv.close()
    assert r["status"] == "DC_ERR_OOM" and r["slot"] == -1


@pytest.mark.parametrize("max_batch", [1, 4])
def test_server_bad_request_fails_alone(max_batch):
    """A request with an out-of-range triangle index fails with DC_ERR_INVALID; the
    requests around it (also those packed into the same batch) still finish with
    the same results as alone."""
    import paper_2106_05306_gb300 as dc
    reqs = _requests()[:3]
    srv = dc.Server(n_slots=2, n_prep_threads=2, max_batch=max_batch)
    t_ok1 = _submit_all(srv, reqs[:1])[0]
    sc, gv, kw = reqs[1]
    bad_tris = sc.tris.copy()
    bad_tris[0, 0] = sc.m + 5
    t_bad = srv.submit(sc.rest_pos, bad_tris, sc.pins, sc.x0, sc.v0, sc.loss_w, sc.n_steps, kw)
    t_ok2 = _submit_all(srv, reqs[2:3])[0]
    r1, rb, r2 = srv.wait(t_ok1), srv.wait(t_bad), srv.wait(t_ok2)
    st = srv.stats()
    srv.close()
    assert rb["status"] == "DC_ERR_INVALID" and rb["slot"] == -1, rb
    assert r1["status"] == "DC_OK" and r2["status"] == "DC_OK"
    assert st["failed"] == 1 and st["completed"] == 2
    for (sc, gv, kw), r in ((reqs[0], r1), (reqs[2], r2)):
        cl = make_cloth(sc, checkpoint_every=2)
        xN, _ = cl.rollout(cuda(sc.x0), cuda(sc.v0), sc.n_steps)
        dx0, _, _ = cl.backward(cuda(sc.loss_w), cuda(gv))
        cl.close()
        assert np.array_equal(r["x_final"], xN.cpu().numpy()) and np.array_equal(r["dL_dx0"], dx0.cpu().numpy())


def test_failing_request_does_not_fail_its_batch():
    """A request whose x0 holds a NaN fails its whole batch context (the forward's
    non-finite flag is per context); the server then runs that batch's requests
    again one per context, so only the bad request fails and the others are
    bitwise their alone results."""
    import paper_2106_05306_gb300 as dc
    reqs = _requests()[:4]
    bad_sc, bad_gv, bad_kw = reqs[0]
    x0_bad = bad_sc.x0.copy()
    x0_bad[1, 0] = np.nan
    srv = dc.Server(n_slots=1, n_prep_threads=1, max_batch=8)
    tickets = _submit_all(srv, reqs)
    t_bad = srv.submit(bad_sc.rest_pos, bad_sc.tris, bad_sc.pins, x0_bad, bad_sc.v0, bad_sc.loss_w, bad_sc.n_steps,
                       bad_kw, dL_dv=bad_gv)
    res = [srv.wait(t) for t in tickets]
    r_bad = srv.wait(t_bad)
    st = srv.stats()
    srv.close()
    assert r_bad["status"] == "DC_ERR_NONFINITE", r_bad["status"]
    assert st["batch_retries"] >= 1 and st["completed"] == len(reqs) and st["failed"] == 1
    for i, ((sc, gv, kw), r) in enumerate(zip(reqs, res)):
        assert r["status"] == "DC_OK", (i, r["status"], r["message"])
        cl = make_cloth(sc, checkpoint_every=2)
        xN, vN = cl.rollout(cuda(sc.x0), cuda(sc.v0), sc.n_steps)
        dx0, dv0, dth = cl.backward(cuda(sc.loss_w), cuda(gv))
        cl.close()
        assert np.array_equal(r["x_final"], xN.cpu().numpy()), i
        assert np.array_equal(r["dL_dx0"], dx0.cpu().numpy()), i
        assert np.array_equal(r["dL_dparams"], dth.cpu().numpy()), i
