"""Triangle-mesh obstacles on the GPU (closest-triangle query, pseudo-normal sign,
per-region normal Jacobian) against the oracle, and the continuity study of
triangulated vs analytic obstacles (Sec. "Continuity and Smoothness"): sweeping
where a cloth lands, the adjoint gradient changes smoothly over an analytic
sphere and jumps over its triangulation, whose normal is discontinuous across
edges and whose curvature concentrates at edges and vertices."""
import numpy as np
import pytest

import scenes
from oracle import cloth as oc
from tests._helpers import GRAD_TOL, STATE_TOL, cuda, make_cloth, oracle_model, rel_inf, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sub,offset", [(1, 0.0), (1, 0.037), (2, 0.02)])
def test_mesh_obstacle_step_parity(sub, offset):
    sc = scenes.sphere_drop(offset, mesh_subdivisions=sub, n_steps=8)
    cloth = make_cloth(sc)
    M = oracle_model(sc)
    xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps)
    assert sum(len(r.contacts) for r in recs) > 0
    for n in range(sc.n_steps):
        x1, v1 = cloth.step(cuda(xs[n]), cuda(vs[n]))
        assert rel_inf(x1.cpu().numpy(), xs[n + 1]) <= STATE_TOL, n
        assert rel_inf(v1.cpu().numpy(), vs[n + 1]) <= STATE_TOL, n
    cloth.close()


def test_mesh_obstacle_gradient_parity():
    sc = scenes.sphere_drop(0.02, mesh_subdivisions=1, n_steps=8)
    cloth = make_cloth(sc, adj_tol=1e-12)
    M = oracle_model(sc)
    xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps)
    want = oc.rollout_gradient(M, recs, sc.loss_w)
    cloth.rollout(cuda(sc.x0), cuda(sc.v0), sc.n_steps)
    dx0, dv0, dth = cloth.backward(cuda(sc.loss_w))
    assert rel_l2(dx0.cpu().numpy(), want[0]) <= GRAD_TOL
    assert rel_l2(dv0.cpu().numpy(), want[1]) <= GRAD_TOL
    assert rel_l2(dth.cpu().numpy(), want[2]) <= GRAD_TOL
    cloth.close()


def _sweep(sub, offsets):
    """dL/d(offset) of L = mean final x over a sweep of landing offsets: the sum of
    the x components of dL/dx0 (all nodes move with the offset)."""
    g = []
    for d in offsets:
        sc = scenes.sphere_drop(float(d), mesh_subdivisions=sub, n_steps=8)
        cloth = make_cloth(sc, adj_tol=1e-12)
        w = np.zeros((sc.m, 3))
        w[:, 0] = 1.0 / sc.m
        cloth.rollout(cuda(sc.x0), cuda(sc.v0), sc.n_steps)
        dx0, _, _ = cloth.backward(cuda(w), allow_nonconverged=True)
        g.append(float(dx0[:, 0].sum()))
        cloth.close()
    return np.array(g)


def test_triangulated_obstacle_gradients_are_discontinuous():
    offsets = np.linspace(0.0, 0.12, 49)
    g_s = _sweep(-1, offsets)
    g_m = _sweep(1, offsets)
    js, jm = np.abs(np.diff(g_s)), np.abs(np.diff(g_m))
    print(f"total variation analytic {js.sum():.3g}, triangulated {jm.sum():.3g}; "
          f"median |jump| {np.median(js):.3g} / {np.median(jm):.3g}; max {js.max():.3g} / {jm.max():.3g}")
    assert jm.sum() > 10.0 * js.sum()
    # three points of the sweep against the oracle's adjoint
    for d in offsets[[5, 20, 40]]:
        sc = scenes.sphere_drop(float(d), mesh_subdivisions=1, n_steps=8)
        M = oracle_model(sc)
        xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps)
        w = np.zeros((sc.m, 3))
        w[:, 0] = 1.0 / sc.m
        gx, _, _ = oc.rollout_gradient(M, recs, w)
        k = int(np.argmin(np.abs(offsets - d)))
        assert abs(g_m[k] - gx[:, 0].sum()) <= GRAD_TOL * max(1.0, abs(gx[:, 0].sum()))


def test_mesh_registration_rejects_open_meshes():
    import paper_2106_05306_gb300 as dc
    sc = scenes.sphere_drop(0.0, mesh_subdivisions=1)
    ob = sc.obstacles[0]
    open_mesh = scenes.Obstacle("mesh", vertices=ob.vertices, triangles=ob.triangles[:-1])
    cloth = dc.Cloth(sc.rest_pos, sc.tris, sc.pins)
    with pytest.raises(dc.DCError, match="closed"):
        cloth.set_params(obstacles=[open_mesh])
    flipped = scenes.Obstacle("mesh", vertices=ob.vertices, triangles=np.concatenate(
        [ob.triangles[:1, ::-1], ob.triangles[1:]]))
    with pytest.raises(dc.DCError, match="closed"):
        cloth.set_params(obstacles=[flipped])
    cloth.close()
