"""Pins for the CPU oracle: each test checks it against something other than itself
(closed forms, invariants the paper states, library routines, finite differences).
"""
import dataclasses

import numpy as np
import pytest

import scenes
from oracle import cloth as oc


def _model(pos, tris, pins=(), obst=(), **kw):
    prm = dataclasses.replace(scenes.Params(), **kw)
    return oc.Model(pos, tris, list(pins), list(obst), prm)


# --------------------------------------------------------------------- local step

def test_polar_matches_svd():
    """Closed-form 2x2 polar factor = U V^T of the SVD (the closest matrix with
    orthonormal columns, reading R1)."""
    rng = np.random.default_rng(0)
    F = rng.standard_normal((200, 3, 2))
    R, S = oc.polar(F)
    U, _, Vt = np.linalg.svd(F, full_matrices=False)
    np.testing.assert_allclose(R, U @ Vt, atol=1e-12)
    np.testing.assert_allclose(np.einsum("tck,tcl->tkl", R, R), np.broadcast_to(np.eye(2), (200, 2, 2)), atol=1e-12)
    np.testing.assert_allclose(np.einsum("tck,tkl->tcl", R, S), F, atol=1e-12)


def test_polar_derivative_matches_fd():
    rng = np.random.default_rng(1)
    for _ in range(20):
        F = rng.standard_normal((3, 2))
        dF = rng.standard_normal((3, 2))
        R, S = oc.polar(F[None])
        dR = oc.polar_derivative(R[0], S[0], dF)
        e = 1e-6
        Rp, _ = oc.polar((F + e * dF)[None])
        Rm, _ = oc.polar((F - e * dF)[None])
        np.testing.assert_allclose(dR, (Rp[0] - Rm[0]) / (2 * e), atol=1e-8)


def test_cotan_laplacian_on_grid_is_five_point_stencil():
    """On the split regular grid the cotangent weights are 1 on axis edges and 0 on
    diagonals, so A_b is the textbook 5-point Laplacian / a^2 in the interior."""
    n, side = 6, 0.5
    a = side / (n - 1)
    pos, tris = scenes.grid_mesh(n, side=side)
    G, area = oc.triangle_rest(pos, tris)
    Lb, abar = oc.cotan_laplacian(pos, tris, area)
    np.testing.assert_allclose(area, a * a / 2)
    assert abs(abar.sum() - side * side) < 1e-14
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            b = j * n + i
            row = Lb[b].toarray().ravel() * a * a
            expect = np.zeros(n * n)
            expect[b] = -4
            for nb in (b - 1, b + 1, b - n, b + n):
                expect[nb] = 1
            np.testing.assert_allclose(row, expect, atol=1e-12)


def test_mass_and_translation_kernel():
    """Total lumped mass = density * area (R3); rigid translations lie in the kernel of
    every A_i, so P t = M t for a translation t (Eq. pd_global)."""
    pos, tris = scenes.grid_mesh(7, side=0.8)
    M = _model(pos, tris, density=0.3)
    assert abs(M.mass.sum() - 0.3 * 0.64) < 1e-14
    t = np.ones(M.m)
    np.testing.assert_allclose(M.P @ t, M.mass, rtol=1e-11, atol=1e-14)


def test_banded_cholesky_solve_residual():
    sc = scenes.hanging_cloth()
    M = oc.model_from_scene(sc)
    rng = np.random.default_rng(2)
    b = rng.standard_normal((len(M.free), 3))
    x = M.solve_P(b)
    r = M.Pff @ x - b
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-13


# --------------------------------------------------------------------- forward step

def test_free_fall_is_exact():
    """No contact: translation is in the kernel of every A_i, so v_{n+1} = v_n + h g."""
    pos, tris = scenes.grid_mesh(5, side=0.4, height=1.0)
    M = _model(pos, tris)
    v0 = np.tile([0.3, -0.2, 0.1], (M.m, 1))
    x1, v1, _ = oc.step(M, pos, v0, n_iters=20)
    np.testing.assert_allclose(v1, v0 + M.h * M.g, rtol=0, atol=1e-13)
    np.testing.assert_allclose(x1, pos + M.h * v1, rtol=0, atol=1e-15)


def test_rigid_rest_state_stays_at_rest():
    pos, tris = scenes.grid_mesh(5, side=0.4, height=1.0)
    M = _model(pos, tris, gravity=(0.0, 0.0, 0.0), k_bend=1e-2)
    th = 0.7
    Rz = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    x0 = pos @ Rz.T + np.array([0.3, -0.1, 0.2])
    x1, v1, _ = oc.step(M, x0, np.zeros_like(pos), n_iters=20)
    assert np.max(np.abs(v1)) < 1e-12


def test_surrogate_energy_decreases_monotonically():
    """Alternating local and global steps never increases g~ (Sec. 3.1)."""
    sc = scenes.small_scene(5, seed=3, contact="none", pinned=True)
    M = oc.model_from_scene(sc)
    tr = []
    oc.step(M, sc.x0, sc.v0, n_iters=40, trace=tr)
    d = np.diff(np.asarray(tr))
    assert np.all(d <= 1e-14 * np.abs(np.asarray(tr[:-1])))


def _energy_svd(M, x):
    """W(x) evaluated independently of the oracle's projections: stretch from the
    singular values (distance to orthonormal columns), bending from |q|."""
    F = M.deformation_gradients(x)
    sig = np.linalg.svd(F, compute_uv=False)
    ws = 0.5 * np.sum(M.w_t * np.sum((sig - 1.0) ** 2, axis=1))
    q = M.Lb @ x
    nq = np.linalg.norm(q, axis=1)
    wb = 0.5 * np.sum(M.w_b * (nq - M.s_b) ** 2)
    return ws + wb


def test_converged_pd_solves_implicit_euler():
    """At convergence the PD iterate is a stationary point of g (Eq. implicit_energy):
    M (x - y)/h^2 + grad W(x) = 0, grad W by central differences of an SVD energy."""
    sc = scenes.small_scene(3, seed=4, contact="none", pinned=True)
    M = oc.model_from_scene(sc)
    x1, v1, _ = oc.step(M, sc.x0, sc.v0, tol=1e-15, max_iters=20000)
    y = sc.x0 + M.h * np.where(M.is_pin[:, None], 0.0, sc.v0) + M.h ** 2 * M.g
    grad = np.zeros_like(x1)
    e = 1e-7
    for j in M.free:
        for c in range(3):
            xp = x1.copy(); xp[j, c] += e
            xm = x1.copy(); xm[j, c] -= e
            grad[j, c] = (_energy_svd(M, xp) - _energy_svd(M, xm)) / (2 * e)
    res = M.mass[:, None] * (x1 - y) / M.h ** 2 + grad
    scale = np.max(np.abs(M.mass[:, None] * (x1 - y) / M.h ** 2))
    assert np.max(np.abs(res[M.free])) < 1e-6 * scale


# --------------------------------------------------------------------- contact

def _check_contact_law(M, rec, tol=1e-12):
    for a, j in enumerate(rec.contacts.nodes):
        n = rec.contacts.normals[a]
        f = rec.forces[a]
        v = rec.v_np1[j]
        fN = np.dot(f, n)
        fT = f - fN * n
        uN = np.dot(n, v) + rec.contacts.betas[a]
        uT = v - np.dot(n, v) * n
        scale = max(1.0, np.linalg.norm(f))
        vs = max(1.0, np.linalg.norm(v))
        case = rec.cases[a]
        assert fN >= -tol * scale
        assert np.linalg.norm(fT) <= M.mu * fN + tol * scale
        if case == oc.TAKEOFF:
            assert np.linalg.norm(f) == 0.0 and uN >= -tol * vs
        elif case == oc.STICK:
            assert abs(uN) <= tol * vs and np.linalg.norm(uT) <= tol * vs
        else:
            assert abs(uN) <= tol * vs
            assert abs(np.linalg.norm(fT) - M.mu * fN) <= tol * scale
            assert np.dot(fT, uT) <= tol * scale * vs
            assert np.linalg.norm(np.cross(fT, uT)) <= 1e-9 * scale * vs


def test_contact_law_holds_at_every_contact_node():
    """Eq. contact_1-3 hold after every step (the per-node solve is exact), and
    the plane is never penetrated (Eq. implicit_with_contact with R4's bias)."""
    sc = scenes.hanging_cloth(n_steps=40)
    M = oc.model_from_scene(sc)
    xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps)
    n_cases = np.zeros(3, int)
    for rec in recs:
        _check_contact_law(M, rec)
        n_cases += np.bincount(rec.cases, minlength=3)
    assert n_cases[oc.SLIP] > 0
    for x in xs:
        assert np.min(x[:, 1]) >= -1e-12
    sc2 = scenes.small_scene(4, seed=3, contact="plane", drop=True, n_steps=3)
    M2 = oc.model_from_scene(sc2)
    _, _, recs2 = oc.rollout(M2, sc2.x0, sc2.v0, 3)
    for rec in recs2:
        _check_contact_law(M2, rec)
        n_cases += np.bincount(rec.cases, minlength=3)
    assert n_cases[oc.STICK] > 0 and n_cases[oc.TAKEOFF] > 0


@pytest.mark.parametrize("side", [-1, 1])
def test_inclined_plane_stick_slip_threshold(side):
    """Rigid cloth on a slope: it sticks iff tan(theta) <= mu, otherwise it slides
    with v_n = n h g (sin(theta) - mu cos(theta)) (the Slope scene, Sec. 5.3)."""
    mu = 0.4
    theta = np.arctan(mu) + side * 0.05
    sc = scenes.inclined_plane(theta, mu)
    M = oc.model_from_scene(sc)
    x, v = sc.x0.copy(), sc.v0.copy()
    down = np.array([-np.cos(theta), -np.sin(theta), 0.0])   # down-slope unit vector
    gm = 9.8
    for n in range(1, 6):
        x, v, rec = oc.step(M, x, v, tol=1e-15, max_iters=5000)
        expect = max(0.0, n * M.h * gm * (np.sin(theta) - mu * np.cos(theta)))
        np.testing.assert_allclose(v @ down, expect, rtol=0, atol=1e-10)
        nrm = np.asarray(sc.obstacles[0].normal)
        np.testing.assert_allclose(v @ nrm, 0.0, atol=1e-12)
        assert np.all(rec.cases == (oc.STICK if side < 0 else oc.SLIP))


def test_cloth_resting_on_ground_stays_at_rest():
    pos, tris = scenes.grid_mesh(6, side=0.5, height=0.0)
    M = _model(pos, tris, obst=[scenes.Obstacle("plane")], mu=0.3)
    x, v = pos.copy(), np.zeros_like(pos)
    for _ in range(3):
        x, v, rec = oc.step(M, x, v, n_iters=20)
        assert np.max(np.abs(v)) < 1e-13
        assert np.all(rec.cases == oc.STICK)


# --------------------------------------------------------------------- adjoint

def _run(sc, tol=1e-14, **ov):
    M = oc.model_from_scene(sc, **ov)
    xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps, tol=tol)
    return M, xs, vs, recs


def _sig(recs):
    return [(tuple(r.contacts.nodes), tuple(r.cases)) for r in recs]


@pytest.mark.parametrize("contact,seed", [("sphere", 3), ("plane", 1), ("capsule", 0), ("none", 2)])
def test_adjoint_matches_central_differences(contact, seed):
    """The KKT adjoint (R7) agrees with central finite differences of the converged
    forward map, for x0, v0, k_stretch, k_bend and mu, where the contact set and
    the case of every contact node are the same at +-eps (Sec. 5.1)."""
    sc = scenes.small_scene(4, seed=seed, contact=contact, drop=(contact != "none"), n_steps=2)
    M, xs, vs, recs = _run(sc)
    base = _sig(recs)
    xi = sc.loss_w
    gx0, gv0, dth = oc.rollout_gradient(M, recs, xi)

    def loss_at(**kw):
        x0 = kw.pop("x0", sc.x0)
        v0 = kw.pop("v0", sc.v0)
        sc2 = dataclasses.replace(sc, x0=x0, v0=v0)
        _, xs2, _, recs2 = _run(sc2, **kw)
        assert _sig(recs2) == base
        return np.sum(xi * xs2[-1])

    p = sc.params
    for idx, (name, val) in enumerate([("k_stretch", p.k_stretch), ("k_bend", p.k_bend), ("mu", p.mu)]):
        e = 1e-6 * val
        fd = (loss_at(**{name: val + e}) - loss_at(**{name: val - e})) / (2 * e)
        assert abs(dth[idx] - fd) <= 2e-6 * max(abs(fd), 1e-3 * np.abs(dth).max())
    rng = np.random.default_rng(7)
    for which in ("x0", "v0"):
        d = rng.standard_normal(sc.x0.shape)
        d[sc.pins] = 0.0
        e = 1e-6
        base_v = getattr(sc, which)
        fd = (loss_at(**{which: base_v + e * d}) - loss_at(**{which: base_v - e * d})) / (2 * e)
        adj = np.sum((gx0 if which == "x0" else gv0) * d)
        assert abs(adj - fd) <= 1e-6 * abs(fd)


def test_mu_gradient_vanishes_without_slip():
    sc = scenes.small_scene(4, seed=0, contact="none", n_steps=2)
    M, xs, vs, recs = _run(sc, tol=1e-12)
    _, _, dth = oc.rollout_gradient(M, recs, sc.loss_w)
    assert dth[2] == 0.0
