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
    """With contacts that stick or take off but never slip, the converged step does
    not depend on mu (it only enters the slip branch and the stick test): the
    adjoint's dL/dmu is exactly 0, and the central difference in mu is 0 up to
    rounding (intermediate PD iterations may pass through a slip case, so the
    iterates, though not the fixed point, see mu)."""
    sc = scenes.liftoff_scene(mu=1.2)
    M, xs, vs, recs = _run(sc, tol=1e-14)
    cases = np.zeros(3, int)
    for r in recs:
        cases += np.bincount(r.cases, minlength=3)
    assert cases[oc.STICK] > 0 and cases[oc.TAKEOFF] > 0 and cases[oc.SLIP] == 0
    _, _, dth = oc.rollout_gradient(M, recs, sc.loss_w)
    assert dth[2] == 0.0
    assert abs(dth[0]) > 0.0 and abs(dth[1]) > 0.0
    e = 1e-6 * sc.params.mu
    lp = np.sum(sc.loss_w * _run(sc, tol=1e-14, mu=sc.params.mu + e)[1][-1])
    lm = np.sum(sc.loss_w * _run(sc, tol=1e-14, mu=sc.params.mu - e)[1][-1])
    assert abs(lp - lm) / (2 * e) <= 1e-8 * max(1.0, abs(lp))


# --------------------------------------------------------------------- degenerate triangles (R1)

def test_polar_of_collapsed_triangles():
    """A 3x2 F of rank <= 1 is flagged degenerate; its polar factor still has
    orthonormal columns and is a closest one: |F - R|_F^2 = sum_i (sigma_i - 1)^2
    with the singular values of numpy's SVD (the minimum over all matrices with
    orthonormal columns)."""
    rng = np.random.default_rng(11)
    Fs = [np.outer(rng.standard_normal(3), rng.standard_normal(2)) for _ in range(20)]
    Fs.append(np.zeros((3, 2)))
    Fs.append(np.array([[1.0, 2.0], [0.0, 0.0], [0.0, 0.0]]))
    Fs.append(np.array([[0.3, 0.3], [-1.0, -1.0], [2.0, 2.0]]))
    F = np.stack(Fs)
    assert np.all(oc.polar_degenerate(F))
    R, _ = oc.polar(F)
    np.testing.assert_allclose(np.einsum("tck,tcl->tkl", R, R), np.broadcast_to(np.eye(2), (len(F), 2, 2)),
                               atol=1e-14)
    sig = np.linalg.svd(F, compute_uv=False)
    np.testing.assert_allclose(np.sum((F - R) ** 2, axis=(1, 2)), np.sum((sig - 1.0) ** 2, axis=1), atol=1e-12)
    # nearly collapsed but above the threshold: the closed form, equal to the SVD factor
    F2 = np.stack([np.outer(rng.standard_normal(3), rng.standard_normal(2)) for _ in range(20)])
    U, s, Vt = np.linalg.svd(F2, full_matrices=False)
    F2 = np.einsum("tck,tk,tkl->tcl", U, np.stack([s[:, 0], 1e-9 * s[:, 0]], axis=1), Vt)
    assert not np.any(oc.polar_degenerate(F2))
    R2, _ = oc.polar(F2)
    np.testing.assert_allclose(R2, U @ Vt, atol=1e-6)


def test_step_with_a_collapsed_triangle():
    """A cloth that starts with one triangle collapsed onto a line: the first local
    step meets the degenerate case, the step stays finite, the surrogate g~ still
    decreases after every local and global step (the collapsed projection is still
    a closest point), and the triangle is no longer collapsed afterwards."""
    sc = scenes.collapsed_triangle_scene()
    M = oc.model_from_scene(sc)
    assert oc.polar_degenerate(M.deformation_gradients(sc.x0))[0]
    tr = []
    x1, v1, _ = oc.step(M, sc.x0, sc.v0, n_iters=30, trace=tr)
    assert np.all(np.isfinite(x1)) and np.all(np.isfinite(v1))
    t = np.asarray(tr)
    assert np.all(np.diff(t) <= 1e-14 * np.abs(t[:-1]))
    assert not np.any(oc.polar_degenerate(M.deformation_gradients(x1)))


# --------------------------------------------------------------------- rest operators and P

def test_rest_deformation_gradient_is_a_rotation():
    """F(x_rest) has orthonormal columns for every triangle (G = E D_m^-1 maps the
    rest triangle to itself), and a uniform scaling by s has singular values (s, s)."""
    pos, tris = scenes.grid_mesh(5, side=0.4)
    rng = np.random.default_rng(3)
    pos = pos + 0.02 * rng.standard_normal(pos.shape)          # a non-flat, irregular rest shape
    G, area = oc.triangle_rest(pos, tris)
    X = pos[tris]
    F = np.einsum("tac,tak->tck", X, G)
    np.testing.assert_allclose(np.einsum("tck,tcl->tkl", F, F), np.broadcast_to(np.eye(2), (len(tris), 2, 2)),
                               atol=1e-12)
    F2 = np.einsum("tac,tak->tck", 2.5 * X, G)
    np.testing.assert_allclose(np.linalg.svd(F2, compute_uv=False), 2.5, rtol=1e-12)
    e1, e2 = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]
    np.testing.assert_allclose(area, 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1), rtol=1e-14)


def test_P_is_the_hessian_of_the_quadratic_energy():
    """P = M + h^2 sum_i w_i A_i^T A_i (Eq. pd_global) is the Hessian of
    |x|_M^2/2 + h^2 sum_i w_i |A_i x|^2 / 2 per coordinate; central differences of
    that quadratic (written here from the per-triangle edge vectors and the bending
    rows) recover every entry of the scalar P_s."""
    pos, tris = scenes.grid_mesh(4, side=0.3)
    rng = np.random.default_rng(5)
    pos = pos + 0.01 * rng.standard_normal(pos.shape)
    M = _model(pos, tris, k_stretch=70.0, k_bend=3e-3, density=0.2)
    h = M.h

    def energy(u):                     # u: one coordinate of every node
        e = 0.5 * np.sum(M.mass * u * u)
        ut = u[M.tris]
        F = np.einsum("ta,tak->tk", ut, M.G)
        e += 0.5 * h * h * np.sum(M.w_t * np.sum(F * F, axis=1))
        q = M.Lb @ u
        e += 0.5 * h * h * np.sum(M.w_b * q * q)
        return e

    P = M.P.toarray()
    eps = 1e-3
    for i in range(M.m):
        for j in range(M.m):
            ei = np.zeros(M.m); ei[i] = eps
            ej = np.zeros(M.m); ej[j] = eps
            fd = (energy(ei + ej) - energy(ei - ej) - energy(ej - ei) + energy(-ei - ej)) / (4 * eps * eps)
            assert abs(fd - P[i, j]) <= 1e-9 * abs(P).max()


def test_compliance_is_the_row_sum_of_the_contact_block_of_h_P_inverse():
    """c_j = h (P^-1 1_I)_j (reading R5): the banded solve against the explicit dense
    inverse of P_ff (numpy inverse, i.e. unit-vector solves)."""
    sc = scenes.hanging_cloth(n=8, n_steps=1)
    M = oc.model_from_scene(sc)
    nodes = M.free[[3, 4, 5, 17, 40, 41]]
    ctr = oc.Contacts(nodes, np.zeros(len(nodes), int), np.zeros((len(nodes), 3)), np.zeros(len(nodes)))
    c = M.compliance(ctr)
    Pinv = np.linalg.inv(M.Pff.toarray())
    pos = np.searchsorted(M.free, nodes)
    expect = M.h * Pinv[np.ix_(pos, pos)].sum(axis=1)
    np.testing.assert_allclose(c, expect, rtol=1e-12)
    assert np.all(c > 0)


# --------------------------------------------------------------------- curved obstacles (R4)

def test_sphere_and_capsule_signed_distance():
    """phi and its gradient against points placed at known distances: along random
    directions from a sphere's centre; across a capsule's barrel (perpendicular to
    the axis) and beyond its end caps; plus a brute-force distance to the segment
    (dense sampling) for random points."""
    rng = np.random.default_rng(8)
    c = np.array([0.1, -0.2, 0.3])
    sph = scenes.Obstacle("sphere", center=tuple(c), radius=0.4)
    for _ in range(50):
        u = rng.standard_normal(3); u /= np.linalg.norm(u)
        d = rng.uniform(-0.35, 0.5)
        ph, n = oc.signed_distance(sph, c + (0.4 + d) * u)
        assert abs(ph - d) < 1e-14 and np.allclose(n, u, atol=1e-12)
    a, b = np.array([-0.3, 0.1, 0.0]), np.array([0.5, 0.3, 0.2])
    cap = scenes.Obstacle("capsule", a=tuple(a), b=tuple(b), radius=0.15)
    e = (b - a) / np.linalg.norm(b - a)
    for _ in range(50):
        w = rng.standard_normal(3); w -= np.dot(w, e) * e; w /= np.linalg.norm(w)
        t = rng.uniform(0.0, 1.0)
        d = rng.uniform(-0.14, 0.3)
        ph, n = oc.signed_distance(cap, a + t * (b - a) + (0.15 + d) * w)            # barrel
        assert abs(ph - d) < 1e-13 and np.allclose(n, w, atol=1e-12)
        u = rng.standard_normal(3); u /= np.linalg.norm(u)
        end, sgn = (a, -1.0) if rng.uniform() < 0.5 else (b, 1.0)
        if sgn * np.dot(u, e) < 0:
            u -= 2 * np.dot(u, e) * e                                                # point into the cap's half-space
        ph, n = oc.signed_distance(cap, end + (0.15 + d) * u)                        # end cap
        assert abs(ph - d) < 1e-13 and np.allclose(n, u, atol=1e-12)
    seg = a[None, :] + np.linspace(0.0, 1.0, 200001)[:, None] * (b - a)[None, :]
    for _ in range(20):
        x = a + rng.uniform(-0.5, 1.5) * (b - a) + 0.4 * rng.standard_normal(3)
        brute = np.min(np.linalg.norm(seg - x, axis=1)) - 0.15
        ph, _ = oc.signed_distance(cap, x)
        assert abs(ph - brute) < 1e-11


def test_obstacle_normal_jacobian_matches_central_differences():
    rng = np.random.default_rng(9)
    obs = [scenes.Obstacle("sphere", center=(0.0, 0.1, 0.2), radius=0.3),
           scenes.Obstacle("capsule", a=(-0.3, 0.0, 0.0), b=(0.4, 0.1, 0.3), radius=0.1)]
    for ob in obs:
        for _ in range(30):
            x = rng.uniform(-0.6, 0.6, 3)
            J = oc.normal_jacobian(ob, x)
            fd = np.zeros((3, 3))
            for k in range(3):
                d = np.zeros(3); d[k] = 1e-6
                fd[:, k] = (oc.signed_distance(ob, x + d)[1] - oc.signed_distance(ob, x - d)[1]) / 2e-6
            np.testing.assert_allclose(J, fd, atol=1e-6)
            g = np.array([(oc.signed_distance(ob, x + 1e-6 * np.eye(3)[k])[0] -
                           oc.signed_distance(ob, x - 1e-6 * np.eye(3)[k])[0]) / 2e-6 for k in range(3)])
            np.testing.assert_allclose(oc.signed_distance(ob, x)[1], g, atol=1e-8)


@pytest.mark.parametrize("contact,seed", [("sphere", 0), ("sphere", 5), ("capsule", 1), ("capsule", 4)])
def test_curved_obstacles_are_not_penetrated(contact, seed):
    """Every contact node ends its step on or outside the tangent plane at its
    closest surface point (stick and slip put u_N = 0 with the bias phi(x_n)/h,
    take-off u_N >= 0), so on a convex obstacle phi(x_{n+1}) >= 0 up to rounding
    (reading R4); nodes outside the contact set may move in by at most about
    h^2 |a| for this step's acceleration a."""
    sc = scenes.small_scene(4, seed=seed, contact=contact, drop=True, n_steps=4)
    M = oc.model_from_scene(sc)
    xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps)
    n_contacts = 0
    for n, rec in enumerate(recs):
        for a, j in enumerate(rec.contacts.nodes):
            ph, _ = oc.signed_distance(M.obstacles[rec.contacts.obs[a]], rec.x_np1[j])
            assert ph >= -1e-12
            n_contacts += 1
        for j in M.free:
            ph = min(oc.signed_distance(ob, rec.x_np1[j])[0] for ob in M.obstacles)
            acc = np.linalg.norm(vs[n + 1][j] - vs[n][j]) / M.h
            assert ph >= -(M.h ** 2) * acc - 1e-12
    assert n_contacts > 0


# --------------------------------------------------------------------- contact compliance choices (R5)

def _soft_contact_scene():
    sc = scenes.small_scene(5, seed=3, contact="both", drop=True, n_steps=1)
    return dataclasses.replace(sc, params=dataclasses.replace(sc.params, k_stretch=0.15, k_bend=1e-7))


def test_compliance_choices_share_the_fixed_point():
    """Every compliance choice of the per-node contact solve, the printed mass
    splitting of Eq. ly_et_al_govrningEq included, converges to the same solution
    of Eq. implicit_with_contact where it converges at all (a soft cloth, where
    h^2 rho(M^-1 (P - M)) < 1)."""
    sc = _soft_contact_scene()
    M0 = oc.model_from_scene(sc)
    A = M0.Pff.toarray()
    m = M0.mass[M0.free]
    assert np.max(np.abs(np.linalg.eigvals((A - np.diag(m)) / m[:, None]))) < 1.0
    ref = None
    for mode in ("rowsum", "diag_pinv", "diag_p", "mass"):
        M = oc.model_from_scene(sc, contact_compliance=mode)
        x1, v1, rec = oc.step(M, sc.x0, sc.v0, tol=1e-13, max_iters=20000)
        assert rec.iters < 20000 and len(rec.contacts) > 0
        _check_contact_law(M, rec, tol=1e-10)
        if ref is None:
            ref = v1
        else:
            np.testing.assert_allclose(v1, ref, rtol=0, atol=1e-11)


def test_mass_splitting_diverges_at_cloth_stiffness():
    """At the hanging cloth's stiffness h^2 rho(M^-1 (P - M)) is about 1.3e3, so the
    printed splitting blows up within one step of 20 iterations (the reason the
    default reading uses the prefactorised P)."""
    sc = scenes.hanging_cloth(n_steps=1)
    M = oc.model_from_scene(sc, contact_compliance="mass")
    A = M.Pff.toarray()
    m = M.mass[M.free]
    assert np.max(np.abs(np.linalg.eigvals((A - np.diag(m)) / m[:, None]))) > 1e3
    with np.errstate(all="ignore"):
        _, v1, _ = oc.step(M, sc.x0, sc.v0, n_iters=20)
    assert not np.all(np.abs(v1) < 1e20)


def test_diagonal_compliances_match_the_dense_matrices():
    """diag_pinv: c_j = h (P_ff^-1)_jj from unit-vector solves against numpy's dense
    inverse; diag_p: h / (P_ff)_jj; mass: h / m_j."""
    sc = scenes.hanging_cloth(n=7, n_steps=1)
    nodes = np.array([3, 9, 10, 30, 44])
    ctr = oc.Contacts(nodes, np.zeros(5, int), np.zeros((5, 3)), np.zeros(5))
    M = oc.model_from_scene(sc, contact_compliance="diag_pinv")
    pos = np.searchsorted(M.free, nodes)
    dense = M.Pff.toarray()
    np.testing.assert_allclose(M.compliance(ctr), M.h * np.diag(np.linalg.inv(dense))[pos], rtol=1e-12)
    M = oc.model_from_scene(sc, contact_compliance="diag_p")
    np.testing.assert_allclose(M.compliance(ctr), M.h / np.diag(dense)[pos], rtol=1e-14)
    M = oc.model_from_scene(sc, contact_compliance="mass")
    np.testing.assert_allclose(M.compliance(ctr), M.h / M.mass[nodes], rtol=1e-14)


# --------------------------------------------------------------------- triangle-mesh obstacles

def _ray_inside(V, F, x, d=np.array([0.5377, 0.8310, -0.1424])):
    """Inside test by ray parity (Moller-Trumbore crossings of a fixed ray)."""
    n = 0
    for a, b, c in F:
        e1, e2 = V[b] - V[a], V[c] - V[a]
        p = np.cross(d, e2)
        det = np.dot(e1, p)
        if abs(det) < 1e-14:
            continue
        t0 = x - V[a]
        u = np.dot(t0, p) / det
        q = np.cross(t0, e1)
        v = np.dot(d, q) / det
        t = np.dot(e2, q) / det
        n += (u >= 0) and (v >= 0) and (u + v <= 1) and (t > 0)
    return n % 2 == 1


def test_mesh_signed_distance_against_sampling_and_ray_parity():
    """|phi| equals the distance to a dense sampling of the mesh surface (to the
    sampling's resolution), and its sign agrees with a ray-crossing inside test."""
    ob = scenes.mesh_sphere((0.1, -0.2, 0.3), 0.4, 1)
    V, F = np.asarray(ob.vertices), np.asarray(ob.triangles)
    k = 40
    bary = np.array([(i / k, j / k) for i in range(k + 1) for j in range(k + 1 - i)])
    pts = np.concatenate([V[a] + bary[:, :1] * (V[b] - V[a]) + bary[:, 1:] * (V[c] - V[a]) for a, b, c in F])
    spacing = max(np.linalg.norm(V[a] - V[b]) for a, b, _ in F) / k
    rng = np.random.default_rng(12)
    n_in = 0
    for _ in range(60):
        x = np.array([0.1, -0.2, 0.3]) + rng.uniform(-0.6, 0.6, 3)
        ph, n = oc.signed_distance(ob, x)
        brute = np.min(np.linalg.norm(pts - x, axis=1))
        assert brute - spacing <= abs(ph) <= brute + 1e-12
        inside = _ray_inside(V, F, x)
        n_in += inside
        assert (ph < 0) == inside
        assert abs(np.linalg.norm(n) - 1.0) < 1e-12
    assert 5 < n_in < 55


def test_mesh_normal_and_jacobian_match_differences():
    """grad phi and d n/d x by central differences, away from region boundaries
    (points are kept only where the closest feature is the same at +-1e-6)."""
    ob = scenes.mesh_sphere((0.0, 0.0, 0.0), 0.5, 1)
    rng = np.random.default_rng(13)
    kinds = set()
    tested = 0
    while tested < 40:
        x = rng.uniform(-0.8, 0.8, 3)
        _, _, feat, _ = oc._mesh_closest(ob, x)
        same = all(oc._mesh_closest(ob, x + s * 1e-6 * np.eye(3)[q])[2] == feat for q in range(3) for s in (-1, 1))
        if not same:
            continue
        kinds.add(feat[0])
        tested += 1
        ph, n = oc.signed_distance(ob, x)
        g = np.array([(oc.signed_distance(ob, x + 1e-6 * np.eye(3)[q])[0] -
                       oc.signed_distance(ob, x - 1e-6 * np.eye(3)[q])[0]) / 2e-6 for q in range(3)])
        np.testing.assert_allclose(n, g, atol=1e-8)
        J = oc.normal_jacobian(ob, x)
        fd = np.stack([(oc.signed_distance(ob, x + 1e-6 * np.eye(3)[q])[1] -
                        oc.signed_distance(ob, x - 1e-6 * np.eye(3)[q])[1]) / 2e-6 for q in range(3)], axis=1)
        np.testing.assert_allclose(J, fd, atol=1e-6)
    assert kinds == {"face", "edge", "vertex"}


def test_mesh_normal_on_the_surface_and_exact_ties():
    """The readings for points on a mesh's surface and for exact distance ties, on
    the regular icosahedron (circumradius 0.5), whose symmetry fixes the answers:
    on the surface (|x - c| below 1e-12 m: a vertex, an edge midpoint, a face
    centre, each also displaced by 1e-14 m) the normal is the feature's
    pseudo-normal, which the 5-fold, 2-fold and 3-fold symmetry makes radial; at
    the centre all 20 faces tie at the inradius R sqrt((5 + 2 sqrt 5)/15), and the
    lowest face index wins (also 1e-13 m off centre, inside the tie band)."""
    R = 0.5
    ob = scenes.mesh_sphere((0.0, 0.0, 0.0), R, 0)
    V, F = np.asarray(ob.vertices), np.asarray(ob.triangles)
    rng = np.random.default_rng(3)
    pts = [V[0], V[7], 0.5 * (V[F[3][0]] + V[F[3][1]]), 0.5 * (V[1] + V[8]), V[F[5]].mean(axis=0)]
    for p in pts:
        for x in (p, p + 1e-14 * rng.standard_normal(3)):
            ph, n = oc.signed_distance(ob, x)
            assert abs(ph) < 1e-13
            np.testing.assert_allclose(n, p / np.linalg.norm(p), atol=1e-12)
            assert np.all(oc.normal_jacobian(ob, x) == 0.0)
    a, b, c = V[F[0]]
    n0 = np.cross(b - a, c - a)
    n0 /= np.linalg.norm(n0)
    for x in (np.zeros(3), 1e-13 * rng.standard_normal(3)):
        ph, n = oc.signed_distance(ob, x)
        assert abs(ph + R * np.sqrt((5 + 2 * np.sqrt(5)) / 15)) < 1e-12
        np.testing.assert_allclose(n, n0, atol=1e-11)
        assert oc._mesh_closest(ob, x)[3] == 0


def test_fine_mesh_sphere_approaches_the_analytic_sphere():
    """A subdivided icosphere's phi is within its sagitta of the analytic sphere's
    (vertices lie on the sphere, faces at most r (1 - cos(theta/2)) inside it, theta
    the largest edge angle)."""
    c, r = np.array([0.0, 0.1, 0.0]), 0.3
    sph = scenes.Obstacle("sphere", center=tuple(c), radius=r)
    for sub in (1, 2):
        ob = scenes.mesh_sphere(tuple(c), r, sub)
        V, F = np.asarray(ob.vertices), np.asarray(ob.triangles)
        ang = max(np.arccos(np.clip(np.dot(V[a] - c, V[b] - c) / r ** 2, -1, 1)) for a, b, _ in F)
        sag = r * (1 - np.cos(ang / 2)) * 1.2
        rng = np.random.default_rng(sub)
        for _ in range(20):
            u = rng.standard_normal(3)
            u /= np.linalg.norm(u)
            x = c + rng.uniform(0.2, 0.6) * u
            dm, _ = oc.signed_distance(ob, x)
            ds, _ = oc.signed_distance(sph, x)
            assert -1e-12 <= dm - ds <= sag


def test_continuity_study_analytic_vs_triangulated_sphere():
    """Sec. "Continuity and Smoothness": sweep where a cloth lands on a sphere; the
    gradient of its final mean x w.r.t. the landing offset varies little over the
    analytic sphere and by large jumps over a coarse triangulation of it (normals
    jump across edges, curvature concentrates at edges and vertices): the total
    variation of the gradient over the sweep is ten times larger (both sweeps also
    jump where contacts begin at another step)."""
    offsets = np.linspace(0.0, 0.12, 13)

    def sweep(sub):
        g = []
        for d in offsets:
            sc = scenes.sphere_drop(float(d), mesh_subdivisions=sub)
            M = oc.model_from_scene(sc)
            _, _, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps)
            w = np.zeros((sc.m, 3))
            w[:, 0] = 1.0 / sc.m
            gx, _, _ = oc.rollout_gradient(M, recs, w)
            g.append(gx[:, 0].sum())
        return np.abs(np.diff(np.array(g)))
    js, jm = sweep(-1), sweep(1)
    assert jm.sum() > 10.0 * js.sum()


# ----------------------------------------------------------------- self-collision (R13)

def _pairs_sig(recs):
    return [(tuple(r.pairs.i), tuple(r.pairs.j), tuple(r.pair_cases)) for r in recs] + _sig(recs)


@pytest.mark.parametrize("kw", [dict(), dict(slide=0.0, mu=2.0), dict(approach=3.0)])
def test_self_contact_conserves_momentum_and_keeps_the_thickness(kw):
    """Two cloth patches driven into each other without gravity or obstacles:
    the pair impulses are equal and opposite and the PD forces are internal, so
    the total momentum is unchanged by every step; and a converged step leaves
    every detected pair at least the thickness apart (u_N = d'(t) + (d -
    thickness)/h >= 0 holds along the pair's normal, R13)."""
    sc = scenes.two_patches_scene(**kw)
    M = oc.model_from_scene(sc)
    for tol in (None, 1e-13):
        xs, vs, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps, tol=tol)
        assert sum(len(r.pairs) for r in recs) > 0
        assert any(np.any(r.pair_cases != oc.TAKEOFF) for r in recs)
        p0 = (M.mass[:, None] * sc.v0).sum(axis=0)
        for v in vs[1:]:
            p = (M.mass[:, None] * v).sum(axis=0)
            assert np.max(np.abs(p - p0)) <= 1e-13 * np.max(np.abs(p0))
        if tol is not None:
            for n, r in enumerate(recs):
                if len(r.pairs):
                    d = np.linalg.norm(xs[n + 1][r.pairs.i] - xs[n + 1][r.pairs.j], axis=1)
                    assert np.min(d) >= sc.params.self_thickness - 1e-12


def test_self_contact_without_pairs_is_the_plain_step():
    """Self-collision on, but the patches too far apart for any pair: every
    step is bitwise the step with self-collision off."""
    sc = scenes.two_patches_scene(gap=0.3, approach=0.5)
    on = oc.model_from_scene(sc)
    off = oc.model_from_scene(sc, self_thickness=0.0)
    xa, va, ra = oc.rollout(on, sc.x0, sc.v0, sc.n_steps)
    xb, vb, rb = oc.rollout(off, sc.x0, sc.v0, sc.n_steps)
    assert sum(len(r.pairs) for r in ra) == 0
    assert all(np.array_equal(a, b) for a, b in zip(xa, xb)) and all(np.array_equal(a, b) for a, b in zip(va, vb))


@pytest.mark.parametrize("kw", [dict(n_steps=2), dict(slide=0.0, mu=2.0, n_steps=2),
                                dict(pinned=True, gravity=True, n_steps=1), dict(ground=True, n_steps=1)])
def test_self_contact_adjoint_matches_central_differences(kw):
    """The KKT adjoint with pair rows (slip pairs; a mix of stick and slip pairs)
    agrees with central differences of the converged forward map for x0, v0,
    k_stretch, k_bend and mu, where the pairs and their cases are unchanged at
    +-eps (the derivatives of the pair normal and bias with respect to both
    nodes, and the friction term on the relative velocity, are all exercised);
    also with gravity and pinned nodes among the pairs (a pinned node has no
    row in the adjoint system), and with nodes in contact with the ground and
    with the other patch at once (the two kinds of rows in one KKT system)."""
    sc = scenes.two_patches_scene(**kw)
    M, xs, vs, recs = _run(sc)
    base = _pairs_sig(recs)
    assert any(np.any(r.pair_cases == oc.SLIP) for r in recs)
    xi = sc.loss_w
    gx0, gv0, dth = oc.rollout_gradient(M, recs, xi)

    def loss_at(**kw2):
        x0 = kw2.pop("x0", sc.x0)
        v0 = kw2.pop("v0", sc.v0)
        _, xs2, _, recs2 = _run(dataclasses.replace(sc, x0=x0, v0=v0), **kw2)
        assert _pairs_sig(recs2) == base
        return np.sum(xi * xs2[-1])

    p = sc.params
    # relative steps of 1e-4: the tolerance-mode forward (thousands of Jacobi
    # iterations over the pairs) leaves ~1e-14 of noise in the loss, which a
    # 1e-6 step of the small bending stiffness would amplify past the bound
    for idx, (name, val) in enumerate([("k_stretch", p.k_stretch), ("k_bend", p.k_bend), ("mu", p.mu)]):
        e = 1e-4 * val
        fd = (loss_at(**{name: val + e}) - loss_at(**{name: val - e})) / (2 * e)
        assert abs(dth[idx] - fd) <= 2e-6 * max(abs(fd), 1e-3 * np.abs(dth).max()), (name, dth[idx], fd)
    rng = np.random.default_rng(7)
    for which in ("x0", "v0"):
        d = rng.standard_normal(sc.x0.shape)
        d[sc.pins] = 0.0
        e = 1e-7
        b = getattr(sc, which)
        fd = (loss_at(**{which: b + e * d}) - loss_at(**{which: b - e * d})) / (2 * e)
        adj = np.sum((gx0 if which == "x0" else gv0) * d)
        assert abs(adj - fd) <= 1e-6 * abs(fd), (which, adj, fd)


def test_self_contact_detection_rules():
    """R13's detection on the two patches with a thickness above the
    node spacing: every returned pair has i < j, at least one free node, nodes
    that share no triangle, predicted distance within thickness + delta, a unit
    normal from j to i and the bias (|x_i - x_j| - thickness)/h; and no pair of
    triangle neighbours is returned although all of them are within range."""
    sc = scenes.two_patches_scene(thickness=0.15, gap=0.3, approach=0.0, slide=0.0, pinned=True)
    M = oc.model_from_scene(sc)
    pr = M.detect_self(sc.x0, sc.v0)
    assert len(pr) > 0
    adjacent = {(min(a, b), max(a, b)) for t in sc.tris for a in t for b in t if a != b}
    xp = sc.x0 + M.h * sc.v0
    for a in range(len(pr)):
        i, j = int(pr.i[a]), int(pr.j[a])
        assert i < j and (i, j) not in adjacent and not (M.is_pin[i] and M.is_pin[j])
        assert np.linalg.norm(xp[i] - xp[j]) <= 0.15 + M.delta
        d = sc.x0[i] - sc.x0[j]
        np.testing.assert_allclose(pr.normals[a], d / np.linalg.norm(d), rtol=0, atol=1e-15)
        assert abs(pr.betas[a] - (np.linalg.norm(d) - 0.15) / M.h) <= 1e-12
    # every non-adjacent pair within range is found
    want = {(i, j) for i in range(sc.m) for j in range(i + 1, sc.m)
            if (i, j) not in adjacent and not (M.is_pin[i] and M.is_pin[j])
            and np.linalg.norm(xp[i] - xp[j]) <= 0.15 + M.delta}
    assert want == set(zip(pr.i.tolist(), pr.j.tolist()))
    assert any(np.linalg.norm(xp[i] - xp[j]) <= 0.15 for i, j in adjacent)
