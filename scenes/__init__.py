"""Seeded synthetic cloth scenes: the inputs shared by the oracle, the tests and the benchmark.

This module only builds inputs -- rest meshes, pins, obstacles, material and
solver parameters, initial states and loss weights.  It holds none of the
simulation arithmetic (no rest-shape operators, no masses, no system matrix,
no projections): both the CPU oracle and the CUDA library derive those from
the raw mesh on their own.

Geometry conventions (the paper fixes none of them):
  * y is up; gravity is (0, -9.8, 0) m/s^2.
  * An n x n grid cloth of side ``side`` lies in the x-z plane at height
    ``height``; node (i, j) has index j*n + i and rest position
    (x0 + i*a, height, z0 + j*a) with a = side/(n-1).
  * Each grid quad (i, j)-(i+1, j+1) is split along that diagonal into the
    triangles (v00, v10, v11) and (v00, v11, v01).
  * Obstacles are analytic (planes {x : n.x = d}, spheres and capsules) or
    closed triangle meshes with outward (counter-clockwise) orientation.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

GRAVITY = (0.0, -9.8, 0.0)


@dataclasses.dataclass
class Obstacle:
    kind: str                      # "plane" | "sphere" | "capsule" | "mesh"
    normal: tuple = (0.0, 1.0, 0.0)  # plane: unit normal
    offset: float = 0.0            # plane: n.x = offset
    center: tuple = (0.0, 0.0, 0.0)  # sphere centre
    radius: float = 0.0            # sphere / capsule radius
    a: tuple = (0.0, 0.0, 0.0)     # capsule segment end points
    b: tuple = (0.0, 0.0, 0.0)
    vertices: Optional[np.ndarray] = None   # mesh: (V, 3) positions
    triangles: Optional[np.ndarray] = None  # mesh: (F, 3) int32, counter-clockwise seen from outside


def icosphere(center=(0.0, 0.0, 0.0), radius: float = 1.0, subdivisions: int = 1):
    """A closed triangle mesh of a sphere: the icosahedron, each face split into 4
    subdivisions times, vertices pushed onto the sphere.  Outward orientation."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
             (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
             (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdivisions):
        mid = {}

        def midpoint(i, j):
            key = (min(i, j), max(i, j))
            if key not in mid:
                p = verts[i] + verts[j]
                verts.append(p / np.linalg.norm(p))
                mid[key] = len(verts) - 1
            return mid[key]
        nf = []
        for a, b, c in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.asarray(center, dtype=np.float64) + radius * np.stack(verts)
    return V, np.asarray(faces, dtype=np.int32)


def mesh_sphere(center, radius, subdivisions=1) -> Obstacle:
    V, F = icosphere(center, radius, subdivisions)
    return Obstacle("mesh", vertices=V, triangles=F)


@dataclasses.dataclass
class Params:
    k_stretch: float = 1e3
    k_bend: float = 1e-3
    density: float = 0.1           # kg / m^2
    mu: float = 0.3
    h: float = 1.0 / 120.0
    gravity: tuple = GRAVITY
    n_pd_iters: int = 20
    contact_margin: float = 1e-6   # detection margin delta (m)
    # compliance of the per-node contact solve: "rowsum", "diag_pinv", "diag_p" or "mass"
    contact_compliance: str = "rowsum"
    # node-node self-collision: the distance two nodes keep (m); 0 turns it off
    self_thickness: float = 0.0


@dataclasses.dataclass
class Scene:
    name: str
    n: int                         # grid resolution (n x n nodes)
    rest_pos: np.ndarray           # (m, 3) float64
    tris: np.ndarray               # (T, 3) int32
    pins: np.ndarray               # (p,) int32, sorted
    obstacles: List[Obstacle]
    params: Params
    x0: np.ndarray                 # (m, 3) initial positions
    v0: np.ndarray                 # (m, 3) initial velocities
    n_steps: int
    loss_w: Optional[np.ndarray] = None   # (m, 3) loss weights xi, L = sum(xi * x_N)
    checkpoint_every: int = 0

    @property
    def m(self) -> int:
        return self.rest_pos.shape[0]


def grid_mesh(n: int, side: float = 1.0, height: float = 0.6,
              x0: float = -0.5, z0: float = 0.0):
    """Rest positions (n*n, 3) and triangles (2(n-1)^2, 3) of a flat n x n grid."""
    a = side / (n - 1)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    pos = np.zeros((n * n, 3))
    pos[:, 0] = x0 + a * ii.reshape(-1)
    pos[:, 1] = height
    pos[:, 2] = z0 + a * jj.reshape(-1)
    tris = []
    for j in range(n - 1):
        for i in range(n - 1):
            v00 = j * n + i
            v10 = v00 + 1
            v01 = v00 + n
            v11 = v01 + 1
            tris.append((v00, v10, v11))
            tris.append((v00, v11, v01))
    return pos, np.asarray(tris, dtype=np.int32)


def loss_weights(m: int, seed: int) -> np.ndarray:
    """Standard-normal loss weights xi (m, 3); the loss is sum(xi * x_final)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x10557]))
    return rng.standard_normal((m, 3))


def _log_uniform(rng, lo, hi):
    return float(np.exp(rng.uniform(np.log(lo), np.log(hi))))


def hanging_cloth(n: int = 16, seed: int = 0, n_steps: int = 50) -> Scene:
    """16x16 cloth pinned at two corners, falling onto a sphere and the ground.

    Side 1 m, mu 0.3, h 1/120 s, 20 PD iterations, stretch 1e3, bend 1e-3,
    density 0.1 kg/m^2; sphere of radius 0.3 m under the cloth centre.
    """
    pos, tris = grid_mesh(n, side=1.0, height=0.7)
    pins = np.array([0, n - 1], dtype=np.int32)
    obst = [Obstacle("plane", normal=(0.0, 1.0, 0.0), offset=0.0),
            Obstacle("sphere", center=(0.0, 0.35, 0.55), radius=0.3)]
    prm = Params(k_stretch=1e3, k_bend=1e-3, density=0.1, mu=0.3, h=1.0 / 120.0)
    return Scene("hanging_16", n, pos, tris, pins, obst, prm, pos.copy(),
                 np.zeros_like(pos), n_steps, loss_weights(n * n, seed))


def draped_cloth(n: int = 61, seed: int = 0, n_steps: int = 125,
                 checkpoint_every: int = 25) -> Scene:
    """Unpinned n x n cloth dropped over a sphere (r 0.3 m) and the ground.

    mu ~ U[0.1, 0.6], k_stretch ~ logU[1e2, 1e4], k_bend ~ logU[1e-4, 1e-2]
    drawn from the seed; h 1/120 s; 20 PD iterations.
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xD7A9E]))
    mu = float(rng.uniform(0.1, 0.6))
    ks = _log_uniform(rng, 1e2, 1e4)
    kb = _log_uniform(rng, 1e-4, 1e-2)
    pos, tris = grid_mesh(n, side=1.0, height=0.8)
    obst = [Obstacle("plane", normal=(0.0, 1.0, 0.0), offset=0.0),
            Obstacle("sphere", center=(0.0, 0.35, 0.5), radius=0.3)]
    prm = Params(k_stretch=ks, k_bend=kb, density=0.1, mu=mu, h=1.0 / 120.0)
    return Scene(f"draped_{n}", n, pos, tris, np.zeros(0, np.int32), obst, prm,
                 pos.copy(), np.zeros_like(pos), n_steps, loss_weights(n * n, seed),
                 checkpoint_every)


def batch_instance(seed: int, n_lo: int = 16, n_hi: int = 64, n_steps: int = 50) -> Scene:
    """One member of the batched workload: random grid size, material, sphere."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xBA7C4]))
    n = int(rng.integers(n_lo, n_hi + 1))
    mu = float(rng.uniform(0.1, 0.6))
    ks = _log_uniform(rng, 1e2, 1e4)
    kb = _log_uniform(rng, 1e-4, 1e-2)
    r = float(rng.uniform(0.2, 0.5))
    cy = r + float(rng.uniform(0.0, 0.2))
    pos, tris = grid_mesh(n, side=1.0, height=cy + r + 0.1)
    obst = [Obstacle("plane", normal=(0.0, 1.0, 0.0), offset=0.0),
            Obstacle("sphere", center=(0.0, cy, 0.5), radius=r)]
    prm = Params(k_stretch=ks, k_bend=kb, density=0.1, mu=mu, h=1.0 / 120.0)
    return Scene(f"batch_{seed}_{n}", n, pos, tris, np.zeros(0, np.int32), obst, prm,
                 pos.copy(), np.zeros_like(pos), n_steps, loss_weights(n * n, seed))


def capsule_field(n: int = 200, seed: int = 0, n_steps: int = 100, n_capsules: int = 8) -> Scene:
    """Large cloth dropped onto random capsules and the ground (mu 0.4, h 1/240)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xCA95]))
    pos, tris = grid_mesh(n, side=1.0, height=0.5)
    obst = [Obstacle("plane", normal=(0.0, 1.0, 0.0), offset=0.0)]
    for _ in range(n_capsules):
        c = np.array([rng.uniform(-0.4, 0.4), rng.uniform(0.1, 0.35), rng.uniform(0.1, 0.9)])
        th = rng.uniform(0, np.pi)
        half = rng.uniform(0.05, 0.2)
        d = np.array([np.cos(th), 0.0, np.sin(th)]) * half
        obst.append(Obstacle("capsule", a=tuple(c - d), b=tuple(c + d),
                             radius=float(rng.uniform(0.02, 0.1))))
    prm = Params(k_stretch=1e3, k_bend=1e-3, density=0.1, mu=0.4, h=1.0 / 240.0)
    return Scene(f"capsules_{n}", n, pos, tris, np.zeros(0, np.int32), obst, prm,
                 pos.copy(), np.zeros_like(pos), n_steps, loss_weights(n * n, seed), 10)


def inclined_plane(theta: float, mu: float, n: int = 4, side: float = 0.3) -> Scene:
    """A flat cloth resting on a plane tilted by theta about the z axis (no pins)."""
    pos, tris = grid_mesh(n, side=side, height=0.0, x0=0.0, z0=0.0)
    c, s = np.cos(theta), np.sin(theta)
    rot = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    pos = pos @ rot.T
    nrm = rot @ np.array([0.0, 1.0, 0.0])
    obst = [Obstacle("plane", normal=tuple(nrm), offset=0.0)]
    prm = Params(k_stretch=1e3, k_bend=1e-3, density=0.1, mu=mu, h=1.0 / 100.0)
    return Scene("slope", n, pos, tris, np.zeros(0, np.int32), obst, prm, pos.copy(),
                 np.zeros_like(pos), 10)


def sliding_breathing_scene(n: int = 8, n_steps: int = 24) -> Scene:
    """A cloth on a plane tilted 0.15 rad past the friction angle of mu = 0.5,
    started with a uniform in-plane expansion velocity (0.5 s^-1 about its centre):
    it slides down (rate set by mu) while it breathes (frequency set by
    k_stretch).  Both motions are smooth, so a handful of PD iterations per step
    reach the step's fixed point (the system-identification scene)."""
    sc = inclined_plane(float(np.arctan(0.5) + 0.15), 0.5, n=n, side=0.4)
    nrm = np.asarray(sc.obstacles[0].normal)
    c = sc.x0.mean(axis=0)
    v0 = 0.5 * (sc.x0 - c)
    v0 -= np.outer(v0 @ nrm, nrm)
    return dataclasses.replace(sc, name="sliding_breathing", v0=v0, n_steps=n_steps,
                               loss_w=loss_weights(n * n, 2))


def sphere_drop(offset: float = 0.0, mesh_subdivisions: int = -1, n: int = 5, n_steps: int = 8) -> Scene:
    """A small cloth (side 0.2 m, 5x5) falling at 0.5 m/s onto a sphere of radius
    0.3 m centred at the origin, shifted by `offset` along x: the analytic sphere,
    or (mesh_subdivisions >= 0) an icosphere of that many subdivisions with its
    vertices on the sphere (the scene of the continuity study)."""
    pos, tris = grid_mesh(n, side=0.2, height=0.32, x0=-0.1 + offset, z0=-0.1)
    ob = (Obstacle("sphere", center=(0.0, 0.0, 0.0), radius=0.3) if mesh_subdivisions < 0
          else mesh_sphere((0.0, 0.0, 0.0), 0.3, mesh_subdivisions))
    prm = Params(k_stretch=100.0, k_bend=1e-3, density=0.1, mu=0.2, h=1.0 / 100.0)
    v0 = np.tile([0.0, -0.5, 0.0], (n * n, 1))
    return Scene(f"sphere_drop_{offset:.4f}_{mesh_subdivisions}", n, pos, tris, np.zeros(0, np.int32), [ob], prm,
                 pos.copy(), v0, n_steps, loss_weights(n * n, 3))


def small_scene(n: int = 4, seed: int = 0, contact: str = "sphere", pinned: bool = True,
                n_steps: int = 3, drop: bool = False) -> Scene:
    """Tiny seeded scenes for brute-force and finite-difference checks.

    ``drop`` gives every node a downward velocity with little tangential noise
    and a high friction coefficient, so that contacts stick.
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5A11]))
    pos, tris = grid_mesh(n, side=0.3, height=0.2, x0=-0.15, z0=0.0)
    x0 = pos + 0.01 * rng.standard_normal(pos.shape)
    v0 = 0.2 * rng.standard_normal(pos.shape)
    if drop:
        v0 = 0.01 * rng.standard_normal(pos.shape) + np.array([0.0, -0.6, 0.0])
    pins = np.array([0, n - 1], dtype=np.int32) if pinned else np.zeros(0, np.int32)
    v0[pins] = 0.0
    x0[pins] = pos[pins]
    obst: List[Obstacle] = []
    if contact in ("plane", "both"):
        obst.append(Obstacle("plane", normal=(0.0, 1.0, 0.0), offset=0.185))
    if contact in ("sphere", "both"):
        obst.append(Obstacle("sphere", center=(0.0, -0.1, 0.15), radius=0.3))
    if contact == "capsule":
        obst.append(Obstacle("capsule", a=(-0.3, -0.05, 0.15), b=(0.3, -0.02, 0.15), radius=0.25))
    prm = Params(k_stretch=float(rng.uniform(50, 200)), k_bend=float(rng.uniform(1e-3, 1e-2)),
                 density=0.1, mu=float(rng.uniform(0.1, 0.6)), h=1.0 / 60.0)
    if drop:
        prm.mu = float(rng.uniform(0.8, 1.5))
    return Scene(f"small_{n}_{contact}", n, pos, tris, pins, obst, prm, x0, v0, n_steps,
                 loss_weights(n * n, seed))


def liftoff_scene(mu: float = 1.2, n: int = 4, n_steps: int = 3) -> Scene:
    """A flat, unstretched cloth lying on the ground at rest, three of its nodes
    moving straight up at 0.4 m/s, with a 1 cm detection margin so that they are
    still in the contact set: their neighbours stick under gravity, they take off,
    and (at this friction) no node slips."""
    pos, tris = grid_mesh(n, side=0.3, height=0.0, x0=-0.15, z0=0.0)
    v0 = np.zeros_like(pos)
    v0[[n + 1, n + 2, 2 * n + 2]] = (0.0, 0.4, 0.0)
    prm = Params(k_stretch=100.0, k_bend=5e-3, density=0.1, mu=mu, h=1.0 / 60.0, contact_margin=0.01)
    return Scene("liftoff", n, pos, tris, np.zeros(0, np.int32), [Obstacle("plane")], prm, pos.copy(), v0,
                 n_steps, loss_weights(n * n, 0))


def collapsed_triangle_scene(n: int = 5, n_steps: int = 3) -> Scene:
    """A small pinned cloth whose first triangle starts collapsed onto a line:
    node (1, 1) is moved onto the segment between nodes (0, 0) and (1, 0)."""
    pos, tris = grid_mesh(n, side=0.3, height=0.3, x0=-0.15, z0=0.0)
    x0 = pos.copy()
    x0[n + 1] = 0.5 * (pos[0] + pos[1])
    pins = np.array([n - 1, n * n - 1], dtype=np.int32)
    prm = Params(k_stretch=200.0, k_bend=1e-3, density=0.1, mu=0.3, h=1.0 / 120.0)
    return Scene("collapsed", n, pos, tris, pins, [Obstacle("plane")], prm, x0, np.zeros_like(pos), n_steps,
                 loss_weights(n * n, 1))


def serve_request(seed: int, dof_lo: float = 1e3, dof_hi: float = 3e4, steps_lo: int = 25,
                  steps_hi: int = 150) -> Scene:
    """One request of the served workload: a square cloth of log-uniform DOF count
    (3 n^2 in [dof_lo, dof_hi]), a uniform step count, random material and friction,
    dropped onto a random sphere and the ground."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5E4E]))
    dof = _log_uniform(rng, dof_lo, dof_hi)
    n = max(4, int(round(np.sqrt(dof / 3.0))))
    n_steps = int(rng.integers(steps_lo, steps_hi + 1))
    mu = float(rng.uniform(0.1, 0.6))
    ks = _log_uniform(rng, 1e2, 1e4)
    kb = _log_uniform(rng, 1e-4, 1e-2)
    r = float(rng.uniform(0.2, 0.5))
    cy = r + float(rng.uniform(0.0, 0.2))
    cx, cz = float(rng.uniform(-0.2, 0.2)), float(rng.uniform(0.3, 0.7))
    pos, tris = grid_mesh(n, side=1.0, height=cy + r + 0.1)
    obst = [Obstacle("plane", normal=(0.0, 1.0, 0.0), offset=0.0),
            Obstacle("sphere", center=(cx, cy, cz), radius=r)]
    prm = Params(k_stretch=ks, k_bend=kb, density=0.1, mu=mu, h=1.0 / 120.0)
    return Scene(f"request_{seed}_{n}_{n_steps}", n, pos, tris, np.zeros(0, np.int32), obst, prm,
                 pos.copy(), np.zeros_like(pos), n_steps, loss_weights(n * n, seed))


def two_patches_scene(n: int = 4, gap: float = 0.025, approach: float = 1.0, slide: float = 0.3,
                      thickness: float = 0.02, mu: float = 0.3, gravity: bool = False, seed: int = 0,
                      n_steps: int = 3, pinned: bool = False, ground: bool = False) -> Scene:
    """Node-node self-collision: two n x n patches (side 0.3 m) in one mesh, the
    upper `gap` above the lower and shifted sideways by a fifth of the thickness, moving
    down at `approach` m/s and sideways at `slide` m/s with small seeded noise; no
    obstacle and, by default, no gravity (so that momentum is conserved).  With
    `pinned`, the lower patch's four corners are pinned at their rest positions.
    With `ground`, gravity is on and the lower patch falls at 0.1 m/s from half a
    millimetre above a ground plane, so that nodes meet the ground and the other
    patch at once."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5E1F]))
    lo, tris = grid_mesh(n, side=0.3, height=0.0, x0=-0.15, z0=0.0)
    hi = lo.copy()
    hi[:, 1] = gap
    hi[:, 0] += 0.2 * thickness
    pos = np.vstack([lo, hi])
    tris = np.vstack([tris, tris + n * n]).astype(np.int32)
    m = 2 * n * n
    v0 = np.zeros((m, 3))
    v0[n * n:, 1] = -approach
    v0[n * n:, 0] = slide
    v0 += 0.02 * rng.standard_normal((m, 3))
    x0 = pos + 0.002 * rng.standard_normal((m, 3))
    obst: List[Obstacle] = []
    if ground:
        gravity = True
        x0[:, 1] += 0.0005
        v0[:n * n, 1] = -0.1
        obst = [Obstacle("plane", normal=(0.0, 1.0, 0.0), offset=0.0)]
    pins = np.zeros(0, np.int32)
    if pinned:
        pins = np.array([0, n - 1, n * n - n, n * n - 1], dtype=np.int32)
        x0[pins] = pos[pins]
        v0[pins] = 0.0
    prm = Params(k_stretch=200.0, k_bend=1e-3, density=0.1, mu=mu, h=1.0 / 120.0,
                 gravity=GRAVITY if gravity else (0.0, 0.0, 0.0), self_thickness=thickness)
    return Scene(f"two_patches_{n}_{seed}", n, pos, tris, pins, obst, prm, x0, v0, n_steps, loss_weights(m, seed))
