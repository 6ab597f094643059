"""Seeded synthetic cloth workloads.

This module only builds inputs: vertex positions, triangle lists, pinned
vertex sets, scripted pin / obstacle motion and initial velocities, all from a
seeded ``numpy.random.Generator``.  It holds none of the projective-dynamics
arithmetic (no masses, rest operators, projections, solves or collision
tests); the FP64 oracle and the CUDA library both derive those on their own
from the arrays returned here.

The scenes stand in for the paper's cloth scenes (Tab. 1: drape on a sphere,
just folding, fashion show), whose meshes are not public.  Every scene is a
square grid or a conical tube triangulated with two triangles per quad and
alternating diagonals, in SI units, z up.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

__all__ = [
    "Obstacle", "Scene", "grid_mesh", "icosphere", "box_mesh", "cylinder_mesh",
    "cone_skirt", "drape_sphere", "fold_on_box", "hanging_swept", "batched_drape",
    "skirt_on_body", "tiny_scene", "beam_strip", "seed_for",
]


def seed_for(config_id: int) -> int:
    """Seed convention of the synthetic workloads: 1000 + config id."""
    return 1000 + int(config_id)


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------

def grid_mesh(nx: int, ny: int, size_x: float, size_y: float):
    """Regular nx-by-ny vertex grid in the local (u, v) plane.

    Vertex (i, j) has index j*nx + i and local coordinates
    (i*size_x/(nx-1), j*size_y/(ny-1)).  Each quad is split into two triangles;
    the diagonal alternates in a checkerboard pattern.  Triangles are listed
    counter-clockwise seen from +w.
    Returns (uv float64 [n,2], tris int32 [m,3]).
    """
    i = np.arange(nx, dtype=np.float64) * (size_x / (nx - 1))
    j = np.arange(ny, dtype=np.float64) * (size_y / (ny - 1))
    uu, vv = np.meshgrid(i, j)
    uv = np.stack([uu.ravel(), vv.ravel()], axis=1)
    qi, qj = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1))
    qi = qi.ravel()
    qj = qj.ravel()
    a = qj * nx + qi
    b = a + 1
    c = a + nx
    d = c + 1
    flip = ((qi + qj) % 2) == 1
    t1 = np.where(flip[:, None], np.stack([a, b, c], 1), np.stack([a, b, d], 1))
    t2 = np.where(flip[:, None], np.stack([b, d, c], 1), np.stack([a, d, c], 1))
    tris = np.empty((2 * len(a), 3), dtype=np.int32)
    tris[0::2] = t1
    tris[1::2] = t2
    return uv, tris


def icosphere(subdiv: int, radius: float, center):
    """Icosahedron refined ``subdiv`` times, projected to a sphere.

    5 refinements give 10,242 vertices and 20,480 triangles.  Outward
    counter-clockwise triangles.  Returns (verts float64, tris int32).
    """
    t = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9),
         (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2),
         (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts) * radius + np.asarray(center, dtype=np.float64)
    return V, np.array(faces, dtype=np.int32)


def box_mesh(lo, hi, subdiv: int):
    """Closed axis-aligned box surface, each face a subdiv-by-subdiv grid.

    Faces are refined so that obstacle triangles stay comparable in size to
    cloth triangles.  Outward counter-clockwise triangles; shared edge
    vertices are merged.
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    uv, tris = grid_mesh(subdiv + 1, subdiv + 1, 1.0, 1.0)
    verts = []
    faces = []
    # (axis held fixed, value side, u axis, v axis); u x v points outward
    specs = [(2, 1, 0, 1), (2, 0, 1, 0), (0, 1, 1, 2), (0, 0, 2, 1), (1, 1, 2, 0), (1, 0, 0, 2)]
    off = 0
    for ax, side, ua, va in specs:
        p = np.empty((len(uv), 3))
        p[:, ax] = hi[ax] if side else lo[ax]
        p[:, ua] = lo[ua] + uv[:, 0] * (hi[ua] - lo[ua])
        p[:, va] = lo[va] + uv[:, 1] * (hi[va] - lo[va])
        verts.append(p)
        faces.append(tris + off)
        off += len(p)
    V = np.concatenate(verts)
    F = np.concatenate(faces)
    key = np.round(V * 1e9).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    Vu = V[first]
    Fu = inv.ravel()[F]
    return Vu, Fu.astype(np.int32)


def cylinder_mesh(radius: float, length: float, n_theta: int, n_axial: int, center):
    """Open cylinder surface along z, centred at ``center``; outward normals."""
    th = np.arange(n_theta) * (2 * np.pi / n_theta)
    zz = np.linspace(-length / 2, length / 2, n_axial)
    T, Z = np.meshgrid(th, zz)
    V = np.stack([radius * np.cos(T).ravel(), radius * np.sin(T).ravel(), Z.ravel()], 1)
    V += np.asarray(center, dtype=np.float64)
    tris = []
    for j in range(n_axial - 1):
        for i in range(n_theta):
            a = j * n_theta + i
            b = j * n_theta + (i + 1) % n_theta
            c = a + n_theta
            d = b + n_theta
            tris += [(a, b, d), (a, d, c)]
    return V, np.array(tris, dtype=np.int32)


def cone_skirt(n_radial: int, n_axial: int, r_top: float, r_hem: float, length: float,
               pleats: int, pleat_amp: float, rng: np.random.Generator, top_z: float = 0.0):
    """Open conical tube (a skirt): ring j at height top_z - j*length/(n_axial-1).

    Radius varies linearly from r_top (j=0) to r_hem, modulated by
    pleat_amp*sin(pleats*theta + phase)*(axial fraction) with a seeded phase.
    Returns (verts, tris, top ring indices).
    """
    phase = rng.uniform(0, 2 * np.pi)
    th = np.arange(n_radial) * (2 * np.pi / n_radial)
    s = np.linspace(0.0, 1.0, n_axial)
    T, S = np.meshgrid(th, s)
    R = r_top + (r_hem - r_top) * S + pleat_amp * np.sin(pleats * T + phase) * S
    V = np.stack([(R * np.cos(T)).ravel(), (R * np.sin(T)).ravel(), (top_z - S * length).ravel()], 1)
    j, i = np.meshgrid(np.arange(n_axial - 1), np.arange(n_radial), indexing="ij")
    a = (j * n_radial + i).ravel()
    b = (j * n_radial + (i + 1) % n_radial).ravel()
    c = a + n_radial
    d = b + n_radial
    flip = ((i + j).ravel() % 2) == 1
    t1 = np.where(flip[:, None], np.stack([a, c, b], 1), np.stack([a, d, b], 1))
    t2 = np.where(flip[:, None], np.stack([b, c, d], 1), np.stack([a, c, d], 1))
    tris = np.empty((2 * len(a), 3), dtype=np.int32)
    tris[0::2] = t1
    tris[1::2] = t2
    return V, tris, np.arange(n_radial, dtype=np.int32)


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------

@dataclass
class Obstacle:
    """Kinematic triangle mesh.  ``transform(t)`` gives a 4x4 rigid transform
    applied to ``verts`` at time t (identity for a static obstacle)."""
    verts: np.ndarray
    tris: np.ndarray
    transform: Optional[Callable[[float], np.ndarray]] = None

    def positions(self, t: float) -> np.ndarray:
        if self.transform is None:
            return self.verts.astype(np.float32)
        m = self.transform(t)
        p = self.verts @ m[:3, :3].T + m[:3, 3]
        return p.astype(np.float32)


@dataclass
class Scene:
    """One synthetic cloth workload.

    verts float32 [n,3]; tris int32 [m,3]; pins int32 [p]; v0 float32 [n,3];
    ``pin_targets(t)`` gives float32 [p,3] pinned positions at time t.
    Material: density (kg/m^2), k_stretch, k_bend.  Solver settings listed
    in ``settings`` are scene-specific defaults (time step, iteration
    counts, subspace size, precision).
    """
    name: str
    verts: np.ndarray
    tris: np.ndarray
    pins: np.ndarray
    v0: np.ndarray
    density: float
    k_stretch: float
    k_bend: float
    obstacles: List[Obstacle] = field(default_factory=list)
    pin_targets: Optional[Callable[[float], np.ndarray]] = None
    settings: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.verts.shape[0])

    @property
    def m(self) -> int:
        return int(self.tris.shape[0])

    def pins_at(self, t: float) -> np.ndarray:
        if self.pin_targets is None:
            return self.verts[self.pins].astype(np.float32)
        return self.pin_targets(t).astype(np.float32)


def _jitter(rng, shape, amp):
    return rng.uniform(-amp, amp, size=shape)


def drape_sphere(side: int = 32, size: float = 1.0, seed: int = seed_for(0), sphere_subdiv: int = 4,
                 with_sphere: bool = True, jitter: float = 1e-4) -> Scene:
    """Square cloth draping over a fixed sphere (the paper's drape-on-a-sphere
    scene, Tab. 1, at 32x32 resolution): grid at z=0 over [0,1]^2, the two
    corners with j = side-1 pinned, sphere r=0.3 centred (0.5, 0.5, -0.35),
    density 0.1, stretch 1e3, bend 1e-2, gravity -9.8, dt 1/200, 32 LG
    iterations per step, seeded uniform jitter of +-1e-4 m on all coordinates."""
    rng = np.random.default_rng(seed)
    uv, tris = grid_mesh(side, side, size, size)
    V = np.zeros((len(uv), 3))
    V[:, :2] = uv
    V += _jitter(rng, V.shape, jitter)
    pins = np.array([(side - 1) * side, side * side - 1], dtype=np.int32)
    obs = []
    if with_sphere:
        sv, st = icosphere(sphere_subdiv, 0.3, (0.5 * size, 0.5 * size, -0.35))
        obs.append(Obstacle(sv, st))
    return Scene("drape_sphere_%d" % side, V.astype(np.float32), tris, pins,
                 np.zeros_like(V, dtype=np.float32), 0.1, 1e3, 1e-2, obs,
                 settings=dict(dt=1 / 200, steps=200, lg_iters=32))


def beam_strip(nx: int = 250, ny: int = 40, length: float = 1.0, width: float = 0.16, k_bend: float = 1.0,
               seed: int = seed_for(5), jitter: float = 1e-5) -> Scene:
    """Horizontal strip clamped at one end (the paper's bending-strip scene,
    Fig. beam: about 30 K DOFs, stiff bending, no collisions): an nx-by-ny
    grid over length x width at z = 0 with the first two columns (x = 0 and
    the next) pinned, so the clamp resists the bending moment of gravity.
    density 0.1, stretch 1e3, bend k_bend, dt 1/200; seeded jitter of
    +-1e-5 m on z only (the rest stays nearly flat)."""
    rng = np.random.default_rng(seed)
    uv, tris = grid_mesh(nx, ny, length, width)
    V = np.zeros((len(uv), 3))
    V[:, :2] = uv
    V[:, 2] = _jitter(rng, len(uv), jitter)
    pins = np.array([j * nx + i for j in range(ny) for i in range(2)], dtype=np.int32)
    return Scene("beam_strip_%dx%d" % (nx, ny), V.astype(np.float32), tris, pins,
                 np.zeros_like(V, dtype=np.float32), 0.1, 1e3, k_bend, [],
                 settings=dict(dt=1 / 200, steps=100, lg_iters=20))


def fold_on_box(side: int = 256, size: float = 2.0, seed: int = seed_for(1), box_subdiv: int = 32) -> Scene:
    """Cloth dropped flat onto the edge of a static unit box so that it folds
    over itself (a synthetic stand-in for the paper's folding scene): grid
    over 2x2 m, centre (0.5, 0, 1.0) i.e. 0.5 m above the box top face, box
    [-0.5,0.5]^3, no pins, per-vertex velocity noise N(0, 0.01) m/s."""
    rng = np.random.default_rng(seed)
    uv, tris = grid_mesh(side, side, size, size)
    V = np.zeros((len(uv), 3))
    V[:, 0] = uv[:, 0] - size / 2 + 0.5
    V[:, 1] = uv[:, 1] - size / 2
    V[:, 2] = 1.0
    v0 = rng.normal(0.0, 0.01, size=V.shape)
    bv, bt = box_mesh((-0.5, -0.5, -0.5), (0.5, 0.5, 0.5), box_subdiv)
    return Scene("fold_on_box_%d" % side, V.astype(np.float32), tris, np.zeros(0, np.int32),
                 v0.astype(np.float32), 0.1, 1e3, 1e-2, [Obstacle(bv, bt)],
                 settings=dict(dt=1 / 200, steps=500, lg_iters=64))


def hanging_swept(side: int = 512, size: float = 1.0, seed: int = seed_for(2), amp: float = 0.2,
                  freq: float = 1.0, jitter: float = 1e-4) -> Scene:
    """Vertical cloth in the x-z plane, top row (j = side-1, z = size) pinned
    and swept along x by amp*sin(2*pi*freq*t).  A seeded +-jitter offset in y
    keeps the sheet from being exactly planar."""
    rng = np.random.default_rng(seed)
    uv, tris = grid_mesh(side, side, size, size)
    V = np.zeros((len(uv), 3))
    V[:, 0] = uv[:, 0] - size / 2
    V[:, 2] = uv[:, 1]
    V[:, 1] = _jitter(rng, len(uv), jitter)
    pins = np.arange((side - 1) * side, side * side, dtype=np.int32)
    base = V[pins].copy()

    def targets(t):
        p = base.copy()
        p[:, 0] += amp * np.sin(2 * np.pi * freq * t)
        return p

    return Scene("hanging_swept_%d" % side, V.astype(np.float32), tris, pins,
                 np.zeros_like(V, dtype=np.float32), 0.1, 1e3, 1e-2, [], targets,
                 settings=dict(dt=1 / 200, r=256))


def batched_drape(count: int = 64, seed: int = seed_for(3), lo: int = 16, hi: int = 192) -> List[Scene]:
    """Independent square cloths of seeded sides in [lo, hi], 1 m wide, stretch
    stiffness log-uniform in [1e2, 1e4], each over its own sphere of radius
    uniform in [0.2, 0.4]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        side = int(rng.integers(lo, hi + 1))
        ks = float(10 ** rng.uniform(2, 4))
        rad = float(rng.uniform(0.2, 0.4))
        uv, tris = grid_mesh(side, side, 1.0, 1.0)
        V = np.zeros((len(uv), 3))
        V[:, :2] = uv
        V += _jitter(rng, V.shape, 1e-4)
        sv, st = icosphere(3, rad, (0.5, 0.5, -rad - 0.05))
        out.append(Scene("batched_%d_side%d" % (k, side), V.astype(np.float32), tris,
                         np.zeros(0, np.int32), np.zeros_like(V, dtype=np.float32),
                         0.1, ks, 1e-2, [Obstacle(sv, st)], settings=dict(dt=1 / 200, lg_iters=32)))
    return out


def skirt_on_body(n_radial: int = 1024, n_axial: int = 332, seed: int = seed_for(4)) -> Scene:
    """Garment-scale skirt: open cone (radius 0.15 at the top ring to 0.45 at
    the hem, length 0.6 m, 12 seeded pleats) whose top ring is pinned to a
    kinematic cylinder 'body' of radius 0.15 that translates at 0.5 m/s along
    x and rotates 180 degrees about z over 2 s."""
    rng = np.random.default_rng(seed)
    V, tris, top = cone_skirt(n_radial, n_axial, 0.15, 0.45, 0.6, 12, 0.02, rng, top_z=1.0)
    base = V[top].copy()
    cv, ct = cylinder_mesh(0.145, 0.8, 128, 32, (0.0, 0.0, 1.2))

    def rigid(t):
        ang = np.pi * min(t, 2.0) / 2.0
        c, s = np.cos(ang), np.sin(ang)
        m = np.eye(4)
        m[:3, :3] = [[c, -s, 0], [s, c, 0], [0, 0, 1]]
        m[0, 3] = 0.5 * t
        return m

    def targets(t):
        m = rigid(t)
        return base @ m[:3, :3].T + m[:3, 3]

    return Scene("skirt_%dx%d" % (n_radial, n_axial), V.astype(np.float32), tris, top,
                 np.zeros_like(V, dtype=np.float32), 0.1, 1e3, 1e-2,
                 [Obstacle(cv, ct, rigid)], targets, settings=dict(dt=1 / 200, steps=400, r=512))


def tiny_scene(side: int = 6, seed: int = 7, curved: bool = False, pinned: bool = True) -> Scene:
    """Very small jittered grid used by unit tests (optionally with a curved
    rest shape so that bending targets are non-zero)."""
    rng = np.random.default_rng(seed)
    uv, tris = grid_mesh(side, side, 0.5, 0.5)
    V = np.zeros((len(uv), 3))
    V[:, :2] = uv
    if curved:
        V[:, 2] = 0.15 * np.sin(2.0 * uv[:, 0]) * np.cos(1.5 * uv[:, 1])
    V += _jitter(rng, V.shape, 1e-3)
    pins = np.array([side * (side - 1), side * side - 1], dtype=np.int32) if pinned else np.zeros(0, np.int32)
    return Scene("tiny_%d" % side, V.astype(np.float32), tris, pins,
                 np.zeros_like(V, dtype=np.float32), 0.1, 1e3, 1e-2, settings=dict(dt=1 / 200))
