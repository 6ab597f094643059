"""FP64 projective-dynamics cloth stepper -- the ORACLE.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
the cpu_baseline leg of bench.py.  The CUDA library never calls it and shares
no code with it; the only shared module is ``workloads`` (seeded inputs).

Everything is double precision, written for a reader to check against the
paper (Lan et al., "Efficient GPU Cloth Simulation with Non-distance
Barriers and Subspace Reuse", arXiv 2403.19272):

  * implicit Euler as a minimisation, Sec. 3 Eq. (var) / (var_barrier), with
    the inertial target z of Eq. (z);
  * PD local step, Eq. (local): per-triangle stretch projection (closest
    column-orthonormal 3x2 to the deformation gradient) and per-hinge
    bending projection (quadratic cotangent stencil, keeps the rest
    magnitude);
  * PD global step, Eq. (global), assembled literally and solved EXACTLY by a
    sparse direct factorisation (this is what the GPU's subspace + Jacobi
    iteration approximates);
  * non-distance barrier weights w = k*K^a, Eq. (exp), with a counting
    consecutive active LG iterations, collision constraints with
    A_i = B_i = Id (Sec. 5.1), partial CCD (Sec. 4.1) and exact CCD;
  * the step pipeline of Alg. 1 / Sec. 7 (warm start, initial CCD filter,
    outer/inner loops, exit line search with alpha * t_TOI).

Readings where the paper is silent (stretch model, bending stencil, contact
target, thresholds) are documented beside the code that takes them.

Pins (tests/test_oracle_pins.py; each checks the oracle against something
other than itself):
  Model (masses, H)        total mass = density * area; H symmetric positive
                           definite, elastic rows sum to zero
  stretch_targets          polar factor orthonormal, rotation-equivariant,
                           minimal against random rotations (brute force)
  bend_targets             planar null space and a fold identity of the stencil
  rhs / solve / residual   dense Cholesky; closed-form free fall; rest states
                           (rotated, pinned) are fixed points; PD energy
                           decreases per LG iteration
  contact_terms (R6)       targets land exactly on C = 0, least-norm among
                           random feasible moves, identity when inactive
  ndb_* (Eq. exp)          life-span counters and weights of a scripted
                           active/inactive sequence written out by hand
                           (consecutive count, reset, cap, w = k K^a), driven
                           by the partial CCD of a vertex moved across the
                           activity threshold; the step's own trace obeys them
  CollisionMesh.candidates contains every pair that collides (brute force)
  Oracle.step              the closed forms above through the whole step, no
                           triangle intersections on a drape, residual
                           forwarding: exact 2 dx shift of the next z, dx ~ 0
                           after an exact free fall, residual decrease
  collide (C)              closest points against dense search; CCD golden
                           cases and dense time sampling; partial-CCD identity
  pccd_adaptive            rho* scale/translation invariant; lattice covers its
                           domain to h/sqrt(2); flags every crossing with
                           t* <= alpha (the argument of Eq. sample_bound)
The production mode (1e-3 relative residual, mixed precision) is parity
unpinned: its error against this oracle is reported, not gated.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import collide, pccd_adaptive


# ----------------------------------------------------------------------------
# parameters
# ----------------------------------------------------------------------------

@dataclass
class Params:
    """Solver settings (same meaning as the C-ABI's pdc_params)."""
    dt: float = 1.0 / 200
    gravity: Tuple[float, float, float] = (0.0, 0.0, -9.8)
    k_ndb_scale: float = 1.0       # k = k_ndb_scale * mean(diag H) over free vertices
    K_ndb: float = 2.0             # growth base K of Eq. (exp)
    a_max: int = 20                # cap on the life-span counter a
    alpha: float = 0.8             # line-search factor of Sec. 4.1 / Sec. 6
    dhat: float = 1e-3             # gap of the activity test and contact target
    eta: float = 1e-9              # exact-CCD contact distance
    tol_outer: float = 1e-3        # ||dx||_inf / L between outer passes (Sec. 7)
    tol_inner: float = 5e-2        # ||dx||_inf / L between inner iterations (Sec. 7)
    tol_rel_residual: float = 0.0  # > 0: inner loop stops on relative PD residual instead
    max_outer: int = 4
    max_inner: int = 32
    warm_iters: int = 5
    samples_vt: int = 3
    samples_ee: int = 4
    collisions: bool = True
    fixed_iters: bool = False      # parity mode: run exactly warm/max_outer/max_inner
    rf_toi: float = 0.0            # residual forwarding (Sec. 6) when the exit TOI is below this (0: off)
    rf_iters: int = 8              # cap on its LG iterations (exact count in parity mode)
    pccd_adaptive: bool = False    # partial-CCD samples from Eq. (sample_bound) instead of fixed patterns
    pccd_max_axis: int = 64        # cap on the per-axis lattice size of the adaptive samples


# ----------------------------------------------------------------------------
# rest model
# ----------------------------------------------------------------------------

def _cot(u, v):
    """cot of the angle between vectors u and v (rows)."""
    c = np.einsum("ij,ij->i", u, v)
    s = np.linalg.norm(np.cross(u, v), axis=1)
    return c / s


class Model:
    """Rest-state quantities of one cloth mesh (Sec. 3, Eq. (local)/(global)).

    stretch: F_t = [x1-x0, x2-x0] Dm^-1 (3x2, Dm from an orthonormal frame of
             the rest triangle), weight w_t = k_stretch * A_t.  F_t = sum_j
             x_j g_{t,j}^T with g1, g2 the rows of Dm^-1 and g0 = -g1-g2.
    bend:    hinge (x0, x1 | x2, x3) with shared edge x0-x1 and opposite
             vertices x2 (triangle A) and x3 (triangle B); stencil
             K = (cot a_A1 + cot a_B1, cot a_A0 + cot a_B0, -cot a_A0 - cot a_A1,
                  -cot a_B0 - cot a_B1), a_Ti the rest angle at x_i in triangle
             T (the quadratic bending model of Bergou et al. 2006 cited in
             Sec. 2); weight w_h = 3 k_bend / (A_A + A_B); rest magnitude
             |sum_j K_j X_j|.
    mass:    lumped, m_v = density * sum_{t contains v} A_t / 3.
    H:       M/h^2 + sum_t w_t G_t G_t^T + sum_h w_h K_h K_h^T (scalar n x n,
             shared by x, y, z), Eq. (global) without contacts.
    """

    def __init__(self, verts, tris, pins, density, k_stretch, k_bend, dt):
        X = np.asarray(verts, dtype=np.float64)
        T = np.asarray(tris, dtype=np.int64)
        self.X, self.T = X, T
        self.n, self.m = len(X), len(T)
        self.h = float(dt)
        self.pins = np.asarray(pins, dtype=np.int64)
        self.free = np.ones(self.n, dtype=bool)
        self.free[self.pins] = False

        # --- triangles
        e1 = X[T[:, 1]] - X[T[:, 0]]
        e2 = X[T[:, 2]] - X[T[:, 0]]
        nrm = np.cross(e1, e2)
        self.area = 0.5 * np.linalg.norm(nrm, axis=1)
        t1 = e1 / np.linalg.norm(e1, axis=1)[:, None]
        t2 = np.cross(nrm, t1)
        t2 /= np.linalg.norm(t2, axis=1)[:, None]
        Dm = np.empty((self.m, 2, 2))
        Dm[:, 0, 0] = np.einsum("ij,ij->i", e1, t1)
        Dm[:, 0, 1] = np.einsum("ij,ij->i", e2, t1)
        Dm[:, 1, 0] = np.einsum("ij,ij->i", e1, t2)
        Dm[:, 1, 1] = np.einsum("ij,ij->i", e2, t2)
        Dinv = np.linalg.inv(Dm)
        G = np.empty((self.m, 3, 2))
        G[:, 1] = Dinv[:, 0]
        G[:, 2] = Dinv[:, 1]
        G[:, 0] = -G[:, 1] - G[:, 2]
        self.G = G
        self.w_t = k_stretch * self.area

        # --- edges and hinges
        ed = {}
        for ti, (a, b, c) in enumerate(T):
            for (u, v, o) in ((a, b, c), (b, c, a), (c, a, b)):
                key = (min(u, v), max(u, v))
                ed.setdefault(key, []).append((ti, o))
        self.edges = np.array(sorted(ed.keys()), dtype=np.int64).reshape(-1, 2)
        hin = []
        for (u, v), lst in sorted(ed.items()):
            if len(lst) == 2:
                hin.append((u, v, lst[0][1], lst[1][1], lst[0][0], lst[1][0]))
        hin = np.array(hin, dtype=np.int64).reshape(-1, 6)
        self.hinges = hin[:, :4]
        if len(hin):
            x0, x1, x2, x3 = (X[hin[:, i]] for i in range(4))
            cA0 = _cot(x1 - x0, x2 - x0)
            cA1 = _cot(x0 - x1, x2 - x1)
            cB0 = _cot(x1 - x0, x3 - x0)
            cB1 = _cot(x0 - x1, x3 - x1)
            K = np.stack([cA1 + cB1, cA0 + cB0, -cA0 - cA1, -cB0 - cB1], axis=1)
            self.Kh = K
            self.w_h = 3.0 * k_bend / (self.area[hin[:, 4]] + self.area[hin[:, 5]])
            s_rest = np.einsum("hj,hjd->hd", K, X[self.hinges])
            self.s_rest = s_rest
            self.s_rest_len = np.linalg.norm(s_rest, axis=1)
        else:
            self.Kh = np.zeros((0, 4))
            self.w_h = np.zeros(0)
            self.s_rest = np.zeros((0, 3))
            self.s_rest_len = np.zeros(0)

        # --- mass
        self.mass = np.zeros(self.n)
        np.add.at(self.mass, T.ravel(), np.repeat(density * self.area / 3.0, 3))

        # --- H
        rows, cols, vals = [], [], []
        for a in range(3):
            for b in range(3):
                rows.append(T[:, a])
                cols.append(T[:, b])
                vals.append(self.w_t * np.einsum("ij,ij->i", G[:, a], G[:, b]))
        for a in range(4):
            for b in range(4):
                rows.append(self.hinges[:, a])
                cols.append(self.hinges[:, b])
                vals.append(self.w_h * self.Kh[:, a] * self.Kh[:, b])
        rows.append(np.arange(self.n))
        cols.append(np.arange(self.n))
        vals.append(self.mass / self.h ** 2)
        self.H = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.n, self.n))
        self.H.sum_duplicates()
        self.diagH = self.H.diagonal()
        lo, hi = X.min(0), X.max(0)
        self.L = float(np.linalg.norm(hi - lo))  # bounding-box diagonal

    # ------------------------------------------------------------------ local
    def stretch_targets(self, x):
        """R_t = closest 3x2 matrix with orthonormal columns to F_t (polar
        factor, via thin SVD F = U S V^T -> R = U V^T).  Rank-deficient F
        (sigma_2 <= 1e-12 sigma_1): Gram-Schmidt of F's columns, completed
        with the direction orthogonal to column 1 inside the rest frame when
        column 2 vanishes."""
        F = np.einsum("tjd,tjk->tdk", x[self.T], self.G)
        U, S, Vt = np.linalg.svd(F, full_matrices=False)
        R = U @ Vt
        bad = S[:, 1] <= 1e-12 * np.maximum(S[:, 0], 1e-300)
        for t in np.nonzero(bad)[0]:
            R[t] = _gram_schmidt(F[t])
        return R

    def bend_targets(self, x):
        """s_hat = |s_rest| * s/|s|, s = sum_j K_j x_j (zero when the rest
        magnitude is zero; the rest vector when s vanishes)."""
        if len(self.hinges) == 0:
            return np.zeros((0, 3))
        s = np.einsum("hj,hjd->hd", self.Kh, x[self.hinges])
        ln = np.linalg.norm(s, axis=1)
        out = np.where(ln[:, None] > 1e-300, s * (self.s_rest_len / np.where(ln > 1e-300, ln, 1.0))[:, None],
                       self.s_rest)
        return out

    def rhs(self, x, z, contact_w=None, contact_y=None):
        """b of Eq. (global): M z/h^2 + sum_t w_t S^T A^T B y + sum_h ... +
        sum_c w_c y_c.  Contacts enter as per-vertex weights and weighted
        targets (A_i = B_i = Id, Sec. 5.1)."""
        b = (self.mass / self.h ** 2)[:, None] * z
        R = self.stretch_targets(x)
        contrib = self.w_t[:, None, None] * np.einsum("tdk,tjk->tjd", R, self.G)
        for a in range(3):
            np.add.at(b, self.T[:, a], contrib[:, a])
        if len(self.hinges):
            sh = self.bend_targets(x)
            for a in range(4):
                np.add.at(b, self.hinges[:, a], (self.w_h * self.Kh[:, a])[:, None] * sh)
        if contact_y is not None:
            b += contact_y
        return b

    def solve(self, b, x_pinned_src, contact_w=None):
        """Exact solution of (H + dH) x = b over free vertices, pinned rows
        held at x_pinned_src (Dirichlet)."""
        A = self.H
        if contact_w is not None and np.any(contact_w):
            A = A + sp.diags(contact_w)
        A = A.tocsr()
        f = self.free
        x = x_pinned_src.copy()
        rhs = b[f] - A[f][:, ~f] @ x_pinned_src[~f]
        lu = spla.splu(A[f][:, f].tocsc())
        x[f] = lu.solve(rhs)
        return x

    def residual(self, x, z, contact_w=None, contact_y=None):
        """PD residual (H + dH) x - b(x) over free vertices (Eq. (global)
        with the projections evaluated at x)."""
        b = self.rhs(x, z, contact_w, contact_y)
        A = self.H
        r = A @ x - b
        if contact_w is not None:
            r += contact_w[:, None] * x
        return r[self.free]

    def energy(self, x, z, R=None, sh=None, contact_w=None, contact_y=None):
        """PD energy E(x; y) with fixed projections (R, s_hat, contact
        targets): inertia + sum_t w_t/2 |F_t - R_t|^2 + sum_h w_h/2 |s_h -
        s_hat_h|^2 + sum_c w_c/2 |x_c - y_c|^2 (contact_y holds w_c*y_c)."""
        if R is None:
            R = self.stretch_targets(x)
        if sh is None:
            sh = self.bend_targets(x)
        d = x - z
        E = 0.5 / self.h ** 2 * np.sum(self.mass[:, None] * d * d)
        F = np.einsum("tjd,tjk->tdk", x[self.T], self.G)
        E += 0.5 * np.sum(self.w_t * np.sum((F - R) ** 2, axis=(1, 2)))
        if len(self.hinges):
            s = np.einsum("hj,hjd->hd", self.Kh, x[self.hinges])
            E += 0.5 * np.sum(self.w_h * np.sum((s - sh) ** 2, axis=1))
        if contact_w is not None:
            nz = contact_w > 0
            y = contact_y[nz] / contact_w[nz][:, None]
            E += 0.5 * np.sum(contact_w[nz][:, None] * (x[nz] - y) ** 2)
        return E


def _gram_schmidt(F):
    c1 = F[:, 0]
    n1 = np.linalg.norm(c1)
    if n1 <= 1e-300:
        c1 = np.array([1.0, 0.0, 0.0])
    else:
        c1 = c1 / n1
    c2 = F[:, 1] - np.dot(F[:, 1], c1) * c1
    n2 = np.linalg.norm(c2)
    if n2 <= 1e-12 * max(n1, 1e-300):
        a = np.eye(3)[np.argmin(np.abs(c1))]
        c2 = a - np.dot(a, c1) * c1
        c2 /= np.linalg.norm(c2)
    else:
        c2 = c2 / n2
    return np.stack([c1, c2], axis=1)


# ----------------------------------------------------------------------------
# collision bookkeeping
# ----------------------------------------------------------------------------

class CollisionMesh:
    """Cloth + kinematic obstacles as one vertex / triangle / edge set.

    Vertex ids: cloth vertices first, then each obstacle's vertices in the
    order the obstacles were added.  Triangle ids likewise.  Vertices with id
    >= n_cloth are kinematic (infinite mass)."""

    def __init__(self, model: Model, obstacles):
        self.model = model
        self.nc = model.n
        tris = [model.T]
        off = model.n
        self.obs_slices = []
        for ob in obstacles:
            tris.append(np.asarray(ob.tris, dtype=np.int64) + off)
            self.obs_slices.append((off, off + len(ob.verts)))
            off += len(ob.verts)
        self.nv = off
        self.tris = np.concatenate(tris)
        ed = set()
        for a, b, c in self.tris:
            for u, v in ((a, b), (b, c), (c, a)):
                ed.add((min(u, v), max(u, v)))
        self.edges = np.array(sorted(ed), dtype=np.int64).reshape(-1, 2)
        self.fixed_v = np.zeros(self.nv, dtype=bool)  # infinite mass (obstacle or pinned)
        self.fixed_v[self.nc:] = True
        self.fixed_v[model.pins] = True

    def candidates(self, X0, X1, dhat):
        """All candidate pairs as an array [k,4] of vertex ids and kind [k]
        plus dict keys; VT keys ('vt', v, t), EE keys ('ee', a, b, c, d)."""
        vt, ee = collide.broadphase(X0, X1, self.nc, self.tris, self.edges, dhat)
        quads, kind, keys = [], [], []
        for v, t in vt:
            a, b, c = self.tris[t]
            quads.append((v, a, b, c))
            kind.append(0)
            keys.append(("vt", int(v), int(t)))
        for e, f in ee:
            a, b = self.edges[e]
            c, d = self.edges[f]
            quads.append((a, b, c, d))
            kind.append(1)
            keys.append(("ee", int(a), int(b), int(c), int(d)))
        return np.array(quads, dtype=np.int64).reshape(-1, 4), np.array(kind, dtype=np.int64), keys


def contact_normal(q0, kind, coef):
    """n0 = unit gap vector at the t=0 closest points; fallback to the
    triangle normal (VT) or the edge cross product (EE) when the gap is 0."""
    d = coef @ q0
    ln = np.linalg.norm(d)
    if ln > 1e-300:
        return d / ln
    if kind == 0:
        nn = np.cross(q0[2] - q0[1], q0[3] - q0[1])
    else:
        nn = np.cross(q0[1] - q0[0], q0[3] - q0[2])
    ln = np.linalg.norm(nn)
    return nn / ln if ln > 1e-300 else np.array([0.0, 0.0, 1.0])


def contact_terms(cm: CollisionMesh, Xall0, xall, active, quads, kinds, weights, dhat):
    """Collision constraint projections (Sec. 5.1: A_i = B_i = Id).

    For an active pair with gap vector d(x) = sum_j c_j x_j (c from the t=0
    closest points on x^-) and unit start direction n0 = d(x^-)/|d(x^-)|,
    the constraint is C(x) = d(x).n0 - dhat >= 0.  Its projection moves each
    non-fixed vertex j by -min(C,0) c_j n0 / sum_k c_k^2 (sum over non-fixed
    k): the least-norm displacement that satisfies C = 0.  Every non-fixed
    vertex of the pair gets a spring of weight w_i to its target (A_i = B_i =
    Id on the pair's vertices; a vertex with c_j = 0 is held at its current
    position), so the per-vertex sums are  dH_jj = sum_i w_i  and
    (w y)_j = sum_i w_i y_ij.
    Returns (contact_w [n], contact_wy [n,3]) over cloth vertices."""
    n = cm.nc
    cw = np.zeros(n)
    cy = np.zeros((n, 3))
    for i in np.nonzero(active)[0]:
        q = quads[i]
        kind = kinds[i]
        q0 = Xall0[q].astype(np.float64)
        coef = collide.closest_coef(q0, kind)
        n0 = contact_normal(q0, kind, coef)
        qx = xall[q]
        C = float(coef @ qx @ n0) - dhat
        movable = [(j, coef[j]) for j in range(4) if not cm.fixed_v[q[j]]]
        S = sum(c * c for _, c in movable)
        if S <= 0:
            continue
        for j, c in movable:
            y = qx[j] - min(C, 0.0) * c * n0 / S
            cw[q[j]] += weights[i]
            cy[q[j]] += weights[i] * y
    return cw, cy


# ----------------------------------------------------------------------------
# non-distance barrier bookkeeping (Sec. 4, Eq. exp)
# ----------------------------------------------------------------------------

def ndb_weight(k, K, a):
    """Eq. (exp): the weight of a constraint whose life-span counter is a,
    w = k * K^a (a may be an array)."""
    return k * np.power(float(K), np.asarray(a, dtype=np.float64))


def ndb_after_partial_ccd(state, keys, flags, a_max):
    """Constraint set after one partial CCD (Sec. 4.1) of one LG iteration.

    state maps a pair key to (active, a).  a counts the consecutive LG
    iterations in which the pair has been active (Sec. 4, text of Eq. exp):
    a pair flagged now that was active before keeps counting, a <- a + 1
    (capped at a_max); a pair flagged now that was not active starts at 0;
    a pair not flagged is inactive and leaves the set, so its counter starts
    again from 0 when it is next flagged."""
    new_state = {}
    for i, kk in enumerate(keys):
        if flags[i]:
            was, a = state.get(kk, (False, 0))
            new_state[kk] = (True, min(a + 1, a_max) if was else 0)
    return new_state


def ndb_after_full_ccd(state, keys, toi):
    """Constraint set after a full CCD over the fresh candidate list keys
    (Alg. 1, FullCCD): a pair with an impact in [0, 1] becomes active and
    keeps the counter it had (0 when it was not active); an active pair
    without an impact stays active with its counter; pairs that are no
    longer candidates leave the set."""
    new_state = {}
    for i, kk in enumerate(keys):
        act, a = state.get(kk, (False, 0))
        if toi[i] <= 1.0:
            act = True
        if act:
            new_state[kk] = (act, a)
    return new_state


# ----------------------------------------------------------------------------
# the step (Alg. 1, Sec. 7)
# ----------------------------------------------------------------------------

@dataclass
class StepStats:
    warm_iters: int = 0
    outer_iters: int = 0
    inner_iters: int = 0
    t_toi: float = 1.0
    s: float = 1.0
    n_candidates: int = 0
    n_active: int = 0
    rf_iters: int = 0              # residual-forwarding LG iterations run after this step
    rf_res0: float = 0.0           # |residual| of the forwarding problem at the filtered x
    rf_res1: float = 0.0           # ... and after its iterations
    rel_residual: float = 0.0     # relative PD residual (R11); with collisions on, the last one the
                                  # stopping test of the relative-residual mode measured
    constraints: dict = field(default_factory=dict)  # the constraint set (key -> (active, a)) at the exit
    log: list = field(default_factory=list)


class Oracle:
    """FP64 stepper.  State: x, v (cloth), obstacle positions."""

    def __init__(self, scene, params: Params):
        self.p = params
        self.scene = scene
        self.model = Model(scene.verts, scene.tris, scene.pins, scene.density, scene.k_stretch,
                           scene.k_bend, params.dt)
        self.cm = CollisionMesh(self.model, scene.obstacles)
        self.x = scene.verts.astype(np.float64).copy()
        self.v = scene.v0.astype(np.float64).copy()
        self.t = 0.0
        self.obs = [o.positions(0.0).astype(np.float64) for o in scene.obstacles]
        f = self.model.free
        self.k = params.k_ndb_scale * float(np.mean(self.model.diagH[f])) if np.any(f) else 1.0
        self.rf = None  # residual-forwarding displacement dx for the next step (Sec. 6)

    # --- helpers
    def _all(self, x_cloth, obs):
        if not obs:
            return x_cloth
        return np.concatenate([x_cloth] + list(obs))

    def _lg(self, x, z, pin_x, contact=None):
        """One LG iteration: local projections at x, exact global solve."""
        cw, cy = (None, None) if contact is None else contact
        b = self.model.rhs(x, z, cw, cy)
        src = x.copy()
        src[~self.model.free] = pin_x
        return self.model.solve(b, src, cw)

    def rel_residual(self, x, z, contact=None):
        cw, cy = (None, None) if contact is None else contact
        return float(np.linalg.norm(self.model.residual(x, z, cw, cy)))

    def step(self, x_star=None, v_star=None, pin_next=None, obs_next=None, trace=None):
        """Advance one time step; returns (x_new, v_new, stats).

        trace (a list, optional) receives one record per inner LG iteration:
        the constraint set it started from, the NDB weights and activity each
        candidate pair had in its contact springs, the partial-CCD flags after
        its global solve (and each pair's activity margin, min over samples of
        Q - dhat |p2^0 - p1^0|) and the constraint set those flags produced."""
        p, M = self.p, self.model
        h = p.dt
        if x_star is None:
            x_star, v_star = self.x, self.v
        x_star = np.asarray(x_star, dtype=np.float64)
        v_star = np.asarray(v_star, dtype=np.float64)
        if pin_next is None:
            pin_next = self.scene.pins_at(self.t + h).astype(np.float64)
        if obs_next is None:
            obs_next = [o.positions(self.t + h).astype(np.float64) for o in self.scene.obstacles]
        L = M.L
        st = StepStats()

        # Eq. (z): z = x* + h v* + h^2 M^-1 f_ext with f_ext = m g; with residual
        # forwarding (Eq. z_rf) h^2 M^-1 df = 2 dx of the previous step's RF
        z = x_star + h * v_star + h * h * np.asarray(p.gravity)[None, :]
        if self.rf is not None:
            z = z + 2.0 * self.rf
            self.rf = None
        z[~M.free] = pin_next
        x = z.copy()
        rho0 = self.rel_residual(x, z)
        st.log.append(("rho0", rho0))

        # warm start: LG iterations of I + Psi without collisions (Alg. 1)
        for it in range(p.warm_iters):
            if p.tol_rel_residual > 0 and not p.fixed_iters:
                if self.rel_residual(x, z) <= p.tol_rel_residual * rho0:
                    break
            xn = self._lg(x, z, pin_next)
            dx = np.max(np.abs(xn - x)) if len(x) else 0.0
            x = xn
            st.warm_iters += 1
            if not p.fixed_iters and p.tol_rel_residual <= 0 and dx <= p.tol_inner * L:
                break

        if not p.collisions:
            # without collision handling the inner LG loop of Alg. 1 still runs,
            # with no springs, partial CCD or full CCD
            for it in range(p.max_inner):
                if p.tol_rel_residual > 0 and not p.fixed_iters:
                    if self.rel_residual(x, z) <= p.tol_rel_residual * rho0:
                        break
                xn = self._lg(x, z, pin_next)
                st.inner_iters += 1
                dx = np.max(np.abs(xn - x)) if len(x) else 0.0
                x = xn
                if not p.fixed_iters and p.tol_rel_residual <= 0 and dx <= p.tol_inner * L:
                    break
            x_new = x
            st.rel_residual = self.rel_residual(x_new, z) / max(rho0, 1e-300)
            v_new = (x_new - x_star) / h
            self.x, self.v, self.t = x_new, v_new, self.t + h
            return x_new, v_new, st

        cm = self.cm
        obs0 = self.obs
        X0 = self._all(x_star, obs0).astype(np.float32)

        # initial full CCD from x* to the warm-start result and filter
        X1 = self._all(x, obs_next).astype(np.float32)
        quads, kinds, keys = cm.candidates(X0, X1, p.dhat)
        toi = collide.ccd(X0, X1, quads, kinds, p.eta)
        t0 = float(toi.min()) if len(toi) else 2.0
        s0 = 1.0 if t0 > 1.0 else p.alpha * t0
        xm_all = X0.astype(np.float64) + s0 * (X1.astype(np.float64) - X0.astype(np.float64))
        # x^- of the constrained solve (Alg. 1: x^- <- x after the filter)
        xm = xm_all[: cm.nc].copy()
        obs_m = [xm_all[a:b] for a, b in cm.obs_slices]
        pin_m = xm[~M.free].copy()
        state: Dict = ndb_after_full_ccd({}, keys, toi)
        # the iterate starts at x^- with pinned rows at their targets
        x = xm.copy()
        x[~M.free] = pin_next
        Xm32 = xm_all.astype(np.float32)

        def full_ccd(xp):
            Xp = self._all(xp, obs_next).astype(np.float32)
            qd, kd, ky = cm.candidates(Xm32, Xp, p.dhat)
            tt = collide.ccd(Xm32, Xp, qd, kd, p.eta)
            tmin = float(tt.min()) if len(tt) else 2.0
            return qd, kd, ky, ndb_after_full_ccd(state, ky, tt), tmin

        # the first inner loop uses the candidates of the initial full CCD; the
        # first outer pass always ends with a full CCD (pinned rows of x^+ sit
        # at their targets even if no inner iteration ran); later passes
        # without an inner iteration leave x^+ unchanged and reuse the result
        t_toi = 2.0
        x_outer_prev = xm.copy()
        for o in range(p.max_outer):
            st.outer_iters += 1
            inner_done = 0
            for it in range(p.max_inner):
                act = np.array([state.get(kk, (False, 0))[0] for kk in keys], dtype=bool)
                aa = np.array([state.get(kk, (False, 0))[1] for kk in keys], dtype=np.int64)
                w = ndb_weight(self.k, p.K_ndb, aa)
                xall = self._all(x, obs_next)
                contact = contact_terms(cm, xm_all, xall, act, quads, kinds, w, p.dhat)
                if p.tol_rel_residual > 0 and not p.fixed_iters:
                    rho = self.rel_residual(x, z, contact)
                    st.rel_residual = rho / max(rho0, 1e-300)  # the last value the stopping test saw
                    if rho <= p.tol_rel_residual * rho0:
                        break
                xn = self._lg(x, z, pin_next, contact)
                st.inner_iters += 1
                inner_done += 1
                # partial CCD (Sec. 4.1) on the candidates over (x^-, x^+)
                Xp = self._all(xn, obs_next).astype(np.float32)
                if p.pccd_adaptive:
                    flags, margin = pccd_adaptive.partial_ccd_adaptive(Xm32, Xp, quads, kinds, p.dhat, p.alpha,
                                                                       p.pccd_max_axis)[:2]
                else:
                    flags, margin = collide.partial_ccd(Xm32, Xp, quads, kinds, p.samples_vt, p.samples_ee, p.dhat)
                if trace is not None:
                    trace.append(dict(state_in=dict(state), weights=dict(zip(keys, w)), active=dict(zip(keys, act)),
                                      flags=dict(zip(keys, np.asarray(flags, dtype=bool))),
                                      margins=dict(zip(keys, np.asarray(margin, dtype=np.float64)))))
                state = ndb_after_partial_ccd(state, keys, flags, p.a_max)
                if trace is not None:
                    trace[-1]["state"] = dict(state)
                dx = np.max(np.abs(xn - x))
                x = xn
                if not p.fixed_iters and p.tol_rel_residual <= 0 and dx <= p.tol_inner * L:
                    break
            if inner_done > 0 or o == 0:
                quads, kinds, keys, state, t_toi = full_ccd(x)
            dxo = np.max(np.abs(x - x_outer_prev))
            x_outer_prev = x.copy()
            if not p.fixed_iters and dxo <= p.tol_outer * L:
                break

        # exit line search (Alg. 1): x <- x^- + s (x^+ - x^-)
        s = 1.0 if t_toi > 1.0 else p.alpha * t_toi
        xall_p = self._all(x, obs_next).astype(np.float32).astype(np.float64)
        xall_new = xm_all + s * (xall_p - xm_all)
        x_new = xall_new[: cm.nc]
        self.obs = [xall_new[a:b] for a, b in cm.obs_slices]
        st.t_toi, st.s = t_toi, s
        st.constraints = dict(state)
        st.n_candidates = len(keys)
        st.n_active = sum(1 for v in state.values() if v[0])

        # residual forwarding (Sec. 6, end of Alg. 1): after a small exit TOI,
        # more LG iterations of this step's problem from the filtered x, with
        # every active constraint at weight k (a = 0) and no CCD; the change
        # dx is carried to the next step's z (Eq. z_rf, h^2 M^-1 df = 2 dx).
        # Pinned rows stay where the filter left them.
        if p.rf_toi > 0 and t_toi < p.rf_toi:
            act = np.array([state.get(kk, (False, 0))[0] for kk in keys], dtype=bool)
            w = np.full(len(keys), self.k)
            pin_f = x_new[~M.free].copy()
            xr = x_new.copy()
            rf_contact = lambda xx: contact_terms(cm, xm_all, self._all(xx, self.obs), act, quads, kinds, w, p.dhat)
            st.rf_res0 = self.rel_residual(xr, z, rf_contact(xr))
            for it in range(p.rf_iters):
                contact = rf_contact(xr)
                xn = self._lg(xr, z, pin_f, contact)
                st.rf_iters += 1
                dx = np.max(np.abs(xn - xr)) if len(xr) else 0.0
                xr = xn
                if not p.fixed_iters and dx <= p.tol_inner * L:
                    break
            st.rf_res1 = self.rel_residual(xr, z, rf_contact(xr))
            self.rf = xr - x_new
            self.rf[~M.free] = 0.0
        v_new = (x_new - x_star) / h
        self.x, self.v, self.t = x_new, v_new, self.t + h
        return x_new, v_new, st
