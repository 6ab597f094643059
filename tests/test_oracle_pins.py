"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test ties an oracle function to something other than itself: a closed
form of the paper's equations, a geometric identity, a hand-built case with
a known answer (tests/golden) or an exhaustive search.  CPU only.
"""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import collide, pd, subspace

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rot(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


# ----------------------------------------------------------------------------
# rest model
# ----------------------------------------------------------------------------

def test_lumped_mass_total_is_density_times_area():
    sc = wl.tiny_scene(side=9)
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    uv, _ = wl.grid_mesh(9, 9, 0.5, 0.5)
    assert abs(m.mass.sum() - 0.1 * m.area.sum()) < 1e-15
    assert abs(m.area.sum() - 0.25) < 5e-4  # jittered 0.5 x 0.5 sheet


def test_H_rows_and_definiteness():
    sc = wl.tiny_scene(side=7, curved=True)
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    H = m.H.toarray()
    assert np.allclose(H, H.T, atol=1e-9)
    # stiffness rows annihilate translations: H 1 = M / h^2  (Eq. (global))
    assert np.allclose(H.sum(1), m.mass / m.h ** 2, rtol=1e-9, atol=1e-9 * np.abs(H).max())
    ev = np.linalg.eigvalsh(H)
    assert ev.min() > 0


def test_deformation_gradient_is_isometry_at_rest_and_equivariant():
    rng = np.random.default_rng(3)
    sc = wl.tiny_scene(side=5, curved=True)
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    X = m.X
    F = np.einsum("tjd,tjk->tdk", X[m.T], m.G)
    FtF = np.einsum("tdk,tdl->tkl", F, F)
    assert np.allclose(FtF, np.eye(2)[None], atol=1e-12)
    Q = _rot(rng)
    Y = X @ Q.T + rng.normal(size=3)
    F2 = np.einsum("tjd,tjk->tdk", Y[m.T], m.G)
    assert np.allclose(F2, np.einsum("de,tek->tdk", Q, F), atol=1e-12)


def test_polar_projection_orthonormal_equivariant_minimal():
    rng = np.random.default_rng(4)
    sc = wl.tiny_scene(side=5)
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    x = m.X + 0.02 * rng.normal(size=m.X.shape)
    R = m.stretch_targets(x)
    assert np.allclose(np.einsum("tdk,tdl->tkl", R, R), np.eye(2)[None], atol=1e-12)
    Q = _rot(rng)
    R2 = m.stretch_targets(x @ Q.T)
    assert np.allclose(R2, np.einsum("de,tek->tdk", Q, R), atol=1e-10)
    F = np.einsum("tjd,tjk->tdk", x[m.T], m.G)
    best = np.sum((F - R) ** 2, axis=(1, 2))
    for _ in range(200):
        Rr, _ = np.linalg.qr(rng.normal(size=(len(F), 3, 2)))
        # compare with random frames nudged toward R: still not closer
        Rn, _ = np.linalg.qr(R + 0.05 * rng.normal(size=R.shape))
        for cand in (Rr, Rn):
            assert np.all(np.sum((F - cand) ** 2, axis=(1, 2)) >= best - 1e-12)


def test_bending_stencil_planar_nullspace_and_fold_identity():
    """For a hinge the stencil sum_j K_j x_j vanishes on planar shapes and
    has length 2|e| sin(theta/2) when the rest-flat hinge is folded
    isometrically by dihedral angle theta (cotangent-weight identity)."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        P = rng.normal(size=(4, 3))
        P[:, 2] = 0
        e = P[1] - P[0]
        nrm = np.array([-e[1], e[0], 0.0])
        if np.dot(P[2] - P[0], nrm) * np.dot(P[3] - P[0], nrm) > 0:
            P[3] -= 2 * np.dot(P[3] - P[0], nrm) / np.dot(nrm, nrm) * nrm
        m = pd.Model(P, np.array([[0, 1, 2], [1, 0, 3]]), [], 1, 1, 1, 0.01)
        assert m.hinges.tolist() == [[0, 1, 2, 3]]
        K = m.Kh[0]
        assert abs(K.sum()) < 1e-12
        assert np.linalg.norm(K @ P) < 1e-12 * np.abs(K).max()
        Q3 = _rot(rng)
        Pp = P @ Q3.T + 1.0
        assert np.linalg.norm(K @ Pp) < 1e-11 * np.abs(K).max()
        a = e / np.linalg.norm(e)
        for th in (0.05, 0.7, 2.0):
            v = P[3] - P[0]
            vr = v * np.cos(th) + np.cross(a, v) * np.sin(th) + a * np.dot(a, v) * (1 - np.cos(th))
            Qp = P.copy()
            Qp[3] = P[0] + vr
            assert abs(np.linalg.norm(K @ Qp) - 2 * np.linalg.norm(e) * np.sin(th / 2)) < 1e-11 * np.abs(K).max()


# ----------------------------------------------------------------------------
# whole-step closed forms
# ----------------------------------------------------------------------------

def _params(**kw):
    p = pd.Params(collisions=False, warm_iters=3, tol_inner=1e-14)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_free_fall_matches_closed_form_with_elasticity_on():
    """Eq. (var) with a rigidly translating rest-shape cloth: every
    projection is exact, so each step returns x = z of Eq. (z) and
    x_n = x_0 + n h v_0 + h^2 g n (n+1) / 2,  v_n = v_0 + n h g."""
    sc = wl.tiny_scene(side=6, curved=True, pinned=False)
    v0 = np.array([0.3, -0.1, 0.2])
    sc.v0 = np.tile(v0, (sc.n, 1)).astype(np.float32)
    v0 = sc.v0[0].astype(np.float64)  # the state is stored in float32
    p = _params()
    o = pd.Oracle(sc, p)
    x0 = sc.verts.astype(np.float64)
    g = np.array(p.gravity)
    h = p.dt
    for n in range(1, 9):
        x, v, _ = o.step()
        xe = x0 + n * h * v0 + h * h * g * n * (n + 1) / 2
        ve = v0 + n * h * g
        assert np.max(np.abs(x - xe)) < 1e-12
        assert np.max(np.abs(v - ve)) < 1e-9


def test_rotated_rest_shape_is_stationary():
    rng = np.random.default_rng(6)
    sc = wl.tiny_scene(side=6, curved=True, pinned=False)
    Q = _rot(rng)
    sc.verts = sc.verts.astype(np.float64)
    p = _params(gravity=(0.0, 0.0, 0.0))
    o = pd.Oracle(sc, p)
    xr = o.model.X @ Q.T + np.array([0.1, 0.2, 0.3])
    x, v, _ = o.step(xr, np.zeros_like(xr), pin_next=np.zeros((0, 3)), obs_next=[])
    assert np.max(np.abs(x - xr)) < 1e-12


def test_rest_state_with_pins_and_no_gravity_is_fixed_point():
    sc = wl.tiny_scene(side=7, curved=True)
    p = _params(gravity=(0.0, 0.0, 0.0))
    o = pd.Oracle(sc, p)
    X = o.model.X.copy()
    for _ in range(3):
        x, v, _ = o.step()
    assert np.max(np.abs(x - X)) < 1e-12


def test_pd_energy_monotone_per_lg_iteration():
    """Local step = exact minimisation over projections, global step = exact
    minimisation over x (Eq. (global)): the PD energy never increases."""
    rng = np.random.default_rng(7)
    sc = wl.tiny_scene(side=8, curved=True)
    m = pd.Model(sc.verts, sc.tris, sc.pins, sc.density, sc.k_stretch, sc.k_bend, 0.005)
    z = m.X + 0.03 * rng.normal(size=m.X.shape)
    x = m.X + 0.05 * rng.normal(size=m.X.shape)
    x[~m.free] = m.X[~m.free]
    z[~m.free] = m.X[~m.free]
    E_prev = m.energy(x, z)
    for _ in range(12):
        b = m.rhs(x, z)
        R, sh = m.stretch_targets(x), m.bend_targets(x)
        xn = m.solve(b, x)
        E_mid = m.energy(xn, z, R, sh)  # new x, old projections
        E_new = m.energy(xn, z)  # new projections
        assert E_mid <= E_prev * (1 + 1e-12)
        assert E_new <= E_mid * (1 + 1e-12)
        E_prev, x = E_new, xn


def test_exact_global_solve_matches_dense():
    rng = np.random.default_rng(8)
    sc = wl.tiny_scene(side=6)
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    b = rng.normal(size=(m.n, 3))
    cw = np.where(rng.random(m.n) < 0.3, 50.0, 0.0)
    x = m.solve(b, m.X, cw)
    A = m.H.toarray() + np.diag(cw)
    f = m.free
    xe = m.X.copy()
    xe[f] = np.linalg.solve(A[np.ix_(f, f)], b[f] - A[np.ix_(f, ~f)] @ m.X[~f])
    assert np.max(np.abs(x - xe)) < 1e-10 * np.max(np.abs(xe))


# ----------------------------------------------------------------------------
# CCD
# ----------------------------------------------------------------------------

def test_ccd_golden_cases():
    cases = json.load(open(os.path.join(GOLDEN, "ccd_cases.json")))["cases"]
    for c in cases:
        t = collide.ccd_single(np.array(c["x0"], float), np.array(c["x1"], float), c["kind"], 1e-9)
        if c["toi"] is None:
            assert t > 1.0, c["name"]
        else:
            assert abs(t - c["toi"]) < 1e-12, (c["name"], t)


def _vt_first_crossing(q0, q1, ts):
    """First sample time at which the vertex has crossed the (moving)
    triangle's plane at a point inside the triangle (vectorised over ts)."""
    Q = q0[None] + ts[:, None, None] * (q1 - q0)[None]
    n = np.cross(Q[:, 2] - Q[:, 1], Q[:, 3] - Q[:, 1])
    s = np.einsum("ij,ij->i", Q[:, 0] - Q[:, 1], n)
    flip = np.nonzero(np.signbit(s[1:]) != np.signbit(s[:-1]))[0] + 1
    for k in flip:
        q = Q[k]
        # the crossing point at the interval's midpoint must be inside
        qm = 0.5 * (Q[k - 1] + Q[k])
        nm = np.cross(qm[2] - qm[1], qm[3] - qm[1])
        p = qm[0] - np.dot(qm[0] - qm[1], nm) / np.dot(nm, nm) * nm
        a, b, c = qm[1], qm[2], qm[3]
        s1 = np.dot(np.cross(b - a, p - a), nm)
        s2 = np.dot(np.cross(c - b, p - b), nm)
        s3 = np.dot(np.cross(a - c, p - c), nm)
        m = min(abs(s1), abs(s2), abs(s3)) / np.dot(nm, nm)
        if ((s1 > 0 and s2 > 0 and s3 > 0) or (s1 < 0 and s2 < 0 and s3 < 0)) and m > 1e-3:
            return ts[k]
    return None


def test_ccd_vt_against_dense_time_sampling():
    """A vertex that crosses the triangle's plane well inside the triangle
    between two sample times must get a TOI no later than that interval; a
    reported TOI must put the vertex on the triangle's plane."""
    rng = np.random.default_rng(9)
    ts = np.linspace(0, 1, 4001)
    hits = 0
    for _ in range(400):
        q0 = rng.normal(size=(4, 3))
        q0[0] = q0[1:].mean(0) + rng.normal(size=3) * 0.7
        q1 = q0 + rng.normal(size=(4, 3)) * 1.2
        toi = collide.ccd_single(q0, q1, 0, 1e-9)
        first = _vt_first_crossing(q0, q1, ts)
        if first is not None:
            hits += 1
            assert toi <= first + 1e-12
        if toi <= 1.0:
            q = q0 + toi * (q1 - q0)
            n = np.cross(q[2] - q[1], q[3] - q[1])
            assert abs(np.dot(q[0] - q[1], n)) / np.linalg.norm(n) < 1e-8
    assert hits > 20


def test_ccd_ee_against_dense_time_sampling():
    rng = np.random.default_rng(10)
    ts = np.linspace(0, 1, 4001)
    hits = 0
    for _ in range(400):
        q0 = rng.normal(size=(4, 3))
        q1 = q0 + rng.normal(size=(4, 3)) * 1.5
        toi = collide.ccd_single(q0, q1, 1, 1e-9)
        Q = q0[None] + ts[:, None, None] * (q1 - q0)[None]
        s = np.einsum("ij,ij->i", np.cross(Q[:, 1] - Q[:, 0], Q[:, 3] - Q[:, 2]), Q[:, 2] - Q[:, 0])
        first = None
        for k in np.nonzero(np.signbit(s[1:]) != np.signbit(s[:-1]))[0] + 1:
            q = 0.5 * (Q[k - 1] + Q[k])
            d1, d2, r = q[1] - q[0], q[3] - q[2], q[0] - q[2]
            A = np.array([[d1 @ d1, -d1 @ d2], [-d1 @ d2, d2 @ d2]])
            st = np.linalg.solve(A, [-d1 @ r, d2 @ r])
            if 1e-3 < st[0] < 1 - 1e-3 and 1e-3 < st[1] < 1 - 1e-3:
                first = ts[k]
                break
        if first is not None:
            hits += 1
            assert toi <= first + 1e-12
    assert hits > 20


def test_partial_ccd_query_identity_at_crossing():
    """Eq. (collision_judge): at the contact point lambda* of a pair that
    meets at t*, Q(lambda*) = (t*-1)/t* |p2^0 - p1^0|^2 <= 0."""
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(400):
        q0 = rng.normal(size=(4, 3))
        q1 = q0 + rng.normal(size=(4, 3)) * 1.5
        t = collide.ccd_single(q0, q1, 0, 1e-9)
        if not (1e-3 < t <= 1.0):
            continue
        qt = q0 + t * (q1 - q0)
        c = collide.closest_coef(qt, 0)  # contact point barycentrics at t*
        d0 = c @ q0
        d1 = c @ q1
        Q = float(d1 @ d0)
        assert abs(Q - (t - 1) / t * float(d0 @ d0)) < 1e-7 * max(1.0, float(d0 @ d0) / t)
        assert Q <= 1e-9
        checked += 1
    assert checked > 20


def test_partial_ccd_flags_crossing_and_not_separating():
    # vertex crosses the triangle: active for every sample pattern
    q0 = np.array([[0.2, 0.2, 1.0], [0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    q1 = q0.copy()
    q1[0, 2] = -1.0
    for ns in (0, 1, 3):
        act, mar = collide.partial_ccd(q0, q1, np.array([[0, 1, 2, 3]]), np.array([0]), ns, 4, 0.0)
        assert act[0] and mar[0] < 0
    # vertex moves away: inactive
    q1 = q0.copy()
    q1[0, 2] = 2.0
    act, _ = collide.partial_ccd(q0, q1, np.array([[0, 1, 2, 3]]), np.array([0]), 3, 4, 0.0)
    assert not act[0]
    # within dhat and not separating: active (sufficiently close, Sec. 4)
    q0[0, 2] = 5e-4
    q1 = q0.copy()
    act, _ = collide.partial_ccd(q0, q1, np.array([[0, 1, 2, 3]]), np.array([0]), 3, 4, 1e-3)
    assert act[0]


# ----------------------------------------------------------------------------
# broad phase, non-penetration
# ----------------------------------------------------------------------------

def _facing_sheets(n1, d):
    """Two parallel sheets whose gap is exactly fl32(z + d_hat), shifted so
    that facing primitives satisfy the FP32 predicate with equality on z."""
    g = np.linspace(0.0, 0.5, n1, dtype=np.float32)
    xx, yy = np.meshgrid(g, g, indexing="ij")
    za = np.float32(0.3)
    zb = np.float32(za + np.float32(d))
    A = np.stack([xx.ravel(), yy.ravel(), np.full(n1 * n1, za, np.float32)], 1)
    B = np.stack([xx.ravel() + np.float32(0.013), yy.ravel(), np.full(n1 * n1, zb, np.float32)], 1)
    T = []
    for i in range(n1 - 1):
        for j in range(n1 - 1):
            a, b, c, e = i * n1 + j, (i + 1) * n1 + j, i * n1 + j + 1, (i + 1) * n1 + j + 1
            T += [[a, b, c], [b, e, c]]
    T = np.array(T, np.int32)
    return np.concatenate([A, B]).astype(np.float32), np.concatenate([T, T + n1 * n1]).astype(np.int32)


def test_broadphase_grid_equals_the_brute_force():
    """The grid-culled lists (for sizes the brute force cannot reach) equal
    the brute-force definition: a swept drape with an obstacle, and two
    sheets exactly d_hat apart (pairs on the predicate boundary), for grid
    cells far smaller and far larger than the primitives."""
    rng = np.random.default_rng(31)
    sc = wl.drape_sphere(side=12, sphere_subdiv=2)
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    cm = pd.CollisionMesh(m, sc.obstacles)
    X0 = np.concatenate([sc.verts] + [o.positions(0.0) for o in sc.obstacles]).astype(np.float32)
    X1 = X0.copy()
    X1[: sc.n] += (rng.normal(size=(sc.n, 3)) * 0.01 + np.array([0, 0, -0.05])).astype(np.float32)
    cases = [(X0, X1, cm.nc, cm.tris, cm.edges, 1e-3)]
    V, T = _facing_sheets(9, 1e-3)
    ms = pd.Model(V, T, np.zeros(0, np.int32), 0.1, 1e3, 1e-2, 0.005)
    cs = pd.CollisionMesh(ms, [])
    cases.append((V, V, cs.nc, cs.tris, cs.edges, 1e-3))
    for X0_, X1_, nc, tris, edges, d in cases:
        vt_b, ee_b = collide.broadphase(X0_, X1_, nc, tris, edges, d)
        assert len(vt_b) > 50 and len(ee_b) > 50
        vt_b = vt_b[np.lexsort((vt_b[:, 1], vt_b[:, 0]))]
        ee_b = ee_b[np.lexsort((ee_b[:, 1], ee_b[:, 0]))]
        for cell in (None, 2e-3, 0.02, 0.3, 2.0):
            vt_g, ee_g = collide.broadphase_grid(X0_, X1_, nc, tris, edges, d, cell)
            assert np.array_equal(vt_g, vt_b), cell
            assert np.array_equal(ee_g, ee_b), cell


def test_broadphase_contains_every_colliding_pair():
    rng = np.random.default_rng(12)
    sc = wl.tiny_scene(side=6)
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    X0 = m.X.astype(np.float32)
    X1 = (m.X + 0.08 * rng.normal(size=m.X.shape)).astype(np.float32)
    cm = pd.CollisionMesh(m, [])
    quads, kinds, keys = cm.candidates(X0, X1, 1e-3)
    cand = set(keys)
    # every VT / EE pair of the mesh that collides must be a candidate
    allq, allk, allkeys = [], [], []
    for v in range(m.n):
        for t, (a, b, c) in enumerate(m.T):
            if v in (a, b, c):
                continue
            allq.append((v, a, b, c)); allk.append(0); allkeys.append(("vt", v, t))
    E = cm.edges
    for i in range(len(E)):
        for j in range(i + 1, len(E)):
            if set(E[i]) & set(E[j]):
                continue
            allq.append((*E[i], *E[j])); allk.append(1); allkeys.append(("ee", *E[i], *E[j]))
    toi = collide.ccd(X0, X1, np.array(allq), np.array(allk), 1e-9)
    hit = [allkeys[i] for i in np.nonzero(toi <= 1.0)[0]]
    assert len(hit) > 0
    assert all(h in cand for h in hit)


def test_oracle_drape_is_penetration_free():
    """Sec. 7: the exit CCD line search keeps every step intersection free
    (cloth-cloth and cloth-sphere)."""
    sc = wl.drape_sphere(side=12, sphere_subdiv=2)
    p = pd.Params(max_outer=2, max_inner=6)
    o = pd.Oracle(sc, p)
    allT = o.cm.tris
    for k in range(25):
        x, v, st = o.step()
        X = np.concatenate([x] + o.obs)
        assert len(collide.intersecting_triangle_pairs(X, allT)) == 0
    assert x[:, 2].min() < -0.04  # it did reach the sphere


# ----------------------------------------------------------------------------
# closest points and the contact projection (Sec. 4.1, Sec. 5.1 / R6)
# ----------------------------------------------------------------------------

def _dense_vt(p, a, b, c, m=400):
    u, v = np.meshgrid(np.linspace(0, 1, m + 1), np.linspace(0, 1, m + 1))
    keep = (u + v) <= 1.0
    u, v = u[keep], v[keep]
    pts = a[None, :] + u[:, None] * (b - a)[None, :] + v[:, None] * (c - a)[None, :]
    return float(np.min(np.linalg.norm(pts - p[None, :], axis=1)))


def _dense_ee(a0, a1, b0, b1, m=600):
    s_, t_ = np.meshgrid(np.linspace(0, 1, m + 1), np.linspace(0, 1, m + 1))
    s_, t_ = s_.ravel(), t_.ravel()
    pa = a0[None, :] + s_[:, None] * (a1 - a0)[None, :]
    pb = b0[None, :] + t_[:, None] * (b1 - b0)[None, :]
    return float(np.min(np.linalg.norm(pa - pb, axis=1)))


def test_closest_points_match_a_dense_search():
    """The gap vector sum_j c_j q_j of closest_coef has the length of the
    minimum distance found by a dense barycentric (VT) or (s, t) (EE) search,
    its coefficients sum to zero (translation invariance) and the closest
    points lie on the primitives; cases include projections outside the
    triangle (clamped to an edge or a corner) and nearly parallel edges."""
    rng = np.random.default_rng(11)
    cases_vt = [rng.normal(size=(4, 3)) for _ in range(12)]
    cases_vt.append(np.array([[2.0, 2.0, 0.3], [0, 0, 0], [1, 0, 0], [0, 1, 0]]))   # beyond the hypotenuse
    cases_vt.append(np.array([[-1.0, -1.0, 0.2], [0, 0, 0], [1, 0, 0], [0, 1, 0]]))  # beyond a corner
    for q in cases_vt:
        c = collide.closest_coef(q, 0)
        assert abs(c.sum()) < 1e-12 and c[0] == -1.0
        assert np.all(c[1:] >= -1e-12) and abs(c[1:].sum() - 1.0) < 1e-12
        d = float(np.linalg.norm(c @ q))
        dd = _dense_vt(q[0], q[1], q[2], q[3])
        scale = float(np.max(np.linalg.norm(q[1:] - q[1], axis=1)))
        assert d <= dd + 1e-12 and dd - d <= 2e-3 * scale
    cases_ee = [rng.normal(size=(4, 3)) for _ in range(12)]
    cases_ee.append(np.array([[0, 0, 0], [1, 0, 0], [0.2, 0.5, 1e-9], [1.2, 0.5, 0.0]]))  # nearly parallel
    for q in cases_ee:
        c = collide.closest_coef(q, 1)
        assert abs(c.sum()) < 1e-12
        s_, t_ = -c[1], c[3]
        assert -1e-12 <= s_ <= 1 + 1e-12 and -1e-12 <= t_ <= 1 + 1e-12
        d = float(np.linalg.norm(c @ q))
        dd = _dense_ee(q[0], q[1], q[2], q[3])
        scale = float(max(np.linalg.norm(q[1] - q[0]), np.linalg.norm(q[3] - q[2])))
        assert d <= dd + 1e-12 and dd - d <= 2e-3 * scale


def test_contact_projection_is_the_least_norm_move_onto_the_gap_plane():
    """R6 (Sec. 5.1 with A = B = Id): for an active pair whose gap along the
    start direction is below dhat, the spring targets put the pair exactly on
    C = 0, and no other displacement of the movable vertices that does so is
    shorter (random feasible alternatives); an obstacle vertex gets no
    spring; on the inactive side (C >= 0) each target is the vertex itself."""
    from types import SimpleNamespace
    dhat = 1e-3
    # vertex 0 above triangle (1, 2, 3); all cloth (movable), or 3 = obstacle
    X0 = np.array([[0.3, 0.3, 2 * dhat], [0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
    x = X0.copy()
    x[0, 2] = 0.3 * dhat            # moved into the gap band
    x[1:, 2] += 0.1 * dhat           # the triangle rose a little
    quads = np.array([[0, 1, 2, 3]])
    kinds = np.array([0])
    w = np.array([5.0])
    for fixed in ([False, False, False, False], [False, False, False, True]):
        cm = SimpleNamespace(nc=4, fixed_v=np.array(fixed))
        cw, cy = pd.contact_terms(cm, X0, x, np.array([True]), quads, kinds, w, dhat)
        coef = collide.closest_coef(X0, 0)
        n0 = pd.contact_normal(X0, 0, coef)
        mov = [j for j in range(4) if not fixed[j]]
        assert all(cw[j] == 5.0 for j in mov) and all(cw[j] == 0.0 for j in range(4) if fixed[j])
        y = x.copy()
        for j in mov:
            y[j] = cy[j] / cw[j]
        assert abs(float(coef @ y @ n0) - dhat) < 1e-15
        move = y - x
        base = float(np.sum(move ** 2))
        rng = np.random.default_rng(5)
        for _ in range(200):
            eta = np.zeros_like(x)
            eta[mov] = rng.normal(size=(len(mov), 3)) * 1e-3
            # keep the alternative on the plane: remove the component of eta that changes C
            g = np.zeros_like(x)
            g[mov] = coef[mov][:, None] * n0[None, :]
            eta -= (np.sum(g * eta) / np.sum(g * g)) * g
            assert float(np.sum((move + eta) ** 2)) >= base - 1e-18
    # inactive side: C >= 0 at x leaves every target at its vertex
    x2 = X0.copy()
    cm = SimpleNamespace(nc=4, fixed_v=np.zeros(4, bool))
    cw, cy = pd.contact_terms(cm, X0, x2, np.array([True]), quads, kinds, w, dhat)
    assert np.allclose(cy / cw[:, None], x2, rtol=0, atol=1e-15)


# ----------------------------------------------------------------------------
# adaptive partial-CCD sample density (Eq. sample_bound)
# ----------------------------------------------------------------------------

def test_sample_bound_is_scale_and_translation_invariant():
    """rho* is a length ratio in parameter space: scaling or translating the
    pair (both times) leaves it unchanged."""
    from oracle import pccd_adaptive as pa
    rng = np.random.default_rng(4)
    for kind in (0, 1):
        for _ in range(5):
            q0, q1 = rng.normal(size=(4, 3)), rng.normal(size=(4, 3))
            r = pa.sample_bound(q0, q1, kind, 0.8)
            sh = rng.normal(size=3)
            assert pa.sample_bound(3.7 * q0 + sh, 3.7 * q1 + sh, kind, 0.8) == pytest.approx(r, rel=1e-10)


def test_sample_lattice_covers_its_domain():
    """Every point of the parameter domain (VT: b1, b2 >= 0, b1 + b2 <= 1;
    EE: the unit square) lies within h / sqrt(2) of a lattice sample."""
    from oracle import pccd_adaptive as pa
    rng = np.random.default_rng(9)
    for kind in (0, 1):
        for m in (1, 3, 7):
            L = pa.lattice(kind, m)
            P = rng.uniform(size=(2000, 2))
            if kind == 0:
                P = P[P.sum(axis=1) <= 1.0]
            d = np.min(np.linalg.norm(P[:, None, :] - L[None, :, :], axis=2), axis=1)
            assert d.max() <= (1.0 / m) / np.sqrt(2.0) + 1e-12


def test_adaptive_density_flags_every_crossing_before_alpha():
    """Sec. 4.1: a pair whose exact time of impact is at most alpha has
    Q < 0 on a disc of radius rho* around the contact parameters, so the
    lattice of spacing <= sqrt(2) rho* flags it (random VT and EE crossings
    whose elements are comparable in size to their distance, so that the
    lattice stays below its cap)."""
    from oracle import pccd_adaptive as pa
    rng = np.random.default_rng(7)
    alpha, checked = 0.8, 0
    for trial in range(700):
        kind = trial % 2
        if kind == 0:
            q0 = np.zeros((4, 3))
            q0[1:] = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]]) + rng.normal(size=(3, 3)) * 0.05
            q0[0] = [rng.uniform(-0.2, 1.0), rng.uniform(-0.2, 1.0), rng.uniform(0.3, 1.5)]
            q1 = q0.copy()
            q1[0] = [rng.uniform(-0.2, 1.0), rng.uniform(-0.2, 1.0), -rng.uniform(0.3, 1.5)]
            q1[1:] += rng.normal(size=(3, 3)) * 0.05
        else:
            q0 = np.array([[0, 0, 0], [1, 0, 0], [0, 0, 0], [0, 1, 0]], dtype=float) + rng.normal(size=(4, 3)) * 0.05
            q0[2:] += [rng.uniform(0, 0.5), rng.uniform(-0.5, 0), rng.uniform(0.3, 1.2)]
            q1 = q0.copy()
            q1[2:, 2] -= rng.uniform(0.6, 2.5)
            q1 += rng.normal(size=(4, 3)) * 0.05
        q0, q1 = q0.astype(np.float32), q1.astype(np.float32)
        toi = collide.ccd(q0, q1, np.arange(4)[None, :], np.array([kind]), 1e-9)[0]
        if not (0.0 < toi <= alpha):
            continue
        act, _, m, cap = pa.partial_ccd_adaptive(q0, q1, np.arange(4)[None, :], [kind], 0.0, alpha, 64)
        if cap[0]:
            continue
        assert act[0], (trial, kind, toi, m[0])
        checked += 1
    assert checked >= 100


def test_oracle_drape_with_adaptive_samples_is_penetration_free():
    """The step with adaptive partial-CCD samples (Eq. sample_bound) still
    keeps every step intersection free (the exit line search guarantees it)
    and reaches the sphere."""
    sc = wl.drape_sphere(side=10, sphere_subdiv=2)
    o = pd.Oracle(sc, pd.Params(max_outer=2, max_inner=4, pccd_adaptive=True, pccd_max_axis=16))
    allT = o.cm.tris
    for k in range(22):
        x, v, st = o.step()
        X = np.concatenate([x] + o.obs)
        assert len(collide.intersecting_triangle_pairs(X, allT)) == 0
    assert x[:, 2].min() < -0.04


# ----------------------------------------------------------------------------
# residual forwarding (Sec. 6, Eq. z_rf, end of Alg. 1)
# ----------------------------------------------------------------------------

def test_residual_forwarding_shifts_the_next_z_by_twice_dx():
    """Eq. z_rf with h^2 M^-1 df = 2 dx: with no LG iteration the step
    returns z, which must be x* + h v* + h^2 g + 2 dx on free rows (pins at
    their targets); the forwarded dx is used once."""
    sc = wl.tiny_scene(side=6, curved=True, pinned=True)
    p = pd.Params(collisions=False, fixed_iters=True, warm_iters=0, max_inner=0)
    o = pd.Oracle(sc, p)
    rng = np.random.default_rng(3)
    D = rng.normal(size=(sc.n, 3)) * 1e-3
    D[~o.model.free] = 0.0
    o.rf = D.copy()
    xs, vs = o.x.copy(), o.v.copy()
    h, g = p.dt, np.array(p.gravity)
    x, v, _ = o.step()
    ze = xs + h * vs + h * h * g + 2.0 * D
    ze[~o.model.free] = sc.pins_at(h)
    assert np.max(np.abs(x - ze)) < 1e-14
    assert o.rf is None
    x2, _, _ = o.step()
    ze2 = x + h * v + h * h * g
    ze2[~o.model.free] = sc.pins_at(2 * h)
    assert np.max(np.abs(x2 - ze2)) < 1e-14


def test_residual_forwarding_leaves_an_exact_free_fall_unchanged():
    """A rigidly translating rest shape ends every step at the minimiser
    x = z (up to the FP32 rounding of the filtered state on the collision
    path, ~1e-8 m here), so forwarding (forced after every step: rf_toi above
    the no-impact value 2) must find dx ~ 0 (a dx measured from x* instead of
    the filtered x would be ~h|v| = 2 mm) and keep the closed-form trajectory
    x_n = x_0 + n h v_0 + h^2 g n (n+1) / 2."""
    sc = wl.tiny_scene(side=6, curved=True, pinned=False)
    v0 = np.array([0.3, -0.1, 0.2])
    sc.v0 = np.tile(v0, (sc.n, 1)).astype(np.float32)
    v0 = sc.v0[0].astype(np.float64)
    p = _params(collisions=True, rf_toi=3.0, rf_iters=4)
    o = pd.Oracle(sc, p)
    x0 = sc.verts.astype(np.float64)
    g = np.array(p.gravity)
    h = p.dt
    for n in range(1, 7):
        x, v, st = o.step()
        assert st.rf_iters > 0
        assert np.max(np.abs(o.rf)) < 1e-7
        xe = x0 + n * h * v0 + h * h * g * n * (n + 1) / 2
        assert np.max(np.abs(x - xe)) < 1e-6


def test_residual_forwarding_lowers_the_residual_of_its_problem():
    """After a filtered step with a small exit TOI (a drape thrown at the
    sphere, two inner iterations), the forwarding iterations decrease the
    PD residual of their problem (weights k, no CCD) and leave pinned rows
    unmoved."""
    sc = wl.drape_sphere(side=10, sphere_subdiv=2)
    v0 = sc.v0.copy()
    v0[:, 2] -= 20.0
    sc.v0 = v0.astype(np.float32)
    p = pd.Params(max_outer=1, max_inner=2, rf_toi=1.01, rf_iters=20, tol_inner=1e-14)
    o = pd.Oracle(sc, p)
    x, v, st = o.step()
    assert st.t_toi < 1.0 and st.rf_iters == 20
    assert st.rf_res1 < 0.6 * st.rf_res0
    assert np.all(o.rf[~o.model.free] == 0.0) and np.all(np.isfinite(o.rf))
    assert np.max(np.abs(o.rf)) > 0.0


# ----------------------------------------------------------------------------
# subspace reference
# ----------------------------------------------------------------------------

def test_subspace_correction_exact_for_in_span_solution():
    rng = np.random.default_rng(13)
    sc = wl.tiny_scene(side=7)
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    f = m.free
    H = m.H.tocsr()
    cw = np.where(rng.random(m.n) < 0.2, 30.0, 0.0) * f
    A = m.H.toarray() + np.diag(cw)
    # U has the exact solution direction in its span
    sol = np.zeros((m.n, 3))
    sol[f] = rng.normal(size=(f.sum(), 3))
    r = A @ sol
    r[~f] = 0
    B = np.concatenate([sol, rng.normal(size=(m.n, 5))], axis=1)
    B[~f] = 0
    U, _ = np.linalg.qr(B)
    delta, q = subspace.subspace_correction(U, H, cw, r)
    assert np.max(np.abs(delta - sol)) < 1e-9 * np.max(np.abs(sol))
    # Galerkin: q minimises 1/2 y^T A y - r^T y over y = U q
    def J(qq):
        y = U @ qq
        return 0.5 * np.sum(y * (A @ y)) - np.sum(r * y)
    for _ in range(20):
        assert J(q) <= J(q + 1e-3 * rng.normal(size=q.shape)) + 1e-12


def test_jacobi_relaxes_high_frequencies_and_the_subspace_the_low_modes():
    """Sec. 5 / Fig. error_projection on a clamped bending strip: the error of
    a gravity load lies in the lowest modes of H (eigenvectors from scipy's
    shift-invert Lanczos), 100 damped Jacobi sweeps leave it untouched while
    the Galerkin correction in the 30 lowest modes removes it; an error made
    only of modes above the 60th is relaxed by the same sweeps."""
    import scipy.sparse.linalg as sla
    sc = wl.beam_strip(nx=100, ny=16)
    m = pd.Model(sc.verts, sc.tris, sc.pins, sc.density, sc.k_stretch, sc.k_bend, 0.005)
    f = m.free
    Hf = m.H.tocsr()[f][:, f].tocsc()
    rhs = m.mass[f, None] * np.array([0.0, 0.0, -9.8])[None, :]
    ex = np.column_stack([sla.spsolve(Hf, rhs[:, k]) for k in range(3)])
    w, V = sla.eigsh(Hf, k=60, sigma=0, which="LM")
    d = Hf.diagonal()
    om = min(1.0, 1.8 / np.max(np.abs(Hf).sum(axis=1).A1 / d))
    free = np.ones(len(d), dtype=bool)
    assert np.linalg.norm(V[:, :10].T @ ex) >= 0.99 * np.linalg.norm(ex)  # low-frequency load
    jac = subspace.jacobi(Hf, None, rhs, np.zeros_like(rhs), 100, om, free)
    assert np.linalg.norm(jac - ex) >= 0.99 * np.linalg.norm(ex)
    d0, _ = subspace.subspace_correction(V[:, :30], Hf, None, rhs)
    assert np.linalg.norm(d0 - ex) <= 1e-3 * np.linalg.norm(ex)
    rng = np.random.default_rng(0)
    xh = rng.normal(size=(Hf.shape[0], 3))
    xh -= V @ (V.T @ xh)  # only modes above the 60th
    jh = subspace.jacobi(Hf, None, Hf @ xh, np.zeros_like(xh), 100, om, free)
    assert np.linalg.norm(jh - xh) <= 0.2 * np.linalg.norm(xh)


def test_jacobi_reference_converges_to_exact_solve():
    rng = np.random.default_rng(14)
    sc = wl.tiny_scene(side=5)
    m = pd.Model(sc.verts, sc.tris, sc.pins, 1.0, 1.0, 1e-4, 0.005)  # diagonally dominant
    r = rng.normal(size=(m.n, 3))
    r[~m.free] = 0
    d = subspace.jacobi(m.H, None, r, np.zeros_like(r), 400, 1.0, m.free)
    A = m.H.toarray()
    f = m.free
    ex = np.zeros_like(r)
    ex[f] = np.linalg.solve(A[np.ix_(f, f)], r[f])
    assert np.max(np.abs(d - ex)) < 1e-8 * np.max(np.abs(ex))


# ----------------------------------------------------------------------------
# non-distance barrier life span (Sec. 4, Eq. exp)
# ----------------------------------------------------------------------------

def test_ndb_counter_and_weight_follow_a_scripted_flag_sequence():
    """Eq. (exp): w = k K^a with a the number of consecutive LG iterations a
    constraint has been active.  Seven partial-CCD results for three pairs,
    with the counters and weights written out by hand (k = 5, K = 2,
    a_max = 3): A stays flagged (0, 1, 2, 3, then held at the cap), drops
    out once and restarts at 0; B comes and goes; C is never flagged."""
    flags = [  # A, B, C
        (1, 0, 0),
        (1, 1, 0),
        (1, 0, 0),
        (1, 1, 0),
        (1, 1, 0),
        (0, 1, 0),
        (1, 1, 0),
    ]
    expect_a = [
        {"A": 0},
        {"A": 1, "B": 0},
        {"A": 2},
        {"A": 3, "B": 0},
        {"A": 3, "B": 1},
        {"B": 2},
        {"A": 0, "B": 3},
    ]
    expect_w = [
        {"A": 5.0},
        {"A": 10.0, "B": 5.0},
        {"A": 20.0},
        {"A": 40.0, "B": 5.0},
        {"A": 40.0, "B": 10.0},
        {"B": 20.0},
        {"A": 5.0, "B": 40.0},
    ]
    keys = ["A", "B", "C"]
    state = {}
    for f, ea, ew in zip(flags, expect_a, expect_w):
        state = pd.ndb_after_partial_ccd(state, keys, f, 3)
        assert {k: a for k, (act, a) in state.items() if act} == ea
        assert set(state) == set(ea)  # inactive pairs leave the set
        got_w = {k: float(pd.ndb_weight(5.0, 2.0, a)) for k, (act, a) in state.items()}
        assert got_w == ew


def test_ndb_full_ccd_keeps_counters_and_activates_impacts_at_zero():
    """Alg. 1 FullCCD: a pair with an impact in [0, 1] joins the set at a = 0,
    an active pair keeps its counter whether or not it has an impact, a pair
    that is no longer a candidate leaves, and a candidate without an impact
    that was not active stays out."""
    state = {"A": (True, 2), "B": (True, 1), "F": (True, 4)}
    keys = ["A", "C", "D", "E", "F"]
    toi = [2.0, 0.5, 1.5, 1.0, 0.25]
    got = pd.ndb_after_full_ccd(state, keys, toi)
    assert got == {"A": (True, 2), "C": (True, 0), "E": (True, 0), "F": (True, 4)}
    # the next partial CCD flags A, C and D
    got = pd.ndb_after_partial_ccd(got, keys, [1, 1, 1, 0, 0], 20)
    assert got == {"A": (True, 3), "C": (True, 1), "D": (True, 0)}


def test_ndb_schedule_of_a_vertex_moved_across_the_activity_threshold():
    """One VT pair: a vertex 5 mm above a static triangle (x^-), its end
    position x^+ scripted per LG iteration.  With p2 - p1 vertical the
    closest-point sample gives Q = 5 mm * z1, so the pair is active exactly
    when the end height z1 <= d_hat (Eq. collision_judge with the gap of
    R7); the other samples of the pattern lie > 8 cm away sideways and never
    fire.  The partial CCD of collide.c decides, the NDB rule counts: heights
    3, 0.5, 0.8, -1, 2, 0.2, 0.1 mm give flags 0 1 1 1 0 1 1, counters
    -, 0, 1, 2, -, 0, 1 and weights -, k, 2k, 4k, -, k, 2k."""
    dhat = 1e-3
    X0 = np.array([[0.25, 0.25, 0.005], [0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    quads = np.array([[0, 1, 2, 3]])
    kinds = np.array([0])
    heights = [3e-3, 5e-4, 8e-4, -1e-3, 2e-3, 2e-4, 1e-4]
    expect_flag = [False, True, True, True, False, True, True]
    expect_a = [None, 0, 1, 2, None, 0, 1]
    k = 7.5
    expect_w = [None, 7.5, 15.0, 30.0, None, 7.5, 15.0]
    state = {}
    for z1, ef, ea, ew in zip(heights, expect_flag, expect_a, expect_w):
        X1 = X0.copy()
        X1[0, 2] = z1
        flags, margin = collide.partial_ccd(X0, X1, quads, kinds, 3, 4, dhat)
        assert bool(flags[0]) == ef, (z1, margin)
        state = pd.ndb_after_partial_ccd(state, [("vt", 0, 0)], flags, 20)
        if ea is None:
            assert state == {}
        else:
            assert state == {("vt", 0, 0): (True, ea)}
            assert float(pd.ndb_weight(k, 2.0, state[("vt", 0, 0)][1])) == ew


def test_oracle_step_applies_the_ndb_schedule_in_every_inner_iteration():
    """A drape thrown at the sphere with 8 inner iterations: in every inner
    LG iteration of Oracle.step the springs carry w = k K^a of the set the
    iteration started from (and no spring on a pair outside it), the set
    after the partial CCD is the consecutive count of the flags, and some
    counters pass 2, so the growth of Eq. (exp) is exercised."""
    import dataclasses
    sc = wl.drape_sphere(side=10, sphere_subdiv=2)
    v0 = sc.v0.copy()
    v0[:, 2] -= 20.0
    sc = dataclasses.replace(sc, v0=v0.astype(np.float32))
    p = pd.Params(fixed_iters=True, warm_iters=1, max_outer=1, max_inner=8, a_max=6)
    o = pd.Oracle(sc, p)
    amax_seen = 0
    for step in range(3):
        tr = []
        o.step(trace=tr)
        assert len(tr) == 8
        for rec in tr:
            s_in, w, act, fl, s_out = rec["state_in"], rec["weights"], rec["active"], rec["flags"], rec["state"]
            for kk in w:
                if kk in s_in:
                    assert act[kk] and w[kk] == o.k * 2.0 ** s_in[kk][1]
                else:
                    assert not act[kk]
            for kk in w:
                if fl[kk]:
                    a_prev = s_in[kk][1] if kk in s_in else None
                    assert s_out[kk] == (True, 0 if a_prev is None else min(a_prev + 1, 6))
                else:
                    assert kk not in s_out
            amax_seen = max([amax_seen] + [a for _, a in s_out.values()])
    assert amax_seen >= 3


# ----------------------------------------------------------------------------
# the non-penetration checker (Sec. 7 invariant)
# ----------------------------------------------------------------------------

def test_intersection_checker_on_hand_built_pairs():
    """Two triangles crossing in an X, a triangle pierced by another that
    shares one vertex with it, a pair sharing an edge (never counted), two
    disjoint parallel triangles and two coplanar overlapping ones (the
    coplanar case is not counted)."""
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0],            # 0-2: in z = 0
                  [0.2, 0.2, -0.5], [0.3, 0.2, 0.5], [0.2, 0.3, 0.5],  # 3-5: pierces 0-2
                  [2, 0, 0], [3, 0, 0], [2, 1, 0],             # 6-8
                  [2, 0, 0.1], [3, 0, 0.1], [2, 1, 0.1],       # 9-11: parallel above 6-8
                  [0.1, 0.1, 0], [0.9, 0.05, 0], [0.1, 0.8, 0]], float)  # 12-14: coplanar with 0-2
    T = np.array([[0, 1, 2], [3, 4, 5], [6, 7, 8], [9, 10, 11], [12, 13, 14]])
    got = collide.intersecting_triangle_pairs(X, T)
    assert sorted(map(tuple, got.tolist())) == [(0, 1), (1, 4)]
    assert np.array_equal(collide.intersecting_triangle_pairs_grid(X, T), np.array([[0, 1], [1, 4]]))
    # sharing vertex 0 and folded through: the far edge of one crosses the other
    X2 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.8, 0.3, -0.4], [0.3, 0.8, 0.4]], float)
    T2 = np.array([[0, 1, 2], [0, 3, 4]])
    assert len(collide.intersecting_triangle_pairs(X2, T2)) == 1
    # sharing an edge: skipped even when folded onto each other
    X3 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.5, 0.5, 0.0]], float)
    assert len(collide.intersecting_triangle_pairs(X3, np.array([[0, 1, 2], [1, 0, 3]]))) == 0


def test_intersection_checker_ignores_exactly_aligned_smooth_sheets():
    """A sheet bent only along x (z a function of x, exactly aligned grid)
    has quadruples of coplanar points whose orientations round to tiny
    values of either sign; it does not intersect itself."""
    uv, tris = wl.grid_mesh(40, 40, 2.0, 2.0)
    for f in (lambda u: 0.01 * np.sin(7 * u[:, 0]), lambda u: 0.2 * u[:, 0] ** 2, lambda u: 0.0 * u[:, 0]):
        V = np.zeros((len(uv), 3))
        V[:, :2] = uv
        V[:, 2] = f(uv)
        assert len(collide.intersecting_triangle_pairs(V, tris)) == 0
        assert len(collide.intersecting_triangle_pairs_grid(V, tris)) == 0


def test_grid_culled_checker_lists_the_brute_force_pairs():
    """The grid-culled checker returns exactly the brute-force list on
    crumpled sheets (hundreds of intersections) with an obstacle through
    them, for several cell sizes."""
    rng = np.random.default_rng(11)
    for seed in range(3):
        rng = np.random.default_rng(seed)
        uv, tris = wl.grid_mesh(28, 28, 1.0, 1.0)
        V = np.zeros((len(uv), 3))
        V[:, :2] = uv + rng.normal(size=(len(uv), 2)) * 0.02
        V[:, 2] = rng.normal(size=len(uv)) * 0.05
        sv, st = wl.icosphere(2, 0.3, (0.5, 0.5, 0.0))
        X = np.concatenate([V, sv])
        T = np.concatenate([tris, np.asarray(st) + len(V)])
        ref = collide.intersecting_triangle_pairs(X, T)
        ref = ref[np.lexsort((ref[:, 1], ref[:, 0]))]
        assert len(ref) > 100
        for cell in (None, 0.01, 0.05, 0.3):
            assert np.array_equal(collide.intersecting_triangle_pairs_grid(X, T, cell), ref), (seed, cell)
