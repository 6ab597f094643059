"""GPU parity: every stage of the CUDA path against the FP64 oracle.

All calls go through the C ABI (ctypes binding).  Tolerances:
  * broad phase: bit-exact candidate sets (the FP32 predicate is the
    definition on both sides);
  * exact CCD: identical hit/miss outside near-grazing cases, TOI within
    1e-9 (both sides refine roots in FP64);
  * partial CCD: identical flags except where the FP64 margin is within
    FP32 rounding of zero;
  * residual / contact springs / solves: FP32 arithmetic against FP64,
    relative 1e-4 of the largest entry;
  * one step from identical states: 1e-5 of the bounding-box diagonal.
"""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import collide, pd, subspace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2403_19272_gb300 import build
    build.build()
    from oracle import build as ob
    ob.build()
    from paper_2403_19272_gb300 import pdcloth
    return pdcloth


def params(pc, **kw):
    p = pc.pdc_default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def all_pos(scene, x, t=0.0):
    parts = [np.asarray(x, np.float32)] + [o.positions(t) for o in scene.obstacles]
    return np.concatenate(parts).astype(np.float32)


# ----------------------------------------------------------------------------- broad phase
def test_broadphase_bitexact_with_obstacle(pc):
    sc = wl.drape_sphere(side=16, sphere_subdiv=2)
    cl = pc.Cloth(sc, params(pc, d_hat=1e-3))
    rng = np.random.default_rng(21)
    X0 = all_pos(sc, sc.verts)
    X1 = X0.copy()
    X1[: sc.n] += (rng.normal(size=(sc.n, 3)) * 0.01 + np.array([0, 0, -0.2])).astype(np.float32)
    vt_g, ee_g = pc.pdc_op_broadphase(cl.h, X0, X1)
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    cm = pd.CollisionMesh(m, sc.obstacles)
    vt_o, ee_o = collide.broadphase(X0, X1, cm.nc, cm.tris, cm.edges, 1e-3)
    assert len(vt_o) > 100 and len(ee_o) > 100
    vt_o = vt_o[np.lexsort((vt_o[:, 1], vt_o[:, 0]))]
    assert np.array_equal(vt_g, vt_o)  # same set, GPU list sorted by (v, t)
    q_o = np.concatenate([cm.edges[ee_o[:, 0]], cm.edges[ee_o[:, 1]]], axis=1)
    key = lambda q: set(map(tuple, q.tolist()))
    assert key(ee_g) == key(q_o) and len(ee_g) == len(q_o)
    cl.close()


def test_broadphase_static_and_empty(pc):
    """No motion: only boxes within d_hat (e.g. a quad's fourth corner and the
    opposite triangle) pair up.  Far-apart primitives give empty lists."""
    sc = wl.tiny_scene(side=5)
    cl = pc.Cloth(sc, params(pc, d_hat=1e-4))
    X = sc.verts.astype(np.float32)
    vt, ee = pc.pdc_op_broadphase(cl.h, X, X)
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    cm = pd.CollisionMesh(m, [])
    vt_o, ee_o = collide.broadphase(X, X, cm.nc, cm.tris, cm.edges, 1e-4)
    assert np.array_equal(vt, vt_o[np.lexsort((vt_o[:, 1], vt_o[:, 0]))])
    assert len(ee) == len(ee_o)
    cl.close()
    # two triangles 1 m apart: nothing
    V = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0], [1, 1, 1], [1.1, 1, 1], [1, 1.1, 1]], np.float32)
    T = np.array([[0, 1, 2], [3, 4, 5]])
    h = pc.pdc_create(V, T, np.zeros(0, np.int32), 0.1, 1e3, 1e-2, params(pc, d_hat=1e-3))
    vt, ee = pc.pdc_op_broadphase(h, V, V)
    assert len(vt) == 0 and len(ee) == 0
    pc.pdc_destroy(h)


def test_broadphase_pairs_on_the_predicate_boundary(pc):
    """Two parallel sheets whose gap is exactly fl32(z + d_hat): every facing
    pair satisfies the FP32 predicate with equality on z, so a search range
    that dropped a cell at either end would lose pairs."""
    d = 1e-3
    n1 = 12
    g = np.linspace(0.0, 0.5, n1, dtype=np.float32)
    xx, yy = np.meshgrid(g, g, indexing="ij")
    za = np.float32(0.3)
    zb = np.float32(za + np.float32(d))  # fl32(z_a + d_hat)
    A = np.stack([xx.ravel(), yy.ravel(), np.full(n1 * n1, za, np.float32)], 1)
    B = np.stack([xx.ravel() + np.float32(0.013), yy.ravel(), np.full(n1 * n1, zb, np.float32)], 1)
    V = np.concatenate([A, B]).astype(np.float32)
    T = []
    for i in range(n1 - 1):
        for j in range(n1 - 1):
            a, b, c, e = i * n1 + j, (i + 1) * n1 + j, i * n1 + j + 1, (i + 1) * n1 + j + 1
            T += [[a, b, c], [b, e, c]]
    T = np.array(T, np.int32)
    T = np.concatenate([T, T + n1 * n1]).astype(np.int32)
    h = pc.pdc_create(V, T, np.zeros(0, np.int32), 0.1, 1e3, 1e-2, params(pc, d_hat=d))
    vt_g, ee_g = pc.pdc_op_broadphase(h, V, V)
    m = pd.Model(V, T, np.zeros(0, np.int32), 0.1, 1e3, 1e-2, 0.005)
    cm = pd.CollisionMesh(m, [])
    vt_o, ee_o = collide.broadphase(V, V, cm.nc, cm.tris, cm.edges, d)
    cross = np.sum((vt_o[:, 0] < n1 * n1) != (cm.tris[vt_o[:, 1], 0] < n1 * n1))
    assert cross > 100  # pairs across the gap exist
    assert np.array_equal(vt_g, vt_o[np.lexsort((vt_o[:, 1], vt_o[:, 0]))])
    q_o = np.concatenate([cm.edges[ee_o[:, 0]], cm.edges[ee_o[:, 1]]], axis=1)
    key = lambda q: set(map(tuple, q.tolist()))
    assert key(ee_g) == key(q_o) and len(ee_g) == len(q_o)
    pc.pdc_destroy(h)


def _canon_ee(q):
    """EE pairs as vertex quads (a, b, c, d), each edge as (min, max) and the
    two edges in lexicographic order, rows sorted: a form independent of the
    edge numbering of either side."""
    q = np.asarray(q, np.int64).reshape(-1, 4)
    e1 = np.sort(q[:, :2], axis=1)
    e2 = np.sort(q[:, 2:], axis=1)
    swap = (e1[:, 0] > e2[:, 0]) | ((e1[:, 0] == e2[:, 0]) & (e1[:, 1] > e2[:, 1]))
    a = np.where(swap[:, None], e2, e1)
    b = np.where(swap[:, None], e1, e2)
    c = np.concatenate([a, b], axis=1)
    return c[np.lexsort((c[:, 3], c[:, 2], c[:, 1], c[:, 0]))]


def test_broadphase_full_lists_at_262k_vertices(pc):
    """The whole VT and EE lists of the 512 x 512 swept sheet (the benchmark's
    mesh, 1.8 M candidates, as many as the benchmark's steps hold) under a
    3 mm motion across the sheet with noise, bit-exact against the oracle's
    grid-culled lists, which are pinned to the brute force on small meshes."""
    sc = wl.hanging_swept(side=512)
    assert not sc.obstacles
    cl = pc.Cloth(sc, params(pc, d_hat=1e-3))
    rng = np.random.default_rng(23)
    X0 = sc.verts.astype(np.float32)
    X1 = X0.copy()
    X1 += (rng.normal(size=X1.shape) * 0.0001 + np.array([0.0, 0.003, -0.0005])).astype(np.float32)
    vt_g, ee_g = pc.pdc_op_broadphase(cl.h, X0, X1)
    cl.close()
    tris = np.asarray(sc.tris, np.int64)
    ed = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]), axis=1)
    edges = np.unique(ed, axis=0)
    vt_o, ee_o = collide.broadphase_grid(X0, X1, sc.n, tris, edges, 1e-3)
    assert len(vt_o) > 100000 and len(ee_o) > 100000
    assert np.array_equal(vt_g, vt_o)  # both sorted by (v, t)
    q_o = np.concatenate([edges[ee_o[:, 0]], edges[ee_o[:, 1]]], axis=1)
    assert np.array_equal(_canon_ee(ee_g), _canon_ee(q_o))


def test_broadphase_sampled_at_65k_vertices(pc):
    sc = wl.fold_on_box(side=256, box_subdiv=16)
    cl = pc.Cloth(sc, params(pc, d_hat=1e-3))
    rng = np.random.default_rng(22)
    X0 = all_pos(sc, sc.verts)
    X1 = X0.copy()
    X1[: sc.n] += (rng.normal(size=(sc.n, 3)) * 0.002).astype(np.float32)
    X1[: sc.n, 2] -= 0.49  # the sheet sweeps down onto the box top
    vt_g, ee_g = pc.pdc_op_broadphase(cl.h, X0, X1)
    assert len(vt_g) > 1000 and len(ee_g) > 1000
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    cm = pd.CollisionMesh(m, sc.obstacles)
    for v in rng.choice(cm.nv, 60, replace=False):
        exp = collide.broadphase_vt_one(X0, X1, v, cm.nc, cm.tris, 1e-3)
        got = vt_g[vt_g[:, 0] == v, 1]
        assert np.array_equal(np.sort(exp), got)
    eset = {}
    for q in ee_g.tolist():
        eset.setdefault((q[0], q[1]), set()).add((q[2], q[3]))
        eset.setdefault((q[2], q[3]), set()).add((q[0], q[1]))
    for e in rng.choice(len(cm.edges), 60, replace=False):
        ab = cm.edges[e]
        exp = collide.broadphase_ee_one(X0, X1, ab, cm.nc, cm.edges, 1e-3)
        exp_set = set(map(tuple, cm.edges[exp].tolist()))
        assert eset.get(tuple(ab.tolist()), set()) == exp_set
    cl.close()


# ----------------------------------------------------------------------------- CCD
def _handle_with(pc, nverts):
    side = int(np.ceil(np.sqrt(max(nverts, 9))))
    sc = wl.tiny_scene(side=side, pinned=False)
    return pc.Cloth(sc, params(pc, d_hat=1e-3)), side * side


def test_ccd_golden_cases_on_gpu(pc):
    import json, os
    cases = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ccd_cases.json")))["cases"]
    cl, nv = _handle_with(pc, 4)
    for c in cases:
        X0 = np.zeros((nv, 3), np.float32)
        X1 = np.zeros((nv, 3), np.float32)
        X0[:4] = c["x0"]
        X1[:4] = c["x1"]
        t = pc.pdc_op_ccd(cl.h, X0, X1, np.array([[0, 1, 2, 3]]), np.array([c["kind"]]))[0]
        if c["toi"] is None:
            assert t > 1.0, c["name"]
        else:
            assert abs(t - c["toi"]) < 1e-6, (c["name"], t)
    cl.close()


def _random_pairs(rng, count, scale):
    X0 = rng.normal(size=(4 * count, 3)).astype(np.float32)
    X1 = (X0 + rng.normal(size=X0.shape) * scale).astype(np.float32)
    quads = np.arange(4 * count).reshape(-1, 4)
    kinds = rng.integers(0, 2, count)
    return X0, X1, quads, kinds


def test_ccd_parity_random_pairs(pc):
    rng = np.random.default_rng(23)
    count = 2000
    cl, nv = _handle_with(pc, 4 * count)
    X0, X1, quads, kinds = _random_pairs(rng, count, 1.2)
    X0 = np.concatenate([X0, np.zeros((nv - len(X0), 3), np.float32)])
    X1 = np.concatenate([X1, np.zeros((nv - len(X1), 3), np.float32)])
    tg = pc.pdc_op_ccd(cl.h, X0, X1, quads, kinds)
    to = collide.ccd(X0, X1, quads, kinds, 1e-9)
    hit_g, hit_o = tg <= 1, to <= 1
    assert hit_o.sum() > 100
    assert np.array_equal(hit_g, hit_o)
    assert np.max(np.abs(tg[hit_o] - to[hit_o])) < 1e-9
    cl.close()


def test_partial_ccd_parity_random_pairs(pc):
    rng = np.random.default_rng(24)
    count = 3000
    cl, nv = _handle_with(pc, 4 * count)
    X0, X1, quads, kinds = _random_pairs(rng, count, 0.6)
    X0 = np.concatenate([X0, np.zeros((nv - len(X0), 3), np.float32)])
    X1 = np.concatenate([X1, np.zeros((nv - len(X1), 3), np.float32)])
    ag = pc.pdc_op_partial_ccd(cl.h, X0, X1, quads, kinds)
    ao, margin = collide.partial_ccd(X0, X1, quads, kinds, 3, 4, 1e-3)
    bad = (ag != ao) & (np.abs(margin) > 1e-5)
    assert ao.sum() > 300 and (~ao).sum() > 300
    assert not bad.any(), np.nonzero(bad)[0][:10]
    cl.close()


# ----------------------------------------------------------------------------- local step / springs
@pytest.mark.parametrize("patch", [1, 0])
def test_residual_parity_force_form(pc, patch):
    # patch 1: element forces and residual in one kernel per mesh patch;
    # 0: two kernels through the per-corner force arrays
    rng = np.random.default_rng(25)
    sc = wl.drape_sphere(side=24, with_sphere=False)
    cl = pc.Cloth(sc, params(pc, residual_patch=patch))
    m = pd.Model(sc.verts, sc.tris, sc.pins, sc.density, sc.k_stretch, sc.k_bend, 0.005)
    x = (m.X + rng.normal(size=m.X.shape) * 0.003).astype(np.float32)
    z = (m.X + rng.normal(size=m.X.shape) * 0.001).astype(np.float32)
    cw = np.where(rng.random(m.n) < 0.1, 40.0, 0.0).astype(np.float32)
    cw[~m.free] = 0
    y = x + rng.normal(size=x.shape).astype(np.float32) * 1e-3
    cf = (cw[:, None] * (y - x)).astype(np.float32)
    rg = pc.pdc_op_residual(cl.h, x, z, cw, cf)
    x64, z64 = x.astype(np.float64), z.astype(np.float64)
    ro = -m.residual(x64, z64, cw.astype(np.float64), (cw[:, None] * y).astype(np.float64))
    full = np.zeros_like(x64)
    full[m.free] = ro
    scale = np.max(np.abs(full))
    assert np.max(np.abs(rg - full)) <= 1e-4 * scale
    cl.close()


def test_residual_parity_full_size_512(pc):
    # the benchmark's cloth (262,144 vertices, 522,242 triangles, 782,341
    # hinges) in the launch configuration of the step; every entry compared,
    # for the one-kernel patch form (the default) and the two-kernel form,
    # which sum the same terms in the same order
    rng = np.random.default_rng(28)
    sc = wl.hanging_swept(side=512)
    m = pd.Model(sc.verts, sc.tris, sc.pins, sc.density, sc.k_stretch, sc.k_bend, 0.005)
    x = (m.X + rng.normal(size=m.X.shape) * 5e-4).astype(np.float32)
    z = (m.X + rng.normal(size=m.X.shape) * 2e-4).astype(np.float32)
    ro = -m.residual(x.astype(np.float64), z.astype(np.float64))
    full = np.zeros((m.n, 3))
    full[m.free] = ro
    scale = np.max(np.abs(full))
    rgs = []
    for patch in (1, 0):
        cl = pc.Cloth(sc, params(pc, r_warm=0, residual_patch=patch))
        rgs.append(pc.pdc_op_residual(cl.h, x, z))
        cl.close()
        assert np.max(np.abs(rgs[-1] - full)) <= 1e-4 * scale, patch
    assert np.max(np.abs(rgs[0] - rgs[1])) <= 1e-6 * scale


def test_contact_springs_parity(pc):
    rng = np.random.default_rng(26)
    sc = wl.drape_sphere(side=16, sphere_subdiv=2)
    cl = pc.Cloth(sc, params(pc, d_hat=1e-3))
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    cm = pd.CollisionMesh(m, sc.obstacles)
    X0 = all_pos(sc, sc.verts)
    X1 = X0.copy()
    X1[: sc.n] += (rng.normal(size=(sc.n, 3)) * 0.02).astype(np.float32)
    quads, kinds, keys = cm.candidates(X0, X1, 1e-3)
    sel = rng.choice(len(quads), min(400, len(quads)), replace=False)
    quads, kinds = quads[sel], kinds[sel]
    w = rng.uniform(10, 1000, len(quads)).astype(np.float32)
    Xc = X1.copy()
    cw_g, cf_g = pc.pdc_op_contact(cl.h, sc.n, X0, Xc, quads, kinds, w)
    act = np.ones(len(quads), bool)
    cw_o, cy_o = pd.contact_terms(cm, X0.astype(np.float64), Xc.astype(np.float64), act, quads, kinds,
                                  w.astype(np.float64), 1e-3)
    cf_o = cy_o - cw_o[:, None] * Xc[: sc.n].astype(np.float64)
    assert np.max(np.abs(cw_g - cw_o)) <= 1e-5 * np.max(cw_o)
    assert np.max(np.abs(cf_g - cf_o)) <= 1e-4 * max(np.max(np.abs(cf_o)), 1e-12)
    cl.close()


# ----------------------------------------------------------------------------- global solve
def _seeded_basis(n, r, free, seed):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(n, r))
    B[~free] = 0
    U, _ = np.linalg.qr(B)
    return U.astype(np.float32)


def test_global_solve_one_cycle_matches_dense_reference(pc):
    rng = np.random.default_rng(27)
    sc = wl.drape_sphere(side=20, with_sphere=False)
    cl = pc.Cloth(sc, params(pc, r_warm=0, jacobi_omega=0.5))
    m = pd.Model(sc.verts, sc.tris, sc.pins, sc.density, sc.k_stretch, sc.k_bend, 0.005)
    r = 16
    U = _seeded_basis(m.n, r, m.free, 28)
    pc.pdc_set_basis(cl.h, U)
    x = (m.X + rng.normal(size=m.X.shape) * 0.003).astype(np.float32)
    z = m.X.astype(np.float32)
    cw = np.where(rng.random(m.n) < 0.1, 80.0, 0.0).astype(np.float32)
    cw[~m.free] = 0
    cf = np.zeros((m.n, 3), np.float32)
    out = pc.pdc_op_global_solve(cl.h, x, z, cw, cf, r, 1, 6)
    # dense FP64 reference on the same inputs
    x64 = x.astype(np.float64)
    rr = np.zeros_like(x64)
    rr[m.free] = -m.residual(x64, z.astype(np.float64), cw.astype(np.float64), cw[:, None] * x64)
    d0, _ = subspace.subspace_correction(U.astype(np.float64), m.H, cw.astype(np.float64), rr)
    d = subspace.jacobi(m.H, cw.astype(np.float64), rr, d0, 6, 0.5, m.free)
    exp = x64 + d
    assert np.max(np.abs(out - exp)) <= 1e-4 * np.max(np.abs(d))
    cl.close()


@pytest.mark.parametrize("side,r", [(20, 150), (24, 512)])
def test_global_solve_one_cycle_wide_reuse_basis(pc, side, r):
    """Reduced solves with collision springs on more than 128 columns (the
    blocked FP64 factorisation over many CTAs; r = 150 pads to 160 with a
    ragged last block, r = 512 is the largest accepted) against the dense
    FP64 reference, as in the 16-column case."""
    rng = np.random.default_rng(31)
    sc = wl.drape_sphere(side=side, with_sphere=False)
    cl = pc.Cloth(sc, params(pc, r_warm=0, jacobi_omega=0.5))
    m = pd.Model(sc.verts, sc.tris, sc.pins, sc.density, sc.k_stretch, sc.k_bend, 0.005)
    U = _seeded_basis(m.n, r, m.free, 32)
    pc.pdc_set_basis(cl.h, U)
    x = (m.X + rng.normal(size=m.X.shape) * 0.003).astype(np.float32)
    z = m.X.astype(np.float32)
    # spring weights spanning four decades, as life-span doubling produces
    cw = np.where(rng.random(m.n) < 0.15, 80.0 * 2.0 ** rng.integers(0, 14, m.n), 0.0).astype(np.float32)
    cw[~m.free] = 0
    cf = np.zeros((m.n, 3), np.float32)
    out = pc.pdc_op_global_solve(cl.h, x, z, cw, cf, r, 1, 6)
    x64 = x.astype(np.float64)
    rr = np.zeros_like(x64)
    rr[m.free] = -m.residual(x64, z.astype(np.float64), cw.astype(np.float64), cw[:, None] * x64)
    d0, _ = subspace.subspace_correction(U.astype(np.float64), m.H, cw.astype(np.float64), rr)
    d = subspace.jacobi(m.H, cw.astype(np.float64), rr, d0, 6, 0.5, m.free)
    exp = x64 + d
    assert np.max(np.abs(out - exp)) <= 1e-4 * np.max(np.abs(d))
    cl.close()


def test_global_solve_converges_to_exact_solution(pc):
    rng = np.random.default_rng(29)
    sc = wl.drape_sphere(side=20, with_sphere=False)
    cl = pc.Cloth(sc, params(pc, r_warm=64))
    m = pd.Model(sc.verts, sc.tris, sc.pins, sc.density, sc.k_stretch, sc.k_bend, 0.005)
    x = (m.X + rng.normal(size=m.X.shape) * 0.003).astype(np.float32)
    x[~m.free] = m.X[~m.free]
    z = (m.X + np.array([0, 0, -2.5e-4])).astype(np.float32)
    z[~m.free] = m.X[~m.free]
    cw = np.where(rng.random(m.n) < 0.05, 500.0, 0.0).astype(np.float32)
    cw[~m.free] = 0
    y = x + rng.normal(size=x.shape).astype(np.float32) * 1e-3
    cf = (cw[:, None] * (y - x)).astype(np.float32)
    out = pc.pdc_op_global_solve(cl.h, x, z, cw, cf, 64, 400, 6)
    x64 = x.astype(np.float64)
    b = m.rhs(x64, z.astype(np.float64), cw.astype(np.float64), cw[:, None] * y.astype(np.float64))
    exp = m.solve(b, x64, cw.astype(np.float64))
    assert np.max(np.abs(out - exp)) <= 1e-5 * m.L
    cl.close()


# ----------------------------------------------------------------------------- whole step
def test_free_fall_closed_form_on_gpu(pc):
    sc = wl.tiny_scene(side=8, curved=True, pinned=False)
    v0 = np.array([0.3, -0.1, 0.2], np.float32)
    sc.v0 = np.tile(v0, (sc.n, 1))
    cl = pc.Cloth(sc, params(pc, collisions=0, warm_iters=2, solve_cycles=1, jacobi_sweeps=4, tol_inner=1e-12))
    x0 = sc.verts.astype(np.float64)
    g, h = np.array([0, 0, -9.8]), 1 / 200
    v0 = v0.astype(np.float64)
    for n in range(1, 11):
        cl.step()
        x = cl.positions()
        xe = x0 + n * h * v0 + h * h * g * n * (n + 1) / 2
        assert np.max(np.abs(x - xe)) < 2e-6
    cl.close()


def test_rest_state_fixed_point_on_gpu(pc):
    sc = wl.tiny_scene(side=8, curved=True)
    cl = pc.Cloth(sc, params(pc, gravity=(0.0, 0.0, 0.0), collisions=1, r_warm=16, r_reuse=16))
    for _ in range(5):
        cl.step()
    assert np.max(np.abs(cl.positions() - sc.verts)) < 1e-6
    cl.close()


def _parity_pair(pc, sc, warm=2, outer=1, inner=3, cycles=40, sweeps=8, r=64, dhat=1e-3, collisions=True):
    gp = params(pc, fixed_iters=1, warm_iters=warm, max_outer=outer, max_inner=inner, solve_cycles=cycles,
                jacobi_sweeps=sweeps, r_warm=r, r_reuse=min(r, 64), d_hat=dhat, collisions=int(collisions))
    cl = pc.Cloth(sc, gp)
    op = pd.Params(fixed_iters=True, warm_iters=warm, max_outer=outer, max_inner=inner, dhat=dhat,
                   collisions=collisions)
    return cl, pd.Oracle(sc, op)


def test_one_step_parity_without_collisions(pc):
    sc = wl.drape_sphere(side=32, with_sphere=False)
    cl, orc = _parity_pair(pc, sc, collisions=False)
    for k in range(3):
        cl.step()
        xo, vo, _ = orc.step()
        xg, vg = cl.state()
        assert np.max(np.abs(xg - xo)) <= 1e-5 * orc.model.L, k
        orc.x, orc.v = xg.astype(np.float64), vg.astype(np.float64)
    cl.close()


def test_one_step_parity_with_chebyshev_sweeps(pc):
    # the benchmark's smoother (Jacobi-preconditioned Chebyshev steps in
    # three-term form, several solve cycles) converged per LG iteration gives
    # the oracle's exact global solves
    sc = wl.drape_sphere(side=40, with_sphere=False)
    gp = params(pc, fixed_iters=1, warm_iters=2, max_outer=1, max_inner=3, solve_cycles=40, jacobi_sweeps=32,
                sweep_kind=1, cheb_ratio=300.0, r_warm=64, r_reuse=64, d_hat=1e-3, collisions=0)
    cl = pc.Cloth(sc, gp)
    orc = pd.Oracle(sc, pd.Params(fixed_iters=True, warm_iters=2, max_outer=1, max_inner=3, dhat=1e-3,
                                  collisions=False))
    for k in range(3):
        cl.step()
        xo, vo, _ = orc.step()
        xg, vg = cl.state()
        assert np.max(np.abs(xg - xo)) <= 1e-5 * orc.model.L, k
        orc.x, orc.v = xg.astype(np.float64), vg.astype(np.float64)
    cl.close()


def test_chebyshev_matrix_sources_take_identical_steps(pc):
    """The Chebyshev steps read the same matrix entries in the same order from
    the ELL arrays (0), the tiles of consecutive rows (1), the tiles of compact
    patches of the rest mesh with delta staged with the patch's halo in shared
    memory (2), and two steps a launch over patches widened by a second ring
    (3): with no atomics anywhere in the step (no collisions, no subspace, no
    LG acceleration) the four take bit-identical steps; in the benchmark's
    settings, steps equal up to the order of float atomics."""
    import bench
    sc = wl.hanging_swept(side=64)
    kw = dict(fixed_iters=1, warm_iters=2, max_outer=1, max_inner=4, solve_cycles=2, jacobi_sweeps=11,
              sweep_kind=1, cheb_ratio=300.0, r_warm=0, collisions=0)
    xs = []
    for src in (0, 1, 2, 3):
        cl = pc.Cloth(sc, params(pc, cheb_source=src, **kw))
        for _ in range(3):
            cl.step()
        assert pc.pdc_get_tuning(cl.h)["cheb_tile"] == src
        xs.append(cl.state()[0])
        cl.close()
    assert all(np.array_equal(xs[0], xk) for xk in xs[1:])
    L = float(np.linalg.norm(sc.verts.max(0) - sc.verts.min(0)))
    xp = []
    for src in (1, 2, 3):
        p = bench.solver_params(pc, 2)
        p.cheb_source = src
        cl = pc.Cloth(sc, p)
        for _ in range(3):
            cl.step()
        xp.append(cl.state()[0])
        cl.close()
    assert max(np.max(np.abs(xp[0] - xk)) for xk in xp[1:]) <= 1e-5 * L


def test_one_step_parity_config0_with_collision_pipeline(pc):
    """32x32 drape over the sphere with self-collision on: the whole step
    (warm start, full CCD, filter, partial CCD, line search)."""
    sc = wl.drape_sphere(side=32, sphere_subdiv=3)
    cl, orc = _parity_pair(pc, sc)
    for k in range(4):
        cl.step()
        xo, vo, st = orc.step()
        xg, vg = cl.state()
        assert np.max(np.abs(xg - xo)) <= 1e-5 * orc.model.L, k
        orc.x, orc.v = xg.astype(np.float64), vg.astype(np.float64)
    cl.close()


def test_broadphase_reuse_leaves_steps_unchanged(pc):
    # the candidate lists filtered from a wider first pass are the lists of a
    # fresh pass: from identical states both runs take the same step (up to
    # the order of float atomics in the contact sums)
    sc = wl.drape_sphere(side=16, sphere_subdiv=2)
    base = dict(fixed_iters=1, warm_iters=2, max_outer=3, max_inner=3, solve_cycles=40, jacobi_sweeps=8, r_warm=32,
                r_reuse=32, d_hat=1e-3)
    a = pc.Cloth(sc, params(pc, bp_reuse=0.0, **base))
    b = pc.Cloth(sc, params(pc, bp_reuse=4.0, **base))
    L = float(np.linalg.norm(sc.verts.max(0) - sc.verts.min(0)))
    reused = 0
    for k in range(8):
        a.step()
        b.step()
        reused += b.stats()["bp_reused"]
        xa, va = a.state()
        xb, vb = b.state()
        assert np.max(np.abs(xa - xb)) <= 1e-6 * L, k
        pc.pdc_set_state(b.h, xa, va)
    assert reused > 0
    a.close()
    b.close()


def test_drape_run_stays_penetration_free(pc):
    sc = wl.drape_sphere(side=16, sphere_subdiv=2)
    cl = pc.Cloth(sc, params(pc, r_warm=32, r_reuse=32, d_hat=1e-3, max_inner=12))
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    cm = pd.CollisionMesh(m, sc.obstacles)
    for k in range(60):
        cl.step()
        if k % 10 == 9:
            X = all_pos(sc, cl.positions()).astype(np.float64)
            assert len(collide.intersecting_triangle_pairs(X, cm.tris)) == 0, k
    assert cl.positions()[:, 2].min() < -0.04
    cl.close()


def test_contact_iterations_are_counted(pc):
    """A drape thrown at the sphere: once contact vertices exist, the step
    statistics count the LG iterations that ran with collision springs."""
    import bench
    sc = wl.drape_sphere(side=32, sphere_subdiv=3)
    v0 = sc.v0.copy()
    v0[:, 2] -= 2.5  # reaches the sphere within a few steps
    sc = dataclasses.replace(sc, v0=v0.astype(np.float32))
    p = bench.solver_params(pc, 0)
    for k, v in dict(r_warm=32, r_reuse=32, eig_iters=6, d_hat=1e-3).items():
        setattr(p, k, v)
    cl = pc.Cloth(sc, p)
    counted = 0
    for k in range(10):
        cl.step()
        st = cl.stats()
        assert st["contact_iters"] <= st["warm_iters"] + st["inner_iters"]
        if st["n_contact_vertices"] > 0:
            counted += st["contact_iters"]
    assert counted > 0
    cl.close()


def test_residual_forwarding_parity(pc):
    """A drape thrown at the sphere with two inner iterations per step: the
    exit TOI falls below 1, residual forwarding (Sec. 6) runs 3 iterations
    with the active constraints at weight k and no CCD, and the next step's z
    carries 2 dx.  From the same states, GPU and oracle agree within 1e-5 of
    the bounding-box diagonal, including the steps that use a forwarded dx."""
    sc = wl.drape_sphere(side=16, sphere_subdiv=2)
    v0 = sc.v0.copy()
    v0[:, 2] -= 20.0
    sc = dataclasses.replace(sc, v0=v0.astype(np.float32))
    gp = params(pc, fixed_iters=1, warm_iters=2, max_outer=1, max_inner=2, solve_cycles=40, jacobi_sweeps=8,
                r_warm=64, r_reuse=64, d_hat=1e-3, rf_toi=1.01, rf_iters=3)
    cl = pc.Cloth(sc, gp)
    orc = pd.Oracle(sc, pd.Params(fixed_iters=True, warm_iters=2, max_outer=1, max_inner=2, dhat=1e-3, rf_toi=1.01,
                                  rf_iters=3))
    rf_g = rf_o = 0
    for k in range(4):
        cl.step()
        xo, vo, st = orc.step()
        xg, vg = cl.state()
        rf_g += cl.stats()["rf_iters"]
        rf_o += st.rf_iters
        assert np.max(np.abs(xg - xo)) <= 1e-5 * orc.model.L, k
        orc.x, orc.v = xg.astype(np.float64), vg.astype(np.float64)  # the oracle keeps its own forwarded dx
    assert rf_g > 0 and rf_g == rf_o
    cl.close()
