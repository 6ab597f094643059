"""ctypes wrapper around the oracle's C collision routines (collide.c).

Test infrastructure only.  See collide.c for the definitions (Sec. 4 and
Sec. 4.1 of the paper: exact CCD, partial CCD, brute-force candidates).
"""
import ctypes
import numpy as np

from .build import build

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, dbl, flt = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_float
        L.oc_ccd_batch.argtypes = [P, P, i64, P, P, dbl, P]
        L.oc_partial_ccd_batch.argtypes = [P, P, i64, P, P, ctypes.c_int, ctypes.c_int, dbl, P, P]
        L.oc_closest_coef.argtypes = [P, ctypes.c_int, P]
        L.oc_broadphase_vt.argtypes = [P, P, i32, i32, P, i32, flt, i64, P]
        L.oc_broadphase_vt.restype = i64
        L.oc_broadphase_ee.argtypes = [P, P, i32, P, i32, flt, i64, P]
        L.oc_broadphase_ee.restype = i64
        L.oc_broadphase_vt_one.argtypes = [P, P, i32, i32, P, i32, flt, i64, P]
        L.oc_broadphase_vt_one.restype = i64
        L.oc_broadphase_ee_one.argtypes = [P, P, P, i32, P, i32, flt, i64, P]
        L.oc_broadphase_ee_one.restype = i64
        L.oc_count_tri_tri.argtypes = [P, P, i32, i64, P]
        L.oc_count_tri_tri.restype = i64
        L.oc_count_tri_tri_grid.argtypes = [P, P, i32, dbl, i64, P]
        L.oc_count_tri_tri_grid.restype = i64
        L.oc_broadphase_grid.argtypes = [P, P, i32, i32, P, i32, P, i32, flt, dbl, i64, P, i64, P, P, P]
        L.oc_broadphase_grid.restype = ctypes.c_int
        L.oc_ccd_vt.argtypes = [P, P, dbl]
        L.oc_ccd_vt.restype = dbl
        L.oc_ccd_ee.argtypes = [P, P, dbl]
        L.oc_ccd_ee.restype = dbl
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def ccd(X0, X1, pairs, kind, eta):
    """Exact time of impact per pair (2.0 = none).  pairs [np,4] vertex ids:
    VT (v, a, b, c), EE (a, b, c, d); kind 0 = VT, 1 = EE."""
    X0, X1, pairs, kind = _f32(X0), _f32(X1), _i32(pairs).reshape(-1, 4), _i32(kind)
    out = np.empty(len(pairs), dtype=np.float64)
    if len(pairs):
        lib().oc_ccd_batch(_p(X0), _p(X1), len(pairs), _p(pairs), _p(kind), float(eta), _p(out))
    return out


def ccd_single(q0, q1, kind, eta):
    a = np.ascontiguousarray(q0, dtype=np.float64).reshape(12)
    b = np.ascontiguousarray(q1, dtype=np.float64).reshape(12)
    f = lib().oc_ccd_ee if kind else lib().oc_ccd_vt
    return f(_p(a), _p(b), float(eta))


def partial_ccd(X0, X1, pairs, kind, nsamp_vt, nsamp_ee, dhat):
    """Active flag and margin min_s(Q - dhat*|d0|) per pair (Sec. 4.1)."""
    X0, X1, pairs, kind = _f32(X0), _f32(X1), _i32(pairs).reshape(-1, 4), _i32(kind)
    act = np.empty(len(pairs), dtype=np.int32)
    mar = np.empty(len(pairs), dtype=np.float64)
    if len(pairs):
        lib().oc_partial_ccd_batch(_p(X0), _p(X1), len(pairs), _p(pairs), _p(kind), int(nsamp_vt),
                                   int(nsamp_ee), float(dhat), _p(act), _p(mar))
    return act.astype(bool), mar


def closest_coef(q, kind):
    """Gap-vector coefficients c (p2 - p1 = sum_j c_j q_j) at the closest points."""
    a = np.ascontiguousarray(q, dtype=np.float64).reshape(12)
    c = np.empty(4, dtype=np.float64)
    lib().oc_closest_coef(_p(a), int(kind), _p(c))
    return c


def broadphase(X0, X1, n_dyn, tris, edges, dhat):
    """All VT pairs (v, t) and EE pairs (e, f) (e < f) whose swept boxes meet
    under the FP32 predicate (brute force).  Returns (vt [k,2], ee [l,2])."""
    X0, X1, tris, edges = _f32(X0), _f32(X1), _i32(tris), _i32(edges)
    nv = len(X0)
    L = lib()
    cap = 1 << 16
    while True:
        out = np.empty((cap, 2), dtype=np.int32)
        n = L.oc_broadphase_vt(_p(X0), _p(X1), nv, int(n_dyn), _p(tris), len(tris), np.float32(dhat), cap, _p(out))
        if n <= cap:
            vt = out[:n].copy()
            break
        cap = int(n)
    cap = 1 << 16
    while True:
        out = np.empty((cap, 2), dtype=np.int32)
        n = L.oc_broadphase_ee(_p(X0), _p(X1), int(n_dyn), _p(edges), len(edges), np.float32(dhat), cap, _p(out))
        if n <= cap:
            ee = out[:n].copy()
            break
        cap = int(n)
    return vt, ee


def broadphase_grid(X0, X1, n_dyn, tris, edges, dhat, cell=None):
    """The pairs of broadphase (same predicate and exclusions), culled by a
    uniform grid of side `cell` (default: the mean largest swept-box extent
    of the triangles, at least 2 d_hat): for lists too large for the brute
    force.  Returns (vt [k,2], ee [l,2]), sorted."""
    X0, X1, tris, edges = _f32(X0), _f32(X1), _i32(tris), _i32(edges)
    if cell is None:
        if len(tris):
            P = np.concatenate([X0[tris], X1[tris]], axis=1).astype(np.float64)
            cell = float(np.mean(np.max(P.max(1) - P.min(1), axis=1)))
        else:
            cell = 1.0
        cell = max(cell, 2.0 * float(dhat), 1e-9)
    cap_vt = cap_ee = 1 << 16
    while True:
        ovt = np.empty((cap_vt, 2), dtype=np.int32)
        oee = np.empty((cap_ee, 2), dtype=np.int32)
        nvt, nee = ctypes.c_int64(0), ctypes.c_int64(0)
        rc = lib().oc_broadphase_grid(_p(X0), _p(X1), len(X0), int(n_dyn), _p(tris), len(tris), _p(edges),
                                      len(edges), np.float32(dhat), float(cell), cap_vt, _p(ovt), cap_ee, _p(oee),
                                      ctypes.byref(nvt), ctypes.byref(nee))
        if rc != 0:
            raise MemoryError("broadphase_grid: grid too large")
        if nvt.value <= cap_vt and nee.value <= cap_ee:
            return ovt[:nvt.value].copy(), oee[:nee.value].copy()
        cap_vt, cap_ee = max(cap_vt, int(nvt.value)), max(cap_ee, int(nee.value))


def broadphase_vt_one(X0, X1, v, n_dyn, tris, dhat):
    X0, X1, tris = _f32(X0), _f32(X1), _i32(tris)
    out = np.empty(len(tris), dtype=np.int32)
    n = lib().oc_broadphase_vt_one(_p(X0), _p(X1), int(v), int(n_dyn), _p(tris), len(tris), np.float32(dhat),
                                   len(tris), _p(out))
    return out[:n].copy()


def broadphase_ee_one(X0, X1, e2, n_dyn, edges, dhat):
    X0, X1, edges = _f32(X0), _f32(X1), _i32(edges)
    q = _i32(e2)
    out = np.empty(len(edges), dtype=np.int32)
    n = lib().oc_broadphase_ee_one(_p(X0), _p(X1), _p(q), int(n_dyn), _p(edges), len(edges), np.float32(dhat),
                                   len(edges), _p(out))
    return out[:n].copy()


def intersecting_triangle_pairs(X, tris):
    """Brute-force list of intersecting triangle pairs (no shared edge)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    tris = _i32(tris)
    cap = 1024
    while True:
        out = np.empty((cap, 2), dtype=np.int32)
        n = lib().oc_count_tri_tri(_p(X), _p(tris), len(tris), cap, _p(out))
        if n <= cap:
            return out[:n].copy()
        cap = int(n)


def intersecting_triangle_pairs_grid(X, tris, cell=None):
    """The pairs of intersecting_triangle_pairs (same exact test), culled by
    a uniform grid of side `cell` (default: the mean largest box extent of
    the triangles): for the invariant check of large meshes.  Sorted pairs."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    tris = _i32(tris)
    if cell is None:
        P3 = X[tris]
        cell = float(np.mean(np.max(P3.max(1) - P3.min(1), axis=1))) if len(tris) else 1.0
        cell = max(cell, 1e-9)
    cap = 1024
    while True:
        out = np.empty((cap, 2), dtype=np.int32)
        n = lib().oc_count_tri_tri_grid(_p(X), _p(tris), len(tris), float(cell), cap, _p(out))
        if n < 0:
            raise MemoryError("intersecting_triangle_pairs_grid: grid too large")
        if n <= cap:
            return out[:n].copy()
        cap = int(n)
