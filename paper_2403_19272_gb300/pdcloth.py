"""ctypes binding of libpdcloth.so (include/pdcloth.h).

Argument marshalling only: every step of the cloth solve runs in the CUDA
library.  Importing this module loads the library; if it is missing the
import raises (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdcloth.so")

PDC_OK, PDC_ERR_ARG, PDC_ERR_CUDA, PDC_ERR_NUMERIC, PDC_ERR_TIMEOUT, PDC_ERR_DEGENERATE, PDC_ERR_STATE, \
    PDC_ERR_CAPACITY = range(8)
STATUS_NAMES = ["PDC_OK", "PDC_ERR_ARG", "PDC_ERR_CUDA", "PDC_ERR_NUMERIC", "PDC_ERR_TIMEOUT",
                "PDC_ERR_DEGENERATE", "PDC_ERR_STATE", "PDC_ERR_CAPACITY"]

c_i32, c_i64, c_dbl, c_flt, c_u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_float, ctypes.c_uint64
P = ctypes.c_void_p


class pdc_mesh_desc(ctypes.Structure):
    _fields_ = [("verts", P), ("nv", c_i32), ("tris", P), ("nt", c_i32), ("pins", P), ("npins", c_i32)]


class pdc_material(ctypes.Structure):
    _fields_ = [("density", c_dbl), ("k_stretch", c_dbl), ("k_bend", c_dbl)]


class pdc_params(ctypes.Structure):
    _fields_ = [("dt", c_dbl), ("gravity", c_dbl * 3), ("k_ndb_scale", c_dbl), ("K_ndb", c_dbl), ("a_max", c_i32),
                ("alpha_ls", c_dbl), ("d_hat", c_dbl), ("eta_ccd", c_dbl), ("tol_outer", c_dbl),
                ("tol_inner", c_dbl), ("tol_rel_residual", c_dbl), ("max_outer", c_i32), ("max_inner", c_i32),
                ("warm_iters", c_i32), ("jacobi_sweeps", c_i32), ("jacobi_omega", c_dbl), ("solve_cycles", c_i32),
                ("r_warm", c_i32), ("r_reuse", c_i32), ("precision", c_i32), ("samples_vt", c_i32),
                ("samples_ee", c_i32), ("collisions", c_i32), ("fixed_iters", c_i32), ("eig_iters", c_i32),
                ("seed", c_u64), ("accel", c_i32), ("accel_rho", c_dbl), ("sweep_kind", c_i32),
                ("cheb_ratio", c_dbl), ("aa_depth", c_i32),
                ("tensor_cores", c_i32), ("bp_reuse", c_dbl), ("launch_overlap", c_i32),
                ("rf_toi", c_dbl), ("rf_iters", c_i32), ("loop_control", c_i32), ("pccd_adaptive", c_i32),
                ("pccd_max_axis", c_i32), ("instance_line_search", c_i32), ("autotune", c_i32),
                ("graph_unroll", c_i32), ("loop_ahead", c_i32), ("cheb_source", c_i32),
                ("residual_patch", c_i32)]


class pdc_stats(ctypes.Structure):
    _fields_ = [("warm_iters", c_i32), ("outer_iters", c_i32), ("inner_iters", c_i32), ("contact_iters", c_i32),
                ("n_candidates", c_i64), ("n_active", c_i64), ("n_contact_vertices", c_i64), ("t_toi", c_dbl),
                ("s_line_search", c_dbl), ("rho0", c_dbl), ("rel_residual", c_dbl), ("ms_step", c_dbl),
                ("ms_broad", c_dbl), ("ms_narrow", c_dbl), ("ms_lg", c_dbl), ("overflow_retries", c_i32),
                ("bp_reused", c_i32), ("rf_iters", c_i32), ("device_loops", c_i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pdc_tuning(ctypes.Structure):
    _fields_ = [("tuned", c_i32), ("residual_block", c_i32), ("cheb_tile", c_i32), ("pair_blocks", c_i32),
                ("cell_warps", c_i32), ("residual_ms", c_flt * 3), ("cheb_ms", c_flt * 4), ("pair_ms", c_flt * 4),
                ("cell_ms", c_flt * 3), ("cell_grid", c_flt), ("grid_ms", c_flt * 3)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k.endswith("_ms") else getattr(self, k)) for k, _ in self._fields_}


class pdc_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", c_i64), ("total_ms", c_dbl), ("algo_bytes", c_dbl)]


# every entry point declared in include/pdcloth.h: name -> (restype, argtypes)
SIGNATURES = {
    "pdc_default_params": (None, [P]),
    "pdc_create": (c_i32, [P, P, P, P, P]),
    "pdc_create_batch": (c_i32, [c_i32, P, P, P, P, P]),
    "pdc_add_obstacle": (c_i32, [P, P, c_i32, P, c_i32, P]),
    "pdc_set_obstacle_transform": (c_i32, [P, c_i32, P]),
    "pdc_set_obstacle_instance": (c_i32, [P, c_i32, c_i32]),
    "pdc_set_pin_targets": (c_i32, [P, P, c_i32]),
    "pdc_set_state": (c_i32, [P, P, P, c_i32]),
    "pdc_get_state": (c_i32, [P, P, P, c_i32]),
    "pdc_set_basis": (c_i32, [P, P, c_i32]),
    "pdc_get_basis": (c_i32, [P, P, P]),
    "pdc_step": (c_i32, [P, c_dbl]),
    "pdc_get_positions": (c_i32, [P, P, c_i32]),
    "pdc_get_displacement": (c_i32, [P, P, c_i32]),
    "pdc_get_stats": (c_i32, [P, P]),
    "pdc_get_tuning": (c_i32, [P, P]),
    "pdc_get_pairs": (c_i32, [P, P, P, P, c_i64, P]),
    "pdc_destroy": (None, [P]),
    "pdc_measure_copy_bandwidth": (c_i32, [c_i64, c_i32, P, P]),
    "pdc_last_error": (ctypes.c_char_p, [P]),
    "pdc_set_profiling": (c_i32, [P, c_i32]),
    "pdc_get_kernel_times": (c_i32, [P, P, c_i32, P]),
    "pdc_op_broadphase": (c_i32, [P, P, P, P, c_i64, P, P, c_i64, P]),
    "pdc_op_ccd": (c_i32, [P, P, P, P, P, c_i64, P]),
    "pdc_op_partial_ccd": (c_i32, [P, P, P, P, P, c_i64, P]),
    "pdc_op_contact": (c_i32, [P, P, P, P, P, P, c_i64, P, P]),
    "pdc_op_residual": (c_i32, [P, P, P, P, P, P]),
    "pdc_op_global_solve": (c_i32, [P, P, P, P, P, c_i32, c_i32, c_i32, P]),
    "pdc_op_contact_noalloc": (c_i32, [P, P, P, P, P, P, c_i64, P, P, P]),
    "pdc_op_project": (c_i32, [P, P, c_i32, P]),
    "pdc_op_lift": (c_i32, [P, P, c_i32, P]),
}

_lib = None


def lib():
    """Load libpdcloth.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libpdcloth.so not built: run paper_2403_19272_gb300/build.py (or __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PdcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))
        self.status = status


def _ptr(a):
    return None if a is None else a.ctypes.data_as(P)


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ----------------------------------------------------------------------------- same names as the C ABI
def pdc_default_params() -> pdc_params:
    p = pdc_params()
    lib().pdc_default_params(ctypes.byref(p))
    return p


def _check(h, st):
    if st != PDC_OK:
        msg = lib().pdc_last_error(h)
        raise PdcError(st, msg.decode() if msg else "")


def pdc_create(verts, tris, pins, density, k_stretch, k_bend, params: pdc_params, stream=None):
    verts, tris, pins = _f32(verts, (-1, 3)), _i32(tris).reshape(-1, 3), _i32(pins).reshape(-1)
    mesh = pdc_mesh_desc(_ptr(verts), len(verts), _ptr(tris), len(tris), _ptr(pins) if len(pins) else None, len(pins))
    mat = pdc_material(density, k_stretch, k_bend)
    h = P()
    st = lib().pdc_create(ctypes.byref(mesh), ctypes.byref(mat), ctypes.byref(params), stream, ctypes.byref(h))
    if st != PDC_OK:
        raise PdcError(st, lib().pdc_last_error(None).decode())
    return h


def pdc_create_batch(instances, params: pdc_params, stream=None):
    """instances: sequence of (verts, tris, pins, density, k_stretch, k_bend).
    Returns (handle, vertex offsets of the instances in the union)."""
    keep, meshes, mats, offs = [], [], [], []
    nv = 0
    for verts, tris, pins, density, k_stretch, k_bend in instances:
        verts, tris, pins = _f32(verts, (-1, 3)), _i32(tris).reshape(-1, 3), _i32(pins).reshape(-1)
        keep += [verts, tris, pins]
        meshes.append(pdc_mesh_desc(_ptr(verts), len(verts), _ptr(tris), len(tris), _ptr(pins) if len(pins) else None,
                                    len(pins)))
        mats.append(pdc_material(density, k_stretch, k_bend))
        offs.append(nv)
        nv += len(verts)
    marr = (pdc_mesh_desc * len(meshes))(*meshes)
    tarr = (pdc_material * len(mats))(*mats)
    h = P()
    st = lib().pdc_create_batch(len(meshes), marr, tarr, ctypes.byref(params), stream, ctypes.byref(h))
    if st != PDC_OK:
        raise PdcError(st, lib().pdc_last_error(None).decode())
    return h, np.array(offs + [nv], dtype=np.int64)


def pdc_destroy(h):
    lib().pdc_destroy(h)


def pdc_measure_copy_bandwidth(nbytes, passes, stream=None) -> float:
    out = c_dbl()
    st = lib().pdc_measure_copy_bandwidth(int(nbytes), int(passes), stream, ctypes.byref(out))
    if st != PDC_OK:
        raise PdcError(st, lib().pdc_last_error(None).decode())
    return out.value


def pdc_add_obstacle(h, verts, tris) -> int:
    verts, tris = _f32(verts, (-1, 3)), _i32(tris).reshape(-1, 3)
    oid = c_i32()
    _check(h, lib().pdc_add_obstacle(h, _ptr(verts), len(verts), _ptr(tris), len(tris), ctypes.byref(oid)))
    return oid.value


def pdc_set_obstacle_instance(h, oid, instance):
    _check(h, lib().pdc_set_obstacle_instance(h, int(oid), int(instance)))


def pdc_set_obstacle_transform(h, oid, m4x4):
    m = _f32(m4x4, (16,))
    _check(h, lib().pdc_set_obstacle_transform(h, int(oid), _ptr(m)))


def pdc_set_pin_targets(h, xyz):
    xyz = _f32(xyz, (-1, 3))
    _check(h, lib().pdc_set_pin_targets(h, _ptr(xyz), 0))


def pdc_set_pin_targets_device(h, dev_ptr: int):
    _check(h, lib().pdc_set_pin_targets(h, P(dev_ptr), 1))


def pdc_set_state(h, x, v=None):
    x = _f32(x, (-1, 3))
    v = None if v is None else _f32(v, (-1, 3))
    _check(h, lib().pdc_set_state(h, _ptr(x), _ptr(v), 0))


def pdc_set_state_device(h, x_ptr: int, v_ptr: Optional[int]):
    _check(h, lib().pdc_set_state(h, P(x_ptr), P(v_ptr) if v_ptr else None, 1))


def pdc_get_state(h, n):
    x = np.empty((n, 3), np.float32)
    v = np.empty((n, 3), np.float32)
    _check(h, lib().pdc_get_state(h, _ptr(x), _ptr(v), 0))
    return x, v


def pdc_set_basis(h, U):
    U = _f32(U)
    _check(h, lib().pdc_set_basis(h, _ptr(U), U.shape[1]))


def pdc_get_basis(h, n, r):
    U = np.empty((n, r), np.float32)
    A0 = np.empty((r, r), np.float64)
    _check(h, lib().pdc_get_basis(h, _ptr(U), _ptr(A0)))
    return U, A0


def pdc_step(h, dt):
    _check(h, lib().pdc_step(h, float(dt)))


def pdc_get_positions(h, n):
    out = np.empty((n, 3), np.float32)
    _check(h, lib().pdc_get_positions(h, _ptr(out), 0))
    return out


def pdc_get_displacement(h, n):
    out = np.empty((n, 3), np.float32)
    _check(h, lib().pdc_get_displacement(h, _ptr(out), 0))
    return out


def pdc_get_positions_device(h, dev_ptr: int):
    _check(h, lib().pdc_get_positions(h, P(dev_ptr), 1))


def pdc_get_stats(h) -> dict:
    s = pdc_stats()
    _check(h, lib().pdc_get_stats(h, ctypes.byref(s)))
    return s.as_dict()


def pdc_get_pairs(h):
    """(prim [k,2] int32, kinds [k] int32, state [k] uint8) of the last step's candidate pairs."""
    cnt = c_i64()
    _check(h, lib().pdc_get_pairs(h, None, None, None, 0, ctypes.byref(cnt)))
    k = cnt.value
    prim = np.empty((max(k, 1), 2), np.int32)
    kinds = np.empty(max(k, 1), np.int32)
    state = np.empty(max(k, 1), np.uint8)
    _check(h, lib().pdc_get_pairs(h, _ptr(prim), _ptr(kinds), _ptr(state), k, ctypes.byref(cnt)))
    return prim[:k].copy(), kinds[:k].copy(), state[:k].copy()


def pdc_get_tuning(h) -> dict:
    t = pdc_tuning()
    _check(h, lib().pdc_get_tuning(h, ctypes.byref(t)))
    return t.as_dict()


def pdc_set_profiling(h, enable: bool):
    _check(h, lib().pdc_set_profiling(h, 1 if enable else 0))


def pdc_get_kernel_times(h) -> dict:
    """{name: {"launches", "total_ms", "algo_bytes"}} of the profiled launches."""
    cnt = c_i32()
    _check(h, lib().pdc_get_kernel_times(h, None, 0, ctypes.byref(cnt)))
    arr = (pdc_kernel_time * max(cnt.value, 1))()
    _check(h, lib().pdc_get_kernel_times(h, arr, cnt.value, ctypes.byref(cnt)))
    return {arr[i].name.decode(): dict(launches=arr[i].launches, total_ms=arr[i].total_ms,
                                       algo_bytes=arr[i].algo_bytes) for i in range(cnt.value)}


def pdc_op_broadphase(h, x0, x1):
    x0, x1 = _f32(x0, (-1, 3)), _f32(x1, (-1, 3))
    nvt, nee = c_i64(), c_i64()
    _check(h, lib().pdc_op_broadphase(h, _ptr(x0), _ptr(x1), None, 0, ctypes.byref(nvt), None, 0, ctypes.byref(nee)))
    vt = np.empty((max(nvt.value, 1), 2), np.int32)
    ee = np.empty((max(nee.value, 1), 4), np.int32)
    _check(h, lib().pdc_op_broadphase(h, _ptr(x0), _ptr(x1), _ptr(vt), nvt.value, ctypes.byref(nvt), _ptr(ee),
                                      nee.value, ctypes.byref(nee)))
    return vt[: nvt.value].copy(), ee[: nee.value].copy()


def pdc_op_ccd(h, x0, x1, quads, kinds):
    x0, x1, quads, kinds = _f32(x0, (-1, 3)), _f32(x1, (-1, 3)), _i32(quads).reshape(-1, 4), _i32(kinds)
    out = np.empty(len(quads), np.float64)
    _check(h, lib().pdc_op_ccd(h, _ptr(x0), _ptr(x1), _ptr(quads), _ptr(kinds), len(quads), _ptr(out)))
    return out


def pdc_op_partial_ccd(h, x0, x1, quads, kinds):
    x0, x1, quads, kinds = _f32(x0, (-1, 3)), _f32(x1, (-1, 3)), _i32(quads).reshape(-1, 4), _i32(kinds)
    out = np.empty(len(quads), np.int32)
    _check(h, lib().pdc_op_partial_ccd(h, _ptr(x0), _ptr(x1), _ptr(quads), _ptr(kinds), len(quads), _ptr(out)))
    return out.astype(bool)


def pdc_op_contact(h, n, x0, x, quads, kinds, w):
    x0, x = _f32(x0, (-1, 3)), _f32(x, (-1, 3))
    quads, kinds, w = _i32(quads).reshape(-1, 4), _i32(kinds), _f32(w)
    cw = np.empty(n, np.float32)
    cf = np.empty((n, 3), np.float32)
    _check(h, lib().pdc_op_contact(h, _ptr(x0), _ptr(x), _ptr(quads), _ptr(kinds), _ptr(w), len(quads), _ptr(cw),
                                   _ptr(cf)))
    return cw, cf


def pdc_op_residual(h, x, z, cw=None, cf=None):
    x, z = _f32(x, (-1, 3)), _f32(z, (-1, 3))
    cw = None if cw is None else _f32(cw)
    cf = None if cf is None else _f32(cf, (-1, 3))
    r = np.empty_like(x)
    _check(h, lib().pdc_op_residual(h, _ptr(x), _ptr(z), _ptr(cw), _ptr(cf), _ptr(r)))
    return r


def pdc_op_global_solve(h, x, z, cw, cf, r, cycles, sweeps):
    x, z = _f32(x, (-1, 3)), _f32(z, (-1, 3))
    cw = None if cw is None else _f32(cw)
    cf = None if cf is None else _f32(cf, (-1, 3))
    out = np.empty_like(x)
    _check(h, lib().pdc_op_global_solve(h, _ptr(x), _ptr(z), _ptr(cw), _ptr(cf), int(r), int(cycles), int(sweeps),
                                        _ptr(out)))
    return out


def pdc_op_project(h, v, r):
    v = _f32(v, (-1, 3))
    g = np.empty((int(r), 3), np.float64)
    _check(h, lib().pdc_op_project(h, _ptr(v), int(r), _ptr(g)))
    return g


def pdc_op_lift(h, n, q, r):
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 3)
    out = np.empty((n, 3), np.float32)
    _check(h, lib().pdc_op_lift(h, _ptr(q), int(r), _ptr(out)))
    return out


def pdc_op_contact_noalloc(h, x0, x, quads, kinds, w, np_, cw, cf, stream=0):
    """Allocation-free pdc_op_contact: every array argument is an integer
    device pointer (x0, x [nv_all][3] f32; quads [np][4] i32, 16-byte
    aligned; kinds [np] i32; w [np] f32; outputs cw [nv] f32, cf [nv][3]
    f32); stream is a cudaStream_t as an integer (0 = the handle's stream).
    Results are valid once the stream has completed the enqueued work."""
    _check(h, lib().pdc_op_contact_noalloc(h, P(x0), P(x), P(quads) if quads else None, P(kinds) if kinds else None,
                                           P(w) if w else None, int(np_), P(cw), P(cf), P(stream) if stream else None))


# ----------------------------------------------------------------------------- convenience
class Cloth:
    """One simulated cloth (a handle of the C library) built from a
    ``workloads.Scene``-like object: verts, tris, pins, density, k_stretch,
    k_bend, v0, obstacles (verts, tris, positions(t)), pins_at(t)."""

    def __init__(self, scene, params: pdc_params, stream=None):
        self.scene = scene
        self.params = params
        self.n = scene.n
        self.h = pdc_create(scene.verts, scene.tris, scene.pins, scene.density, scene.k_stretch, scene.k_bend,
                            params, stream)
        self.obstacle_ids = [pdc_add_obstacle(self.h, o.verts, o.tris) for o in scene.obstacles]
        self.t = 0.0
        if np.any(scene.v0):
            pdc_set_state(self.h, scene.verts, scene.v0)

    def close(self):
        if self.h:
            pdc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self):
        """Advance one step with the scene's scripted pins / obstacles."""
        dt = self.params.dt
        if len(self.scene.pins):
            pdc_set_pin_targets(self.h, self.scene.pins_at(self.t + dt))
        for oid, o in zip(self.obstacle_ids, self.scene.obstacles):
            if o.transform is not None:
                pdc_set_obstacle_transform(self.h, oid, o.transform(self.t + dt))
        pdc_step(self.h, dt)
        self.t += dt

    def positions(self):
        return pdc_get_positions(self.h, self.n)

    def state(self):
        return pdc_get_state(self.h, self.n)

    def stats(self):
        return pdc_get_stats(self.h)
