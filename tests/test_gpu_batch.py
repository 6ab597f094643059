"""GPU tests of the batched form (pdc_create_batch): several independent
cloths of different sizes and materials advanced as one system.

* Without collisions the instances do not interact, so a batched step must
  reproduce each instance stepped on its own handle (parity mode: fixed
  iteration counts, global solves converged per LG iteration) within the
  one-step tolerance of 1e-5 of the instance's bounding-box diagonal.
* With collisions, two drapes over their own spheres, placed apart, are
  compared with the FP64 oracle stepping their union as one cloth.
"""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import pd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2403_19272_gb300 import build
    build.build()
    from oracle import build as ob
    ob.build()
    from paper_2403_19272_gb300 import pdcloth
    return pdcloth


def _params(pc, collisions):
    p = pc.pdc_default_params()
    for k, v in dict(fixed_iters=1, warm_iters=2, max_outer=1, max_inner=3, solve_cycles=40, jacobi_sweeps=8,
                     r_warm=64, r_reuse=64, d_hat=1e-3, collisions=int(collisions)).items():
        setattr(p, k, v)
    return p


def _shift(sc, dx):
    d = np.array([dx, 0.0, 0.0], np.float32)
    obs = [wl.Obstacle((o.verts + d).astype(np.float32), o.tris) for o in sc.obstacles]
    return dataclasses.replace(sc, verts=(sc.verts + d).astype(np.float32), obstacles=obs, pin_targets=None)


def _union(scenes):
    V, T, Pn, V0, obs = [], [], [], [], []
    off = 0
    for sc in scenes:
        V.append(sc.verts)
        T.append(sc.tris + off)
        Pn.append(sc.pins + off)
        V0.append(sc.v0)
        obs += sc.obstacles
        off += sc.n
    s0 = scenes[0]
    return wl.Scene("union", np.concatenate(V).astype(np.float32), np.concatenate(T).astype(np.int32),
                    np.concatenate(Pn).astype(np.int32), np.concatenate(V0).astype(np.float32), s0.density,
                    s0.k_stretch, s0.k_bend, obs)


class _Batch:
    def __init__(self, pc, scenes, params):
        self.pc, self.scenes, self.params = pc, scenes, params
        inst = [(s.verts, s.tris, s.pins, s.density, s.k_stretch, s.k_bend) for s in scenes]
        self.h, self.off = pc.pdc_create_batch(inst, params)
        for s in scenes:
            for o in s.obstacles:
                pc.pdc_add_obstacle(self.h, o.verts, o.tris)
        self.n = int(self.off[-1])
        self.pins = np.concatenate([s.verts[s.pins] for s in scenes]).astype(np.float32)
        v0 = np.concatenate([s.v0 for s in scenes]).astype(np.float32)
        if np.any(v0):
            pc.pdc_set_state(self.h, np.concatenate([s.verts for s in scenes]).astype(np.float32), v0)

    def step(self):
        if len(self.pins):
            self.pc.pdc_set_pin_targets(self.h, self.pins)
        self.pc.pdc_step(self.h, self.params.dt)

    def state(self):
        return self.pc.pdc_get_state(self.h, self.n)

    def close(self):
        self.pc.pdc_destroy(self.h)


def test_batch_matches_instances_stepped_alone(pc):
    scenes = [
        _shift(dataclasses.replace(wl.tiny_scene(side=6), k_stretch=3e2), 0.0),
        _shift(dataclasses.replace(wl.tiny_scene(side=9, curved=True), k_stretch=5e3, density=0.2), 2.0),
        _shift(wl.drape_sphere(side=11, with_sphere=False), 4.0),
    ]
    p = _params(pc, collisions=False)
    b = _Batch(pc, scenes, p)
    singles = [pc.Cloth(s, _params(pc, collisions=False)) for s in scenes]
    for k in range(3):
        b.step()
        xb, vb = b.state()
        for i, (s, cl) in enumerate(zip(scenes, singles)):
            cl.step()
            xs, vs = cl.state()
            L = float(np.linalg.norm(s.verts.max(0) - s.verts.min(0)))
            part = xb[b.off[i]:b.off[i + 1]]
            assert np.max(np.abs(part - xs)) <= 1e-5 * L, (k, i)
    for cl in singles:
        cl.close()
    b.close()


def test_batch_with_collisions_matches_oracle_on_the_union(pc):
    scenes = [_shift(wl.drape_sphere(side=12, sphere_subdiv=2), 0.0),
              _shift(wl.drape_sphere(side=14, sphere_subdiv=2, seed=77), 2.5)]
    p = _params(pc, collisions=True)
    b = _Batch(pc, scenes, p)
    orc = pd.Oracle(_union(scenes), pd.Params(fixed_iters=True, warm_iters=2, max_outer=1, max_inner=3, dhat=1e-3,
                                              collisions=True))
    for k in range(4):
        b.step()
        xo, vo, _ = orc.step()
        xg, vg = b.state()
        assert np.max(np.abs(xg - xo)) <= 1e-5 * orc.model.L, k
        orc.x, orc.v = xg.astype(np.float64), vg.astype(np.float64)
    b.close()


def test_batch_rejects_bad_instances(pc):
    p = _params(pc, collisions=False)
    sc = wl.tiny_scene(side=5)
    bad = (sc.verts, sc.tris + 100, sc.pins, sc.density, sc.k_stretch, sc.k_bend)
    with pytest.raises(pc.PdcError):
        pc.pdc_create_batch([(sc.verts, sc.tris, sc.pins, sc.density, sc.k_stretch, sc.k_bend), bad], p)


def _thrown(sc, vz):
    v0 = sc.v0.copy()
    v0[:, 2] += vz
    return dataclasses.replace(sc, v0=v0.astype(np.float32))


def test_batch_with_instance_line_search_matches_each_instance_alone(pc):
    """instance_line_search = 1: each instance takes its own step fraction
    alpha * t_k from the pairs that touch it (its sphere attached to it), so
    the batch equals every instance stepped by itself; here one drape is
    thrown fast at its sphere and meets it within the test, the other falls
    slowly, and each is compared with its own FP64 oracle (the oracle's
    NDB base weight k set to the union's).  With one fraction for the union
    the slow drape's steps would be cut short by the fast drape's impacts."""
    scenes = [_shift(_thrown(wl.drape_sphere(side=12, sphere_subdiv=2), -20.0), 0.0),
              _shift(_thrown(wl.drape_sphere(side=14, sphere_subdiv=2, seed=77), -0.5), 2.5)]
    p = _params(pc, collisions=True)
    p.instance_line_search = 1
    b = _Batch(pc, scenes, p)
    for j in range(len(scenes)):
        pc.pdc_set_obstacle_instance(b.h, j, j)
    pu = _params(pc, collisions=True)  # the same batch with one fraction for the union
    bu = _Batch(pc, scenes, pu)
    # the union's k = mean of diag H over all free vertices
    models = [pd.Model(s.verts, s.tris, s.pins, s.density, s.k_stretch, s.k_bend, p.dt) for s in scenes]
    dg = np.concatenate([m.diagH[m.free] for m in models])
    orcs = [pd.Oracle(s, pd.Params(fixed_iters=True, warm_iters=2, max_outer=1, max_inner=3, dhat=1e-3,
                                   collisions=True, k_ndb_scale=float(dg.mean() / m.diagH[m.free].mean())))
            for s, m in zip(scenes, models)]
    impacts = 0
    cut_short = 0.0
    for k in range(5):
        b.step()
        bu.step()
        xg, vg = b.state()
        xu, vu = bu.state()
        impacts += b.pc.pdc_get_stats(b.h)["t_toi"] <= 1.0
        for i, (o, s) in enumerate(zip(orcs, scenes)):
            xo, vo, _ = o.step()
            part = slice(b.off[i], b.off[i + 1])
            assert np.max(np.abs(xg[part] - xo)) <= 1e-5 * o.model.L, (k, i)
            o.x, o.v = xg[part].astype(np.float64), vg[part].astype(np.float64)
        cut_short = max(cut_short, float(np.max(np.abs(xu[b.off[1]:] - xg[b.off[1]:]))))
        pc.pdc_set_state(bu.h, xg, vg)
    assert impacts > 0
    assert cut_short > 1e-4  # the union's single fraction would have moved the slow drape less
    b.close()
    bu.close()


def test_instance_line_search_attachment_is_checked(pc):
    scenes = [_shift(wl.drape_sphere(side=8, sphere_subdiv=1), 0.0), _shift(wl.drape_sphere(side=8, sphere_subdiv=1), 2.0)]
    p = _params(pc, collisions=True)
    p.instance_line_search = 1
    b = _Batch(pc, scenes, p)
    with pytest.raises(pc.PdcError):
        pc.pdc_set_obstacle_instance(b.h, 0, 2)
    with pytest.raises(pc.PdcError):
        pc.pdc_set_obstacle_instance(b.h, 5, 0)
    pc.pdc_set_obstacle_instance(b.h, 0, 0)
    b.step()  # one obstacle unattached: the union's fraction, still a valid step
    b.close()
    sc = wl.drape_sphere(side=8, sphere_subdiv=1)
    cl = pc.Cloth(sc, _params(pc, collisions=True))
    with pytest.raises(pc.PdcError):
        pc.pdc_set_obstacle_instance(cl.h, 0, 0)  # not a batched handle
    cl.close()


def test_autotuned_batch_takes_the_same_steps(pc):
    """autotune = 1: the first step times every candidate launch shape on the
    batch's own data and keeps the fastest of each, the broad phase its grid
    and block shape on its 8th pass; the steps are those of the fixed shapes
    (up to the order of float atomics)."""
    scenes = [_shift(_thrown(wl.drape_sphere(side=12, sphere_subdiv=2), -15.0), 0.0),
              _shift(wl.drape_sphere(side=20, sphere_subdiv=2, seed=5), 2.5)]
    pt = _params(pc, collisions=True)
    pt.autotune = 1
    bt = _Batch(pc, scenes, pt)
    bf = _Batch(pc, scenes, _params(pc, collisions=True))
    L = max(float(np.linalg.norm(s.verts.max(0) - s.verts.min(0))) for s in scenes)
    for k in range(6):
        bt.step()
        bf.step()
        xt, _ = bt.state()
        xf, _ = bf.state()
        assert np.max(np.abs(xt - xf)) <= 1e-6 * L, k
    t = pc.pdc_get_tuning(bt.h)
    assert t["tuned"] == 1
    assert t["residual_block"] in (64, 128, 256) and t["cheb_tile"] in (0, 1, 2, 3)
    assert t["pair_blocks"] in (152 * 2, 152 * 4, 152 * 8, 152 * 16) and t["cell_warps"] in (4, 8, 16)
    assert all(v > 0 for v in t["residual_ms"] + t["pair_ms"] + t["cell_ms"])
    assert t["residual_ms"][(64, 128, 256).index(t["residual_block"])] == min(t["residual_ms"])
    assert t["cell_ms"][(4, 8, 16).index(t["cell_warps"])] == min(t["cell_ms"])
    assert t["cell_grid"] in (1.0, 1.5, 2.0) and all(v > 0 for v in t["grid_ms"])
    assert t["grid_ms"][(1.0, 1.5, 2.0).index(t["cell_grid"])] == min(t["grid_ms"])
    assert pc.pdc_get_tuning(bf.h)["tuned"] == 0
    bt.close()
    bf.close()
