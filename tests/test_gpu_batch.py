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
