"""GPU runs of the larger synthetic workloads in the benchmark's production
settings (relative PD residual 1e-3, Chebyshev sweeps, Anderson mixing, FP16
basis on the tensor cores), checked by properties that hold at any size:

* fold on a box (256 x 256, 65,536 vertices, thrown at the box so that it
  lands within the test): positions stay finite, contacts become active, and
  no cloth vertex ever ends inside the box (obstacles have infinite mass and
  the exit line search keeps every step free of penetration);
* skirt on a moving body (1024 x 332, 339,968 vertices, basis of 512 columns,
  which exceeds the tensor-core kernels' row limit and runs on the CUDA-core
  kernels): the pinned ring follows the body's rigid motion and each step
  ends with a small relative residual.
"""
import dataclasses

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2403_19272_gb300 import build
    build.build()
    from paper_2403_19272_gb300 import pdcloth
    return pdcloth


def _production(pc, **kw):
    import bench
    p = bench.solver_params(pc, 2)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_fold_on_box_lands_without_entering_the_box(pc):
    sc = wl.fold_on_box(side=256)
    v0 = sc.v0.copy()
    v0[:, 2] -= 6.0  # reaches the box top within ~17 steps
    sc = dataclasses.replace(sc, v0=v0.astype(np.float32))
    cl = pc.Cloth(sc, _production(pc, r_warm=128, max_inner=200))
    active = 0
    for k in range(40):
        cl.step()
        st = cl.stats()
        active = max(active, st["n_active"])
        x = cl.positions()
        assert np.all(np.isfinite(x)), k
        inside = np.all((x > -0.5 + 1e-5) & (x < 0.5 - 1e-5), axis=1)
        assert not inside.any(), (k, int(inside.sum()))
    assert active > 0
    assert x[:, 2].min() < 0.5  # the cloth has folded over the box edge
    cl.close()


def test_skirt_on_moving_body_runs_on_the_cuda_core_subspace_path(pc):
    sc = wl.skirt_on_body()
    p = _production(pc, r_warm=512, r_reuse=32, eig_iters=4, max_inner=200)
    cl = pc.Cloth(sc, p)
    for k in range(3):
        cl.step()
        st = cl.stats()
        x = cl.positions()
        assert np.all(np.isfinite(x)), k
        # a 4-pass basis of 512 columns: the iteration ends at the 1e-3 target
        # or where the residual stops decreasing, within the inner-loop cap
        assert st["rel_residual"] <= 2e-2, (k, st)
    ring = x[sc.pins]
    assert np.max(np.abs(ring - sc.pins_at(3 * p.dt))) <= 1e-6
    cl.close()
