"""Several handles in one process (GPU).

Every handle keeps its own device state: two cloths of different sizes,
each on its own CUDA stream, stepped alternately through a regrowth of
their broad-phase candidate lists (created at a capacity of 256 pairs, so
the first pass of each step overflows and the lists are regrown in place),
each against its own FP64 oracle within 1e-5 of the bounding-box diagonal.
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


def test_two_handles_of_different_sizes_through_a_forced_regrow(pc, monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setenv("PDC_BP_CAPACITY", "256")
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    cls, orcs = [], []
    for side, s in zip((16, 21), streams):
        sc = wl.drape_sphere(side=side, sphere_subdiv=2)
        v0 = sc.v0.copy()
        v0[:, 2] -= 20.0
        sc = dataclasses.replace(sc, v0=v0.astype(np.float32))
        p = pc.pdc_default_params()
        for k, v in dict(fixed_iters=1, warm_iters=2, max_outer=1, max_inner=2, solve_cycles=40, jacobi_sweeps=8,
                         r_warm=32 if side == 16 else 48, r_reuse=32, d_hat=1e-3).items():
            setattr(p, k, v)
        cls.append(pc.Cloth(sc, p, stream=s.cuda_stream))
        orcs.append(pd.Oracle(sc, pd.Params(fixed_iters=True, warm_iters=2, max_outer=1, max_inner=2, dhat=1e-3)))
    monkeypatch.delenv("PDC_BP_CAPACITY")
    regrown = [0, 0]
    try:
        for k in range(4):
            for j in (0, 1):
                cls[j].step()
                regrown[j] += cls[j].stats()["overflow_retries"]
            for j in (0, 1):
                xo, vo, _ = orcs[j].step()
                xg, vg = cls[j].state()
                assert np.max(np.abs(xg - xo)) <= 1e-5 * orcs[j].model.L, (k, j)
                orcs[j].x, orcs[j].v = xg.astype(np.float64), vg.astype(np.float64)
    finally:
        for c in cls:
            c.close()
    assert regrown[0] > 0 and regrown[1] > 0, regrown
