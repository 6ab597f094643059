"""GPU partial CCD with the sample density of Eq. (sample_bound) (Sec. 4.1)
against the oracle's adaptive lattice (oracle/pccd_adaptive.py), through
the C ABI.

* Flags on random VT / EE pairs equal the oracle's wherever the oracle's
  FP64 margin is not within FP32 rounding of zero (both sides use the same
  lattice size m, taken from rho* in FP64).
* The guarantee behind the bound: every crossing with an exact time of
  impact at most alpha is flagged (unless m hit its cap).
* One step from identical states with adaptive samples (thrown drape,
  contacts active) agrees with the oracle's within 1e-5 of the bounding-box
  diagonal, with the same number of active constraints.
"""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import collide, pd
from oracle import pccd_adaptive as pa

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2403_19272_gb300 import build
    build.build()
    from oracle import build as ob
    ob.build()
    from paper_2403_19272_gb300 import pdcloth
    return pdcloth


def _handle(pc, nverts, max_axis):
    side = int(np.ceil(np.sqrt(max(nverts, 9))))
    sc = wl.tiny_scene(side=side, pinned=False)
    p = pc.pdc_default_params()
    p.d_hat = 1e-3
    p.pccd_adaptive = 1
    p.pccd_max_axis = max_axis
    return pc.Cloth(sc, p), side * side


def _pad(X, nv):
    return np.concatenate([X, np.zeros((nv - len(X), 3), np.float32)]).astype(np.float32)


def test_adaptive_flags_match_the_oracle_on_random_pairs(pc):
    rng = np.random.default_rng(24)
    count = 3000
    cl, nv = _handle(pc, 4 * count, 64)
    X0 = rng.normal(size=(4 * count, 3)).astype(np.float32)
    X1 = (X0 + rng.normal(size=X0.shape) * 0.6).astype(np.float32)
    quads = np.arange(4 * count).reshape(-1, 4)
    kinds = rng.integers(0, 2, count)
    ag = pc.pdc_op_partial_ccd(cl.h, _pad(X0, nv), _pad(X1, nv), quads, kinds)
    ao, margin, m, cap = pa.partial_ccd_adaptive(X0, X1, quads, kinds, 1e-3, 0.8, 64)
    assert ao.sum() > 300 and (~ao).sum() > 300
    assert len(np.unique(m)) > 5  # the lattice size does vary with the pair
    bad = (ag != ao) & (np.abs(margin) > 1e-5)
    assert not bad.any(), np.nonzero(bad)[0][:10]
    # the adaptive lattice contains the t = 0 closest point, so it flags at
    # least what the closest-point-only pattern flags (away from rounding)
    a0, m0 = collide.partial_ccd(X0, X1, quads, kinds, 0, 0, 1e-3)
    assert not (a0 & ~ag & (np.abs(m0) > 1e-5)).any()
    cl.close()


def test_adaptive_flags_every_crossing_before_alpha_on_the_gpu(pc):
    rng = np.random.default_rng(7)
    alpha, cases = 0.8, []
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
        _, _, m, cap = pa.partial_ccd_adaptive(q0, q1, np.arange(4)[None, :], [kind], 0.0, alpha, 64)
        if not cap[0]:
            cases.append((q0, q1, kind))
    assert len(cases) >= 100
    p = pc.pdc_default_params()
    X0 = np.concatenate([c[0] for c in cases])
    X1 = np.concatenate([c[1] for c in cases])
    quads = np.arange(4 * len(cases)).reshape(-1, 4)
    kinds = np.array([c[2] for c in cases])
    # d_hat ~ 0: the bare Eq. (collision_judge) test, as in the bound's argument
    sc = wl.tiny_scene(side=int(np.ceil(np.sqrt(4 * len(cases)))), pinned=False)
    p.d_hat = 1e-12
    p.pccd_adaptive = 1
    p.pccd_max_axis = 64
    cl = pc.Cloth(sc, p)
    ag = pc.pdc_op_partial_ccd(cl.h, _pad(X0, sc.n), _pad(X1, sc.n), quads, kinds)
    assert ag.all(), np.nonzero(~ag)[0][:10]
    cl.close()


def test_adaptive_whole_step_parity_with_contacts(pc):
    sc = wl.drape_sphere(side=16, sphere_subdiv=2)
    v0 = sc.v0.copy()
    v0[:, 2] -= 20.0
    sc = dataclasses.replace(sc, v0=v0.astype(np.float32))
    p = pc.pdc_default_params()
    for k, v in dict(fixed_iters=1, warm_iters=2, max_outer=1, max_inner=4, solve_cycles=40, jacobi_sweeps=8,
                     r_warm=64, r_reuse=64, d_hat=1e-3, pccd_adaptive=1, pccd_max_axis=16).items():
        setattr(p, k, v)
    cl = pc.Cloth(sc, p)
    orc = pd.Oracle(sc, pd.Params(fixed_iters=True, warm_iters=2, max_outer=1, max_inner=4, dhat=1e-3,
                                  pccd_adaptive=True, pccd_max_axis=16))
    active = 0
    try:
        for k in range(4):
            cl.step()
            xo, vo, st = orc.step()
            xg, vg = cl.state()
            sg = cl.stats()
            assert np.max(np.abs(xg - xo)) <= 1e-5 * orc.model.L, k
            assert sg["n_active"] == st.n_active, (k, sg["n_active"], st.n_active)
            active = max(active, st.n_active)
            orc.x, orc.v = xg.astype(np.float64), vg.astype(np.float64)
    finally:
        cl.close()
    assert active > 0
