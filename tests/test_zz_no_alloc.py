"""GPU test of pdc_op_contact_noalloc, the allocation-free variant of
pdc_op_contact.

It must give what pdc_op_contact gives on the same inputs -- up to the
order of the float atomics that accumulate per-vertex sums, hence the
relative tolerances below -- and what the oracle's contact_terms gives for
the same pairs and weights, on two calls in a row, with the outputs filled
with garbage in between (nothing has to start at zero), and reject inputs
larger than its static scratch before doing any work.  The file name keeps it
last in collection so that it also runs after the other GPU tests.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import pd

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 8 << 20  # PDC_NOALLOC_SCRATCH_BYTES


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2403_19272_gb300 import build
    build.build()
    from paper_2403_19272_gb300 import pdcloth
    return torch, pdcloth


def _mesh(sc):
    m = pd.Model(sc.verts, sc.tris, sc.pins, 0.1, 1e3, 1e-2, 0.005)
    return pd.CollisionMesh(m, sc.obstacles)


def _case(pc, seed):
    rng = np.random.default_rng(seed)
    sc = wl.drape_sphere(side=16, sphere_subdiv=2)
    p = pc.pdc_default_params()
    p.d_hat = 1e-3
    cl = pc.Cloth(sc, p)
    cm = _mesh(sc)
    X0 = np.concatenate([sc.verts] + [o.positions(0.0) for o in sc.obstacles]).astype(np.float32)
    X1 = X0.copy()
    X1[: sc.n] += (rng.normal(size=(sc.n, 3)) * 0.02).astype(np.float32)
    quads, kinds, _ = cm.candidates(X0, X1, 1e-3)
    sel = rng.choice(len(quads), min(400, len(quads)), replace=False)
    quads, kinds = np.ascontiguousarray(quads[sel], np.int32), np.ascontiguousarray(kinds[sel], np.int32)
    w = rng.uniform(10, 1000, len(quads)).astype(np.float32)
    return sc, cl, X0, X1, quads, kinds, w


def _noalloc(torch, pc, cl, n, X0, X1, quads, kinds, w, cw, cf):
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x0d, x1d, qd, kd, wd = d(X0), d(X1), d(quads), d(kinds), d(w)
    stream = torch.cuda.current_stream().cuda_stream
    pc.pdc_op_contact_noalloc(cl.h, x0d.data_ptr(), x1d.data_ptr(), qd.data_ptr(), kd.data_ptr(), wd.data_ptr(),
                              len(quads), cw.data_ptr(), cf.data_ptr(), stream)
    torch.cuda.synchronize()
    return cw.cpu().numpy().copy(), cf.cpu().numpy().copy()


def test_noalloc_contact_matches_contact_twice(env):
    torch, pc = env
    sc, cl, X0, X1, quads, kinds, w = _case(pc, 41)
    assert len(quads) > 50
    cw_ref, cf_ref = pc.pdc_op_contact(cl.h, sc.n, X0, X1, quads, kinds, w)
    assert np.max(cw_ref) > 0 and np.max(np.abs(cf_ref)) > 0
    # the oracle's springs (Sec. 5.1) for the same pairs and weights, every pair active
    cw_o, cy_o = pd.contact_terms(_mesh(sc), X0.astype(np.float64), X1.astype(np.float64),
                                  np.ones(len(quads), bool), quads, kinds, w.astype(np.float64), 1e-3)
    cf_o = cy_o - cw_o[:, None] * X1[: sc.n].astype(np.float64)
    cw = torch.full((sc.n,), float("nan"), device="cuda")
    cf = torch.full((sc.n, 3), float("nan"), device="cuda")
    for _ in range(2):
        got_cw, got_cf = _noalloc(torch, pc, cl, sc.n, X0, X1, quads, kinds, w, cw, cf)
        assert np.all(np.isfinite(got_cw)) and np.all(np.isfinite(got_cf))
        assert np.max(np.abs(got_cw - cw_ref)) <= 1e-5 * np.max(cw_ref)
        assert np.max(np.abs(got_cf - cf_ref)) <= 1e-5 * np.max(np.abs(cf_ref))
        assert np.max(np.abs(got_cw - cw_o)) <= 1e-5 * np.max(cw_o)
        assert np.max(np.abs(got_cf - cf_o)) <= 1e-4 * max(np.max(np.abs(cf_o)), 1e-12)
        cw.fill_(1e30)
        cf.fill_(-1e30)
    cl.close()


def test_noalloc_contact_empty_and_rejections(env):
    torch, pc = env
    sc, cl, X0, X1, quads, kinds, w = _case(pc, 42)
    cw = torch.full((sc.n,), 7.0, device="cuda")
    cf = torch.full((sc.n, 3), 7.0, device="cuda")
    empty = np.zeros((0, 4), np.int32)
    got_cw, got_cf = _noalloc(torch, pc, cl, sc.n, X0, X1, empty, np.zeros(0, np.int32), np.zeros(0, np.float32),
                              cw, cf)
    assert not got_cw.any() and not got_cf.any()
    # more pairs than the static scratch holds: rejected before any launch
    # (every id is valid, so even a run past the check would stay in bounds
    # of the caller's arrays)
    big = SCRATCH_BYTES // 48 + 1
    qd = torch.zeros((big, 4), dtype=torch.int32, device="cuda")
    kd = torch.zeros(big, dtype=torch.int32, device="cuda")
    wd = torch.ones(big, dtype=torch.float32, device="cuda")
    x0d = torch.from_numpy(X0).cuda()
    with pytest.raises(pc.PdcError) as e:
        pc.pdc_op_contact_noalloc(cl.h, x0d.data_ptr(), x0d.data_ptr(), qd.data_ptr(), kd.data_ptr(), wd.data_ptr(),
                                  big, cw.data_ptr(), cf.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.status == pc.PDC_ERR_CAPACITY and "static scratch" in str(e.value)
    # an out-of-range vertex id is caught by the device-side check
    bad = quads.copy()
    bad[3, 1] = len(X0)
    with pytest.raises(pc.PdcError) as e:
        _noalloc(torch, pc, cl, sc.n, X0, X1, bad, kinds, w, cw, cf)
    assert e.value.status == pc.PDC_ERR_ARG
    # the handle still works after the rejections
    cw_ref, cf_ref = pc.pdc_op_contact(cl.h, sc.n, X0, X1, quads, kinds, w)
    got_cw, got_cf = _noalloc(torch, pc, cl, sc.n, X0, X1, quads, kinds, w, cw, cf)
    assert np.max(np.abs(got_cw - cw_ref)) <= 1e-5 * np.max(cw_ref)
    assert np.max(np.abs(got_cf - cf_ref)) <= 1e-5 * np.max(np.abs(cf_ref))
    cl.close()
