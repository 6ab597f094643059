"""CPU checks of the seeded synthetic workloads: the sizes stated for each
configuration, determinism under the seed convention (1000 + config id),
and the pins / obstacles each scene is described with."""
import numpy as np

import workloads as wl


def _edges(tris):
    e = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]), axis=1)
    return np.unique(e, axis=0)


def test_configuration_sizes():
    sc = wl.drape_sphere(32)
    assert (sc.n, len(sc.tris), len(_edges(sc.tris))) == (1024, 1922, 2945)
    assert len(sc.pins) == 2 and len(sc.obstacles) == 1
    sc = wl.fold_on_box(256)
    assert (sc.n, len(sc.tris), len(_edges(sc.tris))) == (65536, 130050, 195585)
    assert len(sc.pins) == 0 and len(sc.obstacles) == 1
    sc = wl.hanging_swept(512)
    assert (sc.n, len(sc.tris), len(_edges(sc.tris))) == (262144, 522242, 784385)
    assert len(sc.pins) == 512
    sc = wl.skirt_on_body()
    assert (sc.n, len(sc.tris)) == (339968, 677888)
    sc = wl.beam_strip()
    assert sc.n == 10000 and len(sc.pins) == 80 and sc.k_bend == 1.0


def test_seeded_and_deterministic():
    a, b = wl.hanging_swept(64), wl.hanging_swept(64)
    assert np.array_equal(a.verts, b.verts) and np.array_equal(a.tris, b.tris)
    c = wl.hanging_swept(64, seed=wl.seed_for(2) + 1)
    assert not np.array_equal(a.verts, c.verts)
    assert wl.seed_for(3) == 1003
    s1 = [s.n for s in wl.batched_drape()]
    s2 = [s.n for s in wl.batched_drape()]
    assert s1 == s2 and len(s1) == 64


def test_pinned_rows_follow_their_script():
    sc = wl.hanging_swept(64)
    p0, p1 = sc.pins_at(0.0), sc.pins_at(0.25)
    # top row swept along x by 0.2 sin(2 pi t): a quarter period moves it 0.2 m
    assert np.allclose(p1[:, 0] - p0[:, 0], 0.2, atol=1e-6)
    assert np.allclose(p1[:, 1:], p0[:, 1:], atol=1e-7)
