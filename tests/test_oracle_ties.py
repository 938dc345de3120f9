"""Pin for the oracle's tie rule (minimum t, ties -> lower triangle index) under
BVH traversal: coincident triangles at exactly the same distance must resolve
to the lowest index, as brute force does."""
import numpy as np

from paper_2508_18071_gb300 import inputs


def test_coincident_triangles_resolve_to_lowest_index(orc):
    base = np.array([[-1, -1, -2, 1, -1, -2, 0, 1, -2]], np.float32)
    rng = np.random.default_rng(0)
    others = (rng.uniform(-3, 3, (200, 1, 3)) + np.array([0, 0, -6]) +
              rng.normal(0, 0.3, (200, 3, 3))).reshape(-1, 9).astype(np.float32)
    tris = np.concatenate([others[:100], np.repeat(base, 40, 0), others[100:],
                           np.asarray(inputs._quad((-5, -5, -4), (10, 0, 0), (0, 10, 0)), np.float32)])
    s = {"tris": tris, "tri_mat": np.zeros(len(tris), np.uint32),
         "materials": np.asarray([[0.5, 0.5, 0.5, 0.5, 0]], np.float32),
         "lights": np.zeros((0, 12), np.float32), "env": 0.0}
    a = orc.Scene(s["tris"], s["tri_mat"], s["materials"], s["lights"], s["env"], use_bvh=True)
    b = orc.Scene(s["tris"], s["tri_mat"], s["materials"], s["lights"], s["env"], use_bvh=False)
    n = 20000
    o = np.zeros((n, 3))
    d = np.column_stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.6, 0.6, n), -np.ones(n)])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ta, pa = a.intersect(o, d)
    tb, pb = b.intersect(o, d)
    assert np.array_equal(pa, pb) and np.array_equal(ta, tb)
    assert (pa == 100).sum() > 1000          # the first of the 40 copies wins its ties
    assert not np.isin(pa, np.arange(101, 140)).any()
