"""Moving geometry (et_scene_update): the hierarchy keeps its topology and its
boxes are refitted to the new triangles.  An update to the same positions
changes nothing, bit for bit; after real motion (a rigidly moving box, a
deforming triangle soup) closest hits through the refitted hierarchy equal the
oracle's on the moved geometry (brute force), and the annotations agree."""
import numpy as np
import pytest
import torch

from paper_2508_18071_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available()
    from paper_2508_18071_gb300 import api as A
    return A


def test_update_to_same_positions_is_bitwise_neutral(api):
    s = inputs.city_block(seed=21)
    g = api.Scene(s)
    path = inputs.city_path(3, first=200)
    _, before, rec0 = api.render_frames(g, path, 160, 90, 2, 5, 7, records=True, want_rgb=False)
    before = before.clone()
    g.update(s["tris"])
    _, after, rec1 = api.render_frames(g, path, 160, 90, 2, 5, 7, records=True, want_rgb=False)
    assert torch.equal(rec0, rec1)
    assert torch.equal(before, after)


def _first_hits(api, orc, s_moved, g, cams, W, H):
    _, _, rec = api.render_frames(g, cams, W, H, 2, 1, 5, records=True)
    o = orc.Scene(s_moved["tris"], s_moved["tri_mat"], s_moved["materials"], s_moved["lights"],
                  s_moved["env"], use_bvh=False)
    _, orec = o.render(cams, W, H, 2, 1, 5, records=True)
    return (rec.cpu().numpy()[..., 0, 0] == orec[..., 0, 0]).mean()


def test_moving_box_matches_oracle(api, orc):
    s = inputs.cornell_box()
    g = api.Scene(s)
    cams = inputs.cornell_path(2)
    base = np.asarray(s["tris"], np.float32).reshape(-1, 3, 3)
    for step in range(1, 4):
        moved = base.copy()
        moved[10:20] += np.array([0.07 * step, 0.0, -0.05 * step], np.float32)   # the first box
        sm = dict(s, tris=moved.reshape(-1, 9))
        g.update(sm["tris"])
        assert _first_hits(api, orc, sm, g, cams, 48, 36) > 0.999
        a = api.render_annotations(g, cams, 48, 36)
        o = orc.Scene(sm["tris"], sm["tri_mat"], sm["materials"], sm["lights"], sm["env"]).annotations(cams, 48, 36)
        prim = a["prim"].cpu().numpy()
        d = a["depth"].cpu().numpy()
        with np.errstate(invalid="ignore"):
            ok = (prim == o["prim"]) | ((prim >= 0) & (o["prim"] >= 0) &
                                         (np.abs(d - o["depth"]) <= 1e-4 * o["depth"]))
        assert ok.mean() >= 0.999


def test_deforming_soup_matches_oracle(api, orc):
    rng = np.random.default_rng(2)
    c = rng.uniform(-3, 3, (2000, 1, 3)) + np.array([0, 0, -6])
    tris = (c + rng.normal(0, 0.3, (2000, 3, 3))).astype(np.float32)
    s = {"tris": tris.reshape(-1, 9), "tri_mat": np.zeros(2000, np.uint32),
         "materials": np.asarray([[0.5, 0.5, 0.5, 0.5, 0]], np.float32),
         "lights": np.zeros((0, 12), np.float32), "env": 0.0}
    g = api.Scene(s)
    cams = np.stack([inputs.camera((0, 0, 0), np.eye(3), 60.0)])
    for step in range(3):
        tris = tris + rng.normal(0, 0.05, tris.shape).astype(np.float32)
        sm = dict(s, tris=tris.reshape(-1, 9))
        g.update(sm["tris"])
        assert _first_hits(api, orc, sm, g, cams, 48, 48) > 0.999
