"""Pins of the oracle's primary-hit annotations (depth, normal, triangle and
material ids, screen-space flow to the next frame) by closed forms of the
pinhole camera: a fronto-parallel plane at distance Z has depth Z everywhere
and normal +z; a sideways camera step dx moves it by -dx H / (2 Z tan(fov/2))
pixels; a forward step scales the offset from the image centre by Z / (Z - dz);
a pure rotation moves every depth alike."""
import math

import numpy as np

from paper_2508_18071_gb300 import inputs


def _plane_scene(Z, size=400.0):
    tris = np.asarray(inputs._quad((-size / 2, -size / 2, -Z), (size, 0, 0), (0, size, 0)), np.float32)
    return {"tris": tris, "tri_mat": np.array([3, 3], np.uint32),
            "materials": np.asarray([[0.5, 0.5, 0.5, 0.5, 0]] * 4, np.float32),
            "lights": np.zeros((0, 12), np.float32), "env": 0.0}


def _scene(orc, s, use_bvh=True):
    return orc.Scene(s["tris"], s["tri_mat"], s["materials"], s["lights"], s["env"], use_bvh=use_bvh)


def test_plane_depth_normal_and_ids(orc):
    s = _scene(orc, _plane_scene(5.0))
    cam = inputs.camera((0, 0, 0), np.eye(3), 60.0)
    a = s.annotations(np.stack([cam]), 32, 24)
    assert (a["prim"] >= 0).all()
    np.testing.assert_allclose(a["depth"], 5.0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(a["normal"][..., 2], 1.0, atol=1e-12)
    np.testing.assert_allclose(a["normal"][..., :2], 0.0, atol=1e-12)
    assert (a["material"] == 3).all()
    assert np.isnan(a["flow"]).all()                # no next camera


def test_sideways_step_flow(orc):
    Z, dx, H, W = 5.0, 0.05, 24, 32
    s = _scene(orc, _plane_scene(Z))
    c0 = inputs.camera((0, 0, 0), np.eye(3), 60.0)
    c1 = inputs.camera((dx, 0, 0), np.eye(3), 60.0)
    a = s.annotations(np.stack([c0]), W, H, next_cam=c1)
    th = math.tan(math.radians(float(np.float32(60.0))) / 2)
    dx32 = float(np.float32(dx))
    np.testing.assert_allclose(a["flow"][..., 0], -dx32 * H / (2 * Z * th), rtol=1e-9)
    np.testing.assert_allclose(a["flow"][..., 1], 0.0, atol=1e-9)


def test_forward_step_flow(orc):
    Z, dz, H, W = 5.0, 0.25, 24, 32
    s = _scene(orc, _plane_scene(Z))
    c0 = inputs.camera((0, 0, 0), np.eye(3), 60.0)
    c1 = inputs.camera((0, 0, -dz), np.eye(3), 60.0)
    a = s.annotations(np.stack([c0]), W, H, next_cam=c1)
    xs = np.arange(W) + 0.5 - W / 2
    ys = np.arange(H) + 0.5 - H / 2
    k = Z / (Z - float(np.float32(dz))) - 1.0
    np.testing.assert_allclose(a["flow"][0, :, :, 0], np.broadcast_to(xs * k, (H, W)), atol=1e-9)
    np.testing.assert_allclose(a["flow"][0, :, :, 1], np.broadcast_to(ys[:, None] * k, (H, W)), atol=1e-9)


def test_rotation_flow_does_not_depend_on_depth(orc):
    H, W = 24, 32
    phi = 0.02
    c0 = inputs.camera((0, 0, 0), np.eye(3), 60.0)
    c1 = inputs.camera((0, 0, 0), inputs.look_rot((math.sin(phi), 0, -math.cos(phi))), 60.0)
    flows = []
    for Z in (3.0, 40.0):
        a = _scene(orc, _plane_scene(Z, size=2000.0)).annotations(np.stack([c0]), W, H, next_cam=c1)
        flows.append(a["flow"][0])
    np.testing.assert_allclose(flows[0], flows[1], atol=1e-6)
    th = math.tan(math.radians(float(np.float32(60.0))) / 2)
    # the image centre moves by -tan(phi) H / (2 th) pixels: the view turned right
    # by phi (to second order, the centre pixels lie a half pixel off the axis)
    assert abs(np.mean(flows[0][:, W // 2 - 1:W // 2 + 1, 0]) - (-math.tan(phi) * H / (2 * th))) < 0.05


def test_ids_match_brute_force_and_misses(orc):
    s = inputs.cornell_box()
    cams = np.stack([inputs.camera((0.0, 1.0, 3.4), np.eye(3), 60.0)])
    a = _scene(orc, s).annotations(cams, 40, 30)
    b = _scene(orc, s, use_bvh=False).annotations(cams, 40, 30)
    np.testing.assert_array_equal(a["prim"], b["prim"])
    n_user = len(s["tri_mat"])
    user = (a["prim"] >= 0) & (a["prim"] < n_user)
    light = a["prim"] >= n_user                 # the builder's two triangles per light
    assert user.any() and light.any()
    np.testing.assert_array_equal(a["material"][user], np.asarray(s["tri_mat"], np.int64)[a["prim"][user]])
    np.testing.assert_array_equal(a["material"][light],
                                  0x80000000 | ((a["prim"][light].astype(np.int64) - n_user) // 2))
    # an empty direction: looking away from a small scene
    away = np.stack([inputs.camera((0.0, 1.0, 50.0), inputs.look_rot((0, 0, 1)), 60.0)])
    m = _scene(orc, s).annotations(away, 8, 6)
    assert (m["prim"] == -1).all() and np.isinf(m["depth"]).all() and (m["material"] == -1).all()
