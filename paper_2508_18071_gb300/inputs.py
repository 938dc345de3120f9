"""Seeded synthetic inputs: scenes, camera paths, EvSNet weights, log-frame clips.

This module generates inputs only; it holds none of the method's arithmetic and
is shared by the library's callers, the tests and the benchmark.  Scenes stand
in for the paper's Bistro / Kitchen / Staircase / Classroom assets (Sec. 4.1),
which are not available: the same resolution (1280x720), rate (1 kHz) and clip
lengths, with procedural geometry.

Scene dictionaries hold:
  tris      float32 [n, 9]   (v0, v1, v2)
  tri_mat   uint32  [n]      material index per triangle
  materials float32 [m, 5]   (albedo r, g, b, roughness, type 0 Lambert / 1 GGX)
  lights    float32 [l, 12]  (p0, e1, e2, radiance rgb); one-sided, normal e1 x e2
  env       float            constant environment radiance on a miss
Camera records are float32 [13]: position, 3x3 camera-to-world rotation stored
row-major (columns: right, up, backward), vertical field of view in degrees.
"""
from __future__ import annotations

import math

import numpy as np


# ------------------------------------------------------------------ geometry
def _quad(p0, e1, e2):
    p0, e1, e2 = (np.asarray(v, np.float64) for v in (p0, e1, e2))
    a, b, c, d = p0, p0 + e1, p0 + e1 + e2, p0 + e2
    return [np.concatenate([a, b, c]), np.concatenate([a, c, d])]


def _box(lo, hi, rot_y=0.0, subdiv=1, bottom=True):
    """Axis-aligned box (optionally rotated about its vertical axis), faces split
    into subdiv x subdiv quads of two triangles."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    c = 0.5 * (lo + hi)
    h = 0.5 * (hi - lo)
    cs, sn = math.cos(rot_y), math.sin(rot_y)
    R = np.array([[cs, 0, sn], [0, 1, 0], [-sn, 0, cs]])
    faces = []
    # (origin corner, edge u, edge v) in unit-box coordinates, outward normal u x v
    unit = [
        ((-1, -1, 1), (2, 0, 0), (0, 2, 0)),     # +z
        ((1, -1, -1), (-2, 0, 0), (0, 2, 0)),    # -z
        ((1, -1, 1), (0, 0, -2), (0, 2, 0)),     # +x
        ((-1, -1, -1), (0, 0, 2), (0, 2, 0)),    # -x
        ((-1, 1, 1), (2, 0, 0), (0, 0, -2)),     # +y
        ((-1, -1, -1), (2, 0, 0), (0, 0, 2)),    # -y
    ]
    if not bottom:
        unit = unit[:5]
    tris = []
    for o, u, v in unit:
        o, u, v = np.array(o, float), np.array(u, float), np.array(v, float)
        for i in range(subdiv):
            for j in range(subdiv):
                p0 = o + u * i / subdiv + v * j / subdiv
                for t in _quad(p0, u / subdiv, v / subdiv):
                    t = t.reshape(3, 3) * h
                    t = t @ R.T + c
                    tris.append(t.reshape(9))
    return tris


def _sphere(center, radius, slices=8, stacks=7):
    """UV sphere: 2 * slices * (stacks - 1) triangles (96 for 8 x 7)."""
    c = np.asarray(center, np.float64)
    P = {}
    for i in range(stacks + 1):
        th = math.pi * i / stacks
        for j in range(slices):
            ph = 2 * math.pi * j / slices
            P[i, j] = c + radius * np.array([math.sin(th) * math.cos(ph), math.cos(th),
                                             math.sin(th) * math.sin(ph)])
    tris = []
    for i in range(stacks):
        for j in range(slices):
            j1 = (j + 1) % slices
            a, b, cc, d = P[i, j], P[i, j1], P[i + 1, j1], P[i + 1, j]
            if i > 0:
                tris.append(np.concatenate([a, b, d]))
            if i < stacks - 1:
                tris.append(np.concatenate([b, cc, d]))
    return tris


def _pack(groups, materials, lights, env):
    tris, mats = [], []
    for tlist, m in groups:
        tris.extend(tlist)
        mats.extend([m] * len(tlist))
    return {
        "tris": np.asarray(tris, np.float32).reshape(-1, 9),
        "tri_mat": np.asarray(mats, np.uint32),
        "materials": np.asarray(materials, np.float32).reshape(-1, 5),
        "lights": np.asarray(lights, np.float32).reshape(-1, 12),
        "env": float(env),
    }


# -------------------------------------------------------------------- cameras
def camera(pos, rot, vfov_deg=60.0):
    return np.concatenate([np.asarray(pos, np.float64), np.asarray(rot, np.float64).reshape(9),
                           [vfov_deg]]).astype(np.float32)


def look_rot(forward, up=(0.0, 1.0, 0.0)):
    """Rotation whose columns are (right, up, backward) for a camera looking along `forward`."""
    f = np.asarray(forward, np.float64)
    f = f / np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r = r / np.linalg.norm(r)
    u = np.cross(r, f)
    return np.stack([r, u, -f], axis=1)


def yaw_rot(deg):
    a = math.radians(deg)
    return look_rot((-math.sin(a), 0.0, -math.cos(a)))


# --------------------------------------------------------------------- scenes
def cornell_box(seed=1):
    """Tiny scene: 5 walls (10 triangles) + 2 boxes without bottoms (10 triangles
    each) + one 0.5 m x 0.5 m ceiling quad light of radiance 15 (2 triangles added
    by the scene builder) = 32 triangles.  Lambertian albedos U[0.2, 0.8]^3."""
    rng = np.random.default_rng(seed)
    mats = [list(rng.uniform(0.2, 0.8, 3)) + [0.5, 0] for _ in range(7)]
    walls = [
        _quad((-1, 0, 1), (0, 0, -2), (2, 0, 0)),        # floor, normal +y
        _quad((-1, 2, -1), (0, 0, 2), (2, 0, 0)),        # ceiling, normal -y
        _quad((-1, 0, -1), (0, 2, 0), (2, 0, 0)),        # back, normal +z
        _quad((-1, 0, 1), (0, 2, 0), (0, 0, -2)),        # left, normal +x
        _quad((1, 0, -1), (0, 2, 0), (0, 0, 2)),         # right, normal -x
    ]
    groups = [(w, i) for i, w in enumerate(walls)]
    groups.append((_box((-0.7, 0, -0.6), (-0.1, 0.6, 0.0), rot_y=0.3, bottom=False), 5))
    groups.append((_box((0.1, 0, -0.8), (0.6, 1.2, -0.3), rot_y=-0.3, bottom=False), 6))
    lights = [[-0.25, 1.98, -0.25, 0.5, 0, 0, 0, 0, 0.5, 15, 15, 15]]
    return _pack(groups, mats, lights, env=0.0)


def cornell_path(n_frames=8, first=0, step=0.001):
    """Pinhole at 60 deg vertical FOV inside the box, translating +1 mm per frame along x."""
    R = look_rot((0, 0, -1))
    return np.stack([camera((step * (first + f), 1.0, 0.9), R) for f in range(n_frames)])


def random_scene(seed=11, n_boxes=100, n_spheres=100, cube=10.0):
    """~20k triangles: boxes with 3x3-subdivided faces (108 triangles) and UV spheres
    (96 triangles), sizes U[0.2, 1] m, centres uniform in a 10 m cube; 30 % GGX
    (roughness U[0.05, 0.5]), 70 % Lambertian; two 1 m^2 quad lights of radiance 20;
    environment 0.1."""
    rng = np.random.default_rng(seed)
    groups, mats = [], []
    for i in range(n_boxes + n_spheres):
        ggx = rng.uniform() < 0.3
        alb = rng.uniform(0.2, 0.8, 3)
        mats.append(list(alb) + [rng.uniform(0.05, 0.5) if ggx else 0.5, 1 if ggx else 0])
        c = rng.uniform(0, cube, 3)
        s = rng.uniform(0.2, 1.0)
        if i < n_boxes:
            ext = s * rng.uniform(0.5, 1.0, 3)
            groups.append((_box(c - ext / 2, c + ext / 2, rot_y=rng.uniform(0, math.pi),
                                subdiv=3), i))
        else:
            groups.append((_sphere(c, s / 2), i))
    lights = []
    for _ in range(2):
        x, z = rng.uniform(2, cube - 2, 2)
        lights.append([x, cube + 0.5, z, 1.0, 0, 0, 0, 0, 1.0, 20, 20, 20])
    return _pack(groups, mats, lights, env=0.1)


def random_scene_path(n_frames=100, first=0, cube=10.0, deg_per_frame=0.09):
    """Camera at the cube centre yawing at 90 deg/s (0.09 deg per 1 kHz frame)."""
    c = (cube / 2, cube / 2, cube / 2)
    return np.stack([camera(c, yaw_rot(deg_per_frame * (first + f))) for f in range(n_frames)])


def random_scene_clip_path(seed, n_frames=65, cube=10.0):
    """Random smooth camera motion through the random scene (training clips)."""
    rng = np.random.default_rng(seed)
    p0 = rng.uniform(3, cube - 3, 3)
    v = rng.normal(0, 1, 3)
    v = v / np.linalg.norm(v) * rng.uniform(1.0, 4.0) / 1000.0      # 1-4 m/s
    yaw0 = rng.uniform(0, 360)
    yaw_rate = rng.uniform(-120, 120) / 1000.0                       # deg per frame
    pitch = rng.uniform(-15, 15)
    out = []
    for f in range(n_frames):
        a = math.radians(yaw0 + yaw_rate * f)
        pt = math.radians(pitch)
        fwd = (-math.sin(a) * math.cos(pt), math.sin(pt), -math.cos(a) * math.cos(pt))
        out.append(camera(p0 + v * f, look_rot(fwd)))
    return np.stack(out)


def city_block(seed=21, n_boxes=40000, street_half=6.0, lot=9.0):
    """~500k triangles: n_boxes closed boxes (12 triangles each, 480k) on a street
    grid along -z, building heights log-normal; a 4 km ground in 40 m tiles (20k);
    four 1 m x 1 m street lights of radiance 50 at 8 m; environment 0.1."""
    rng = np.random.default_rng(seed)
    mats = [[0.5, 0.5, 0.5, 0.5, 0]]                                  # ground
    for _ in range(64):
        ggx = rng.uniform() < 0.3
        mats.append(list(rng.uniform(0.2, 0.8, 3)) +
                    [rng.uniform(0.05, 0.5) if ggx else 0.5, 1 if ggx else 0])
    n_small = n_boxes // 5
    n_build = n_boxes - n_small
    cols = max(2, int(round(math.sqrt(n_build / 4))))                # lots per side along x
    rows = int(math.ceil(n_build / (2 * cols)))
    groups = []
    k = 0
    for r in range(rows):
        z = 10.0 - lot * r
        for side in (-1, 1):
            for c in range(cols):
                if k >= n_build:
                    break
                x = side * (street_half + lot * (c + 0.5))
                w, d = rng.uniform(3.0, 8.0, 2)
                h = float(np.clip(rng.lognormal(math.log(12.0), 0.6), 3.0, 120.0))
                x += rng.uniform(-0.5, 0.5) * (lot - w)
                groups.append((_box((x - w / 2, 0, z - d / 2), (x + w / 2, h, z + d / 2),
                                    rot_y=rng.uniform(-0.1, 0.1)), 1 + int(rng.integers(64))))
                k += 1
    zmin = 10.0 - lot * rows
    for _ in range(n_small):                                          # street furniture
        x = rng.uniform(-street_half + 0.5, street_half - 0.5)
        if abs(x) < 1.5:
            x = math.copysign(1.5 + rng.uniform(0, 4), x if x != 0 else 1.0)
        z = rng.uniform(zmin, 10.0)
        s = rng.uniform(0.3, 2.0, 3) * np.array([1.0, 0.8, 1.0])
        groups.append((_box((x - s[0] / 2, 0, z - s[2] / 2), (x + s[0] / 2, s[1], z + s[2] / 2),
                            rot_y=rng.uniform(0, math.pi)), 1 + int(rng.integers(64))))
    # ground: 4 km x 4 km in 40 m tiles (100 x 100 quads); kilometre-sized
    # triangles would put FP32 hit points ~1e-4 m off near the camera
    L, tile = 2000.0, 40.0
    n = int(2 * L / tile)
    ground = []
    for i in range(n):
        for j in range(n):
            x0, z0 = -L + tile * i, L - tile * j
            ground.extend(_quad((x0, 0, z0), (0, 0, -tile), (tile, 0, 0)))
    groups.append((ground, 0))
    lights = [[-0.5, 8.0, -5.0 - 10.0 * i - 0.5, 1.0, 0, 0, 0, 0, 1.0, 50, 45, 40]
              for i in range(4)]
    return _pack(groups, mats, lights, env=0.1)


def city_path(n_frames=1000, first=0, speed_per_frame=0.01, height=1.7):
    """Forward motion along -z at 10 m/s (1 cm per 1 kHz frame), 1.7 m above the street."""
    R = look_rot((0, -0.05, -1))
    return np.stack([camera((0.0, height, -speed_per_frame * (first + f)), R)
                     for f in range(n_frames)])


# -------------------------------------------------------------------- EvSNet
def layer_shape(net, i):
    """(Cin, kt, ks) of conv layer i of an EvSNet dictionary: layer 0 of a net
    with a spatial stem (ks0 > 0) is one step by ks0 x ks0."""
    ks0 = int(net.get("ks0", 0))
    if i == 0:
        return (1, 1, ks0) if ks0 > 0 else (1, net["kt"], net["ks"])
    return net["C"], net["kt"], net["ks"]


def random_evsnet(kind=0, n_layers=2, C=8, kt=1, ks=3, seed=2, std=0.1, beta=1.0,
                  vth=0.2, reset=None, ks0=0, delay=0):
    """Random-init EvSNet weights N(0, std) in the packed layout: conv layers in
    order, each [Cout][Cin][kt][ks][ks] (Cin = 1 for the first; a stem layer 0,
    ks0 > 0, is [C][1][1][ks0][ks0]), then the projection [C]; biases C per conv
    layer then 1.  `delay` labels the events of step k with t0 + k - delay."""
    rng = np.random.default_rng(seed)
    net = {"kind": kind, "n_layers": n_layers, "C": C, "kt": kt, "ks": ks, "ks0": int(ks0),
           "delay": int(delay), "beta": float(beta), "vth": float(vth),
           "reset": float(vth if reset is None else reset)}
    nw = 0
    for i in range(n_layers):
        cin, t, k = layer_shape(net, i)
        nw += C * cin * t * k * k
    nw += C
    nb = C * n_layers + 1
    net["w"] = rng.normal(0, std, nw).astype(np.float32)
    net["b"] = rng.normal(0, std, nb).astype(np.float32)
    return net


def identity_evsnet(kind=0, n_layers=2, C=2, kt=1, ks=3, vth=0.2, ks0=0):
    """Hand-set weights whose projection reproduces X exactly: the first layer
    splits X into (ReLU(X), ReLU(-X)) with centre taps (+1, -1), inner layers pass
    channels through (centre-tap identity, or zero residual branches) and the
    projection is (+1, -1)."""
    net = random_evsnet(kind, n_layers, C, kt, ks, seed=0, vth=vth, ks0=ks0)
    w = np.zeros_like(net["w"])
    b = np.zeros_like(net["b"])
    r = ks // 2
    off = 0
    for i in range(n_layers):
        cin, t, k = layer_shape(net, i)
        Wl = np.zeros((C, cin, t, k, k), np.float32)
        if i == 0:
            Wl[0, 0, t - 1, k // 2, k // 2] = 1.0
            Wl[1, 0, t - 1, k // 2, k // 2] = -1.0
        elif kind == 0:
            for c in range(2):
                Wl[c, c, kt - 1, r, r] = 1.0
        w[off:off + Wl.size] = Wl.ravel()
        off += Wl.size
    w[off] = 1.0
    w[off + 1] = -1.0
    net["w"], net["b"] = w, b
    return net


# ------------------------------------------------------------ log-frame clips
def random_logl_clip(seed, F, H, W, step_std=0.08, jump_p=0.02, jump_std=0.8):
    """float32 [F,H,W] log-luminance clip: per-pixel random walk with occasional jumps."""
    rng = np.random.default_rng(seed)
    base = rng.normal(-1.0, 0.5, (H, W))
    steps = rng.normal(0, step_std, (F, H, W))
    jumps = (rng.uniform(size=(F, H, W)) < jump_p) * rng.normal(0, jump_std, (F, H, W))
    steps[0] = 0
    jumps[0] = 0
    return (base + np.cumsum(steps + jumps, 0)).astype(np.float32)
