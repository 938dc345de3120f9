"""Pins for the oracle's BVH, intersection, BSDFs and path tracer.

Each test checks the oracle against something other than itself: brute force,
watertightness on shared edges, a closed form (Lambert's polygon irradiance
formula, the weak white furnace of GGX), zero-variance furnace cases, or
quadrature."""
import math

import numpy as np
import pytest

from paper_2508_18071_gb300 import inputs


def _scene(orc, s, use_bvh=True):
    return orc.Scene(s["tris"], s["tri_mat"], s["materials"], s["lights"], s["env"], use_bvh)


def _random_dirs(rng, n):
    d = rng.normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


# ------------------------------------------------------------------ P4 brute
def test_bvh_equals_brute_force_cornell(orc):
    s = inputs.cornell_box()
    a, b = _scene(orc, s, True), _scene(orc, s, False)
    rng = np.random.default_rng(0)
    n = 20000
    o = np.column_stack([rng.uniform(-0.99, 0.99, n), rng.uniform(0.01, 1.99, n),
                         rng.uniform(-0.99, 0.99, n)])
    d = _random_dirs(rng, n)
    ta, pa = a.intersect(o, d)
    tb, pb = b.intersect(o, d)
    assert np.array_equal(pa, pb)
    assert np.array_equal(ta, tb)
    assert (pa >= 0).mean() > 0.7           # five walls: only the open front lets rays out


def test_bvh_equals_brute_force_random_scene(orc):
    s = inputs.random_scene(seed=11, n_boxes=20, n_spheres=20)
    a, b = _scene(orc, s, True), _scene(orc, s, False)
    rng = np.random.default_rng(1)
    n = 3000
    o = rng.uniform(0, 10, (n, 3))
    d = _random_dirs(rng, n)
    ta, pa = a.intersect(o, d)
    tb, pb = b.intersect(o, d)
    assert np.array_equal(pa, pb) and np.array_equal(ta, tb)
    assert (pa >= 0).sum() > 100
    occ_a = a.occluded(o, d, np.full(n, 3.0))
    occ_b = b.occluded(o, d, np.full(n, 3.0))
    assert np.array_equal(occ_a, occ_b)
    assert np.array_equal(occ_a, tb < 3.0)


def test_bvh_invariants(orc):
    s = inputs.random_scene(seed=3, n_boxes=10, n_spheres=10)
    sc = _scene(orc, s)
    bounds, links, perm = sc.bvh()
    tris = np.concatenate([s["tris"].astype(np.float64).reshape(-1, 3, 3)], 0)
    seen = np.zeros(sc.ntris, int)
    for i, (l, r, first, cnt) in enumerate(links):
        if cnt > 0:
            assert cnt <= 4
            seen[perm[first:first + cnt]] += 1
            for t in perm[first:first + cnt]:
                if t < len(tris):
                    v = tris[t]
                    assert np.all(v.min(0) >= bounds[i, :3]) and np.all(v.max(0) <= bounds[i, 3:])
        else:
            for c in (l, r):
                assert np.all(bounds[c, :3] >= bounds[i, :3]) and np.all(bounds[c, 3:] <= bounds[i, 3:])
    assert np.all(seen == 1)
    assert sc.sah_cost() > 0


def test_watertight_on_shared_edges_and_vertices(orc):
    # a closed box: rays from an interior point aimed exactly at every vertex and
    # edge midpoint must hit some triangle (no cracks between triangles)
    tris = np.asarray(inputs._box((-1, -1, -1), (1, 1, 1)), np.float32)
    s = {"tris": tris, "tri_mat": np.zeros(len(tris), np.uint32),
         "materials": np.array([[0.5, 0.5, 0.5, 0.5, 0]], np.float32),
         "lights": np.zeros((0, 12), np.float32), "env": 0.0}
    sc = _scene(orc, s, False)
    V = tris.reshape(-1, 3, 3).astype(np.float64)
    targets = np.concatenate([V.reshape(-1, 3), 0.5 * (V[:, 0] + V[:, 1]),
                              0.5 * (V[:, 1] + V[:, 2]), 0.5 * (V[:, 2] + V[:, 0])])
    for origin in [(0.1, 0.2, 0.3), (0, 0, 0), (-0.37, 0.51, 0.11)]:
        o = np.tile(np.asarray(origin, float), (len(targets), 1))
        d = targets - o
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        t, p = sc.intersect(o, d)
        assert np.all(p >= 0)
        np.testing.assert_allclose(o + t[:, None] * d, targets, atol=1e-12)


def test_closest_hit_distance_closed_form(orc):
    # ray towards an axis-aligned plane: t = (plane - o_y) / d_y
    s = {"tris": np.asarray(inputs._quad((-500, 0, 500), (0, 0, -1000), (1000, 0, 0)), np.float32),
         "tri_mat": np.zeros(2, np.uint32), "materials": np.array([[0.5, 0.5, 0.5, 0.5, 0]]),
         "lights": np.zeros((0, 12), np.float32), "env": 0.0}
    sc = _scene(orc, s)
    rng = np.random.default_rng(2)
    o = np.column_stack([rng.uniform(-1, 1, 100), rng.uniform(0.5, 2, 100), rng.uniform(-1, 1, 100)])
    d = _random_dirs(rng, 100)
    d[:, 1] = -np.abs(d[:, 1]) - 0.2
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t, p = sc.intersect(o, d)
    np.testing.assert_allclose(t, -o[:, 1] / d[:, 1], rtol=1e-13)


# ------------------------------------------------------------------ BSDF pins
def _hemi_grid(n_th=400, n_ph=800, full=False):
    th_max = math.pi if full else math.pi / 2
    th = (np.arange(n_th) + 0.5) * th_max / n_th
    ph = (np.arange(n_ph) + 0.5) * 2 * math.pi / n_ph
    T, P = np.meshgrid(th, ph, indexing="ij")
    w = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    dA = (np.sin(T) * (th_max / n_th) * (2 * math.pi / n_ph)).reshape(-1)
    return w, dA


@pytest.mark.parametrize("alpha", [0.05, 0.2, 0.5])
@pytest.mark.parametrize("theta_o", [0.1, 0.8, 1.3])
def test_ggx_weak_white_furnace(orc, alpha, theta_o):
    """integral over all wi of G1(wo) D(m) / (4 wo.z) = integral over m of
    G1(wo) D(m) <wo.m> / wo.z = 1 (Heitz 2014): the oracle's pdf, integrated over
    the full sphere of reflected directions, is exactly normalised."""
    mat = [1.0, 1.0, 1.0, alpha, 1]
    wo = np.array([[math.sin(theta_o), 0.0, math.cos(theta_o)]])
    # integrate in the half-vector domain: d omega_i = 4 <wo.m> d omega_m
    m, dA = _hemi_grid(1200 if alpha < 0.1 else 400, 400)
    om = m @ wo[0]
    keep = om > 0
    m, dA, om = m[keep], dA[keep], om[keep]
    wi = 2 * om[:, None] * m - wo
    _, pdf = orc.bsdf_eval(mat, np.tile(wo, (len(wi), 1)), wi)
    total = np.sum(pdf * 4 * om * dA)
    assert abs(total - 1.0) < 2e-3


@pytest.mark.parametrize("mat", [[0.3, 0.5, 0.7, 0.5, 0], [0.9, 0.6, 0.3, 0.1, 1],
                                 [0.9, 0.6, 0.3, 0.4, 1]])
def test_bsdf_sample_matches_eval(orc, mat):
    """The sampling weight equals f cos / pdf from evaluation, and the fraction of
    samples that stay above the horizon equals the quadrature of the pdf."""
    rng = np.random.default_rng(5)
    n = 20000
    th = rng.uniform(0.05, 1.4, n)
    ph = rng.uniform(0, 2 * math.pi, n)
    wo = np.column_stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    wi, wt, pdf, ok = orc.bsdf_sample(mat, wo, rng.uniform(size=(n, 2)))
    fc, pe = orc.bsdf_eval(mat, wo[ok], wi[ok])
    np.testing.assert_allclose(pe, pdf[ok], rtol=1e-9)
    np.testing.assert_allclose(fc / pe[:, None], wt[ok], rtol=1e-9)
    # quadrature of pdf over the upper hemisphere vs. sampled survival, fixed wo
    wo1 = np.array([[math.sin(0.9), 0, math.cos(0.9)]])
    wi_g, dA = _hemi_grid(600 if mat[3] < 0.2 else 300, 600)
    _, pq = orc.bsdf_eval(mat, np.tile(wo1, (len(wi_g), 1)), wi_g)
    q = np.sum(pq * dA)
    m = 200000
    _, _, _, ok1 = orc.bsdf_sample(mat, np.tile(wo1, (m, 1)), rng.uniform(size=(m, 2)))
    assert abs(q - ok1.mean()) < 5e-3
    if mat[4] == 0:
        assert abs(q - 1.0) < 1e-4
        fq, _ = orc.bsdf_eval(mat, np.tile(wo1, (len(wi_g), 1)), wi_g)
        np.testing.assert_allclose((fq * dA[:, None]).sum(0), mat[:3], rtol=1e-4)


# ---------------------------------------------------------- renderer: furnace
def _sphere_scene(mat, env=1.0):
    tris = np.asarray(inputs._sphere((0, 0, -3), 1.0), np.float32)
    return {"tris": tris, "tri_mat": np.zeros(len(tris), np.uint32),
            "materials": np.asarray([mat], np.float32), "lights": np.zeros((0, 12), np.float32),
            "env": env}


@pytest.mark.parametrize("depth", [2, 3, 5])
def test_white_furnace_lambert(orc, depth):
    """Lambert albedo a on a convex object under env = 1 renders a on the object
    and 1 elsewhere, with zero variance (cosine sampling)."""
    a = [0.25, 0.5, 0.75]
    s = _sphere_scene(a + [0.5, 0])
    sc = _scene(orc, s)
    cams = np.stack([inputs.camera((0, 0, 0), np.eye(3), 60.0)])
    rgb, rec = sc.render(cams, 24, 24, 4, depth, seed=9, records=True)
    hit = rec[0, :, :, 0, 0, 0] >= 0                        # all samples of these pixels hit
    allhit = (rec[0, :, :, :, 0, 0] >= 0).all(-1)
    allmiss = (rec[0, :, :, :, 0, 0] < 0).all(-1)
    assert allhit.sum() > 50 and allmiss.sum() > 50
    np.testing.assert_allclose(rgb[0][allhit], np.tile(a, (allhit.sum(), 1)), atol=1e-12)
    np.testing.assert_allclose(rgb[0][allmiss], 1.0, atol=0)
    assert hit.any()


def test_white_furnace_depth1_is_black(orc):
    s = _sphere_scene([0.5, 0.5, 0.5, 0.5, 0])
    sc = _scene(orc, s)
    cams = np.stack([inputs.camera((0, 0, 0), np.eye(3), 20.0)])
    rgb = sc.render(cams, 8, 8, 2, 1, seed=1)
    assert np.all(rgb[0, 3:5, 3:5] == 0.0)


def test_ggx_furnace_energy_bounded(orc):
    s = _sphere_scene([1.0, 1.0, 1.0, 0.3, 1])
    sc = _scene(orc, s)
    cams = np.stack([inputs.camera((0, 0, 0), np.eye(3), 60.0)])
    rgb, rec = sc.render(cams, 16, 16, 64, 2, seed=3, records=True)
    allhit = (rec[0, :, :, :, 0, 0] >= 0).all(-1)
    v = rgb[0][allhit]
    assert np.all(v <= 1.0 + 1e-12)
    assert v.mean() > 0.7


# ------------------------------------------- renderer: quad light over a plane
def _polygon_irradiance(x, n, verts, Le):
    """Lambert's formula: E = (Le / 2) sum_i Theta_i (n . Gamma_i)."""
    E = 0.0
    for i in range(len(verts)):
        a, b = verts[i] - x, verts[(i + 1) % len(verts)] - x
        th = math.acos(np.clip(np.dot(a, b) / np.linalg.norm(a) / np.linalg.norm(b), -1, 1))
        g = np.cross(a, b)
        E += th * np.dot(n, g / np.linalg.norm(g))
    return abs(0.5 * Le * E)


def _plane_light_scene(mat, light_p0=(-0.3, 1.0, -0.5)):
    return {"tris": np.asarray(inputs._quad((-50, 0, 50), (0, 0, -100), (100, 0, 0)), np.float32),
            "tri_mat": np.zeros(2, np.uint32), "materials": np.asarray([mat], np.float32),
            "lights": np.asarray([list(light_p0) + [0.6, 0, 0, 0, 0, 0.4, 10, 10, 10]], np.float32),
            "env": 0.0}


def _pixel_camera(eye, target):
    R = inputs.look_rot(np.asarray(target, float) - np.asarray(eye, float))
    return inputs.camera(eye, R, 1e-4)


@pytest.mark.parametrize("target", [(0.0, 0.0, -0.3), (0.7, 0.0, 0.4)])
def test_emitter_over_diffuse_plane_closed_form(orc, target):
    a = np.array([0.5, 0.6, 0.7])
    s = _plane_light_scene(list(a) + [0.5, 0])
    sc = _scene(orc, s)
    eye = np.array([2.5, 0.8, 0.3])
    F, spp = 48, 512
    cams = np.stack([_pixel_camera(eye, target)] * F)
    rgb = sc.render(cams, 1, 1, spp, 2, seed=17)[:, 0, 0]
    L = s["lights"][0].astype(np.float64)
    verts = [L[0:3], L[0:3] + L[3:6], L[0:3] + L[3:6] + L[6:9], L[0:3] + L[6:9]]
    E = _polygon_irradiance(np.asarray(target, float), np.array([0, 1.0, 0]), verts, 10.0)
    expect = a * E / math.pi
    mean, sd = rgb.mean(0), rgb.std(0, ddof=1) / math.sqrt(F)
    assert np.all(np.abs(mean - expect) <= 4 * sd + 1e-4 * expect), (mean, expect, sd)


def test_emitter_over_glossy_plane_quadrature(orc):
    """GGX plane under the quad light: the renderer's MIS estimate equals the
    light-area quadrature of the (separately pinned) BSDF evaluation."""
    mat = [0.8, 0.7, 0.6, 0.3, 1]
    s = _plane_light_scene(mat)
    sc = _scene(orc, s)
    target = np.array([0.1, 0.0, -0.1])
    eye = np.array([1.5, 0.6, 0.2])
    F, spp = 48, 512
    cams = np.stack([_pixel_camera(eye, target)] * F)
    rgb = sc.render(cams, 1, 1, spp, 2, seed=5)[:, 0, 0]
    L = s["lights"][0].astype(np.float64)
    n = 300
    u = (np.arange(n) + 0.5) / n
    U, V = np.meshgrid(u, u, indexing="ij")
    P = L[0:3] + U.reshape(-1, 1) * L[3:6] + V.reshape(-1, 1) * L[6:9]
    area = np.linalg.norm(np.cross(L[3:6], L[6:9]))
    d = P - target
    r2 = (d * d).sum(1)
    wi = d / np.sqrt(r2)[:, None]
    cos_l = wi[:, 1]                      # light normal is -y
    wo = eye - target
    wo = wo / np.linalg.norm(wo)
    # local frame with normal +y -> z
    to_local = lambda w: np.stack([w[..., 0], w[..., 2], w[..., 1]], -1)
    fc, _ = orc.bsdf_eval(mat, np.tile(to_local(wo), (len(wi), 1)), to_local(wi))
    expect = (fc * 10.0 * (cos_l / r2)[:, None]).sum(0) * area / (n * n)
    mean, sd = rgb.mean(0), rgb.std(0, ddof=1) / math.sqrt(F)
    assert np.all(np.abs(mean - expect) <= 4 * sd + 2e-3 * expect), (mean, expect, sd)


# ---------------------------------------------------- renderer: MC convergence
def test_mc_convergence_and_variance(orc):
    s = inputs.cornell_box()
    sc = _scene(orc, s)
    W = H = 12
    cams1 = np.stack([inputs.cornell_path(1)[0]] * 256)
    r1 = sc.render(cams1, W, H, 1, 4, seed=0)                    # 256 frames x 1 spp
    r4 = sc.render(cams1[:64], W, H, 4, 4, seed=1)               # 64 frames x 4 spp
    ref = sc.render(cams1[:1], W, H, 1024, 4, seed=2)[0]
    lum = lambda x: x @ np.array([0.2126, 0.7152, 0.0722])
    m1, m4, mr = lum(r1.mean(0)), lum(r4.mean(0)), lum(ref)
    assert np.mean(np.abs(m1 - mr)) < 0.1 * np.mean(mr)
    assert np.mean(np.abs(m4 - mr)) < 0.1 * np.mean(mr)
    v1, v4 = lum(r1).var(0).mean(), lum(r4).var(0).mean()
    assert 2.5 < v1 / v4 < 6.0                                    # variance ~ 1 / N


def test_camera_orientation(orc):
    s = inputs.cornell_box()
    sc = _scene(orc, s)
    rgb, rec = sc.render(inputs.cornell_path(1), 16, 16, 1, 1, seed=0, records=True)
    prim = rec[0, :, :, 0, 0, 0]
    frac = lambda v, s: np.isin(v, list(s)).mean()
    assert frac(prim[0, 1:15], {2, 3, 30, 31}) > 0.8               # ceiling / light on top
    assert frac(prim[1:11, 0], {6, 7}) >= 0.7                      # left wall on the left
    assert frac(prim[1:11, 15], {8, 9}) > 0.6                      # right wall on the right
    assert frac(prim[12:16, 0:6], set(range(10, 20))) > 0.8        # box 1 (x < 0) bottom left
    assert frac(prim[12:16, 10:14], set(range(20, 30))) > 0.8      # box 2 (x > 0) bottom right


def test_conditioning_record_of_a_plane_under_a_quad_light(orc):
    """The optional conditioning record (test infrastructure) leaves the
    radiance unchanged and holds the path's geometry: for a GGX plane of
    roughness 0.2 under a parallel quad light at height 1, every next-event
    sample has light-side cosine h / |p - x| >= 1 / sqrt(1 + r_max^2) and the
    same surface-side cosine (the two planes are parallel), and the roughness
    record is 0.2."""
    s = _plane_light_scene([0.8, 0.8, 0.8, 0.2, 1])
    sc = _scene(orc, s)
    target = np.array([0.0, 0.0, -0.3])
    cams = np.stack([_pixel_camera((0.0, 0.5, 1.0), target)])
    rgb0 = sc.render(cams, 1, 1, 64, 2, seed=4)
    rgb, cd = sc.render(cams, 1, 1, 64, 2, seed=4, cond=True)
    np.testing.assert_array_equal(rgb, rgb0)
    cosl, cosi, alpha = cd[0, 0, 0]
    corners = np.array([[-0.3, 1.0, -0.5], [0.3, 1.0, -0.5], [-0.3, 1.0, -0.1], [0.3, 1.0, -0.1]])
    r_max = max(np.hypot(c[0] - target[0], c[2] - target[2]) for c in corners)
    assert 1.0 / math.sqrt(1.0 + r_max ** 2) - 1e-3 <= cosl <= 1.0
    assert abs(cosl - cosi) < 1e-3
    assert alpha == pytest.approx(0.2, rel=1e-6)
