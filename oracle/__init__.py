"""Oracle for the EventTracer hot path (arXiv 2508.18071).

TEST INFRASTRUCTURE ONLY.  A plain, slow FP64 CPU restatement of what the
method computes, used to check the CUDA library.  Only ``tests/``,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import it.
It shares no code with the library: the renderer, BVH, event generator and
EvSNet forward are plain C (``liboracle.so``, built by ``oracle/build.py``); the
losses are NumPy; the training gradients are PyTorch float64 autograd on CPU.

Paper passages followed (section / equation of the paper):
  * Sec. 3.2          frames I_k at t_k = k / F_evt rendered by Monte Carlo
                      path tracing (estimator: the project's, see trace.c)
  * Eq. 1             luminance, log map, X_k = L^log_k - L^log_{k-1}
  * Sec. 3.1          contrast-threshold events
  * Eq. 2-3           LIF charge / fire / reset and the bipolar BiLIF fire
  * Eq. 4             surrogate derivative of the bipolar spike
  * Eq. 5-6           EvSNet encoder, residual blocks, projection
  * Eq. 7-11          1-D EMD, bidirectional EMD, polarity split, count loss,
                      total loss
Every function below is pinned by tests in ``tests/test_oracle_*.py`` against
closed forms, published test vectors, brute force or invariants.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        i64, i32 = C.c_int64, C.c_int
        L.orc_philox4x32_10.argtypes = [P, P, P, i64]
        L.orc_scene_new.argtypes = [P, P, i64, P, i32, P, i32, C.c_double, i32]
        L.orc_scene_new.restype = P
        L.orc_scene_free.argtypes = [P]
        L.orc_scene_ntris.argtypes = [P]
        L.orc_scene_ntris.restype = i64
        L.orc_bvh_sah_cost.argtypes = [P]
        L.orc_bvh_sah_cost.restype = C.c_double
        L.orc_bvh_nodes.argtypes = [P]
        L.orc_bvh_nodes.restype = i64
        L.orc_intersect.argtypes = [P, P, P, P, i64, P, P, P, P]
        L.orc_occluded.argtypes = [P, P, P, P, i64, P]
        L.orc_render.argtypes = [P, P, i32, i32, i32, i32, i32, i32, i32, i32, C.c_uint64, P, P,
                                 P, i32, P]
        L.orc_render.restype = i32
        L.orc_logl.argtypes = [P, i64, i32, C.c_double, P]
        L.orc_threshold_events.argtypes = [P, i32, i32, i32, C.c_double, i32, P, P, P, i64]
        L.orc_threshold_events.restype = i64
        L.orc_evsnet_forward.argtypes = [P, i32, i32, i32, i32, i32, i32, i32, i32, i32, i32,
                                         C.c_double, C.c_double, C.c_double, P, P, i32, P, P, P,
                                         P, P, i64, P, P, i32]
        L.orc_evsnet_forward.restype = i64
        L.orc_sensor_events.argtypes = [P, i32, i32, i32, C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_double, C.c_double, C.c_uint64, i32, P,
                                        P, P, i64]
        L.orc_sensor_events.restype = i64
        L.orc_sensor_thresholds.argtypes = [i64, C.c_double, C.c_double, C.c_uint64, P]
        L.orc_annotations.argtypes = [P, P, i32, P, i32, i32, P, P, P, P, P]
        L.orc_event_matches.argtypes = [P, i64, P, i64, i32]
        L.orc_event_matches.restype = i64
        L.orc_bsdf_eval.argtypes = [P, P, P, i64, P, P]
        L.orc_bsdf_sample.argtypes = [P, P, P, i64, P, P, P, P]
        L.orc_bvh_export.argtypes = [P, P, P, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# --------------------------------------------------------------------- Philox
def philox4x32_10(ctr, key):
    """Philox4x32-10 blocks; ctr [n,4] u32, key [n,2] u32 -> [n,4] u32."""
    ctr = _c(ctr, np.uint32).reshape(-1, 4)
    key = _c(key, np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    lib().orc_philox4x32_10(_p(ctr), _p(key), _p(out), ctr.shape[0])
    return out


def u01(x):
    """u32 -> [0,1) with 24 bits: (x >> 8) * 2^-24."""
    return (np.asarray(x, dtype=np.uint32) >> 8).astype(np.float64) * 2.0 ** -24


# ---------------------------------------------------------------------- scene
class Scene:
    """FP64 scene: user triangles plus two emitting triangles per quad light.

    tris [n,9] float32, tri_mat [n] u32, materials [m,5] (albedo rgb, roughness,
    type 0 Lambert / 1 GGX), lights [l,12] float32 (p0, e1, e2, radiance).
    """

    def __init__(self, tris, tri_mat, materials, lights, env=0.0, use_bvh=True):
        self.tris = _c(tris, np.float32).reshape(-1, 9)
        self.tri_mat = _c(tri_mat, np.uint32).reshape(-1)
        mats = np.zeros((max(len(materials), 1), 8), np.float64)
        m = np.asarray(materials, np.float64).reshape(-1, 5)
        mats[: len(m), :5] = m
        self.mats = mats
        self.lights = _c(lights, np.float32).reshape(-1, 12)
        self.env = float(env)
        self._h = lib().orc_scene_new(_p(self.tris), _p(self.tri_mat), self.tris.shape[0],
                                      _p(self.mats), len(m), _p(self.lights),
                                      self.lights.shape[0], self.env, int(bool(use_bvh)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_scene_free(h)
            self._h = None

    @property
    def ntris(self):
        return lib().orc_scene_ntris(self._h)

    def sah_cost(self):
        return lib().orc_bvh_sah_cost(self._h)

    def bvh_nodes(self):
        return lib().orc_bvh_nodes(self._h)

    def bvh(self):
        """(bounds [n,6], links [n,4] (left, right, first, count), perm [ntris])."""
        n = self.bvh_nodes()
        bounds = np.zeros((n, 6))
        links = np.zeros((n, 4), np.int32)
        perm = np.zeros(self.ntris, np.int32)
        lib().orc_bvh_export(self._h, _p(bounds), _p(links), _p(perm))
        return bounds, links, perm

    def intersect(self, o, d, tmax=None, counts=False):
        o = _c(o, np.float64).reshape(-1, 3)
        d = _c(d, np.float64).reshape(-1, 3)
        n = o.shape[0]
        tm = None if tmax is None else _c(tmax, np.float64).reshape(-1)
        t = np.empty(n, np.float64)
        p = np.empty(n, np.int32)
        nv = np.zeros(1, np.int64)
        nt = np.zeros(1, np.int64)
        lib().orc_intersect(self._h, _p(o), _p(d), _p(tm), n, _p(t), _p(p), _p(nv), _p(nt))
        if counts:
            return t, p, int(nv[0]), int(nt[0])
        return t, p

    def occluded(self, o, d, tmax):
        o = _c(o, np.float64).reshape(-1, 3)
        d = _c(d, np.float64).reshape(-1, 3)
        tm = _c(tmax, np.float64).reshape(-1)
        out = np.empty(o.shape[0], np.uint8)
        lib().orc_occluded(self._h, _p(o), _p(d), _p(tm), o.shape[0], _p(out))
        return out.astype(bool)

    def render(self, cams, W, H, spp, max_depth, seed, first_frame=0, rows=None,
               records=False, nthreads=0, cond=False):
        """Mean radiance per pixel, [F,H,W,3] float64 (rows outside `rows` stay 0).
        records=True adds the per-sample path records; cond=True adds [F,H,W,3]:
        the smallest light-side cosine, next-event surface cosine and GGX
        roughness met by the pixel's paths (see oracle.h)."""
        cams = _c(cams, np.float32).reshape(-1, 13)
        F = cams.shape[0]
        y0, y1 = (0, H) if rows is None else rows
        rgb = np.zeros((F, H, W, 3), np.float64)
        rec = np.full((F, H, W, spp, max_depth, 2), -3, np.int32) if records else None
        cd = np.full((F, H, W, 3), np.inf) if cond else None
        nr = np.zeros(3, np.int64)
        lib().orc_render(self._h, _p(cams), F, first_frame, W, H, y0, y1, spp, max_depth,
                         C.c_uint64(seed), _p(rgb), _p(rec), _p(cd), nthreads, _p(nr))
        # rays traced (closest + shadow), BVH nodes visited, triangles tested
        self.rays_traced, self.node_visits, self.tri_tests = (int(v) for v in nr)
        out = (rgb,) + ((rec,) if records else ()) + ((cd,) if cond else ())
        return out if len(out) > 1 else rgb

    def annotations(self, cams, W, H, next_cam=None):
        """Primary-hit annotations through pixel centres: dict of depth [F,H,W],
        normal [F,H,W,3], prim [F,H,W] (-1 miss), material [F,H,W] (-1 miss),
        flow [F,H,W,2] (pixels to the next frame's image)."""
        cams = _c(cams, np.float32).reshape(-1, 13)
        F = cams.shape[0]
        nxt = None if next_cam is None else _c(next_cam, np.float32).reshape(13)
        out = {"depth": np.empty((F, H, W)), "normal": np.empty((F, H, W, 3)),
               "prim": np.empty((F, H, W), np.int32), "material": np.empty((F, H, W), np.int64),
               "flow": np.empty((F, H, W, 2))}
        lib().orc_annotations(self._h, _p(cams), F, _p(nxt), W, H, _p(out["depth"]), _p(out["normal"]),
                              _p(out["prim"]), _p(out["material"]), _p(out["flow"]))
        return out


def bsdf_eval(material, wo, wi):
    """f cos(theta_i) [n,3] and pdf [n] in a local frame with the normal along +z."""
    m = np.asarray(material, np.float64).reshape(5)
    wo = _c(wo, np.float64).reshape(-1, 3)
    wi = _c(wi, np.float64).reshape(-1, 3)
    n = wo.shape[0]
    fc = np.empty((n, 3))
    pdf = np.empty(n)
    lib().orc_bsdf_eval(_p(m), _p(wo), _p(wi), n, _p(fc), _p(pdf))
    return fc, pdf


def bsdf_sample(material, wo, u):
    """(wi [n,3], weight f cos / pdf [n,3], pdf [n], ok [n]) from uniforms u [n,2]."""
    m = np.asarray(material, np.float64).reshape(5)
    wo = _c(wo, np.float64).reshape(-1, 3)
    u = _c(u, np.float64).reshape(-1, 2)
    n = wo.shape[0]
    wi, wt, pdf = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
    ok = np.empty(n, np.int32)
    lib().orc_bsdf_sample(_p(m), _p(wo), _p(u), n, _p(wi), _p(wt), _p(pdf), _p(ok))
    return wi, wt, pdf, ok.astype(bool)


# ---------------------------------------------------------- Eq. 1 log prologue
def logl(rgb, mode=0, p=1e-3):
    """Eq. 1 luminance + log map, rounded to float32 (mode 0: ln(L+eps))."""
    rgb = _c(rgb, np.float64)
    out = np.empty(rgb.shape[:-1], np.float32)
    lib().orc_logl(_p(rgb), out.size, mode, p, _p(out))
    return out


# ------------------------------------------------------- threshold generator
@dataclass
class ThresholdState:
    ref: np.ndarray
    initialized: int = 0

    @staticmethod
    def new(H, W):
        return ThresholdState(np.zeros(H * W, np.float64), 0)


def threshold_events(logl_frames, C_thr, state: ThresholdState, t0=0):
    """Contrast-threshold events from float32 log frames [F,H,W] -> int32 [n,4] (x,y,t,p).

    The threshold C is a float32 quantity (rounded here), widened to FP64 for the
    decision."""
    lf = _c(logl_frames, np.float32)
    C_thr = float(np.float32(C_thr))
    F, H, W = lf.shape
    ini = C.c_int(state.initialized)
    cap = 1 << 16
    while True:
        ref = state.ref.copy()
        ini = C.c_int(state.initialized)
        ev = np.empty((cap, 4), np.int32)
        n = lib().orc_threshold_events(_p(lf), F, H, W, float(C_thr), t0, _p(ref), C.byref(ini),
                                       _p(ev), cap)
        if n <= cap:
            break
        cap = int(n)
    state.ref[:] = ref
    state.initialized = ini.value
    return ev[:n].copy()


# ------------------------------------------------------------ sensor model
@dataclass
class SensorParams:
    """Event-sensor model (oracle/sensor.c).  Float parameters are float32
    quantities (the library's interface), widened to FP64."""
    C: float = 0.2
    sigma_C: float = 0.0          # relative threshold mismatch (std)
    refractory_us: float = 0.0
    leak_hz: float = 0.0
    shot_hz: float = 0.0
    frame_hz: float = 1000.0
    seed: int = 0

    def f64(self):
        return tuple(float(np.float32(v)) for v in (self.C, self.sigma_C, self.refractory_us,
                                                     self.leak_hz, self.shot_hz, self.frame_hz))


@dataclass
class SensorState:
    s: np.ndarray                 # [H*W][3]: reference, last event time, previous log intensity
    initialized: int = 0

    @staticmethod
    def new(H, W):
        return SensorState(np.zeros((H * W, 3), np.float64), 0)


def sensor_events(logl_frames, prm: SensorParams, state: SensorState, t0=0):
    """Sensor-model events from float32 log frames [F,H,W] -> int64 [n,4]
    (x, y, t in microseconds, p), in pixel order."""
    lf = _c(logl_frames, np.float32)
    F, H, W = lf.shape
    C_, sg, tr, lk, sh, fr = prm.f64()
    cap = 1 << 16
    while True:
        st = state.s.copy()
        ini = C.c_int(state.initialized)
        ev = np.empty((cap, 4), np.int64)
        n = lib().orc_sensor_events(_p(lf), F, H, W, C_, sg, tr, lk, sh, fr, int(prm.seed), t0,
                                    _p(st), C.byref(ini), _p(ev), cap)
        if n <= cap:
            break
        cap = int(n)
    state.s[:] = st
    state.initialized = ini.value
    return ev[:n].copy()


def sensor_thresholds(npix, prm: SensorParams):
    """Per-pixel (C_on, C_off) [npix, 2] of the mismatch model."""
    C_, sg = prm.f64()[:2]
    out = np.empty((npix, 2), np.float64)
    lib().orc_sensor_thresholds(npix, C_, sg, int(prm.seed), _p(out))
    return out


# --------------------------------------------------------------------- EvSNet
@dataclass
class EvsNet:
    """EvSNet weights in the packed layout (see events.c)."""
    kind: int          # 0 plain stack of convs, 1 residual (Eq. 5)
    n_layers: int
    C: int
    kt: int
    ks: int
    beta: float
    vth: float
    reset: float
    w: np.ndarray      # flat float64
    b: np.ndarray      # flat float64
    ks0: int = 0       # > 0: layer 0 is a one-step ks0 x ks0 spatial convolution (a stem)
    delay: int = 0     # events of step k are labelled t0 + k - delay

    @staticmethod
    def from_dict(d):
        """From a weights dictionary (keys as in the package's inputs module)."""
        return EvsNet(int(d["kind"]), int(d["n_layers"]), int(d["C"]), int(d["kt"]), int(d["ks"]),
                      float(d["beta"]), float(d["vth"]), float(d["reset"]),
                      np.asarray(d["w"], np.float64), np.asarray(d["b"], np.float64),
                      int(d.get("ks0", 0)), int(d.get("delay", 0)))

    def layer_shape(self, i):
        """(Cin, kt, ks) of conv layer i."""
        if i == 0:
            return (1, 1, self.ks0) if self.ks0 > 0 else (1, self.kt, self.ks)
        return self.C, self.kt, self.ks

    def n_weights(self):
        n = 0
        for i in range(self.n_layers):
            cin, kt, ks = self.layer_shape(i)
            n += self.C * cin * kt * ks * ks
        return n + self.C

    def layer_weights(self):
        """list of (W [Cout,Cin,kt,ks,ks], b [Cout]) plus the projection (W [C], b [1])."""
        out, wo, bo = [], 0, 0
        for i in range(self.n_layers):
            cin, kt, ks = self.layer_shape(i)
            n = self.C * cin * kt * ks * ks
            out.append((self.w[wo:wo + n].reshape(self.C, cin, kt, ks, ks),
                        self.b[bo:bo + self.C]))
            wo += n
            bo += self.C
        return out, (self.w[wo:wo + self.C], self.b[bo:bo + 1])


@dataclass
class EvsState:
    V: np.ndarray
    hist: np.ndarray
    last_l: np.ndarray
    initialized: int = 0

    @staticmethod
    def new(net: EvsNet, H, W, V0=None):
        nh = net.n_layers * max(net.kt - 1, 0) * net.C * H * W
        V = np.zeros(H * W) if V0 is None else np.asarray(V0, np.float64).reshape(-1).copy()
        return EvsState(V, np.zeros(max(nh, 1)), np.zeros(H * W), 0)


def evsnet_forward(logl_frames, net: EvsNet, state: EvsState, t0=0, want_I=False,
                   want_margin=False, nthreads=0):
    """EvSNet + BiLIF forward over float32 log frames [F,H,W].

    Returns (events int32 [n,4] sorted by (t,y,x), I [K,H,W] or None, margin [H,W] or None).
    `margin` is the smallest distance of V' to +-Vth seen by each pixel.
    """
    lf = _c(logl_frames, np.float32)
    F, H, W = lf.shape
    K = F - (0 if state.initialized else 1)
    I = np.zeros((max(K, 1), H, W)) if want_I else None
    mg = np.full(H * W, np.inf) if want_margin else None
    w = _c(net.w, np.float64)
    b = _c(net.b, np.float64)
    cap = max(1 << 16, H * W * 4)
    while True:
        V, hist, last = state.V.copy(), state.hist.copy(), state.last_l.copy()
        ini = C.c_int(state.initialized)
        ev = np.empty((cap, 4), np.int32)
        if mg is not None:
            mg[:] = np.inf
        n = lib().orc_evsnet_forward(_p(lf), F, H, W, net.kind, net.n_layers, net.C, net.kt,
                                     net.ks, net.ks0, net.delay, net.beta, net.vth, net.reset,
                                     _p(w), _p(b), t0,
                                     _p(V), _p(hist), _p(last), C.byref(ini), _p(ev), cap,
                                     _p(I), _p(mg), nthreads)
        if n <= cap:
            break
        cap = int(n)
    state.V[:], state.hist[:], state.last_l[:] = V, hist, last
    state.initialized = ini.value
    return ev[:n].copy(), (I[:K] if I is not None else None), \
        (mg.reshape(H, W) if mg is not None else None)


# ------------------------------------------------------------------ event F1
def event_matches(A, B, delta):
    A = _c(A, np.int32).reshape(-1, 4)
    B = _c(B, np.int32).reshape(-1, 4)
    return int(lib().orc_event_matches(_p(A), A.shape[0], _p(B), B.shape[0], int(delta)))


def event_f1(pred, ref, delta):
    """F1 of predicted vs reference events; both empty -> 1."""
    npred, nref = len(pred), len(ref)
    if npred == 0 and nref == 0:
        return 1.0
    if npred == 0 or nref == 0:
        return 0.0
    m = event_matches(pred, ref, delta)
    P, R = m / npred, m / nref
    return 0.0 if m == 0 else 2 * P * R / (P + R)


def sort_events(ev):
    ev = np.asarray(ev, np.int32).reshape(-1, 4)
    if len(ev) == 0:
        return ev
    order = np.lexsort((ev[:, 3], ev[:, 0], ev[:, 1], ev[:, 2]))
    return ev[order]


def events_to_dense(ev, K, H, W, t0=1):
    """Signed event count per (step, pixel): [K,H,W] with step = t - t0."""
    E = np.zeros((K, H, W), np.float64)
    ev = np.asarray(ev).reshape(-1, 4)
    np.add.at(E, (ev[:, 2] - t0, ev[:, 1], ev[:, 0]), ev[:, 3])
    return E


# -------------------------------------------------------- Eq. 7-11 losses
def emd_1d(E, S):
    """Eq. 7 per pixel: (1/K) sum_i |cumsum(S)_i - cumsum(E)_i|; axis 0 is time."""
    E = np.asarray(E, np.float64)
    S = np.asarray(S, np.float64)
    K = E.shape[0]
    return np.abs(np.cumsum(S, 0) - np.cumsum(E, 0)).sum(0) / K


def emd_bidir(E, S):
    """Eq. 8: half the forward EMD plus the EMD of the reversed sequences."""
    return 0.5 * (emd_1d(E, S) + emd_1d(E[::-1], S[::-1]))


def total_loss(E, S_on, S_off, lam=0.01):
    """Eq. 9-11 with E signed counts [K,...]; returns (total, emd, count) means over pixels."""
    E = np.asarray(E, np.float64)
    Eon, Eoff = np.maximum(E, 0), np.maximum(-E, 0)
    emd = emd_bidir(Eon, S_on) + emd_bidir(Eoff, S_off)
    cnt = np.abs((np.asarray(S_on) + np.asarray(S_off)).sum(0) - np.abs(E).sum(0))
    return float(np.mean(emd) + lam * np.mean(cnt)), float(np.mean(emd)), float(np.mean(cnt))


# ------------------------------------------------- training (torch float64)
def _torch():
    import torch
    return torch


def surrogate_sigma(x, alpha):
    """Arctangent surrogate sigma(x) = 1/2 + arctan(pi alpha x / 2) / pi."""
    torch = _torch()
    return 0.5 + torch.atan(math.pi * alpha * x / 2) / math.pi


def _heaviside_fn():
    torch = _torch()

    class Heaviside(torch.autograd.Function):
        """Theta(x) (x >= 0 fires) forward; Eq. 4 surrogate d sigma / dx backward."""

        @staticmethod
        def forward(ctx, x, alpha):
            ctx.save_for_backward(x)
            ctx.alpha = alpha
            return (x >= 0).to(x.dtype)

        @staticmethod
        def backward(ctx, g):
            (x,) = ctx.saved_tensors
            a = ctx.alpha
            return g * (a / 2) / (1 + (math.pi * a * x / 2) ** 2), None

    return Heaviside


def torch_forward(X, net: EvsNet, params=None, smooth=False, alpha=2.0, V0=None, round_bf16=False):
    """EvSNet on log differences X [B,K,H,W] (torch float64); returns (S_on, S_off, I, Vp).

    round_bf16: the library's BF16 mode -- the weights of layers 1.. and their
    input activations rounded to BF16 (round to nearest even), every sum exact.

    Spikes (Eq. 3, reading: fire on V'): S_on = Theta(V' - Vth), S_off =
    Theta(-V' - Vth), S = S_on - S_off, reset V = V' - r S (not detached).
    `smooth` replaces Theta by sigma in the forward (the smooth surrogate
    network, whose exact gradient finite differences can check).
    """
    torch = _torch()
    F = torch.nn.functional
    B, K, H, W = X.shape
    layers, (wp, bp) = params if params is not None else torch_params(net)

    def conv(h, Wt, bt):
        # h [B, Cin, K, H, W]; causal in time, zero-padded in space (the
        # kernel's own extent: a stem layer 0 is one step by ks0 x ks0)
        kt, pad = Wt.shape[2], Wt.shape[3] // 2
        h = F.pad(h, (pad, pad, pad, pad, kt - 1, 0))
        return F.conv3d(h, Wt, bt)

    def rb(t):
        return t.to(torch.bfloat16).to(t.dtype) if round_bf16 else t

    def convr(h, Wt, bt):
        # a tensor-core layer: BF16 operands in the library's BF16 mode
        return conv(rb(h), rb(Wt), bt)

    x = X.unsqueeze(1)
    h = torch.relu(conv(x, *layers[0]))
    if net.kind == 0:
        for Wt, bt in layers[1:]:
            h = torch.relu(convr(h, Wt, bt))
    else:
        for j in range(1, net.n_layers - 1, 2):
            a = torch.relu(convr(h, *layers[j]))
            h = torch.relu(h + convr(a, *layers[j + 1]))
    I = torch.einsum("bckhw,c->bkhw", h, wp) + bp[0]
    Hv = _heaviside_fn()
    V = torch.zeros(B, H, W, dtype=X.dtype) if V0 is None else V0
    Son, Soff, Vps = [], [], []
    for k in range(K):
        vp = net.beta * V + I[:, k]
        if smooth:
            son = surrogate_sigma(vp - net.vth, alpha)
            soff = surrogate_sigma(-vp - net.vth, alpha)
        else:
            son = Hv.apply(vp - net.vth, alpha)
            soff = Hv.apply(-vp - net.vth, alpha)
        V = vp - net.reset * (son - soff)
        Son.append(son)
        Soff.append(soff)
        Vps.append(vp)
    return torch.stack(Son, 1), torch.stack(Soff, 1), I, torch.stack(Vps, 1)


def torch_params(net: EvsNet, requires_grad=False):
    torch = _torch()
    layers, (wp, bp) = net.layer_weights()
    L = [(torch.tensor(W, dtype=torch.float64, requires_grad=requires_grad),
          torch.tensor(b, dtype=torch.float64, requires_grad=requires_grad)) for W, b in layers]
    return L, (torch.tensor(wp, dtype=torch.float64, requires_grad=requires_grad),
               torch.tensor(bp, dtype=torch.float64, requires_grad=requires_grad))


def torch_loss(E, S_on, S_off, lam=0.01):
    """Eq. 7-11 on torch tensors; E signed counts [B,K,H,W]; mean over B*H*W pixels."""
    torch = _torch()
    K = E.shape[1]
    Eon, Eoff = torch.clamp(E, min=0), torch.clamp(-E, min=0)

    def L1(e, s):
        return (torch.cumsum(s, 1) - torch.cumsum(e, 1)).abs().sum(1) / K

    def L2(e, s):
        return 0.5 * (L1(e, s) + L1(e.flip(1), s.flip(1)))

    emd = L2(Eon, S_on) + L2(Eoff, S_off)
    cnt = ((S_on + S_off).sum(1) - E.abs().sum(1)).abs()
    return emd.mean() + lam * cnt.mean()


def torch_grads(X, E, net: EvsNet, smooth=False, alpha=2.0, lam=0.01):
    """Loss and its gradient w.r.t. the packed weights (flat w, flat b), float64."""
    torch = _torch()
    params = torch_params(net, requires_grad=True)
    Son, Soff, _, _ = torch_forward(torch.as_tensor(X, dtype=torch.float64), net, params,
                                    smooth=smooth, alpha=alpha)
    loss = torch_loss(torch.as_tensor(E, dtype=torch.float64), Son, Soff, lam)
    loss.backward()
    layers, (wp, bp) = params
    gw = np.concatenate([Wt.grad.numpy().ravel() for Wt, _ in layers] + [wp.grad.numpy().ravel()])
    gb = np.concatenate([bt.grad.numpy().ravel() for _, bt in layers] + [bp.grad.numpy().ravel()])
    return float(loss.detach()), gw, gb


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma & Ba 2015, Algorithm 1), bias-corrected, in float64; returns new p,m,v."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
