"""Python surface of libeventtracer: the same calls as include/eventtracer.h.

PyTorch provides device memory and streams; these functions only marshal
arguments into the C ABI.  All tensors passed as device buffers must be CUDA
tensors on the current device.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import _lib as L


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


# ----------------------------------------------------------------------- scene
class Scene:
    """et_build_scene: geometry + BVH on the device (see inputs.py for the dict layout).
    builder: None (the library's default, "gpu_sweep"), "gpu_sweep", "gpu", "host" or "sweep"
    (et_build_scene_with)."""

    BUILDERS = {"gpu": L.ET_BVH_GPU, "host": L.ET_BVH_HOST, "sweep": L.ET_BVH_SWEEP,
                "gpu_sweep": L.ET_BVH_GPU_SWEEP}

    def __init__(self, scene: dict, stream=None, builder=None):
        lib = L.load()
        tris = np.ascontiguousarray(scene["tris"], np.float32).reshape(-1, 9)
        tri_mat = np.ascontiguousarray(scene["tri_mat"], np.uint32).reshape(-1)
        mats = np.asarray(scene["materials"], np.float32).reshape(-1, 5)
        lights = np.asarray(scene["lights"], np.float32).reshape(-1, 12)
        cm = (L.et_material * max(len(mats), 1))()
        for i, m in enumerate(mats):
            cm[i].albedo[:] = [float(v) for v in m[:3]]
            cm[i].roughness = float(m[3])
            cm[i].type = int(m[4])
        cl = (L.et_quad_light * max(len(lights), 1))()
        for i, q in enumerate(lights):
            cl[i].p0[:] = [float(v) for v in q[0:3]]
            cl[i].e1[:] = [float(v) for v in q[3:6]]
            cl[i].e2[:] = [float(v) for v in q[6:9]]
            cl[i].radiance[:] = [float(v) for v in q[9:12]]
        h = C.c_void_p()
        if builder is None:
            st = lib.et_build_scene(tris.ctypes.data_as(C.c_void_p), tri_mat.ctypes.data_as(C.c_void_p),
                                    tris.shape[0], cm, len(mats), cl, len(lights),
                                    float(scene.get("env", 0.0)), C.byref(h), _stream(stream))
        else:
            st = lib.et_build_scene_with(tris.ctypes.data_as(C.c_void_p),
                                         tri_mat.ctypes.data_as(C.c_void_p), tris.shape[0], cm,
                                         len(mats), cl, len(lights), float(scene.get("env", 0.0)),
                                         self.BUILDERS[builder], C.byref(h), _stream(stream))
        L.check("et_build_scene", st)
        self._h = h
        self.n_user = tris.shape[0]

    def update(self, tris, stream=None):
        """et_scene_update: new positions (float [n_tris, 9], input order) for the
        scene's triangles; the hierarchy is refitted."""
        t = np.ascontiguousarray(tris, np.float32).reshape(-1, 9)
        if t.shape[0] != self.n_user:
            raise ValueError("expected %d triangles" % self.n_user)
        L.check("et_scene_update", L.load().et_scene_update(self._h, t.ctypes.data_as(C.c_void_p),
                                                             _stream(stream)))

    def set_mode(self, mode: int):
        """ET_RENDER_WAVEFRONT_TILES (default), ET_RENDER_WAVEFRONT_SORTED, ET_RENDER_WAVEFRONT or
        ET_RENDER_MEGAKERNEL."""
        L.check("et_render_set_mode", L.load().et_render_set_mode(self._h, int(mode)))

    PROFILE_KINDS = ("raygen", "trace", "shade", "shadow", "accumulate")

    def profile(self, enable: bool):
        """et_render_profile: record per-kernel events in later renders."""
        L.check("et_render_profile", L.load().et_render_profile(self._h, int(bool(enable))))

    def profile_read(self) -> dict:
        """et_render_profile_read: {kind: (ms, launches, items)} since the last read."""
        ms = (C.c_double * 5)()
        n = (C.c_int64 * 5)()
        it = (C.c_int64 * 5)()
        st = L.load().et_render_profile_read(self._h, ms, n, it)
        if st not in (L.ET_OK, L.ET_ERR_CAPACITY):
            L.check("et_render_profile_read", st)
        return {k: (ms[i], n[i], it[i] if st == L.ET_OK else None)
                for i, k in enumerate(self.PROFILE_KINDS)}

    def info(self):
        n, nn, sah = C.c_int64(), C.c_int64(), C.c_double()
        L.check("et_scene_info", L.load().et_scene_info(self._h, C.byref(n), C.byref(nn), C.byref(sah)))
        b = L.load().et_scene_builder(self._h)
        builder = {v: k for k, v in self.BUILDERS.items()}[b]
        return {"n_tris": n.value, "n_nodes": nn.value, "sah_cost": sah.value, "builder": builder}

    def free(self):
        if getattr(self, "_h", None):
            L.load().et_scene_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def cameras(cams) -> C.Array:
    cams = np.asarray(cams, np.float32).reshape(-1, 13)
    arr = (L.et_camera * max(len(cams), 1))()
    C.memmove(arr, np.ascontiguousarray(cams).ctypes.data, cams.nbytes)
    return arr


def render_frames(scene: Scene, cams, W, H, spp, max_depth, seed, first_frame=0, rgb=None,
                  logl=None, want_rgb=True, want_logl=True, log_mode=L.ET_LOG_EPS,
                  log_param=1e-3, records=False, stream=None, rows=None):
    """et_render_frames (or et_render_rows for rows = (y0, y1)); returns
    (rgb [F,h,W,3] or None, logl [F,h,W] or None, records or None), h = H or y1 - y0."""
    F = np.asarray(cams, np.float32).reshape(-1, 13).shape[0]
    cams_c = cameras(cams)
    dev = torch.device("cuda")
    y0, y1 = (0, H) if rows is None else (int(rows[0]), int(rows[1]))
    h = y1 - y0
    if want_rgb and rgb is None:
        rgb = torch.empty((F, h, W, 3), dtype=torch.float32, device=dev)
    if want_logl and logl is None:
        logl = torch.empty((F, h, W), dtype=torch.float32, device=dev)
    rec = torch.empty((F, h, W, spp, max_depth, 2), dtype=torch.int32, device=dev) if records else None
    args = (C.c_uint64(seed), _ptr(rgb if want_rgb else None), _ptr(logl if want_logl else None),
            log_mode, float(log_param), _ptr(rec), _stream(stream))
    if rows is None:
        st = L.load().et_render_frames(scene._h, cams_c, F, first_frame, W, H, spp, max_depth, *args)
    else:
        st = L.load().et_render_rows(scene._h, cams_c, F, first_frame, W, H, y0, y1, spp, max_depth,
                                     *args)
    L.check("et_render_frames", st)
    return (rgb if want_rgb else None), (logl if want_logl else None), rec


def render_annotations(scene: Scene, cams, W: int, H: int, next_cam=None, stream=None,
                       want=("depth", "normal", "prim", "material", "flow")) -> dict:
    """et_render_annotations: device tensors depth [F,H,W], normal [F,H,W,3], prim
    [F,H,W] (int32, -1 miss), material [F,H,W] (int32 holding the uint32 word:
    lights 0x80000000 | index, 0xFFFFFFFF miss) and flow [F,H,W,2] (pixels to
    the next camera's image)."""
    cams = np.ascontiguousarray(cams, np.float32).reshape(-1, 13)
    F = cams.shape[0]
    dev = torch.device("cuda")
    out = {}
    if "depth" in want:
        out["depth"] = torch.empty((F, H, W), dtype=torch.float32, device=dev)
    if "normal" in want:
        out["normal"] = torch.empty((F, H, W, 3), dtype=torch.float32, device=dev)
    if "prim" in want:
        out["prim"] = torch.empty((F, H, W), dtype=torch.int32, device=dev)
    if "material" in want:
        out["material"] = torch.empty((F, H, W), dtype=torch.int32, device=dev)
    if "flow" in want:
        out["flow"] = torch.empty((F, H, W, 2), dtype=torch.float32, device=dev)
    nxt = None if next_cam is None else np.ascontiguousarray(next_cam, np.float32).reshape(13)
    st = L.load().et_render_annotations(scene._h, cams.ctypes.data_as(C.c_void_p), F,
                                        None if nxt is None else nxt.ctypes.data_as(C.c_void_p), W, H,
                                        _ptr(out.get("depth")), _ptr(out.get("normal")),
                                        _ptr(out.get("prim")), _ptr(out.get("material")),
                                        _ptr(out.get("flow")), _stream(stream))
    L.check("et_render_annotations", st)
    return out


# ------------------------------------------------------------------ events
def decode_events(raw: torch.Tensor, n: int) -> np.ndarray:
    """Device et_event buffer (int32 [cap,3]) -> host int32 [n,4] (x, y, t, p)."""
    w = raw[:n].cpu().numpy().astype(np.int64)
    out = np.empty((n, 4), np.int32)
    out[:, 0] = w[:, 0] & 0xFFFF
    out[:, 1] = (w[:, 0] >> 16) & 0xFFFF
    out[:, 2] = w[:, 1]
    out[:, 3] = (w[:, 2] & 0xFF).astype(np.uint8).view(np.int8)
    return out


class EventBuffer:
    """Caller-owned device event buffer and count."""

    def __init__(self, cap: int):
        self.cap = int(cap)
        self.raw = torch.empty((max(self.cap, 1), 3), dtype=torch.int32, device="cuda")
        self.count = torch.zeros(1, dtype=torch.int64, device="cuda")

    TIMEOUT_BIT = 1 << 62

    def n(self) -> int:
        """Event count; raises if a kernel's bounded device-side wait gave up
        (the kernels signal that by setting bit 62 of the count)."""
        v = int(self.count.item())
        if v >= self.TIMEOUT_BIT:
            raise L.ETError("device-side wait", L.ET_ERR_TIMEOUT)
        return v

    def host(self) -> np.ndarray:
        n = self.n()
        if n > self.cap:
            raise L.ETError("event buffer", L.ET_ERR_CAPACITY)
        return decode_events(self.raw, n)


def threshold_events(logl: torch.Tensor, C_thr: float, ref: torch.Tensor, initialized: bool,
                     t0=0, buf: Optional[EventBuffer] = None, stream=None,
                     grow: bool = True) -> EventBuffer:
    """et_threshold_events on device log frames [F,H,W]; ref is device float64 [H*W].

    With grow=True and no caller buffer, an overflowing call is repeated once
    with a buffer of the reported size (the state is restored first); this
    synchronises the stream."""
    F, H, W = logl.shape
    own = buf is None
    if own:
        buf = EventBuffer(max(1 << 16, 4 * F * H * W))
    saved = ref.clone() if (own and grow) else None

    def call(b):
        st = L.load().et_threshold_events(_ptr(logl), F, H, W, float(C_thr), int(t0), _ptr(ref),
                                          int(bool(initialized)), _ptr(b.raw), b.cap,
                                          _ptr(b.count), _stream(stream))
        L.check("et_threshold_events", st)

    call(buf)
    if saved is not None:
        n = buf.n()
        if n > buf.cap:
            ref.copy_(saved)
            buf = EventBuffer(n)
            call(buf)
    return buf


def encode_events(ev: np.ndarray) -> np.ndarray:
    """host int32 [n,4] (x, y, t, p) -> packed et_event records (int32 [n,3])."""
    ev = np.asarray(ev, np.int64).reshape(-1, 4)
    out = np.empty((len(ev), 3), np.uint32)
    out[:, 0] = (ev[:, 0] & 0xFFFF) | ((ev[:, 1] & 0xFFFF) << 16)
    out[:, 1] = ev[:, 2]
    out[:, 2] = ev[:, 3].astype(np.int8).view(np.uint8)
    return out.view(np.int32)


def event_f1(pred: np.ndarray, ref: np.ndarray, delta: int) -> float:
    """Event F1 of two host event lists [n,4] via et_event_matches; both empty -> 1."""
    na, nb = len(pred), len(ref)
    if na == 0 and nb == 0:
        return 1.0
    a = np.ascontiguousarray(encode_events(pred))
    b = np.ascontiguousarray(encode_events(ref))
    m = C.c_int64()
    st = L.load().et_event_matches(a.ctypes.data_as(C.c_void_p), na, b.ctypes.data_as(C.c_void_p),
                                   nb, int(delta), C.byref(m))
    L.check("et_event_matches", st)
    return 2.0 * m.value / (na + nb)


def spike_f1(a: torch.Tensor, b: torch.Tensor, delta: int, stream=None) -> float:
    """Event F1 of two dense spike tensors (device int8 [K, H, W] of -1 / 0 / +1)
    via et_spike_matches; both silent -> 1."""
    assert a.shape == b.shape and a.dtype == torch.int8 and b.dtype == torch.int8
    a, b = a.contiguous(), b.contiguous()
    na, nb = int((a != 0).sum().item()), int((b != 0).sum().item())
    if na + nb == 0:
        return 1.0
    m = torch.zeros(1, dtype=torch.int64, device=a.device)
    K = a.shape[0]
    st = L.load().et_spike_matches(_ptr(a), _ptr(b), K, a.numel() // max(K, 1), int(delta), _ptr(m),
                                   _stream(stream))
    L.check("et_spike_matches", st)
    return 2.0 * int(m.item()) / (na + nb)


# ------------------------------------------------------------ sensor model
@dataclass
class SensorParams:
    """et_sensor_params: threshold C, relative mismatch sigma_C, refractory
    period (us), leak and shot-noise rates (Hz), frame rate (Hz), seed."""
    C: float = 0.2
    sigma_C: float = 0.0
    refractory_us: float = 0.0
    leak_hz: float = 0.0
    shot_hz: float = 0.0
    frame_hz: float = 1000.0
    seed: int = 0

    def c_struct(self):
        return L.et_sensor_params(self.C, self.sigma_C, self.refractory_us, self.leak_hz,
                                  self.shot_hz, self.frame_hz, int(self.seed))


class SensorStateDev:
    """Device state of the sensor model: double [H*W][3] (reference, time of the
    last event, previous log intensity)."""

    def __init__(self, H, W):
        self.H, self.W = H, W
        self.s = torch.zeros((H * W, 3), dtype=torch.float64, device="cuda")
        self.initialized = 0


def sensor_events(logl: torch.Tensor, prm: SensorParams, state: SensorStateDev, t0=0,
                  buf: Optional[EventBuffer] = None, stream=None, grow: bool = True) -> EventBuffer:
    """et_sensor_events on device log frames [F,H,W]; events carry t in
    microseconds.  With grow=True and no caller buffer an overflowing call is
    repeated once with a buffer of the reported size (state restored first)."""
    F, H, W = logl.shape
    own = buf is None
    if own:
        buf = EventBuffer(max(1 << 16, 2 * F * H * W))
    saved = state.s.clone() if (own and grow) else None
    cp = prm.c_struct()
    ini0 = state.initialized

    def call(b):
        st = L.load().et_sensor_events(_ptr(logl), F, H, W, C.byref(cp), int(t0), _ptr(state.s),
                                       int(ini0), _ptr(b.raw), b.cap, _ptr(b.count), _stream(stream))
        L.check("et_sensor_events", st)

    call(buf)
    if saved is not None:
        n = buf.n()
        if n > buf.cap:
            state.s.copy_(saved)
            buf = EventBuffer(n)
            call(buf)
    if F > 0:
        state.initialized = 1
    return buf


def philox4x32_10(ctr: torch.Tensor, key: torch.Tensor, stream=None) -> torch.Tensor:
    """et_philox4x32_10: the device generator on counters [n, 4] and keys [n, 2]
    (uint32 values held in int32 device tensors); returns [n, 4]."""
    ctr, key = ctr.contiguous(), key.contiguous()
    out = torch.empty_like(ctr)
    st = L.load().et_philox4x32_10(_ptr(ctr), _ptr(key), ctr.shape[0], _ptr(out), _stream(stream))
    L.check("et_philox4x32_10", st)
    return out


# ------------------------------------------------------------------ EvSNet
@dataclass
class EvsNetDev:
    kind: int
    n_layers: int
    C: int
    kt: int
    ks: int
    beta: float
    vth: float
    reset: float
    w: torch.Tensor
    b: torch.Tensor
    dtype: int = L.ET_F32
    ks0: int = 0
    delay: int = 0
    scales: Optional[torch.Tensor] = None   # FP8 pixel-wise form: device [n_layers - 1]

    @staticmethod
    def from_dict(d: dict, dtype=L.ET_F32):
        return EvsNetDev(d["kind"], d["n_layers"], d["C"], d["kt"], d["ks"], float(d["beta"]),
                         float(d["vth"]), float(d["reset"]),
                         torch.as_tensor(np.asarray(d["w"], np.float32)).cuda().contiguous(),
                         torch.as_tensor(np.asarray(d["b"], np.float32)).cuda().contiguous(), dtype,
                         int(d.get("ks0", 0)), int(d.get("delay", 0)))

    def c_struct(self, w=None, b=None):
        w = self.w if w is None else w
        b = self.b if b is None else b
        return L.et_evsnet_weights(self.kind, self.n_layers, self.C, self.kt, self.ks, self.beta,
                                   self.vth, self.reset, self.dtype, self.ks0, self.delay,
                                   w.data_ptr(), b.data_ptr(),
                                   self.scales.data_ptr() if self.scales is not None else None)


class EvsStateDev:
    """et_evsnet_state: device V, history and last log frame."""

    def __init__(self, net: EvsNetDev, H, W, V0: Optional[torch.Tensor] = None):
        self.H, self.W = H, W
        self.V = torch.zeros(H * W, dtype=torch.float32, device="cuda") if V0 is None \
            else V0.reshape(-1).float().cuda().clone()
        nh = net.n_layers * max(net.kt - 1, 0) * net.C * H * W
        self.hist = torch.zeros(max(nh, 1), dtype=torch.float32, device="cuda")
        self.last_l = torch.zeros(H * W, dtype=torch.float32, device="cuda")
        self.initialized = 0
        self._has_hist = net.kt > 1

    def c_struct(self):
        return L.et_evsnet_state(self.V.data_ptr(), self.hist.data_ptr() if self._has_hist else None,
                                 self.last_l.data_ptr(), self.H, self.W, self.initialized)

    def save(self, path: str):
        """Checkpoint: the state is plain buffers (V, temporal history, previous
        log frame) and the initialized flag; a clip resumed from it continues
        bit for bit."""
        np.savez(path, V=self.V.cpu().numpy(), hist=self.hist.cpu().numpy(),
                 last_l=self.last_l.cpu().numpy(), H=self.H, W=self.W,
                 initialized=self.initialized)

    @staticmethod
    def load(path: str, net: "EvsNetDev") -> "EvsStateDev":
        z = np.load(path)
        st = EvsStateDev(net, int(z["H"]), int(z["W"]))
        if z["hist"].shape != tuple(st.hist.shape):
            raise ValueError("state checkpoint does not match the network's history size")
        st.V.copy_(torch.as_tensor(z["V"]))
        st.hist.copy_(torch.as_tensor(z["hist"]))
        st.last_l.copy_(torch.as_tensor(z["last_l"]))
        st.initialized = int(z["initialized"])
        return st


def evsnet_fp8_scales(logl: torch.Tensor, net: EvsNetDev, state: EvsStateDev, headroom=4.0,
                      stream=None) -> torch.Tensor:
    """et_evsnet_fp8_scales: the FP8 pixel-wise form's per-layer input scales
    from a calibration clip (device float [n_layers - 1]); the state advances."""
    F = logl.shape[0]
    out = torch.empty(max(net.n_layers - 1, 1), dtype=torch.float32, device="cuda")
    cw = net.c_struct()
    cs = state.c_struct()
    st = L.load().et_evsnet_fp8_scales(_ptr(logl), F, C.byref(cw), C.byref(cs), float(headroom),
                                       _ptr(out), _stream(stream))
    L.check("et_evsnet_fp8_scales", st)
    state.initialized = cs.initialized
    return out[:net.n_layers - 1]


def evsnet_forward(logl: torch.Tensor, net: EvsNetDev, state: EvsStateDev, t0=0,
                   buf: Optional[EventBuffer] = None, want_I=False, want_spikes=False, stream=None):
    """et_evsnet_forward; returns (EventBuffer, I [K,H,W] or None, spikes [K,H,W] or None)."""
    F, H, W = logl.shape
    K = F - (0 if state.initialized else 1)
    if buf is None:
        buf = EventBuffer(max(1 << 16, max(K, 1) * H * W))
    I = torch.empty((max(K, 1), H, W), dtype=torch.float32, device="cuda") if want_I else None
    S = torch.empty((max(K, 1), H, W), dtype=torch.int8, device="cuda") if want_spikes else None
    cw = net.c_struct()
    cs = state.c_struct()
    st = L.load().et_evsnet_forward(_ptr(logl), F, C.byref(cw), C.byref(cs), int(t0), _ptr(buf.raw),
                                    buf.cap, _ptr(buf.count), _ptr(I), _ptr(S), _stream(stream))
    L.check("et_evsnet_forward", st)
    state.initialized = cs.initialized
    return buf, (I[:K] if I is not None else None), (S[:K] if S is not None else None)
